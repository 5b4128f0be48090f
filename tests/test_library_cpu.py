"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads,
exports every entry point include/raspml.h declares, and the ctypes structs
match the header's field order."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "raspml.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("ras_pml", "helmholtz"))))


@pytest.fixture(scope="module")
def lib():
    import paper_2602_00735_gb300 as pkg
    pkg.build()
    return pkg.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("ras_pml_setup", "ras_pml_factor", "ras_pml_apply", "helmholtz_solve"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2602_00735_gb300 as pkg
    names = _declared_functions()
    assert sorted(pkg.SYMBOLS) == names
    for n in names:
        assert getattr(lib, n) is not None


def test_struct_layout_matches_header(lib):
    from paper_2602_00735_gb300 import _lib
    src = open(HEADER).read()
    body = src[src.index("typedef struct {\n  double k;"):]
    body = body[:body.index("} ras_pml_params;")]
    fields = re.findall(r"\b(?:double|int)\s+([\w\s,]+);", body)
    names = [f.strip() for grp in fields for f in grp.split(",")]
    assert names == [n for n, _ in _lib.Params._fields_]
    body = src[src.index("typedef struct {\n  int64_t n;"):]
    body = body[:body.index("} ras_pml_info_t;")]
    fields = re.findall(r"\b(?:double|int64_t|int32_t)\s+([\w\s,]+);", body)
    names = [f.strip() for grp in fields for f in grp.split(",")]
    assert names == [n for n, _ in _lib.Info._fields_]


def _fields(src, start, end):
    body = src[src.index(start):]
    body = body[:body.index(end)]
    fields = re.findall(r"\b(?:double|float|int64_t|int32_t)\s+([\w\s,\[\]]+);", body)
    return [re.sub(r"\[\d+\]", "", f).strip() for grp in fields for f in grp.split(",")]


def _lengths(src, start, end):
    body = src[src.index(start):]
    body = body[:body.index(end)]
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"(\w+)\[(\d+)\]", body)}


def test_tune_and_batch_struct_layouts(lib):
    from paper_2602_00735_gb300 import _lib
    src = open(HEADER).read()
    tune = ("typedef struct {\n  int32_t factor_threads;", "} ras_pml_tune_t;")
    assert _fields(src, *tune) == [n for n, _ in _lib.TuneReport._fields_]
    # array members have the header's lengths (the report is filled by the library)
    arrays = {n: t._length_ for n, t in _lib.TuneReport._fields_ if hasattr(t, "_length_")}
    assert arrays == _lengths(src, *tune)
    assert _fields(src, "typedef struct {\n  int32_t nprob;", "} ras_pml_batch_info_t;") == \
        [n for n, _ in _lib.BatchInfo._fields_]


def test_error_strings_and_null_handling(lib):
    import ctypes
    assert lib.ras_pml_error_string(0) == b"success"
    assert b"pivot" in lib.ras_pml_error_string(-4)
    # argument validation happens before any device call
    assert lib.ras_pml_setup(None, None, None) == -1
    assert lib.ras_pml_apply(None, None, None) == -1
    assert lib.ras_pml_tune(None, None) == -1
    assert lib.ras_pml_num_unknowns(None, None) == -1
    assert lib.ras_pml_batch_setup(None, 1, None, None) == -1
    assert lib.ras_pml_batch_solve(None, None, None, 1e-6, 10, 0, None, None) == -1
    assert lib.ras_pml_batch_apply(None, None, None) == -1
    lib.ras_pml_destroy(None)
    lib.ras_pml_batch_destroy(None)
    from paper_2602_00735_gb300 import _lib
    p = _lib.Params(k=10.0, x0=0, y0=0, x1=1, y1=1, kappa_g=0.1, h=0.013, px=2, py=2, ovlp_cells=2,
                    pml_cells=2, g_amp=20, g_ramp=0.05, local_bc=0, factor_prec=0)
    h = ctypes.c_void_p()
    assert lib.ras_pml_setup(ctypes.byref(p), None, ctypes.byref(h)) == -1   # not whole cells


def test_form_validation_before_any_device_call(lib):
    """form 1 (eq. weak as printed) accepts ortho 0..2 and local half-bandwidths
    up to 112 with complex128 factors; other forms are refused."""
    import ctypes
    from paper_2602_00735_gb300 import _lib
    base = dict(k=10.0, x0=0, y0=0, x1=1, y1=1, kappa_g=0.1, h=0.0125, px=2, py=2, ovlp_cells=2,
                pml_cells=2, g_amp=20, g_ramp=0.05, local_bc=0, factor_prec=0)
    h = ctypes.c_void_p()
    for kw in (dict(form=2), dict(form=-1), dict(form=1, ortho=3), dict(form=1, ortho=4),
               dict(form=1, h=1 / 120, px=1, py=1)):        # b = 144 > 112
        p = _lib.Params(**{**base, **kw})
        assert lib.ras_pml_setup(ctypes.byref(p), None, ctypes.byref(h)) == -1, kw
    p = _lib.Params(**{**base, "form": 1})
    arr = (_lib.Params * 1)(p)
    assert lib.ras_pml_batch_setup(arr, 1, None, ctypes.byref(h)) == -1


def test_product_path_has_no_oracle_import():
    pkgdir = os.path.join(ROOT, "paper_2602_00735_gb300")
    for dirpath, _, files in os.walk(pkgdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "from oracle" not in txt and "import oracle" not in txt
