"""ras_pml_assemble_rhs_noalloc: the load vector without any device
allocation, for callers that cannot call cudaMalloc/cudaFree (a caching
allocator has reserved the device, or the caller must not stall on the
synchronisation cudaFree implies). Its source table lives in a fixed device
array shared by all calls, so the test makes two calls in a row with
different source sets and compares each with ras_pml_assemble_rhs, through
the C ABI. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, s, cen, amp, width, out):
    cen = np.ascontiguousarray(np.asarray(cen, dtype=np.float64).reshape(-1, 2))
    amp = np.ascontiguousarray(np.asarray(amp, dtype=np.float64).ravel())
    return lib.ras_pml_assemble_rhs_noalloc(s._h, cen.ctypes.data_as(ctypes.c_void_p),
                                            amp.ctypes.data_as(ctypes.c_void_p), int(amp.size), float(width),
                                            ctypes.c_void_p(out.data_ptr()))


def test_noalloc_rhs_matches_allocating_entry_point_twice():
    import torch

    import __graft_entry__
    import workloads
    __graft_entry__.build()
    from paper_2602_00735_gb300 import RasPml, load
    lib = load()
    w = workloads.get("tiny3")
    rng = np.random.default_rng(7)
    sets = [(w.centres, w.amps, w.width),
            (rng.uniform(0, 1, size=(5, 2)), rng.uniform(0.5, 2.0, size=5), 0.03),
            (w.centres[:1], w.amps[:1], 0.07)]          # fewer sources than the call before
    with RasPml(w.params()) as s:
        for cen, amp, width in sets:
            ref = s.assemble_rhs(cen, amp, width)
            out = torch.full_like(ref, float("nan"))
            assert _call_noalloc(lib, s, cen, amp, width, out) == 0
            torch.cuda.synchronize()
            scale = float(ref.abs().max())
            assert scale > 0
            assert float((out - ref).abs().max()) <= 1e-13 * scale
        # sizes beyond the table are refused before any device work
        big = np.zeros((1025, 2))
        out = torch.zeros_like(ref)
        assert _call_noalloc(lib, s, big, np.ones(1025), 0.1, out) == -1
