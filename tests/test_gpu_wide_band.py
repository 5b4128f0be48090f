"""Wide local bands: subdomains of 150-230 nodes across (the factor window
stored by diagonals; the largest band is 160 for complex128 factors and 232
for complex64). Parity with the CPU FP64 oracle at the same tolerances as the
narrow-band cases: 1e-10 for complex128, 1e-4 for complex64 (b * eps_32 is
still below 2e-5 at b = 232)."""
import numpy as np
import pytest

from gpu_util import oracle_problem, rel, random_vector, to_dev, variant
from oracle import fem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver_cls():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_00735_gb300 import RasPml
    return RasPml


def test_band_154_apply_matches_oracle(solver_cls):
    w = variant("mid", px=3, py=3)               # middle box: 153 local nodes across
    grid, A, R = oracle_problem(w)
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        with solver_cls(w.params(), factor_prec=prec) as s:
            assert s.info()["max_band"] == 154
            s.factor()
            r = random_vector(grid.n, 5)
            assert rel(s.apply(to_dev(r)).cpu().numpy(), R.apply(r)) <= tol


def test_band_205_complex64_apply_and_solve(solver_cls):
    from paper_2602_00735_gb300 import RasPmlError
    w = variant("mid", px=2, py=2)               # 204 local nodes across
    p = w.params()
    with pytest.raises(RasPmlError):
        solver_cls(p, factor_prec=0)             # above the complex128 limit of 160
    grid, A, R = oracle_problem(w)
    with solver_cls(p, factor_prec=1) as s:
        assert s.info()["max_band"] == 205
        s.factor()
        r = random_vector(grid.n, 6)
        assert rel(s.apply(to_dev(r)).cpu().numpy(), R.apply(r)) <= 1e-4
        b = s.assemble_rhs(w.centres, w.amps, w.width)
        x, it, relres, st = s.solve(b, rtol=1e-11, maxit=200)
        assert st == 0 and relres <= 1e-11
        u = fem.direct_solve(A, fem.assemble_rhs(p, w.centres, w.amps, w.width))
        assert rel(x.cpu().numpy(), u) <= 1e-9


@pytest.mark.parametrize("prec,px,ovlp,pml,limit", [(0, 3, 7, 8, 160), (1, 2, 19, 20, 232), (2, 2, 19, 20, 232)])
def test_band_limits(solver_cls, prec, px, ovlp, pml, limit):
    """384 cells in px boxes: with px = 3 the middle subdomain has
    129 + 2(ovlp + pml) nodes across, with px = 2 each has 192 + ovlp + pml.
    The setup accepts b = nlx + 1 up to the limit and rejects one more cell."""
    from paper_2602_00735_gb300 import RasPmlError
    ok = variant("mid", px=px, py=px, ovlp_cells=ovlp, pml_cells=pml)
    grid, A, R = oracle_problem(ok)
    with solver_cls(ok.params(), factor_prec=prec) as s:
        assert s.info()["max_band"] == limit
        s.factor()                                # the largest window and ring
        r = random_vector(grid.n, 7)
        tol = {0: 1e-10, 1: 1e-4, 2: 2e-2}[prec]
        assert rel(s.apply(to_dev(r)).cpu().numpy(), R.apply(r)) <= tol
    with pytest.raises(RasPmlError):
        solver_cls(ok.with_(pml_cells=pml + 1).params(), factor_prec=prec)
