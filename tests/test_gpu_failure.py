"""Failure detection on the device without a fault: the apply kernels' waits
for their bulk copies are bounded, and a time-out is reported, not hung on.
The limit is injected from the host (ras_pml_set_copy_wait_limit, 1 cycle:
every wait gives up at its first check); each timed-out warp records the
time-out, waits with the full limit for the copies it still has in flight,
and returns. The solve reports RASPML_ETIMEOUT, and once the limit is restored
and the handle refactored the same solve gives the same answer as before."""
import numpy as np
import pytest

from gpu_util import rel, variant

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00735_gb300 as p
    return p


@pytest.mark.parametrize("name,prec", [("small", 1), ("c0", 1), ("tiny3", 0)])
def test_copy_wait_timeout_is_reported_and_the_context_recovers(pkg, name, prec):
    from paper_2602_00735_gb300 import RasPmlError
    w = variant(name)
    lib = pkg.load()
    with pkg.RasPml(w.params(), factor_prec=prec, ortho=3) as s:
        b = s.assemble_rhs(w.centres, w.amps, w.width)
        s.factor()
        x0, it0, r0, st0 = s.solve(b, rtol=1e-8, maxit=300)
        assert st0 == 0
        x0 = x0.cpu().numpy()
        assert lib.ras_pml_set_copy_wait_limit(1) == 0
        try:
            with pytest.raises(RasPmlError) as ei:
                s.solve(b, rtol=1e-8, maxit=20)
            assert ei.value.status == -6          # RASPML_ETIMEOUT
        finally:
            assert lib.ras_pml_set_copy_wait_limit(0) == 0
        s.factor()   # clears the recorded time-out
        x1, it1, r1, st1 = s.solve(b, rtol=1e-8, maxit=300)
        assert st1 == 0 and it1 == it0
        assert rel(x1.cpu().numpy(), x0) <= 1e-12


@pytest.mark.parametrize("prec", [1, 0])
def test_wide_class_copy_wait_timeout_is_reported(pkg, prec):
    """The wide band class (several warps per subdomain sharing one copy ring):
    all warps leave together at the first failed wait, after the copies in
    flight have landed, and the handle solves again once the limit is
    restored."""
    from test_gpu_wide_band import strip
    from paper_2602_00735_gb300 import RasPmlError
    w = strip(300)
    lib = pkg.load()
    with pkg.RasPml(w.params(), factor_prec=prec, ortho=3) as s:
        assert s.info()["max_band"] == 300
        b = s.assemble_rhs(w.centres, w.amps, w.width)
        s.factor()
        x0, it0, r0, st0 = s.solve(b, rtol=1e-8, maxit=100)
        x0 = x0.cpu().numpy()
        assert lib.ras_pml_set_copy_wait_limit(1) == 0
        try:
            with pytest.raises(RasPmlError) as ei:
                s.solve(b, rtol=1e-8, maxit=20)
            assert ei.value.status == -6          # RASPML_ETIMEOUT
        finally:
            assert lib.ras_pml_set_copy_wait_limit(0) == 0
        s.factor()
        x1, it1, r1, st1 = s.solve(b, rtol=1e-8, maxit=100)
        assert st1 == st0 and it1 == it0
        assert rel(x1.cpu().numpy(), x0) <= 1e-12
