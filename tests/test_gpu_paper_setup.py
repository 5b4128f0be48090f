"""The paper's experimental set-up (Section 4) on the GPU: the cubic
stretching g(x) = 10 k x^3 with a three-wavelength global PML, h = 1/(2k),
the smoothed-delta source and the width law of Section 3 (iii) (boxes of at
most ~75 cells here; the paper's have ~300).

- parity with the oracle on a small case;
- the qualitative claims of Tables 1-2: with a PML on the subdomains the
  impedance closure (RAS-PML-Imp) needs no more GMRES iterations than the
  Dirichlet closure (RAS-PML-Drch), and both need fewer than impedance
  closure without PML (RAS-Imp).
"""
import numpy as np
import pytest

import workloads
from gpu_util import oracle_problem, rel, random_vector, to_dev
from oracle import fem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver_cls():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_00735_gb300 import RasPml
    return RasPml


def test_paper_setup_parity(solver_cls):
    w = workloads.paper_setup(160, 64)
    p = w.params()
    grid, A, R = oracle_problem(w)
    with solver_cls(p) as s:
        x = random_vector(grid.n, 21)
        assert rel(s.matvec(to_dev(x)).cpu().numpy(), A @ x) <= 1e-13
        b = s.assemble_rhs(w.centres, w.amps, w.width).cpu().numpy()
        bo = fem.assemble_rhs(p, w.centres, w.amps, w.width)
        assert np.max(np.abs(b - bo)) <= 1e-13 * np.max(np.abs(bo))
        s.factor()
        r = random_vector(grid.n, 22)
        assert rel(s.apply(to_dev(r)).cpu().numpy(), R.apply(r)) <= 1e-10


@pytest.mark.parametrize("k,cells", [(300, 75), (600, 64)])
def test_tables_1_2_ordering_of_local_closures(solver_cls, k, cells):
    its = {}
    for name, kw in (("imp", dict(local_bc=0)), ("drch", dict(local_bc=1)),
                     ("ras_imp", dict(local_bc=0, pml=False))):
        w = workloads.paper_setup(k, cells, C_delta=1 / 6, C_kappa=3 / 8, **kw)
        with solver_cls(w.params(), factor_prec=0, ortho=2) as s:
            b = s.assemble_rhs(w.centres, w.amps, w.width)
            x, it, relres, st = s.solve(b, rtol=1e-10, maxit=600)
            assert st == 0 and relres <= 1e-10
            its[name] = it
    assert its["imp"] <= its["drch"] < its["ras_imp"], its


def _closure_counts(solver_cls, k, cells, prec, ortho, form=0):
    its = {}
    for name, kw in (("imp", dict(local_bc=0)), ("drch", dict(local_bc=1)),
                     ("ras_imp", dict(local_bc=0, pml=False))):
        w = workloads.paper_setup(k, cells, C_delta=1 / 6, C_kappa=3 / 8, **kw).with_(form=form)
        with solver_cls(w.params(), factor_prec=prec, ortho=ortho) as s:
            b = s.assemble_rhs(w.centres, w.amps, w.width)
            x, it, relres, st = s.solve(b, rtol=1e-10, maxit=600)
            assert st == 0 and relres <= 1e-10
            its[name] = it
    return its


def test_tables_1_2_ordering_in_the_papers_own_form_on_the_gpu(solver_cls):
    """eq. weak as printed (form 1) on the paper's set-up, k = 160 with 5 x 5
    boxes of 64 cells: the GPU takes the oracle's own iteration counts (within
    one) for RAS-PML-Imp, RAS-PML-Drch and RAS-Imp, in the ordering of Tables
    1-2."""
    from oracle import krylov, ras
    gpu = _closure_counts(solver_cls, 160, 64, 0, 2, form=1)
    ref = {}
    for name, kw in (("imp", dict(local_bc=0)), ("drch", dict(local_bc=1)),
                     ("ras_imp", dict(local_bc=0, pml=False))):
        w = workloads.paper_setup(160, 64, C_delta=1 / 6, C_kappa=3 / 8, **kw).with_(form=1)
        p = w.params()
        grid, A = fem.assemble_global(p)
        bo = fem.assemble_rhs(p, w.centres, w.amps, w.width)
        _, ref[name], _, _ = krylov.fgmres(A.dot, ras.RAS(p).factor().apply, bo, rtol=1e-10, maxit=300)
    assert all(abs(gpu[n] - ref[n]) <= 1 for n in ref), (gpu, ref)
    assert gpu["imp"] <= gpu["drch"] < gpu["ras_imp"], gpu


@pytest.mark.parametrize("k,paper", [(300, (11, 12, 29)), (600, (19, 19, 41))])
def test_papers_300_cell_boxes(solver_cls, k, paper):
    """The paper's own subdomain size (Section 4: boxes of 300 cells, Table 2:
    k = 300 with 2 x 2 and k = 600 with 4 x 4 of them, h = 1/(2k); local
    half-bandwidths 315 and 333, on the blocked wide-band kernels), headline
    form (complex64 factors, double-float Gram-Schmidt), rtol 1e-10: the
    ordering of Tables 1-2, RAS-PML-Imp <= RAS-PML-Drch < RAS-Imp. The P1
    counts are printed beside the paper's Q1 counts (Table 2, C_kappa = 3/8,
    C_delta = 1/6), which they need not equal (other elements, and the width
    law rounds the PML to 9 and 11 cells where the table prints 8 and 11)."""
    its = _closure_counts(solver_cls, k, 300, 1, 3)
    print(f"\nk = {k}, boxes of 300 cells: P1 {its}; the paper's Q1 counts (imp, drch, ras_imp): {paper}")
    assert its["imp"] <= its["drch"] < its["ras_imp"], its
    assert its["imp"] <= 2 * paper[0] and its["ras_imp"] <= 2 * paper[2]
