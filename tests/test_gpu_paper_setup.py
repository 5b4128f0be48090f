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
