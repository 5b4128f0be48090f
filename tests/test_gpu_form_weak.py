"""Parity of form 1 (the paper's eq. weak as printed, not symmetric) on the
CUDA path, through the C ABI, with the CPU FP64 oracle's form 1.

Form 1 has its own global stencil (seven couplings per row), SpMV, local
rows and L D U band factor; the apply kernel is the one of form 0, reading
the reversed band of U where form 0 reads that of L^T. Tolerances as for
form 0: 1e-13 for the matvec, 1e-10 for complex128 factors, 1e-4 for
complex64 and 2e-2 for half-pair storage of the factors.
"""
import numpy as np
import pytest

from gpu_util import oracle_problem, rel, random_vector, to_dev, variant
from oracle import fem, krylov

pytestmark = pytest.mark.gpu

CASES = [
    ("tiny", {}),
    ("tiny3", {}),
    ("small", {}),
    ("c0", {}),
    ("tiny3", {"local_bc": 1}),                   # RAS-PML-Drch
    ("tiny3", {"pml_cells": 0}),                  # RAS-Imp (no local PML)
    ("small", {"px": 3, "py": 5}),                # uneven boxes
    ("tiny", {"x1": 1.3, "kappa_g": 0.125}),      # rectangle
    ("tiny", {"g_profile": 1, "g_amp": 200.0}),   # cubic profile g = amp d^3
]
IDS = [n + "".join(f"-{k}{v}" for k, v in kw.items()) for n, kw in CASES]


def weak(name, **kw):
    return variant(name, form=1, **kw)


@pytest.fixture(scope="module")
def solver_cls():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_00735_gb300 import RasPml
    return RasPml


@pytest.mark.parametrize("name,kw", CASES, ids=IDS)
def test_weak_matvec_matches_oracle(solver_cls, name, kw):
    w = weak(name, **kw)
    grid, A, _ = oracle_problem(w)
    assert abs(A - A.T).max() > 1e-6 * abs(A).max()        # the form really is not symmetric
    with solver_cls(w.params()) as s:
        x = random_vector(grid.n, 1)
        y = s.matvec(to_dev(x)).cpu().numpy()
        assert rel(y, A @ x) <= 1e-13


@pytest.mark.parametrize("name,kw", CASES, ids=IDS)
def test_weak_apply_fp64_matches_oracle(solver_cls, name, kw):
    w = weak(name, **kw)
    grid, A, R = oracle_problem(w)
    with solver_cls(w.params()) as s:
        s.factor()
        for seed in (2, 3):
            r = random_vector(grid.n, seed)
            z = s.apply(to_dev(r)).cpu().numpy()
            assert rel(z, R.apply(r)) <= 1e-10
        assert s.info()["min_pivot_ratio"] > 0


@pytest.mark.parametrize("prec,tol", [(1, 1e-4), (2, 2e-2)])
@pytest.mark.parametrize("name,kw", CASES[:6], ids=IDS[:6])
def test_weak_low_precision_apply_close_to_oracle(solver_cls, name, kw, prec, tol):
    w = weak(name, **kw)
    grid, A, R = oracle_problem(w)
    with solver_cls(w.params(), factor_prec=prec) as s:
        s.factor()
        r = random_vector(grid.n, 2)
        assert rel(s.apply(to_dev(r)).cpu().numpy(), R.apply(r)) <= tol


@pytest.mark.parametrize("name", ["tiny3", "small", "c0"])
def test_weak_fgmres_fixed_iterations_match_oracle(solver_cls, name):
    w = weak(name)
    p = w.params()
    grid, A, R = oracle_problem(w)
    bo = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    m = 7
    xo, _, _, ho = krylov.fgmres(A.dot, R.apply, bo, rtol=0.0, maxit=m)
    with solver_cls(p) as s:
        b = s.assemble_rhs(w.centres, w.amps, w.width)
        x, it, relres, st = s.solve(b, rtol=0.0, maxit=m)
        assert it == m and st == 1
        assert rel(x.cpu().numpy(), xo) <= 1e-10
        assert np.max(np.abs(s.history() - np.array(ho)) / np.array(ho)) <= 1e-8


@pytest.mark.parametrize("prec,ortho", [(0, 0), (0, 2), (1, 2), (2, 2)])
@pytest.mark.parametrize("name,kw", CASES[:6], ids=IDS[:6])
def test_weak_converged_solve_matches_direct_solve(solver_cls, name, kw, prec, ortho):
    w = weak(name, **kw)
    p = w.params()
    grid, A, _ = oracle_problem(w)
    u = fem.direct_solve(A, fem.assemble_rhs(p, w.centres, w.amps, w.width))
    with solver_cls(p, factor_prec=prec, ortho=ortho) as s:
        b = s.assemble_rhs(w.centres, w.amps, w.width)
        x, it, relres, st = s.solve(b, rtol=1e-11, maxit=400)
        assert st == 0 and relres <= 1e-11
        assert rel(x.cpu().numpy(), u) <= 1e-9


def test_weak_richardson_matches_oracle_algorithm_1(solver_cls):
    w = weak("tiny")
    p = w.params()
    grid, A, R = oracle_problem(w)
    bo = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    uo, _, _, _ = krylov.richardson(A.dot, R.apply, bo, rtol=0.0, maxit=5)
    with solver_cls(p) as s:
        b = s.assemble_rhs(w.centres, w.amps, w.width)
        u, it, relres, st = s.richardson(b, rtol=0.0, maxit=5)
        assert it == 5 and rel(u.cpu().numpy(), uo) <= 1e-10


def test_weak_and_symmetric_solutions_agree_on_the_gpu(solver_cls):
    """Both forms discretise the same problem: on c0 the two GPU solutions
    differ in Omega_int by the discretisation error only (the oracle pins the
    second-order decay of that difference)."""
    w0 = variant("c0")
    grid = fem.make_grid(w0.params())
    xs = {}
    for form in (0, 1):
        with solver_cls(dict(w0.params(), form=form)) as s:
            b = s.assemble_rhs(w0.centres, w0.amps, w0.width)
            x, it, relres, st = s.solve(b, rtol=1e-10, maxit=400)
            assert st == 0
            xs[form] = x.cpu().numpy()
    x, y = fem.unknown_coords(grid)
    m = (x > 0) & (x < 1) & (y > 0) & (y < 1)
    d = rel(xs[1][m], xs[0][m])
    assert 1e-8 < d < 0.2, d


def test_weak_form_restrictions(solver_cls):
    from paper_2602_00735_gb300 import BatchRasPml, RasPmlError
    w = weak("tiny")
    with pytest.raises(RasPmlError):
        solver_cls(w.params(), ortho=3)                   # double-float Arnoldi: symmetric form only
    with pytest.raises(RasPmlError):
        BatchRasPml([w.params()], factor_prec=1)          # batched kernels: symmetric form only
    with solver_cls(w.params()) as s:
        rep = s.tune()                                    # one factor shape: factors, times nothing
        assert s.info()["factored"] == 1 and rep["factor_ms"] == {}
