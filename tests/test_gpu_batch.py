"""Batched form: eight independent problems of uneven size, subdomain grids
and wavenumbers (workloads.batch("c3small")) set up, factored, applied and
solved in the same launches. Each problem is compared with the CPU FP64
oracle on its own, at the tolerances of the one-problem path; the batch
apply is also compared bit for bit with the one-problem handle (the same
kernels run the same arithmetic on every subdomain)."""
import numpy as np
import pytest
import torch

import workloads
from gpu_util import oracle_problem, rel, random_vector
from oracle import fem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2602_00735_gb300 as p
    return p


@pytest.fixture(scope="module")
def probs():
    return workloads.batch("c3small")


def _sources(ws):
    return [(w.centres, w.amps, w.width) for w in ws]


def test_layout_matvec_and_rhs(pkg, probs):
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=1) as B:
        assert B.nprob == len(probs)
        assert np.all(B.offsets % 2048 == 0)
        assert list(B.sizes) == [w.n_unknowns for w in probs]
        xs = [random_vector(int(n), 10 + q) for q, n in enumerate(B.sizes)]
        x = B.join(xs)
        y = B.matvec(x)
        b = B.assemble_rhs(_sources(probs))
        mask = torch.ones(B.ntot, dtype=torch.bool, device=y.device)
        for q, (w, yq, bq) in enumerate(zip(probs, B.split(y), B.split(b))):
            grid, A, _ = oracle_problem(w)
            assert rel(yq.cpu().numpy(), A @ xs[q]) <= 1e-13
            bo = fem.assemble_rhs(w.params(), w.centres, w.amps, w.width)
            assert np.max(np.abs(bq.cpu().numpy() - bo)) <= 1e-13 * np.max(np.abs(bo))
            mask[int(B.offsets[q]):int(B.offsets[q]) + int(B.sizes[q])] = False
        assert torch.count_nonzero(y[mask]) == 0 and torch.count_nonzero(b[mask]) == 0


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
def test_apply_matches_oracle(pkg, probs, prec, tol):
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=prec) as B:
        B.factor()
        inf = B.info()
        assert inf["factored"] == 1 and inf["num_sub"] == sum(w.px * w.py for w in probs)
        rs = [random_vector(int(n), 20 + q) for q, n in enumerate(B.sizes)]
        z = B.apply(B.join(rs))
        for q, (w, zq) in enumerate(zip(probs, B.split(z))):
            _, _, R = oracle_problem(w)
            assert rel(zq.cpu().numpy(), R.apply(rs[q])) <= tol, q


def test_apply_equals_one_problem_handle_bitwise(pkg, probs):
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=1) as B:
        B.factor()
        rs = [random_vector(int(n), 30 + q) for q, n in enumerate(B.sizes)]
        z = B.apply(B.join(rs))
        for q, w in enumerate(probs[:4]):
            with pkg.RasPml(w.params(), factor_prec=1) as s:
                s.factor()
                zs = s.apply(torch.from_numpy(rs[q]).cuda())
                assert torch.equal(zs, B.split(z)[q])


@pytest.mark.parametrize("prec", [0, 1])
def test_lockstep_solve_matches_direct_solves(pkg, probs, prec):
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=prec) as B:
        b = B.assemble_rhs(_sources(probs))
        x, it, relres, st = B.solve(b, rtol=1e-10, maxit=400)
        assert st == 0 and np.all(relres <= 1e-10)
        assert len(set(it.tolist())) > 1            # problems stopped at different steps
        assert B.info()["steps"] >= it.max()
        for q, (w, xq) in enumerate(zip(probs, B.split(x))):
            grid, A, _ = oracle_problem(w)
            p = w.params()
            u = fem.direct_solve(A, fem.assemble_rhs(p, w.centres, w.amps, w.width))
            assert rel(xq.cpu().numpy(), u) <= 1e-8, q


def test_iterations_match_one_problem_solves(pkg, probs):
    """Lockstep FGMRES takes, per problem, the iterations of the one-problem
    solver with the same Gram-Schmidt (double-float CGS on a complex64 basis,
    ortho = 4); sums in a different order may move the stopping step by one."""
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=1) as B:
        b = B.assemble_rhs(_sources(probs))
        _, it, _, st = B.solve(b, rtol=1e-6, maxit=400)
        assert st == 0
        for q, w in enumerate(probs):
            with pkg.RasPml(w.params(), factor_prec=1, ortho=4) as s:
                bq = s.assemble_rhs(w.centres, w.amps, w.width)
                _, its, _, _ = s.solve(bq, rtol=1e-6, maxit=400)
            assert abs(int(it[q]) - its) <= 1, (q, it[q], its)


def test_restarted_and_tuned_solve(pkg, probs):
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=1) as B:
        rep = B.tune()
        assert rep["factor_threads"] in (128, 256, 512, 1024) and rep["apply_cols"] in (4, 8, 16)
        # the tensor-core forms (128 x 8, 128 x 16) are candidates: complex64, every b <= 127
        assert set(rep["factor_ms"]) == {"128x1", "256x1", "512x1", "256x2", "512x2", "1024x2", "128x8", "128x16"}
        assert all(v > 0 for v in rep["factor_ms"].values())
        inf = B.info()
        assert (inf["factor_threads"], inf["factor_rank"], inf["apply_cols"]) == \
            (rep["factor_threads"], rep["factor_rank"], rep["apply_cols"])
        b = B.assemble_rhs(_sources(probs))
        x, it, relres, st = B.solve(b, rtol=1e-8, maxit=600, restart=15)
        assert st == 0 and np.all(relres <= 1e-8)
        assert B.info()["cycles"] >= 2
        w = probs[0]
        grid, A, _ = oracle_problem(w)
        u = fem.direct_solve(A, fem.assemble_rhs(w.params(), w.centres, w.amps, w.width))
        assert rel(B.split(x)[0].cpu().numpy(), u) <= 1e-6


def test_not_converged_and_errors(pkg, probs):
    from paper_2602_00735_gb300 import RasPmlError
    ps = [w.params() for w in probs[:3]]
    with pkg.BatchRasPml(ps, factor_prec=1) as B:
        with pytest.raises(RasPmlError):
            B.apply(B.empty())                    # not factored
        b = B.assemble_rhs(_sources(probs[:3]))
        x, it, relres, st = B.solve(b, rtol=1e-12, maxit=3)
        assert st == 1 and np.all(it == 3) and np.all(relres > 1e-12)
        zero = torch.zeros_like(b)
        x, it, relres, st = B.solve(zero, rtol=1e-6, maxit=10)
        assert st == 0 and np.all(it == 0) and torch.count_nonzero(x) == 0
        bn = b.clone()
        bn[int(B.offsets[1]) + 5] = float("nan")
        with pytest.raises(RasPmlError):
            B.solve(bn, rtol=1e-6, maxit=10)


def test_mixed_variants_in_one_batch(pkg):
    """Problems that differ in closure (impedance / Dirichlet), local PML
    (present / absent), boxes and stretching profile (the paper's g = 10k x^3
    set-up) share the launches; each matches its own oracle."""
    from gpu_util import variant
    probs = [variant("tiny3", local_bc=1), variant("tiny3", pml_cells=0), variant("small", px=3, py=5),
             workloads.paper_setup(160, 40)]
    for prec, tol in ((0, 1e-10), (2, 2e-2)):
        with pkg.BatchRasPml([w.params() for w in probs], factor_prec=prec) as B:
            B.factor()
            rs = [random_vector(int(n), 40 + q) for q, n in enumerate(B.sizes)]
            z = B.apply(B.join(rs))
            for q, (w, zq) in enumerate(zip(probs, B.split(z))):
                _, _, R = oracle_problem(w)
                assert rel(zq.cpu().numpy(), R.apply(rs[q])) <= tol, (prec, q)
            if prec == 0:
                b = B.assemble_rhs(_sources(probs))
                x, it, relres, st = B.solve(b, rtol=1e-10, maxit=400)
                assert st == 0
                for q, (w, xq) in enumerate(zip(probs, B.split(x))):
                    grid, A, _ = oracle_problem(w)
                    u = fem.direct_solve(A, fem.assemble_rhs(w.params(), w.centres, w.amps, w.width))
                    assert rel(xq.cpu().numpy(), u) <= 1e-8, q


@pytest.mark.parametrize("rank", [8, 16])
@pytest.mark.parametrize("prec,tol", [(1, 1e-4), (2, 2e-2)])
def test_tensor_core_factor_in_a_batch(pkg, probs, prec, tol, rank):
    """The blocked tensor-core factorisation over the union of the problems'
    subdomains (uneven bands, LPT order) gives each problem's oracle B^-1."""
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=prec) as B:
        B.set_shapes(128, rank, 8)
        B.factor()
        assert (B.info()["factor_threads"], B.info()["factor_rank"]) == (128, rank)
        rs = [random_vector(int(n), 60 + q) for q, n in enumerate(B.sizes)]
        z = B.apply(B.join(rs))
        for q, (w, zq) in enumerate(zip(probs, B.split(z))):
            _, _, R = oracle_problem(w)
            assert rel(zq.cpu().numpy(), R.apply(rs[q])) <= tol, q


def test_mixed_band_factor_shape(pkg):
    """A batch whose subdomains straddle the tensor-core form's band limit
    (b = 193 in c0 with one box across, b <= 127 elsewhere): the mixed shape
    factors the wide ones on the CUDA cores and the rest on the tensor cores,
    factor_rank 24 the wide ones on the blocked tensor-core kernel (window in
    scratch), and each gives every problem its oracle B^-1 and the CUDA-core
    shape's iteration counts."""
    from gpu_util import variant
    from paper_2602_00735_gb300 import RasPmlError
    probs = [variant("c0", px=1, py=2), variant("tiny3"), variant("small", px=3, py=5)]
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=1) as B:
        assert B.info()["max_band"] > 127
        with pytest.raises(RasPmlError):
            B.set_shapes(128, 8, 8)            # the tensor-core form alone cannot take b > 127
        rs = [random_vector(int(n), 70 + q) for q, n in enumerate(B.sizes)]
        b = B.assemble_rhs(_sources(probs))
        its = {}
        for shape in ((1024, 2), (1024, 8), (512, 16), (128, 24)):
            B.set_shapes(*shape, 8)
            B.factor()
            z = B.apply(B.join(rs))
            for q, (w, zq) in enumerate(zip(probs, B.split(z))):
                _, _, R = oracle_problem(w)
                assert rel(zq.cpu().numpy(), R.apply(rs[q])) <= 1e-4, (shape, q)
            _, its[shape], _, st = B.solve(b, rtol=1e-8, maxit=400)
            assert st == 0
        for shape in ((1024, 8), (512, 16), (128, 24)):
            assert np.all(np.abs(np.asarray(its[shape]) - np.asarray(its[(1024, 2)])) <= 1), its
        rep = B.tune()
        # 128 threads cannot hold the 194 diagonals of the b = 193 window:
        # that shape is skipped, the other seven and the blocked tensor-core
        # shape are timed
        assert {"1024x2", "512x2", "128x24"} <= set(rep["factor_ms"]) and len(rep["factor_ms"]) == 8
        assert "128x1" not in rep["factor_ms"]


def test_blocked_tensor_core_shape_with_half_storage(pkg):
    """Factor shape 24 with half-precision factor storage: the subdomains
    with 127 < b <= 232 on the blocked tensor-core kernel, the others on the
    tensor-core kernel, each problem's B^-1 at the half-storage tolerance."""
    from gpu_util import variant
    probs = [variant("c0", px=1, py=2), variant("small", px=3, py=5)]
    with pkg.BatchRasPml([w.params() for w in probs], factor_prec=2) as B:
        assert 127 < B.info()["max_band"] <= 232
        B.set_shapes(128, 24, 8)
        B.factor()
        rs = [random_vector(int(n), 90 + q) for q, n in enumerate(B.sizes)]
        z = B.apply(B.join(rs))
        for q, (w, zq) in enumerate(zip(probs, B.split(z))):
            _, _, R = oracle_problem(w)
            assert rel(zq.cpu().numpy(), R.apply(rs[q])) <= 2e-2, q
