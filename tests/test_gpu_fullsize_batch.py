"""The batched form at full size (workloads.batch("c3"): 64 problems, k from
20*pi to 113*pi, 19.5M unknowns, 3827 subdomains), in the configuration
bench.py times (complex64 factors, tuned tile shapes, rtol 1e-6):

- every problem converges, and for the smallest problems the oracle's own
  matrix and load vector give the same true residual;
- the solutions of the smallest problems agree with the oracle's direct
  solve to the accuracy that rtol allows;
- rows of A x of the largest problem at sampled nodes (oracle assembly of
  the cells around each node).
"""
import json
import os

import numpy as np
import pytest
import torch

import workloads
from gpu_util import random_vector
from oracle import fem

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_iterations.json")


@pytest.fixture(scope="module")
def c3():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_00735_gb300 import BatchRasPml
    probs = workloads.batch("c3")
    B = BatchRasPml([w.params() for w in probs], factor_prec=1)
    yield probs, B
    B.close()


def test_c3_solve_in_bench_configuration(c3):
    probs, B = c3
    B.tune()
    b = B.assemble_rhs([(w.centres, w.amps, w.width) for w in probs])
    x, it, relres, st = B.solve(b, rtol=1e-6, maxit=400)
    assert st == 0 and np.all(relres <= 1e-6)
    assert it.min() >= 1 and it.max() <= 400
    # every problem takes the oracle's own FGMRES count (tests/golden/oracle_iterations.json)
    gold = np.array(json.load(open(GOLD))["c3"]["iters"])
    assert np.max(np.abs(it - gold)) <= 1, np.abs(it - gold).max()
    order = np.argsort([w.n_unknowns for w in probs])
    for q in order[:3]:
        w = probs[q]
        p = w.params()
        grid, A = fem.assemble_global(p)
        bo = fem.assemble_rhs(p, w.centres, w.amps, w.width)
        xq = B.split(x)[q].cpu().numpy()
        r = np.linalg.norm(bo - A @ xq) / np.linalg.norm(bo)
        assert r <= 1.05e-6, (q, r)
        u = fem.direct_solve(A, bo)
        assert np.linalg.norm(xq - u) <= 1e-3 * np.linalg.norm(u)


def test_c3_matvec_rows_of_largest_problem(c3):
    from test_gpu_fullsize import _oracle_rows, _sample_nodes
    probs, B = c3
    q = int(np.argmax([w.n_unknowns for w in probs]))
    w = probs[q]
    p = w.params()
    grid = fem.make_grid(p)
    xs = [np.zeros(int(n), complex) for n in B.sizes]
    xs[q] = random_vector(int(B.sizes[q]), 41)
    y = B.split(B.matvec(B.join(xs)))[q].cpu().numpy()
    i, j = _sample_nodes(grid, 40, 42)
    rows = _oracle_rows(p, grid, i, j)
    for (ii, jj), (cols, vals) in rows.items():
        r = (jj - 1) * grid.nx + (ii - 1)
        ref = vals @ xs[q][cols]
        assert abs(y[r] - ref) <= 1e-13 * max(1.0, np.abs(vals).sum() * np.abs(xs[q][cols]).max())
