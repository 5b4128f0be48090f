"""The stored oracle solutions (tests/golden/oracle_solution_*.json, written
by tests/golden/make_oracle_iterations.py --solution) are what the oracle
computes: c0 is re-solved here and compared sample by sample; the c2 file
is checked for its own consistency (sample count, seed, strip edges, the
iteration count stored beside it in oracle_iterations.json)."""
import json
import os

import numpy as np

import workloads
from oracle import fem, krylov, ras

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_c0_golden_solution_is_the_oracles():
    g = json.load(open(os.path.join(GOLD, "oracle_solution_c0.json")))
    w = workloads.get("c0")
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    x, it, rel, _ = krylov.fgmres(A.dot, ras.RAS(p).factor().apply, b, rtol=1e-6, maxit=1000)
    assert it == g["iters"] and abs(rel - g["relres"]) <= 1e-6 * g["relres"]
    idx = np.array([t[0] for t in g["samples"]])
    ref = np.array([t[1] + 1j * t[2] for t in g["samples"]])
    assert np.max(np.abs(x[idx] - ref)) <= 1e-9 * np.max(np.abs(ref))
    assert abs(np.linalg.norm(x) - g["norm"]) <= 1e-12 * g["norm"]
    ed = g["strip_edges"]
    strips = [np.linalg.norm(x[ed[q]:ed[q + 1]]) for q in range(len(ed) - 1)]
    assert np.allclose(strips, g["strip_norms"], rtol=1e-12, atol=0)


def test_c2_golden_solution_is_consistent():
    g = json.load(open(os.path.join(GOLD, "oracle_solution_c2.json")))
    it = json.load(open(os.path.join(GOLD, "oracle_iterations.json")))["c2"]
    w = workloads.get("c2")
    assert g["workload"] == "c2" and g["n"] == w.n_unknowns and g["iters"] == it["iters"]
    assert len(g["samples"]) == 2048 and g["sample_seed"] == 20260
    idx = np.array([t[0] for t in g["samples"]])
    expect = np.sort(np.random.default_rng(20260).choice(g["n"], size=2048, replace=False))
    assert np.array_equal(idx, expect)
    assert g["strip_edges"][0] == 0 and g["strip_edges"][-1] == g["n"]
    assert abs(np.sqrt(np.sum(np.square(g["strip_norms"]))) - g["norm"]) <= 1e-12 * g["norm"]
