"""Writes tests/golden/oracle_iterations.json: the CPU oracle's flexible GMRES
iteration counts (rtol 1e-6, x0 = 0, no restart) with the RAS-PML
preconditioner on the named workloads. Calls only oracle/ and workloads.

    python tests/golden/make_oracle_iterations.py c0 c1 c2
    python tests/golden/make_oracle_iterations.py c3     # every problem of the batch
    python tests/golden/make_oracle_iterations.py --solution c2

For a batch the counts are stored per problem, in the batch's order; the
problems run in a pool of processes started with "spawn".

--solution NAME also writes tests/golden/oracle_solution_NAME.json: the
2-norm of the oracle's FGMRES solution x (rtol 1e-6), its 2-norm over each of
16 horizontal strips of unknowns, and x at 2048 indices drawn from
numpy's default_rng(20260) without replacement (sorted), stored as
[index, re, im] triples with 11 significant digits.
"""
import json
import os
import sys
import time

# one BLAS thread per process: batches run one problem per process
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import fem, krylov, ras  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.json")


def run(name):
    return run_workload(workloads.get(name))


def run_workload(w, keep_x=False):
    p = w.params()
    t0 = time.time()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    R = ras.RAS(p).factor()
    t1 = time.time()
    x, it, rel, hist = krylov.fgmres(A.dot, R.apply, b, rtol=1e-6, maxit=1000)
    t2 = time.time()
    out = {"iters": int(it), "relres": float(rel), "rtol": 1e-6, "n": int(grid.n),
           "subdomains": len(R.subs), "setup_factor_s": round(t1 - t0, 2), "solve_s": round(t2 - t1, 2)}
    return (out, x) if keep_x else out


NSAMP, NSTRIP, SAMPLE_SEED = 2048, 16, 20260


def solution_record(name, x, it, rel):
    import numpy as np
    n = x.size
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(n, size=NSAMP, replace=False))
    edges = [n * q // NSTRIP for q in range(NSTRIP + 1)]
    return {"workload": name, "n": int(n), "iters": int(it), "relres": float(rel), "rtol": 1e-6,
            "norm": float(np.linalg.norm(x)),
            "strip_edges": [int(e) for e in edges],
            "strip_norms": [float(np.linalg.norm(x[edges[q]:edges[q + 1]])) for q in range(NSTRIP)],
            "sample_seed": SAMPLE_SEED,
            "samples": [[int(i), float(f"{x[i].real:.10e}"), float(f"{x[i].imag:.10e}")] for i in idx]}


def run_batch(name):
    import multiprocessing as mp
    probs = workloads.batch(name)
    order = sorted(range(len(probs)), key=lambda q: -probs[q].n_unknowns)   # largest first
    with mp.get_context("spawn").Pool(min(len(probs), os.cpu_count() or 1)) as pool:
        res = dict(zip(order, pool.map(run_workload, [probs[q] for q in order], chunksize=1)))
    return {key: [res[q][key] for q in range(len(probs))] for key in ("iters", "relres", "n", "subdomains")} | \
        {"rtol": 1e-6, "solve_s_total": round(sum(res[q]["solve_s"] + res[q]["setup_factor_s"] for q in res), 1)}


if __name__ == "__main__":
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    if sys.argv[1:2] == ["--solution"]:
        for name in sys.argv[2:]:
            rec, x = run_workload(workloads.get(name), keep_x=True)
            sol = solution_record(name, x, rec["iters"], rec["relres"])
            path = os.path.join(os.path.dirname(OUT), f"oracle_solution_{name}.json")
            samples = sol.pop("samples")
            head = json.dumps(sol, indent=1)[:-2]
            with open(path, "w") as f:
                f.write(head + ',\n "samples": [\n' + ",\n".join(json.dumps(t) for t in samples) + "\n ]\n}\n")
            print(name, rec, "->", path, flush=True)
        sys.exit(0)
    for name in sys.argv[1:]:
        data[name] = run_batch(name) if name in workloads.BATCH_NAMES else run(name)
        print(name, data[name], flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
