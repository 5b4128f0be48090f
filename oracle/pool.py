"""Oracle, part 5: the RAS-PML preconditioner on all host cores.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): used by the timed CPU
baseline, never by the product path.

The same B^-1 r = sum_j R_j^T (chi_j * A_j^-1 (R_j r)) as ras.RAS (Section 2,
the equation defining B^-1), computed by worker processes (started with
"spawn") that each own a round-robin share of the subdomains:
  * set-up: a worker builds its subdomains with ras.build_subdomain (local
    assembly with the local stretching and the closure of Section 3 (ii)) and
    factors them with SuperLU (scipy.sparse.linalg.splu), once;
  * apply: the parent puts r in shared memory; every worker writes
    chi_j * A_j^-1 (R_j r) of each of its subdomains into that subdomain's own
    slice of a shared array Y (disjoint writes); the parent then forms
    z_i = sum of the Y entries that hold node i, in increasing subdomain order
    (the sum R_j^T ... over j, written as a gather of at most a few entries
    per node). Entries with chi_j = 0 (the local PML) add nothing and are left
    out of the gather.
Only the order of the final additions differs from ras.RAS.apply.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time
from multiprocessing import shared_memory

import numpy as np


def _worker(p, js, conn, r_name, n):
    # one BLAS thread per worker: the parallelism is over subdomains
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    import scipy.sparse.linalg as spla

    from . import ras
    grid, rxs, rys = ras.covering(p)
    r_shm = shared_memory.SharedMemory(name=r_name)
    r = np.ndarray((n,), dtype=np.complex128, buffer=r_shm.buf)
    t0 = time.perf_counter()
    subs, lus = [], []
    for j in js:
        s = ras.build_subdomain(p, grid, rxs[j % len(rxs)], rys[j // len(rxs)])
        subs.append(s)
        lus.append(spla.splu(s.A.tocsc()))
    conn.send(("built", [(s.glob, s.chi) for s in subs], time.perf_counter() - t0))
    _, y_name, ny, offs = conn.recv()
    y_shm = shared_memory.SharedMemory(name=y_name)
    y = np.ndarray((ny,), dtype=np.complex128, buffer=y_shm.buf)
    try:
        while True:
            cmd = conn.recv()
            if cmd != "apply":
                break
            for s, lu, off in zip(subs, lus, offs):
                y[off:off + s.glob.size] = s.chi * lu.solve(r[s.glob])
            conn.send("done")
    finally:
        del r, y
        r_shm.close()
        y_shm.close()


class PoolRAS:
    """B^-1 of ras.RAS with SuperLU local factors on `nproc` processes.

    factor_s: wall time of the parallel local assembly and factorisation.
    Use as a context manager (the workers and shared memory are released on
    exit)."""

    def __init__(self, p: dict, nproc: int | None = None):
        from . import ras
        grid, rxs, rys = ras.covering(p)
        self.n = grid.n
        nsub = len(rxs) * len(rys)
        self.nproc = max(1, min(nproc or os.cpu_count() or 1, nsub))
        ctx = mp.get_context("spawn")
        self._r_shm = shared_memory.SharedMemory(create=True, size=16 * self.n)
        self.r = np.ndarray((self.n,), dtype=np.complex128, buffer=self._r_shm.buf)
        self._y_shm = None
        shares = [list(range(q, nsub, self.nproc)) for q in range(self.nproc)]
        self._conns, self._procs = [], []
        t0 = time.perf_counter()
        for js in shares:
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_worker, args=(p, js, b, self._r_shm.name, self.n), daemon=True)
            pr.start()
            self._conns.append(a)
            self._procs.append(pr)
        built = [None] * nsub
        for js, c in zip(shares, self._conns):
            tag, data, _ = c.recv()
            assert tag == "built"
            for j, d in zip(js, data):
                built[j] = d
        self.factor_s = time.perf_counter() - t0
        # Y: the local slices in subdomain order; one zero slot at the end
        sizes = np.array([g.size for g, _ in built], dtype=np.int64)
        offs = np.concatenate([[0], np.cumsum(sizes)])
        ny = int(offs[-1])
        self._y_shm = shared_memory.SharedMemory(create=True, size=16 * (ny + 1))
        self.y = np.ndarray((ny + 1,), dtype=np.complex128, buffer=self._y_shm.buf)
        self.y[:] = 0.0
        for js, c in zip(shares, self._conns):
            c.send(("y", self._y_shm.name, ny + 1, [int(offs[j]) for j in js]))
        # gather map: column i lists the Y positions of node i (chi > 0), by subdomain
        g = np.concatenate([gl[ch > 0] for gl, ch in built])
        pos = np.concatenate([offs[j] + np.nonzero(built[j][1] > 0)[0] for j in range(nsub)])
        order = np.argsort(g, kind="stable")
        g, pos = g[order], pos[order]
        counts = np.bincount(g, minlength=self.n)
        starts = np.cumsum(counts) - counts
        rank = np.arange(g.size) - starts[g]
        self.gather = np.full((int(counts.max()), self.n), ny, dtype=np.int64)
        self.gather[rank, g] = pos
        self.nsub = nsub

    def apply(self, r):
        self.r[:] = r
        for c in self._conns:
            c.send("apply")
        for c in self._conns:
            assert c.recv() == "done"
        z = self.y[self.gather[0]].copy()
        for k in range(1, self.gather.shape[0]):
            z += self.y[self.gather[k]]
        return z

    def close(self):
        for c in self._conns:
            try:
                c.send("stop")
            except (BrokenPipeError, OSError):
                pass
        for pr in self._procs:
            pr.join(timeout=10)
            if pr.is_alive():
                pr.terminate()
        self._conns, self._procs = [], []
        for attr in ("r", "y"):
            if hasattr(self, attr):
                delattr(self, attr)
        for shm in (self._r_shm, self._y_shm):
            if shm is not None:
                shm.close()
                shm.unlink()
        self._r_shm = self._y_shm = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
