"""The multi-rank partition of the hot path (paper_2602_00735_gb300.partition)
applied by two gloo ranks on CPU to oracle vectors: each rank holds only its
own unknowns of r and x (every other entry is NaN, so a node missing from an
exchange list poisons the result), receives the halos the plan lists, solves
its own subdomains with the oracle's local operators and SuperLU factors,
sends its prolongation contributions to the owners, and the owners sum them in
subdomain order. Gathered on rank 0, B^-1 r and A x equal the one-rank
oracle's bit for bit; the Arnoldi inner product, all-reduced, agrees to
rounding. Host-side checks of the lists themselves run without ranks."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from paper_2602_00735_gb300.partition import Plan  # noqa: E402

CASES = [("tiny3", 2, 1, {}), ("small", 2, 1, {}), ("small", 1, 2, {}), ("tiny3", 2, 1, {"local_bc": 1}),
         ("small", 2, 1, {"px": 3, "py": 5})]


def _plan(w, Rx, Ry):
    p = w.params()
    return Plan.build(w.cells_x, w.cells_y, p["px"], p["py"], p["ovlp_cells"], p["pml_cells"], p["local_bc"], Rx, Ry)


def _xchg(dist, sends, recvs, get, n_entries):
    """Sends get(idx) to each destination, receives len(idx) complex values
    from each source (non-blocking, then waits); returns {src: values}."""
    import torch
    reqs, bufs = [], {}
    for dst, idx in sends.items():
        t = torch.from_numpy(np.ascontiguousarray(get(dst, idx)).view(np.float64).copy())
        reqs.append(dist.isend(t, dst))
    for src, cnt in recvs.items():
        bufs[src] = torch.empty(2 * n_entries(cnt), dtype=torch.float64)
        reqs.append(dist.irecv(bufs[src], src))
    for q in reqs:
        q.wait()
    return {s: b.numpy().view(np.complex128) for s, b in bufs.items()}


def _rank_main(rank, world, port, case, q):
    import scipy.sparse.linalg as spla
    import torch.distributed as dist

    from oracle import fem, ras
    name, Rx, Ry, kw = CASES[case]
    w = workloads.get(name).with_(**kw)
    p = w.params()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        plan = _plan(w, Rx, Ry)
        grid, rxs, rys = ras.covering(p)
        n = grid.n
        rng = np.random.default_rng(30)
        r_full = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        x_full = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        own = plan.owned[rank]
        r = np.full(n, np.nan + 1j * np.nan)
        r[own] = r_full[own]
        x = np.full(n, np.nan + 1j * np.nan)
        x[own] = x_full[own]
        # restriction halo
        got = _xchg(dist, plan.restrict_send(rank), {s: len(v) for s, v in plan.restrict_recv[rank].items()},
                    lambda d, idx: r[idx], lambda c: c)
        for s, vals in got.items():
            r[plan.restrict_recv[rank][s]] = vals
        # local solves of the rank's subdomains
        contrib = []            # (subdomain, node, value) of every chi_j > 0 entry
        for qd in plan.subdomains[rank]:
            sd = ras.build_subdomain(p, grid, rxs[qd % p["px"]], rys[qd // p["px"]])
            c = sd.chi * spla.splu(sd.A.tocsc()).solve(r[sd.glob])
            m = sd.chi > 0
            contrib.extend(zip([qd] * int(m.sum()), sd.glob[m].tolist(), c[m].tolist()))
        owner = np.empty(n, dtype=np.int64)
        for s in range(world):
            owner[plan.owned[s]] = s
        mine = [t for t in contrib if owner[t[1]] == rank]
        away = {}
        for t in contrib:
            if owner[t[1]] != rank:
                away.setdefault(int(owner[t[1]]), []).append(t)
        # the plan's prolongation lists are exactly the off-rank contributions
        for s, lst in plan.prolong_send[rank].items():
            assert [(a, b) for a, b, _ in away[s]] == [(int(a), int(b)) for a, b in lst]
        assert set(away) == set(plan.prolong_send[rank])
        recv_pairs = plan.prolong_recv(rank)
        got = _xchg(dist, {s: [v for _, _, v in away[s]] for s in away},
                    {s: len(v) for s, v in recv_pairs.items()}, lambda d, vals: np.array(vals, dtype=complex),
                    lambda c: c)
        for s, vals in got.items():
            mine.extend((int(a), int(b), v) for (a, b), v in zip(recv_pairs[s], vals))
        # owners sum every node's contributions in increasing subdomain order
        z = np.zeros(n, dtype=complex)
        for qd, node, v in sorted(mine, key=lambda t: (t[1], t[0])):
            z[node] = z[node] + v
        # SpMV with the 1-cell halo
        got = _xchg(dist, plan.spmv_send(rank), {s: len(v) for s, v in plan.spmv_recv[rank].items()},
                    lambda d, idx: x[idx], lambda c: c)
        for s, vals in got.items():
            x[plan.spmv_recv[rank][s]] = vals
        grid, A = fem.assemble_global(p)
        y_own = A.tocsr()[own] @ x
        # the Arnoldi inner product over owned entries, all-reduced
        import torch
        part = np.vdot(x_full[own], r_full[own])
        t = torch.tensor([part.real, part.imag], dtype=torch.float64)
        dist.all_reduce(t)
        q.put((rank, own, z[own], y_own, complex(t[0].item(), t[1].item())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", range(len(CASES)), ids=[f"{c[0]}-{c[1]}x{c[2]}" + "".join(f"-{k}{v}" for k, v in c[3].items())
                                                         for c in CASES])
def test_two_gloo_ranks_reproduce_the_one_rank_apply_and_product(case):
    import torch.multiprocessing as mp

    from oracle import fem, ras
    name, Rx, Ry, kw = CASES[case]
    w = workloads.get(name).with_(**kw)
    p = w.params()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, case, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=120)
    assert all(pr.exitcode == 0 for pr in procs)
    grid, A = fem.assemble_global(p)
    n = grid.n
    rng = np.random.default_rng(30)
    r = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    z_ref = ras.RAS(p).factor().apply(r)
    y_ref = A @ x
    z, y = np.full(n, np.nan + 0j), np.full(n, np.nan + 0j)
    for rank, own, zo, yo, dot in res:
        z[own] = zo
        y[own] = yo
        assert abs(dot - np.vdot(x, r)) <= 1e-13 * abs(np.vdot(x, r))
    assert np.array_equal(z, z_ref)
    assert np.array_equal(y, y_ref)


@pytest.mark.parametrize("name,Rx,Ry", [("c2", 4, 2), ("c2", 2, 2), ("small", 2, 2)])
def test_plan_covers_every_unknown_once_and_exchanges_only_overlaps(name, Rx, Ry):
    """Ownership partitions the unknowns; the restriction halo of a rank lies
    within ovlp + pml + 1 nodes of its owned ones (the impedance node on the
    artificial boundary; a box's upper edge node belongs to the next box), its
    prolongation contributions within ovlp, its SpMV halo within one node."""
    w = workloads.get(name)
    plan = _plan(w, Rx, Ry)
    n = (w.cells_x - 1) * (w.cells_y - 1)
    allown = np.concatenate(plan.owned)
    assert allown.size == n and np.array_equal(np.sort(allown), np.arange(n))
    nx = w.cells_x - 1
    o, k = w.ovlp_cells, w.pml_cells
    for r in range(plan.nranks):
        own = plan.owned[r]
        i_lo, i_hi = (own % nx).min(), (own % nx).max()
        j_lo, j_hi = (own // nx).min(), (own // nx).max()

        def dist(g):
            i, j = g % nx, g // nx
            return np.maximum(np.maximum(i_lo - i, i - i_hi), np.maximum(j_lo - j, j - j_hi)).max()
        for s, idx in plan.restrict_recv[r].items():
            assert s != r and dist(idx) <= o + k + 1
        for s, pairs in plan.prolong_send[r].items():
            assert dist(np.array([g for _, g in pairs])) <= o
        for s, idx in plan.spmv_recv[r].items():
            assert dist(idx) <= 1
        b = plan.exchange_bytes(r)
        assert b["restrict"] > 0 and b["prolong"] > 0 and b["spmv"] > 0


def test_residual_after_a_sweep_lives_on_the_plans_support():
    """One sweep of Algorithm 1 in the oracle (u = B^-1 F): b - A u vanishes,
    to rounding, outside the plan's residual support (Section 3 (i))."""
    from oracle import fem, ras
    for name, kw in (("tiny3", {}), ("small", {"px": 3, "py": 5}), ("small", {"local_bc": 1})):
        w = workloads.get(name).with_(**kw)
        p = w.params()
        grid, A = fem.assemble_global(p)
        b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
        u = ras.RAS(p).factor().apply(b)
        res = b - A @ u
        sup = _plan(w, 1, 1).residual_support()
        assert np.max(np.abs(res[~sup])) <= 1e-12 * np.max(np.abs(res))
        assert np.max(np.abs(res[sup])) > 1e-3 * np.linalg.norm(b)     # and does not vanish on it
        assert sup.mean() < 0.9


def _richardson_rank(rank, world, port, case, sweeps, q):
    import scipy.sparse.linalg as spla
    import torch.distributed as dist

    from oracle import fem, ras
    name, Rx, Ry, kw = CASES[case]
    w = workloads.get(name).with_(**kw)
    p = w.params()
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        plan = _plan(w, Rx, Ry)
        grid, rxs, rys = ras.covering(p)
        grid, A = fem.assemble_global(p)
        A = A.tocsr()
        n = grid.n
        b_full = fem.assemble_rhs(p, w.centres, w.amps, w.width)
        own = plan.owned[rank]
        owner = np.empty(n, dtype=np.int64)
        for s in range(world):
            owner[plan.owned[s]] = s
        subs = []
        for qd in plan.subdomains[rank]:
            sd = ras.build_subdomain(p, grid, rxs[qd % p["px"]], rys[qd // p["px"]])
            subs.append((qd, sd, spla.splu(sd.A.tocsc())))
        u = np.zeros(n, dtype=complex)          # owned entries meaningful
        sent = 0
        for it in range(sweeps):
            # r = F - A u on owned rows, with the SpMV halo of u
            uh = np.full(n, np.nan + 0j)
            uh[own] = u[own]
            got = _xchg(dist, plan.spmv_send(rank), {s: len(v) for s, v in plan.spmv_recv[rank].items()},
                        lambda d, idx: uh[idx], lambda c: c)
            for s, vals in got.items():
                uh[plan.spmv_recv[rank][s]] = vals
            r = np.full(n, np.nan + 0j)
            r[own] = b_full[own] - A[own] @ uh
            # restriction halo: full before the first sweep, the residual's
            # support after it (zero is taken elsewhere)
            recv = plan.restrict_recv[rank] if it == 0 else plan.restrict_recv_sparse[rank]
            send = plan.restrict_send(rank) if it == 0 else plan.restrict_send_sparse(rank)
            if it > 0:
                full = np.concatenate([v for v in plan.restrict_recv[rank].values()])
                r[full] = 0.0
            got = _xchg(dist, send, {s: len(v) for s, v in recv.items()}, lambda d, idx: r[idx], lambda c: c)
            for s, vals in got.items():
                r[recv[s]] = vals
                sent += len(vals)
            contrib = []
            for qd, sd, lu in subs:
                c = sd.chi * lu.solve(r[sd.glob])
                m = sd.chi > 0
                contrib.extend(zip([qd] * int(m.sum()), sd.glob[m].tolist(), c[m].tolist()))
            mine = [t for t in contrib if owner[t[1]] == rank]
            away = {}
            for t in contrib:
                if owner[t[1]] != rank:
                    away.setdefault(int(owner[t[1]]), []).append(t)
            recv_pairs = plan.prolong_recv(rank)
            got = _xchg(dist, {s: [v for _, _, v in away[s]] for s in away},
                        {s: len(v) for s, v in recv_pairs.items()}, lambda d, vals: np.array(vals, dtype=complex),
                        lambda c: c)
            for s, vals in got.items():
                mine.extend((int(a), int(b), v) for (a, b), v in zip(recv_pairs[s], vals))
            z = np.zeros(n, dtype=complex)
            for qd, node, v in sorted(mine, key=lambda t: (t[1], t[0])):
                z[node] = z[node] + v
            u[own] = u[own] + z[own]
        q.put((rank, own, u[own], sent))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [0, 1, 4], ids=["tiny3-2x1", "small-2x1", "small-2x1-px3-py5"])
def test_algorithm_1_with_the_reduced_restriction_halo(case):
    """Algorithm 1 on two gloo ranks: the first sweep exchanges the full
    restriction halo, the later ones only its part in the residual's support;
    after 4 sweeps the iterate equals the one-rank oracle's to rounding, with
    fewer values exchanged than with the full halo every sweep."""
    import torch.multiprocessing as mp

    from oracle import fem, krylov, ras
    name, Rx, Ry, kw = CASES[case]
    w = workloads.get(name).with_(**kw)
    p = w.params()
    sweeps = 4
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_richardson_rank, args=(r, 2, port, case, sweeps, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in range(2)]
    for pr in procs:
        pr.join(timeout=120)
    assert all(pr.exitcode == 0 for pr in procs)
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    u_ref, it, _, _ = krylov.richardson(A.dot, ras.RAS(p).factor().apply, b, rtol=0.0, maxit=sweeps)
    assert it == sweeps
    u = np.full(grid.n, np.nan + 0j)
    plan = _plan(w, Rx, Ry)
    full = 0
    for rank, own, uo, sent in res:
        u[own] = uo
        full += sweeps * sum(len(v) for v in plan.restrict_recv[rank].values())
    assert np.linalg.norm(u - u_ref) <= 1e-12 * np.linalg.norm(u_ref)
    assert sum(t[3] for t in res) < 0.9 * full
