#!/usr/bin/env python3
"""RAS-PML Helmholtz benchmark on GB300.

One step = the whole hot path on the workload "c2" (k = 160*pi, h = 1/1280,
Omega_int = (0,1)^2 with a 0.1-wide PML, 32 x 32 subdomains, 16 seeded
Gaussian sources, about 2.36M complex unknowns): mesh and global assembly,
load vector, local assembly and LDL^T factorisation of all 1024 PML-extended
subdomains, and flexible GMRES with the RAS-PML preconditioner to a relative
residual of 1e-6.

  value      time per step of the complex64-factor form (local factors and
             solves in complex64, SpMV / Givens / true residual in complex128,
             Gram-Schmidt in double-float arithmetic on a complex64 Krylov
             basis, --ortho 4), seconds, lower is better
  fp64       the same step with complex128 local factors
  e2e        the complex64 form through helmholtz_solve_host: right-hand
             side from pinned host memory in, solution back to the host
  roofline   the apply of B^-1 (k_apply + k_prolong), timed with CUDA events
             inside the timed steps on the handle's stream
  learned    the same step with the learned coarse correction attached (a
             6-layer CNN on a 256^2 grid, tensor-core kernels), trained first
             on this problem's own residual/error pairs (training reported
             apart), and the network's forward / training-step times
  cpu_baseline  the CPU oracle on a bounded sample of the same workload,
             scaled to a full solve (see cpu_sample below)

--workload c3 times the batched form instead: 64 independent problems
(workloads.batch("c3"): k log-uniform in [20*pi, 120*pi], Omega_int sides
0.5-1.5, subdomain grids 2x2..12x12, 19.5M unknowns, 3827 subdomains) set up,
factored and solved to rtol 1e-6 in the same launches (complex64 factors,
lockstep FGMRES in complex128, one Arnoldi step per CUDA graph replay).

--workload net times the learned correction's network alone (forward pass on
one 256^2 image, training steps on 8), against the bf16 tensor peak.

--impl reference times the oracle alone (the reference arm of this repo).
Multi-GPU (torchrun): every rank solves its own replica of the workload; no
data-path collective. Inputs (factors of 4-17 GB) are far larger than L2.
"""
from __future__ import annotations

import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import hashlib  # noqa: E402
import json  # noqa: E402
import math  # noqa: E402
import re  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "RAS-PML time to rtol 1e-6 at k=160*pi, complex64 local factors + complex128 FGMRES (s)"
BATCH_METRIC = ("RAS-PML batched form: 64 independent problems (k 20*pi..120*pi, 19.5M unknowns) to rtol 1e-6, "
                "complex64 local factors + complex128 lockstep FGMRES (s)")
RTOL = 1e-6
MAXIT = 400


def net_channels():
    return (2, 32, 32, 32, 32, 32, 2)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_from_profile(kernel_src: str, algorithmic_bytes: float):
    """DRAM bytes per launch of k_apply for a launch of `algorithmic_bytes`,
    from the committed ncu summary (its measured ratio of DRAM traffic to
    algorithmic bytes: every factor entry is read once per sweep, so traffic
    grows in proportion), or None when the summary is missing or was taken
    on a different apply.cu."""
    path = os.path.join(ROOT, "profiles", "k_apply_sweep_c1.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_h = re.search(r"apply\.cu sha256: ([0-9a-f]{16})", txt)
    m_r = re.search(r"traffic / algorithmic = ([0-9.]+)", txt)
    if not m_h or not m_r:
        return None
    cur = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    return float(f"{float(m_r.group(1)) * algorithmic_bytes:.4g}") if cur == m_h.group(1) else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU oracle baseline on a bounded sample
# ---------------------------------------------------------------------------

def cpu_sample(w, iters: int, n_local: int = 64):
    """Times the oracle on a bounded sample of workload w and scales it to a
    full solve of `iters` FGMRES directions, with the oracle's own code:
      full:   global assembly, load vector, one global SpMV, one norm, and one
              modified Gram-Schmidt step (vdot + w - h v) on length-n vectors;
      sample: for n_local of the subdomains, local assembly + SuperLU factor
              (ras.build_subdomain, splu) and one local apply (gather, solve,
              weighted scatter: ras.local_apply), scaled to all subdomains.
    Estimate = assembly + load + nsub*factor + iters*(nsub*apply + SpMV + norm)
               + MGS steps sum_{j<iters} (j+1) + the final update (iters axpys)."""
    import scipy.sparse.linalg as spla

    from oracle import fem, ras
    p = w.params()
    t0 = time.perf_counter()
    grid, A = fem.assemble_global(p)
    t1 = time.perf_counter()
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    t2 = time.perf_counter()
    x = b / np.linalg.norm(b)
    y = A.dot(x)
    t3 = time.perf_counter()
    nrm = np.linalg.norm(y)
    t4 = time.perf_counter()
    hij = np.vdot(x, y)
    y = y - hij * x
    t5 = time.perf_counter()
    grid, rxs, rys = ras.covering(p)
    nsub = len(rxs) * len(rys)
    picks = np.unique(np.linspace(0, nsub - 1, min(n_local, nsub)).astype(int))
    tf = ta = 0.0
    z = np.zeros(grid.n, dtype=np.complex128)
    for j in picks:
        a = time.perf_counter()
        s = ras.build_subdomain(p, grid, rxs[j % len(rxs)], rys[j // len(rxs)])
        lu = spla.splu(s.A.tocsc())
        c = time.perf_counter()
        ras.local_apply(s, lu, b, z)
        d = time.perf_counter()
        tf += c - a
        ta += d - c
    tf /= len(picks)
    ta /= len(picks)
    t_mgs = t5 - t4
    est = (t1 - t0) + (t2 - t1) + nsub * tf + iters * (nsub * ta + (t3 - t2) + (t4 - t3)) \
        + t_mgs * iters * (iters + 1) / 2 + iters * t_mgs
    sample_s = time.perf_counter() - t0
    return est, sample_s, nsub, nrm


def host_cpus() -> dict:
    """The host's logical CPUs and the ones this process may run on."""
    aff = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None
    return {"host_cpus": os.cpu_count(), "affinity_cpus": aff}


def cpu_baseline_obj(w, iters, n_local: int = 64):
    n_local = min(n_local, w.px * w.py)
    est, sample_s, nsub, _ = cpu_sample(w, iters, n_local)
    return {"value": round(est, 3), "unit": "s", "cores": 1, "kind": "oracle", **host_cpus(),
            "sample": (f"oracle on {w.name}: global assembly, load vector, one SpMV, one norm and one modified "
                       f"Gram-Schmidt step on the full mesh; local assembly + SuperLU factor + one local apply "
                       f"(gather, solve, weighted scatter) on {n_local} of {nsub} subdomains (scaled x{nsub / n_local:g}); "
                       f"scaled to {iters} FGMRES directions; {sample_s:.1f} s of CPU work, one thread")}


def cpu_batch_baseline(probs, iters):
    """The oracle on the batched workload: cpu_sample on the problem of median
    size with its own iteration count, scaled to every problem by unknowns x
    (iterations + 1)."""
    n = np.array([w.n_unknowns for w in probs], dtype=float)
    it = np.asarray(iters, dtype=float)
    q = int(np.argsort(n)[len(n) // 2])
    est_q, sample_s, nsub, _ = cpu_sample(probs[q], int(it[q]))
    est = est_q * float(np.sum(n * (it + 1)) / (n[q] * (it[q] + 1)))
    return {"value": round(est, 3), "unit": "s", "cores": 1, "kind": "oracle", **host_cpus(),
            "sample": (f"oracle cpu_sample on {probs[q].name} ({int(n[q])} unknowns, {nsub} subdomains, "
                       f"{int(it[q])} directions; {sample_s:.1f} s of CPU work, one thread), scaled to all "
                       f"{len(probs)} problems by unknowns x (directions + 1)")}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over the ranks (the step time of the slowest rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_iterations(w) -> int:
    """The oracle's FGMRES iteration count on w (rtol 1e-6): from
    tests/golden/oracle_iterations.json, else by running the oracle."""
    gold = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if os.path.exists(gold):
        d = json.load(open(gold))
        if w.name in d:
            return int(d[w.name]["iters"])
    from oracle import fem, krylov, ras
    p = w.params()
    grid, A = fem.assemble_global(p)
    b = fem.assemble_rhs(p, w.centres, w.amps, w.width)
    R = ras.RAS(p).factor()
    return int(krylov.fgmres(A.dot, R.apply, b, rtol=RTOL, maxit=MAXIT)[1])


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_00735_gb300 import RasPml

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workloads.get(args.workload)
    p = dict(w.params(), form=args.form)
    stream = torch.cuda.current_stream(dev)

    shapes = {}   # tile shapes per factor precision, tuned once on a warm-up handle

    def one_step(prec, timing=False, ortho=None):
        s = RasPml(p, factor_prec=prec, ortho=args.ortho if ortho is None else ortho)
        if prec not in shapes:
            if args.shapes:
                shapes[prec] = tuple(int(v) for v in args.shapes.split(",")) + ({"fixed": args.shapes},)
            else:
                rep = s.tune()
                shapes[prec] = (rep["factor_threads"], rep["factor_rank"], rep["apply_cols"], rep)
        s.set_shapes(*shapes[prec][:3])
        if timing:
            s.set_timing(True)
        b = s.assemble_rhs(w.centres, w.amps, w.width)
        s.factor()
        x, it, rel, st = s.solve(b, rtol=RTOL, maxit=MAXIT)
        return s, x, it, rel, st

    def timed(prec, K, W, timing=True, ortho=None):
        for _ in range(W):
            s, x, it, rel, st = one_step(prec, ortho=ortho)
            s.close()
            del x
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        times, per = [], []
        xs = None
        for k in range(K):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s, x, it, rel, st = one_step(prec, timing, ortho=ortho)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            tm = s.timing()
            per.append(dict(tm, iters=it, relres=rel, status=st, info=s.info()))
            if k == K - 1:
                xs = x
            s.close()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return times, per, xs

    clocks = ClockSampler(local_rank)
    clocks.start()
    t_c64, per_c64, x_c64 = timed(args.prec, args.steps, args.warmup)
    clk = clocks.stop()
    fp64 = None
    x_f64 = None
    gs64 = None
    if not args.skip_fp64 and args.ortho >= 3:
        t_g, per_g, x_g = timed(1, max(1, min(args.steps, 2)), 1, ortho=2)
        gs64 = {"time_s": round(float(np.mean(t_g)), 4), "iters": per_g[-1]["iters"],
                "ortho_ms": round(per_g[-1]["ortho_ms"], 2),
                "error_vs_df": float(torch.linalg.vector_norm(x_g - x_c64) / torch.linalg.vector_norm(x_g))}
        del x_g
    if not args.skip_fp64:
        t_f64, per_f64, x_f64 = timed(0, max(1, min(args.steps, 2)), 1, ortho=2)
        fp64 = {"time_s": round(float(np.mean(t_f64)), 4), "iters": per_f64[-1]["iters"],
                "relres": per_f64[-1]["relres"], "factor_ms": round(per_f64[-1]["factor_ms"], 2),
                "solve_ms": round(per_f64[-1]["solve_ms"], 2),
                "apply_ms_avg": round(per_f64[-1]["apply_ms"] / max(1, per_f64[-1]["applies"]), 4),
                "apply_bytes": per_f64[-1]["info"]["apply_bytes"]}
    err = None
    if x_f64 is not None:
        err = float(torch.linalg.vector_norm(x_c64 - x_f64) / torch.linalg.vector_norm(x_f64))
    del x_c64, x_f64

    # end to end through host buffers
    e2e = None
    if not args.skip_e2e:
        s0 = RasPml(p, factor_prec=args.prec, ortho=args.ortho)
        b_host = s0.assemble_rhs(w.centres, w.amps, w.width).cpu().pin_memory()
        s0.close()
        x_host = torch.zeros_like(b_host).pin_memory()
        te = []
        for k in range(args.warmup + args.steps):
            x_host.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = RasPml(p, factor_prec=args.prec, ortho=args.ortho)
            s.set_shapes(*shapes[args.prec][:3])
            s.factor()
            s.solve_host(b_host, rtol=RTOL, maxit=MAXIT, x_host=x_host)
            t1 = time.perf_counter()
            s.close()
            if k >= args.warmup:
                te.append(t1 - t0)
        nb = b_host.numel() * b_host.element_size()
        e2e = {"value": round(float(np.mean(te)), 4), "unit": "s", "h2d_bytes_per_step": 2 * nb,
               "d2h_bytes_per_step": nb}

    # learned coarse correction (NEXT-2): trained on this problem's own
    # residual/error pairs (training time reported apart), then the same step
    # with the stage attached
    learned = None
    if not args.skip_learned:
        from paper_2602_00735_gb300.net import Net
        net = Net(Nc=256, cap=8, seed=0)
        s0 = RasPml(p, factor_prec=args.prec, ortho=args.ortho)
        s0.set_shapes(*shapes[args.prec][:3])
        s0.factor()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist, gamma = net.train(s0, nrhs=2, m_list=(1, 2, 4, 8, 16, 32), epochs=40, lr=1e-3, seed=7)
        t_train = time.perf_counter() - t0
        s0.close()
        tl, itl, rell = [], None, None
        for k in range(1 + args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s = RasPml(p, factor_prec=args.prec, ortho=args.ortho)
            s.set_shapes(*shapes[args.prec][:3])
            b = s.assemble_rhs(w.centres, w.amps, w.width)
            s.factor()
            s.attach_net(net)
            x, itl, rell, stl = s.solve(b, rtol=RTOL, maxit=MAXIT)
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                tl.append(e0.elapsed_time(e1) / 1e3)
            s.attach_net(None)
            s.close()
            del x, b
        # the network alone: one forward on one 256^2 image; one training step on 8
        xin = torch.randn(8, 2, 256, 256, device=dev, dtype=torch.float32)
        tin = torch.randn(8, 2, 256, 256, device=dev, dtype=torch.float32)
        net.forward(xin[:1])
        net.loss_grad(xin, tin, want_grad=False)
        tf, tb = [], []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            net.forward(xin[:1])
            e1.record(stream)
            net.loss_grad(xin, tin, want_grad=False)
            e2.record(stream)
            e2.synchronize()
            tf.append(e0.elapsed_time(e1) / 1e3)
            tb.append(e1.elapsed_time(e2) / 1e3)
        flop_img = 2 * 256 * 256 * 9 * sum(a * b for a, b in zip(net_channels(), net_channels()[1:]))
        learned = {"time_s": round(float(np.mean(tl)), 4), "iters": int(itl), "relres": float(rell),
                   "iters_plain": int(per_c64[-1]["iters"]), "train_s": round(t_train, 2), "gamma": gamma,
                   "loss_first_epoch": float(hist[0]), "loss_last_epoch": float(hist[-1]),
                   "coarse_grid": 256, "forward_ms_1img": round(1e3 * float(np.median(tf)), 4),
                   "forward_tflops": round(flop_img / float(np.median(tf)) / 1e12, 2),
                   "train_step_ms_8img": round(1e3 * float(np.median(tb)), 3),
                   "note": "complex64 form with the learned stage attached (minimal-residual scaled); "
                           "time excludes training"}
        net.close()

    # max over ranks
    mean_t = max_over_ranks(float(np.mean(t_c64)), world, dev)
    if rank != 0:
        return

    last = per_c64[-1]
    info = last["info"]
    applies = sum(q["applies"] for q in per_c64)
    apply_ms = sum(q["apply_ms"] for q in per_c64)
    avg_apply_s = apply_ms / max(1, applies) / 1e3
    achieved = info["apply_bytes"] / avg_apply_s / 1e9
    peak, peak_kind = peaks()
    traffic = traffic_from_profile(os.path.join(ROOT, "paper_2602_00735_gb300", "csrc", "apply.cu"),
                                   info["apply_bytes"])
    launches_per_step = [q["launches"] + 4 for q in per_c64]   # + setup stencil, rhs, local rows, factor
    out = {
        "metric": METRIC, "value": round(mean_t, 4), "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(mean_t * 1e3, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+c128", "data": "synthetic",
        "config": {"workload": f"{w.name}: k={p['k'] / math.pi:g}*pi, h=1/{round(1 / p['h'])}, "
                               f"Omega_int=({p['x0']:g},{p['x1']:g})x({p['y0']:g},{p['y1']:g}), PML {p['kappa_g']:g}, "
                               f"{p['px']}x{p['py']} subdomains, ovlp={p['ovlp_cells']} pml={p['pml_cells']} cells, "
                               f"{len(w.amps)} Gaussians width {w.width}",
                   "n_unknowns": info["n"], "rtol": RTOL, "parallelism": f"replicas x{world}",
                   "form": args.form,
                   "l2": "inputs larger than L2 (complex64 factors %.1f GB)" % (info["factor_bytes"] / 1e9)},
        "iters": last["iters"], "relres": last["relres"], "ortho": args.ortho, "reorths": last["reorths"],
        "phases_ms": {"factor": round(last["factor_ms"], 2), "solve": round(last["solve_ms"], 2),
                      "apply": round(last["apply_ms"], 2), "spmv": round(last["spmv_ms"], 2),
                      "ortho": round(last["ortho_ms"], 2),
                      "setup_and_rest": round(mean_t * 1e3 - last["factor_ms"] - last["solve_ms"], 2)},
        "apply_gbs": round(achieved, 1),
        "applies_per_s": round(1.0 / avg_apply_s, 1),
        # one timed SpMV per direction: 4 coefficient arrays, x and y (96 bytes per row);
        # 7 arrays with form 1 (144 bytes per row)
        "spmv_gbs": round((96.0 if args.form == 0 else 144.0) * info["n"] * sum(q["applies"] for q in per_c64)
                          / max(1e-9, sum(q["spmv_ms"] for q in per_c64) / 1e3) / 1e9, 1),
        "roofline": {"kernel": "ras_pml_apply (k_apply + k_prolong), complex64", "bound": "hbm",
                     "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "algorithmic_bytes_per_launch": info["apply_bytes"]},
        "fp64": fp64, "error_vs_fp64": err, "c64_fp64_gram_schmidt": gs64,
        "tune": shapes[args.prec][3],
        "learned": learned,
        "gpu_launches": int(sum(launches_per_step)),
        "gpu_launches_per_step": int(launches_per_step[-1]),
        "clocks": clk, "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        it = fp64["iters"] if fp64 else last["iters"]
        out["cpu_baseline"] = cpu_baseline_obj(w, it)
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# Batched form (--workload c3)
# ---------------------------------------------------------------------------

def batch_iterations_golden():
    gold = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if os.path.exists(gold):
        d = json.load(open(gold))
        if "c3" in d:
            return d["c3"]["iters"]
    return None


def run_batch(args, rank, world, local_rank):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_00735_gb300 import BatchRasPml

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    probs = workloads.batch(args.workload)
    params = [w.params() for w in probs]
    srcs = [(w.centres, w.amps, w.width) for w in probs]
    shapes = None

    def one_step():
        B = BatchRasPml(params, factor_prec=args.prec)
        if shapes is not None:
            B.set_shapes(*shapes)
        b = B.assemble_rhs(srcs)
        B.factor()
        x, it, rel, st = B.solve(b, rtol=RTOL, maxit=MAXIT)
        return B, b, x, it, rel, st

    # tile shapes chosen once, on the first warm-up handle (or fixed by --shapes)
    if args.shapes:
        tune = {"fixed": args.shapes}
        shapes = tuple(int(v) for v in args.shapes.split(","))
    else:
        B0 = BatchRasPml(params, factor_prec=args.prec)
        tune = B0.tune()
        shapes = (tune["factor_threads"], tune["factor_rank"], tune["apply_cols"])
        B0.close()
    for _ in range(args.warmup):
        B, b, x, it, rel, st = one_step()
        B.close()
        del b, x
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    times = []
    for k in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B, b, x, it, rel, st = one_step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        info = B.info()
        B.close()          # its Krylov space takes most of the free memory
        del x
    clk = clocks.stop()
    # the batch apply (local solves of all subdomains + prolongation) on a
    # factored handle without a Krylov space
    B = BatchRasPml(params, factor_prec=args.prec)
    B.set_shapes(*shapes)
    B.factor()
    r = b.clone()
    z = B.apply(r)
    ta = []
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.apply(r, out=z)
        e1.record(stream)
        e1.synchronize()
        ta.append(e0.elapsed_time(e1) / 1e3)
    B.close()
    del r, z
    t_apply = float(np.median(ta))
    achieved = info["apply_bytes"] / t_apply / 1e9
    peak, peak_kind = peaks()
    # end to end: right-hand sides from pinned host memory, solutions back
    e2e = None
    if not args.skip_e2e:
        b_host = b.cpu().pin_memory()
        x_host = torch.empty_like(b_host).pin_memory()
        te = []
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Bh = BatchRasPml(params, factor_prec=args.prec)
            Bh.set_shapes(*shapes)
            bd = b_host.to(dev, non_blocking=True)
            Bh.factor()
            xd, _, _, _ = Bh.solve(bd, rtol=RTOL, maxit=MAXIT)
            x_host.copy_(xd)
            t1 = time.perf_counter()
            Bh.close()
            del xd, bd
            if k >= args.warmup:
                te.append(t1 - t0)
        nb = b_host.numel() * b_host.element_size()
        e2e = {"value": round(float(np.mean(te)), 4), "unit": "s", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb}
    mean_t = max_over_ranks(float(np.mean(times)), world, dev)
    if rank != 0:
        return
    nprob = info["nprob"]
    launches = 2 * nprob + 2 + info["cycles"] * 5 + 3 + info["steps"] * 9
    out = {
        "metric": BATCH_METRIC if args.workload == "c3" else f"RAS-PML batched form ({args.workload}) to rtol 1e-6 (s)",
        "value": round(mean_t, 4), "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(mean_t * 1e3, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+c128", "data": "synthetic",
        "config": {"workload": (f"{args.workload}: {nprob} problems, k {min(w.k for w in probs) / math.pi:.1f}*pi.."
                                f"{max(w.k for w in probs) / math.pi:.1f}*pi, 16 points per wavelength, "
                                f"Omega_int sides 0.5..1.5, PML 0.1, grids 2x2..12x12, 1-8 Gaussians each"),
                   "n_unknowns": info["sum_n"], "num_subdomains": info["num_sub"], "rtol": RTOL,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (complex64 factors %.1f GB)" % (info["factor_bytes"] / 1e9)},
        "iters": {"min": int(it.min()), "median": float(np.median(it)), "max": int(it.max())},
        "relres_max": float(rel.max()), "status": st, "lockstep_steps": info["steps"], "cycles": info["cycles"],
        "tune": tune, "shapes": {"factor_threads": shapes[0], "factor_rank": shapes[1], "apply_cols": shapes[2]},
        "apply_ms": round(t_apply * 1e3, 3),
        "roofline": {"kernel": "ras_pml_batch_apply (k_apply + k_bprolong), complex64", "bound": "hbm",
                     "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "algorithmic_bytes_per_launch": info["apply_bytes"]},
        "gpu_launches": int(launches * args.steps), "gpu_launches_per_step": int(launches),
        "clocks": clk, "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_batch_baseline(probs, it)
    print(json.dumps(out), flush=True)



def run_net(args, rank, world, local_rank):
    """The learned correction's network alone (tensor-core 3x3 convolutions):
    forward passes on one 256^2 image and training steps (forward, backward,
    Adam) on batches of 8, random inputs; the roofline object is the forward
    pass against the measured bf16 tensor peak."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_00735_gb300.net import Net

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    Nc, B = 256, 8
    net = Net(Nc=Nc, cap=B, seed=0)
    x = torch.randn(B, 2, Nc, Nc, device=dev, dtype=torch.float32)
    t = torch.randn(B, 2, Nc, Nc, device=dev, dtype=torch.float32)
    for _ in range(args.warmup):
        net.forward(x[:1])
        net.loss_grad(x, t, want_grad=False)
        net.adam_step(1e-4)
    torch.cuda.synchronize()
    tf, tt = [], []
    for _ in range(args.steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        net.forward(x[:1])
        e1.record(stream)
        net.loss_grad(x, t, want_grad=False)
        net.adam_step(1e-4)
        e2.record(stream)
        e2.synchronize()
        tf.append(e0.elapsed_time(e1) / 1e3)
        tt.append(e1.elapsed_time(e2) / 1e3)
    net.close()
    ch = net_channels()
    flop_real = 2 * Nc * Nc * 9 * sum(a * b for a, b in zip(ch, ch[1:]))
    pad = (16, 32, 32, 32, 32, 32, 16)   # channels as the tensor cores run them
    flop_tc = 2 * Nc * Nc * 9 * sum(a * b for a, b in zip(pad, pad[1:]))
    tfw = float(np.median(tf))
    mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(mp.get("bf16_tflops", 1900.0))
    if rank != 0:
        return
    out = {"metric": "learned-correction network: one forward pass on a 256^2 image (ms)",
           "value": round(1e3 * tfw, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * tfw, 4), "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": "net: 6 layers 3x3, channels 2-32-32-32-32-32-2, 256^2 grid, batch 8 for training",
                      "l2": "activations resident in L2 (4 MB per layer)"},
           "train_step_ms_8img": round(1e3 * float(np.median(tt)), 3),
           "roofline": {"kernel": "k_conv_tc (forward, 6 launches)", "bound": "tensor",
                        "achieved": round(flop_tc / tfw / 1e12, 2), "peak": peak,
                        "peak_kind": "measured" if mp else "fallback", "unit": "TFLOP/s",
                        "frac": round(flop_tc / tfw / 1e12 / peak, 4), "traffic": None,
                        "flop_per_launch_set": flop_tc, "flop_real_channels": flop_real},
           "gpu_launches": 6 * args.steps, "e2e": None}
    print(json.dumps(out), flush=True)


def run_reference_batch(args, world):
    probs = workloads.batch("c3")
    iters = batch_iterations_golden()
    if iters is None:
        print(json.dumps({"impl": "reference", "unavailable": "no stored oracle iteration counts for c3"}))
        return
    vals, last = [], None
    for k in range(args.warmup + args.steps):
        obj = cpu_batch_baseline(probs, iters)
        if k >= args.warmup:
            vals.append(obj["value"])
            last = obj
    v = float(np.mean(vals))
    out = {"impl": "reference", "metric": BATCH_METRIC, "value": round(v, 3), "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": {"workload": "c3", "rtol": RTOL},
           "cpu_baseline": dict(last, value=round(v, 3)),
           "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload == "c3":
        run_reference_batch(args, world)
        return
    if args.workload == "net":
        print(json.dumps({"impl": "reference", "unavailable": "the network has no timed reference arm "
                                                             "(the paper has no learned component)"}))
        return
    w = workloads.get(args.workload)
    iters = oracle_iterations(w)
    vals = []
    last = None
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        obj = cpu_baseline_obj(w, iters)
        t1 = time.perf_counter()
        if k >= args.warmup:
            vals.append(obj["value"])
            last = obj
    v = float(np.mean(vals))
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic", "config": {"workload": w.name, "rtol": RTOL, "iters": iters},
           "cpu_baseline": dict(last, value=round(v, 3)),
           "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--ortho", type=int, default=4, choices=[0, 1, 2, 3, 4],
                    help="0: classical Gram-Schmidt twice; 1: once plus the DGKS reorthogonalisation test; "
                         "2: once; 3: once in double-float arithmetic; 4: as 3 on a complex64 basis")
    ap.add_argument("--prec", type=int, default=1, choices=[1, 2],
                    help="local factors of the headline form: 1 complex64, 2 complex64 with half-precision storage")
    ap.add_argument("--form", type=int, default=0, choices=[0, 1],
                    help="bilinear form: 0 the complex-symmetric gamma_1 gamma_2 form (L D L^T factors), "
                         "1 eq. weak as printed (L D U factors; needs --ortho 0..2, no learned stage)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-learned", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shapes", default="",
                    help="fixed tile shapes 'threads,rank,cols' instead of tuning (profiling runs)")
    args = ap.parse_args()
    if args.form == 1:
        if args.ortho > 2 or args.workload in ("c3", "net"):
            ap.error("--form 1 takes --ortho 0..2 and a one-problem workload")
        args.skip_learned = True
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.workload in workloads.BATCH_NAMES:
            run_batch(args, rank, world, local_rank)
        elif args.workload == "net":
            run_net(args, rank, world, local_rank)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
