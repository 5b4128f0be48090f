"""Host-side checks of bench.py (no GPU): the reference arm's JSON line, its
rank handling under torchrun, and the max-over-ranks reduction of the step
time with two gloo ranks on CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_json_line():
    r = _run(["--impl", "reference", "--workload", "tiny3", "--steps", "1", "--warmup", "0"], {})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "s"
    assert d["higher_is_better"] is False
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == min(cores, 9)
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the same config object as the GPU arm's line
    sys.path.insert(0, ROOT)
    import bench
    import workloads
    assert d["config"] == bench.bench_config(workloads.get("tiny3"), 0, 1)
    sp = d["cpu_baseline"]["split"]
    assert abs(sp["total_s"] - (sp["setup_s"] + sp["factor_s"] + sp["solve_s"])) < 2e-3


def test_form_option_is_validated_before_any_device_work():
    """--form 1 (eq. weak as printed) takes the FP64 Gram-Schmidt variants and a
    one-problem workload only; argparse refuses the rest with status 2."""
    for args in (["--form", "1", "--ortho", "4"], ["--form", "1", "--ortho", "2", "--workload", "c3"],
                 ["--form", "2"]):
        r = _run(args, {})
        assert r.returncode == 2 and "form" in r.stderr, (args, r.stderr)


def test_reference_arm_for_the_batched_workload():
    """--workload c3: the oracle's median problem solved on all cores, scaled
    by the oracle's own per-problem iteration counts (tests/golden)."""
    r = _run(["--impl", "reference", "--workload", "c3", "--steps", "1", "--warmup", "0"], {})
    assert r.returncode == 0, r.stderr
    d = json.loads([ln for ln in r.stdout.splitlines() if ln.strip()][0])
    assert d["impl"] == "reference" and d["value"] > 0 and "64 independent problems" in d["metric"]
    assert "scaled to all 64 problems" in d["cpu_baseline"]["sample"]


def test_reference_arm_runs_on_rank_zero_only():
    r = _run(["--impl", "reference", "--workload", "tiny3", "--steps", "1", "--warmup", "0"],
             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def _max_worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(1.5 + rank, world)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 2.5, 1: 2.5}


def test_apply_traffic_scales_with_the_workload(tmp_path):
    """The roofline's traffic figure comes from the committed ncu summary of
    k_apply: its captured DRAM-to-algorithmic ratio times the workload's own
    algorithmic bytes, and None once apply.cu differs from the captured one."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    src = os.path.join(ROOT, "paper_2602_00735_gb300", "csrc", "apply.cu")
    a = bench.traffic_from_profile(src, 1.0e9)
    b = bench.traffic_from_profile(src, 4.0e9)
    assert a is not None and b is not None
    assert 1.0 <= a / 1.0e9 <= 1.2                  # a little above the algorithmic bytes
    assert abs(b / a / 4.0 - 1.0) < 1e-3             # in proportion (both rounded to 4 digits)
    other = tmp_path / "apply.cu"
    other.write_text(open(src).read() + "\n// changed\n")
    assert bench.traffic_from_profile(str(other), 1.0e9) is None
