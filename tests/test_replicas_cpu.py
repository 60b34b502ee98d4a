"""The N > 1 host path of bench.py on CPU (gloo, world size 2).

The method here runs as independent replicas, one per GPU, with no data-path
collective.  The only cross-rank steps are a barrier and the maximum of the
ranks' times, which bounds the whole-job throughput.  These tests exercise those
steps with two gloo ranks on 127.0.0.1, and the reference arm under torchrun:
rank 0 alone works and prints one JSON line, and the other rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # each rank's "time"; every rank must see the slowest
        t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        units = 1000
        v = bench.replica_throughput(world, units, 10, t)
        out.put((rank, t, v))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_throughput_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in got:
        assert t == 2.5  # the slower rank's time on both ranks
        assert v == pytest.approx(2 * 1000 * 10 / 2.5 / 1e6)


def test_single_rank_aggregation_is_the_identity():
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.replica_throughput(1, 4096, 5, 0.5) == pytest.approx(4096 * 5 / 0.5 / 1e6)


def test_reference_arm_under_torchrun_prints_once_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"


def test_secondary_lines_are_compacted_and_failures_recorded(monkeypatch):
    """The default run nests the other configurations' lines: their headline
    fields are kept, and a child that fails or prints no line is recorded as an
    error instead of failing the run."""
    import subprocess
    import types
    line = {"metric": "m", "value": 45621.0, "unit": "MLUPS", "ms_per_step": 0.37, "steps": 20, "dtype": "f16",
            "config": {"workload": "w"}, "status": 0, "e2e": {"value": 30000.0},
            "roofline": {"bound": "hbm", "frac": 0.733, "achieved": 4955.0, "peak": 6760.2, "unit": "GB/s",
                         "peak_kind": "measured", "kernel": "k", "traffic": 1.75e9,
                         "alu": {"bound": "alu", "frac": 0.4, "achieved": 1.0, "peak": 2.0, "unit": "TFLOP/s"}},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}, "passes": {"spread": 0.01}}
    c = bench.compact_line(line)
    assert c["value"] == 45621.0 and c["roofline"]["frac"] == 0.733 and c["roofline"]["alu"]["frac"] == 0.4
    assert c["e2e"] == 30000.0 and c["clocks"]["sm_mhz"] == 2070.0 and c["passes_spread"] == 0.01
    outs = iter([types.SimpleNamespace(returncode=0, stdout="log\n" + json.dumps(line) + "\n", stderr=""),
                 types.SimpleNamespace(returncode=3, stdout="", stderr="boom")])
    calls = []

    def fake_run(cmd, **kw):
        calls.append(cmd)
        try:
            return next(outs)
        except StopIteration:
            raise subprocess.TimeoutExpired(cmd, kw.get("timeout"))

    monkeypatch.setattr(bench.subprocess, "run", fake_run)
    res = bench.run_secondary(types.SimpleNamespace(steps=20, warmup=5))
    assert len(res) == len(bench.SECONDARY) == len(calls)
    assert res[0]["value"] == 45621.0 and "error" not in res[0]
    assert res[1]["error"].startswith("exit 3") and "boom" in res[1]["error"]
    assert all("error" in r for r in res[2:])
    assert all("--no-secondary" in cmd and "--no-cpu-baseline" in cmd for cmd in calls)
    assert calls[0][-2:] == ["--storage", "f16"] and "--steps" in calls[0]
    closure = {"value": 0.8, "unit": "ratio", "result": {
        "plain_coarse": {"n": 128, "steps": 512, "gpu_ms": 42.5, "status": 0, "spectrum_error": 0.99, "E": [1.0]},
        "plain_medium": {"n": 256, "steps": 1024, "gpu_ms": 555.0, "status": 0, "spectrum_error": 0.1},
        "learned": [{"omega_lo": 1.0, "omega_hi": 1.98, "gpu_ms": 76.4, "status": 0, "spectrum_error": 0.72,
                     "time_ratio_at_equal_error": 0.8, "train_loss_first": 205.9}]}}
    c = bench.compact_line(closure)
    assert c["value"] == 0.8 and c["result"]["plain_medium"]["spectrum_error"] == 0.1
    assert c["result"]["learned"][0]["time_ratio_at_equal_error"] == 0.8
    assert "E" not in c["result"]["plain_coarse"] and "train_loss_first" not in c["result"]["learned"][0]
