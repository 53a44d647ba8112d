"""The multi-rank bookkeeping of bench.py on CPU: world-size-2 gloo ranks (replicas, no data-path
collective), the max-over-ranks time and the whole-job value, and the reference arm's rank-0-only
output."""
import os
import socket
import sys
import types

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + 0.5 * rank, dist, torch.device("cpu"))
        v = bench.job_value(1000, 5, world, t)
        out.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, t, v in res:
        assert t == 1.5                        # the slower rank's time on every rank
        assert v == pytest.approx(1000 * 5 * 2 / 1.5)  # all ranks' DOFs over that time


def test_single_process_needs_no_group():
    assert bench.max_over_ranks(2.5, None, None) == 2.5
    assert bench.job_value(10, 3, 1, 2.0) == 15.0


def test_reference_arm_prints_on_rank_zero_only(capsys):
    args = types.SimpleNamespace(gpus=2, steps=1, warmup=1, mesh=1024, rtol=1e-8, cpu_sample_mesh=32)
    bench.reference_arm(args, rank=1)
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys):
    import json
    args = types.SimpleNamespace(gpus=1, steps=1, warmup=1, mesh=1024, rtol=1e-8, cpu_sample_mesh=32)
    bench.reference_arm(args, rank=0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
