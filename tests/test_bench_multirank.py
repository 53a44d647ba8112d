"""The multi-rank bookkeeping of bench.py on CPU: world-size-2 gloo ranks (replicas, no data-path
collective), the max-over-ranks time and the whole-job value, the partition of the batched form's
independent systems over ranks, and the reference arm's rank-0-only output."""
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
from paper_2408_08262_gb300 import shard  # noqa: E402


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


@pytest.mark.parametrize("nparts", [1, 2, 3, 8, 70])
def test_partition_covers_every_system_once_and_balances(nparts):
    import numpy as np
    w = np.random.default_rng(nparts).integers(1, 1000, size=64).tolist()
    parts = shard.partition(w, nparts)
    assert len(parts) == nparts
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(64))
    assert all(p == sorted(p) for p in parts)
    loads = [sum(w[i] for i in p) for p in parts]
    assert max(loads) <= sum(w) / nparts + max(w)  # the greedy bound
    assert shard.partition(w, nparts) == parts     # every rank computes the same one
    if nparts == 1:
        assert parts == [list(range(64))]          # one rank keeps the systems' order


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = [(7 * i) % 13 + 1 for i in range(20)]
        mine = shard.partition(w, world)[rank]
        n = bench.sum_over_ranks(len(mine), dist, torch.device("cpu"))
        got = [None] * world
        dist.all_gather_object(got, mine)
        out.put((rank, n, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_systems_without_overlap():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for _, n, got in res:
        assert n == 20
        assert sorted(i for part in got for i in part) == list(range(20))
        assert set(got[0]).isdisjoint(got[1])


# ---- the batched form's bookkeeping with stand-ins for the library (no GPU) ----

class _Prob:
    def __init__(self, n):
        import numpy as np
        self.n = n
        self.rowptr = np.arange(n + 1, dtype=np.int32)
        self.col = np.arange(n, dtype=np.int32)
        self.val = np.ones(n)
        self.b = np.ones(n)


class _P:
    @staticmethod
    def batched_2d(nsys):
        return [_Prob(10 + 7 * (i % 5)) for i in range(nsys)]


class _H:
    def __init__(self, rp, ci, v, params):
        self.n = rp.numel() - 1

    def solve(self, b, rtol):
        return b, {"iters": 5 + self.n % 3, "status": 0}

    def close(self):
        pass


class _B:
    def __init__(self, Hs):
        self.Hs = Hs
        self.rule = os.environ.get("AIRG_NO_AUTOTUNE") == "1"

    def solve(self, bs, rtol):
        return bs, [{"iters": 6, "status": 0} for _ in bs]

    def tuned(self):
        return [] if self.rule else [(1, 2), (2, 2)]

    def close(self):
        pass


class _Ev:
    def __init__(self, enable_timing=True):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 2.0


def _setup_many(mats, params):
    return [_H(*m, params) for m in mats]


def _fakes():
    airg = types.SimpleNamespace(Hierarchy=_H, Batch=_B, setup_many=_setup_many)
    fake_torch = types.SimpleNamespace(from_numpy=torch.from_numpy,
                                       cuda=types.SimpleNamespace(synchronize=lambda *a: None, Event=_Ev))
    return airg, fake_torch


def test_batched_form_on_one_rank():
    airg, ft = _fakes()
    args = types.SimpleNamespace(rtol=1e-8)
    d = bench.batched_form(args, airg, _P, ft, torch.device("cpu"), None, None, None, 1, 0)
    assert d["systems"] == 64 and d["ranks"] == 1 and d["systems_per_rank_max"] == 64
    assert d["total_dofs"] == sum(p.n for p in _P.batched_2d(64))
    assert d["batched_solve_ms"] == 2.0 and d["sequential_solve_ms"] == 2.0
    assert d["time_to_rtol_batched_ms"] >= d["batched_solve_ms"] and d["setups_concurrent_ms"] >= 0.0
    assert d["iters_min"] == 6 and d["iters_max"] == 6 and d["all_converged"] is True
    assert d["autotuner"]["groups_tuned"] == 2 and d["autotuner"]["changed_from_rule"] == 1
    assert "AIRG_NO_AUTOTUNE" not in os.environ


def _batched_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        airg, ft = _fakes()
        args = types.SimpleNamespace(rtol=1e-8)
        d = bench.batched_form(args, airg, _P, ft, torch.device("cpu"), None, None, dist, world, rank)
        out.put((rank, d["systems"], d["total_dofs"], d["systems_per_rank_max"], d["all_converged"]))
    finally:
        dist.destroy_process_group()


def test_batched_form_shares_the_systems_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batched_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    total = sum(p.n for p in _P.batched_2d(64))
    for _, nsys, ndofs, per_rank, ok in res:
        assert nsys == 64 and ndofs == total and ok
        assert 32 <= per_rank < 64
