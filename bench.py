"""Benchmark: AIRG-preconditioned FGMRES (setup + solve to rtol 1e-8) on one GB300 per rank.

A step is one pass of the whole path over one synthetic system: airg_setup (CF splitting, GMRES
polynomials, restrictor, coarse matrices on every level), airg_solve to rtol 1e-8, airg_free.
The workload is the 2D upwind P1 DG system on 1024 x 1024 jittered squares (6,291,456 DOFs,
sigma piecewise constant on a seeded 8 x 8 block pattern with values {0, 1, 10}, theta = 0.3).

Prints ONE JSON line (rank 0).  Under torchrun every rank runs an independent replica (a single
system does not shard without a halo exchange); value = DOFs of all ranks / max time.

--impl reference times the CPU oracle (plain single-thread FP64 restatement of the method) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "AIRG-GMRES time-to-rtol 1e-8 (DOFs/s, HBM GB/s): mixed/batched vs FP64 on GB300"
UNIT = "DOFs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="airg", choices=["airg", "reference"])
    ap.add_argument("--mesh", type=int, default=1024)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-mesh", type=int, default=320)
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and adjoint form measurements")
    ap.add_argument("--profile-vcycle", action="store_true",
                    help="profiling mode: set up and solve once, then apply one V-cycle inside the NVTX range 'vc' "
                         "(for an ncu capture of the cycle's kernels) and exit")
    ap.add_argument("--profile-setup", action="store_true",
                    help="profiling mode: one warm-up setup + solve, then one setup inside the NVTX range 'setup' "
                         "and one solve inside 'solve', and exit")
    return ap.parse_args()


def workload_name(mesh: int) -> str:
    return (f"2D upwind P1 DG, {mesh}x{mesh} jittered squares ({6 * mesh * mesh:,} DOFs), sigma on a seeded 8x8 "
            f"block pattern from {{0,1,10}}, theta=0.3, q=1; FP64 AIRG setup + FGMRES(30) solve to rtol 1e-8")


def max_over_ranks(x: float, dist, device) -> float:
    """The maximum of a per-rank float over all ranks (x itself without a process group): the
    job's time is that of its slowest rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    """The sum of a per-rank float over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_value(dofs_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the DOFs every rank solved in `steps` steps, over the slowest rank's time."""
    return dofs_per_rank * steps * world / seconds


# top-level SpMV kernels: (ncu summary, source file, the kernel's signature start)
SPMV_KERNELS = {
    "k_spmv_sell": ("k_spmv_sell_top_level_2d_p1dg_640.md", "airg_sell.cu",
                    "__global__ void __launch_bounds__(256, PROLONG ? 6 : 8) k_spmv_sell("),
    "k_spmv_row": ("k_spmv_row_top_level_2d_p1dg_640.md", "airg_prims.cu",
                   "__global__ void __launch_bounds__(256) k_spmv_row("),
}


def spmv_traffic(kernel: str = "k_spmv_sell"):
    """DRAM bytes per top-level SpMV launch from the committed ncu summary, or None when the kernel
    source has changed since that capture (the summary records a hash of the kernel's source)."""
    import hashlib
    prof_name, src_name, sig = SPMV_KERNELS[kernel]
    prof = os.path.join(ROOT, "profiles", prof_name)
    src = os.path.join(ROOT, "paper_2408_08262_gb300", "csrc", src_name)
    try:
        txt = open(prof).read()
        code = open(src).read()
        a = code.index(sig)
        b = code.index("\n}\n", a) + 3
        h = hashlib.sha256(code[a:b].encode()).hexdigest()[:16]
        vals = dict(line.split(": ", 1) for line in txt.splitlines() if ": " in line and line.split(": ")[0].strip().isidentifier())
        if vals.get(f"{kernel}_source_sha256_16", "").strip() != h:
            return None
        return float(vals["traffic_bytes_per_launch_1024"])
    except Exception:
        return None


def family_traffic(n_top: int, n_vc: int):
    """DRAM bytes per launch unit of the SpMV family (V-cycle applications and top-level A z) from the
    committed ncu summary, or None when a source file of the SpMV kernels has changed since the
    capture (the summary records a hash of each file)."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "vcycle_spmv_family_2d_p1dg_640.md")
    try:
        txt = open(prof).read()
        vals = dict(line.split(": ", 1) for line in txt.splitlines()
                    if ": " in line and line.split(": ")[0].strip().isidentifier())
        for name in ("airg_prims.cu", "airg_sell.cu"):
            code = open(os.path.join(ROOT, "paper_2408_08262_gb300", "csrc", name)).read()
            key = name.replace(".", "_") + "_sha256_16"
            if vals.get(key, "").strip() != hashlib.sha256(code.encode()).hexdigest()[:16]:
                return None
        t_vc = float(vals["traffic_bytes_per_vcycle_1024"])
        t_top = float(vals["traffic_bytes_per_top_spmv_1024"])
        return (t_vc * n_vc + t_top * n_top) / max(1, n_vc + n_top)
    except Exception:
        return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons, samples = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            samples += 1
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": samples}


def run_oracle_sample(mesh: int, rtol: float):
    """One oracle step (setup + solve) on a mesh x mesh instance of the workload; returns (dofs, seconds)."""
    from oracle import oracle as O
    from paper_2408_08262_gb300 import problems as P
    p = P.blocked_sigma_2d(mesh)
    t0 = time.perf_counter()
    H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params())
    x, info = H.solve(p.b, rtol=rtol)
    dt = time.perf_counter() - t0
    return p.n, dt, info


def cpu_baselines(args, p) -> dict:
    """The oracle timed on the host cores on the benchmarked system itself: once on one thread, once
    with its SpMV row loop on every core this process may run on (setup otherwise serial; results
    bitwise those of one thread).  Setup and solve are timed separately."""
    from oracle import oracle as O
    O.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    runs = {}
    for t in (1, cores):
        O.set_threads(t)
        t0 = time.perf_counter()
        H = O.Hierarchy(p.rowptr, p.col, p.val, O.Params())
        t1 = time.perf_counter()
        x, info = H.solve(p.b, rtol=args.rtol)
        t2 = time.perf_counter()
        del H
        runs[t] = (t1 - t0, t2 - t1, info)
    O.set_threads(1)
    su, so, info = runs[cores]
    s1, o1, info1 = runs[1]
    return {"value": p.n / (su + so), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one oracle setup + solve to rtol {args.rtol:g} of the benchmarked {args.mesh}x{args.mesh} "
                      f"system ({p.n:,} DOFs); SpMV row loops on {cores} threads, the rest of setup serial: "
                      f"setup {su:.1f} s, solve {so:.2f} s, {info['iters']} iterations",
            "single_thread": {"value": p.n / (s1 + o1), "unit": UNIT, "cores": 1, "setup_s": round(s1, 2),
                              "solve_s": round(o1, 2), "iters": info1["iters"]}}


def reference_arm(args, rank):
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    mesh = args.cpu_sample_mesh
    for _ in range(args.warmup if args.warmup < 1 else 1):
        run_oracle_sample(max(32, mesh // 4), args.rtol)
    tot_dofs, tot_t = 0, 0.0
    for _ in range(args.steps):
        n, dt, info = run_oracle_sample(mesh, args.rtol)
        tot_dofs += n
        tot_t += dt
    value = tot_dofs / tot_t
    sample = (f"oracle setup+solve of the same generator at {mesh}x{mesh} ({6 * mesh * mesh:,} DOFs) per step, "
              f"single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.mesh), "sample_mesh": mesh},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_form(args, airg, P, torch, dev, stream, params, dist, world: int, rank: int) -> dict:
    """The batched form: 64 independent systems of uneven size, grouped kernels and one V-cycle
    graph, against the same systems solved one after another (same hierarchies).  Under torchrun
    the systems are partitioned over the ranks by nonzero count (no data exchange: each rank solves
    its share) and the times are the slowest rank's."""
    from paper_2408_08262_gb300 import shard
    systems_all = P.batched_2d(64)
    mine = shard.partition([len(q.col) for q in systems_all], world)[rank]
    systems = [systems_all[i] for i in mine]
    infos, its_seq, tuned = [], [], []
    tb = ts = tr = 0.0
    tsu = tcr = tsm = 0.0
    if systems:
        mats = [tuple(torch.from_numpy(a).to(dev) for a in (q.rowptr, q.col, q.val)) for q in systems]
        bs = [torch.from_numpy(q.b).to(dev) for q in systems]
        for m in mats[:2]:  # warm-up of the setup path
            airg.Hierarchy(*m, params).close()
        for H in airg.setup_many(mats[:8], params):
            H.close()
        # the batched form's setups: all systems concurrently (airg_setup_many)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Hm = airg.setup_many(mats, params)
        torch.cuda.synchronize(dev)
        tsm = 1e3 * (time.perf_counter() - t0)
        for H in Hm:
            H.close()
        del Hm
        # the same setups one after another (the plain form)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Hs = [airg.Hierarchy(*m, params) for m in mats]
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        Bt = airg.Batch(Hs)
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        tsu, tcr = 1e3 * (t1 - t0), 1e3 * (t2 - t1)
        Bt.solve(bs, rtol=args.rtol)
        for H, bq in zip(Hs, bs):
            H.solve(bq, rtol=args.rtol)
        torch.cuda.synchronize(dev)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        xs, infos = Bt.solve(bs, rtol=args.rtol)
        e1.record(stream)
        for H, bq in zip(Hs, bs):
            _, ii = H.solve(bq, rtol=args.rtol)
            its_seq.append(ii["iters"])
        e2.record(stream)
        torch.cuda.synchronize(dev)
        tb, ts = e0.elapsed_time(e1), e1.elapsed_time(e2)
        # the SpMV autotuner's choices, and the batched solve with the row-length rule alone
        tuned = Bt.tuned()
        Bt.close()
        os.environ["AIRG_NO_AUTOTUNE"] = "1"
        try:
            Br = airg.Batch(Hs)
        finally:
            del os.environ["AIRG_NO_AUTOTUNE"]
        Br.solve(bs, rtol=args.rtol)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        Br.solve(bs, rtol=args.rtol)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        tr = e0.elapsed_time(e1)
        Br.close()
        del Hs
    tb = max_over_ranks(tb, dist, dev)
    ts = max_over_ranks(ts, dist, dev)
    tsu = max_over_ranks(tsu, dist, dev)
    tcr = max_over_ranks(tcr, dist, dev)
    tsm = max_over_ranks(tsm, dist, dev)
    tr = max_over_ranks(tr, dist, dev)
    ndofs = int(sum_over_ranks(sum(q.n for q in systems), dist, dev))
    nsys = int(sum_over_ranks(len(systems), dist, dev))
    it_min = -max_over_ranks(-min((i["iters"] for i in infos), default=10 ** 9), dist, dev)
    it_max = max_over_ranks(max((i["iters"] for i in infos), default=0), dist, dev)
    it_seq = max_over_ranks(max(its_seq, default=0), dist, dev)
    failed = max_over_ranks(float(any(i["status"] != 0 for i in infos)), dist, dev)
    batched = {"workload": "64 P1 DG systems, n x n with n drawn from {64,128,256,512}, theta ~ U[0,2pi), "
                           "sigma ~ U[0,5]", "systems": nsys, "total_dofs": ndofs, "ranks": world,
               "systems_per_rank_max": int(max_over_ranks(len(systems), dist, dev)),
               "batched_solve_ms": round(tb, 2), "sequential_solve_ms": round(ts, 2),
               "speedup_vs_sequential": round(ts / tb, 3), "batched_dofs_per_s": ndofs / (tb / 1e3),
               "setups_concurrent_ms": round(tsm, 2), "setups_sequential_ms": round(tsu, 2),
               "batch_create_and_autotune_ms": round(tcr, 2),
               "time_to_rtol_batched_ms": round(tsm + tcr + tb, 2), "time_to_rtol_sequential_ms": round(tsu + ts, 2),
               "time_to_rtol_speedup_vs_sequential": round((tsu + ts) / max(tsm + tcr + tb, 1e-9), 3),
               "iters_min": int(it_min), "iters_max": int(it_max), "all_converged": failed == 0.0,
               "iters_sequential_max": int(it_seq)}
    batched["autotuner"] = {"groups_tuned": len(tuned), "changed_from_rule": sum(r != c for r, c in tuned),
                            "rule_vs_chosen_lanes": tuned, "batched_solve_ms_rule_lanes": round(tr, 2),
                            "note": "choices of rank 0" if world > 1 else "one rank"}
    return batched


def mixed_forms_3d(args, airg, P, torch, dev, stream, mesh: int = 128) -> dict:
    """The mixed-precision form on its own configuration: 3D upwind P0 DG on mesh^3 cubes of six
    Kuhn tetrahedra (12,582,912 DOFs at 128), FP64 against the FP32 and bf16-value V-cycles, each
    set up and solved to rtol 1e-8 (time-to-rtol = setup + solve), with the per-class SpMV rates
    of one profiled solve and the error against the FP64 GPU solution."""
    import numpy as np
    p3 = P.kuhn_3d(mesh)
    rp3, ci3, v3, b3 = (torch.from_numpy(a).to(dev) for a in (p3.rowptr, p3.col, p3.val, p3.b))
    out = {"workload": f"3D upwind P0 DG, {mesh}^3 cubes x 6 jittered Kuhn tets ({p3.n:,} DOFs, {p3.nnz:,} nnz), "
                       "Omega=(0.48,0.60,0.64), sigma in {0,0.01} by a seeded half-space; setup + FGMRES(30) "
                       "to rtol 1e-8"}
    x64 = None
    for name, prec in (("fp64", 0), ("fp32", 1), ("bf16_values", 2)):
        par = airg.Params(precision=prec)
        Hw = airg.Hierarchy(rp3, ci3, v3, par)
        Hw.solve(b3, rtol=args.rtol, restart=args.restart)
        Hw.close()
        su, so, its = [], [], []
        for _ in range(2):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            Hf = airg.Hierarchy(rp3, ci3, v3, par)
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            xf, inf = Hf.solve(b3, rtol=args.rtol, restart=args.restart)
            t2 = time.perf_counter()
            su.append(1e3 * (t1 - t0))
            so.append(1e3 * (t2 - t1))
            its.append(inf["iters"])
            if _ == 0:
                lvi = Hf.level_info(-1)
                Hf.profile()
                Hf.solve(b3, rtol=args.rtol, restart=args.restart)
                kt = Hf.kernel_times()
            Hf.close()
        ent = {"setup_ms": round(min(su), 2), "solve_ms": round(min(so), 2),
               "time_to_rtol_ms": round(min(su) + min(so), 2), "iters": max(its), "relres": inf["relres"],
               "levels": lvi["levels"], "operator_complexity": round(lvi["operator"], 3),
               "dofs_per_s": p3.n / ((min(su) + min(so)) / 1e3),
               "solve_spmv_GBps": {c: round(kt[c]["bytes"] / max(kt[c]["ms"], 1e-9) / 1e6, 1)
                                   for c in ("smooth_resid", "smooth_update", "restrict", "top_op", "coarsest")}}
        xh = xf.double()
        if prec == 0:
            x64 = xh
        else:
            ent["rel_err_vs_fp64_gpu"] = float(torch.linalg.norm(xh - x64) / torch.linalg.norm(x64))
            ent["solve_speedup_vs_fp64"] = round(out["fp64"]["solve_ms"] / ent["solve_ms"], 3)
            ent["time_to_rtol_speedup_vs_fp64"] = round(out["fp64"]["time_to_rtol_ms"] / ent["time_to_rtol_ms"], 3)
        out[name] = ent
    del rp3, ci3, v3, b3
    return out


def profile_ranges(args, airg, torch, rp, ci, v, b, params, dev):
    """Profiling modes (no bench line): NVTX ranges around one setup and one solve, or around one
    V-cycle, after a warm-up setup + solve, so that an ncu capture can select them."""
    H = airg.Hierarchy(rp, ci, v, params)
    H.solve(b, rtol=args.rtol, restart=args.restart)
    torch.cuda.synchronize(dev)
    if args.profile_vcycle:
        H.vcycle(b)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_push("vc")
        H.vcycle(b)
        torch.cuda.synchronize(dev)
        torch.cuda.nvtx.range_pop()
        H.close()
        return
    H.close()
    torch.cuda.nvtx.range_push("setup")
    H = airg.Hierarchy(rp, ci, v, params)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("solve")
    H.solve(b, rtol=args.rtol, restart=args.restart)
    torch.cuda.synchronize(dev)
    torch.cuda.nvtx.range_pop()
    H.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2408_08262_gb300 import build as B
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_2408_08262_gb300 import airg
    from paper_2408_08262_gb300 import problems as P

    p = P.blocked_sigma_2d(args.mesh)
    rp_h = torch.from_numpy(p.rowptr).pin_memory()
    ci_h = torch.from_numpy(p.col).pin_memory()
    v_h = torch.from_numpy(p.val).pin_memory()
    b_h = torch.from_numpy(p.b).pin_memory()
    rp, ci, v, b = (t.to(dev) for t in (rp_h, ci_h, v_h, b_h))
    stream = torch.cuda.current_stream(dev)
    params = airg.Params()
    classes = airg.PROFILE_CLASSES
    if args.profile_vcycle or args.profile_setup:
        profile_ranges(args, airg, torch, rp, ci, v, b, params, dev)
        return

    def step(profile=False):
        H = airg.Hierarchy(rp, ci, v, params)
        if profile:
            H.profile()
            torch.cuda.nvtx.range_push("airg_solve")
        x, info = H.solve(b, rtol=args.rtol, restart=args.restart)
        if profile:
            torch.cuda.nvtx.range_pop()
        kt = H.kernel_times() if profile else None
        lv = H.level_info(-1)
        H.close()
        return info, kt, lv

    # warm-up; the first warm-up step times every kernel class (reported per class in config)
    info0, kt0, lv0 = step(profile=True)
    for _ in range(max(0, args.warmup - 1)):
        step()
    # The roofline kernel is the SpMV (k_spmv_sell on the large short-row operators, k_spmv_row /
    # k_spmv_vec on the others), the dominant kernel family of the step.  In the
    # timed region its top-level-operator launches (the largest instance, 6.29M rows) are timed
    # with CUDA events; timing every small-level launch inside the V-cycle graph would itself slow
    # the solve.  The warm-up step times every class and is reported in config.
    spmv_classes = ["top_op", "vcycle"]
    all_spmv = ["smooth_resid", "smooth_update", "restrict", "top_op", "coarsest"]

    # timed region: K steps on the device, the SpMV kernel timed with CUDA events
    clk = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk.start()
    launches0 = airg.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dom = {"launches": 0, "ms": 0.0, "bytes": 0.0}  # keys of the per-class sums
    per_class = {c: {"launches": 0, "ms": 0.0, "bytes": 0.0} for c in spmv_classes}
    solve_ms, setup_ms, iters = [], [], []
    ev0.record(stream)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        H = airg.Hierarchy(rp, ci, v, params)
        t1 = time.perf_counter()
        H.profile(spmv_classes)
        x, info = H.solve(b, rtol=args.rtol, restart=args.restart)
        t2 = time.perf_counter()
        kts = H.kernel_times()
        H.close()
        for c in spmv_classes:
            for k in dom:
                per_class[c][k] += kts[c][k]
        setup_ms.append(1e3 * (t1 - t0))
        solve_ms.append(1e3 * (t2 - t1))
        iters.append(info["iters"])
        if info["status"] != 0:
            raise RuntimeError(f"solve did not converge: {info}")
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    launches = airg.launch_count() - launches0
    clocks = clk.stop()
    t_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    value = job_value(p.n, args.steps, world, t_ms / 1e3)

    # end to end through the public API with host buffers: the library copies the matrix
    # (airg_setup_host) and the rhs (airg_solve_host) in from pinned host memory and the solution
    # back, inside the timed region
    x_h = torch.zeros(p.n, dtype=torch.float64).pin_memory()
    h2d = rp_h.numel() * 4 + ci_h.numel() * 4 + v_h.numel() * 8 + b_h.numel() * 8
    d2h = x_h.numel() * 8
    torch.cuda.synchronize(dev)
    e0 = time.perf_counter()
    for _ in range(args.steps):
        H = airg.Hierarchy(rp_h, ci_h, v_h, params, host=True)
        H.solve_host(b_h, x_h, rtol=args.rtol, restart=args.restart)
        H.close()
    torch.cuda.synchronize(dev)
    e_s = max_over_ranks(time.perf_counter() - e0, dist, dev)
    e2e = job_value(p.n, args.steps, world, e_s)

    peak, peak_kind = peaks()
    # The SpMV family as a whole: every V-cycle application (its SpMVs on all levels, timed by one
    # event pair around each graph replay, gaps between its kernels included) and every top-level
    # A z, over the K timed steps.  The top-level launches alone are reported beside it.
    top, vc = per_class["top_op"], per_class["vcycle"]
    agg_bytes, agg_ms = top["bytes"] + vc["bytes"], top["ms"] + vc["ms"]
    achieved = agg_bytes / (agg_ms / 1e3) / 1e9 if agg_ms > 0 else None
    top_ach = top["bytes"] / (top["ms"] / 1e3) / 1e9 if top["ms"] > 0 else None
    fam_bytes = sum(kt0[c]["bytes"] for c in all_spmv)
    fam_ms = sum(kt0[c]["ms"] for c in all_spmv)
    top_kernel = "k_spmv_sell" if lv0.get("top_sell") else "k_spmv_row"
    label = {"k_spmv_sell": "k_spmv_sell (sliced ELL SpMV, one warp per 32-row slice)",
             "k_spmv_row": "k_spmv_row (row-per-thread CSR SpMV)"}[top_kernel]
    units = top["launches"] + vc["launches"]
    roofline = {"bound": "hbm",
                "kernel": "SpMV family of the solve (k_spmv_sell / k_spmv_row / k_spmv_vec): every SpMV of every "
                          f"V-cycle on all {lv0['levels']} levels plus the top-level A z of each FGMRES iteration",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_source": peak_kind,
                "traffic": family_traffic(top["launches"], vc["launches"]) if args.mesh == 1024 else None,
                "traffic_note": "DRAM bytes of the same kernels from one-pass ncu launch lists on the 640x640 case, "
                                "scaled to 1024x1024 by the algorithmic bytes, per launch unit",
                "algorithmic_bytes_per_launch": agg_bytes / max(1, units),
                "launch_unit": "one V-cycle application or one top-level A z (event pairs outside the V-cycle graph; "
                               "gaps between the cycle's kernels count as SpMV time)",
                "launches": units, "avg_launch_us": 1e3 * agg_ms / max(1, units),
                "vcycle": {"applications": vc["launches"], "ms": round(vc["ms"], 3),
                           "GBps": vc["bytes"] / max(vc["ms"], 1e-9) / 1e6,
                           "algorithmic_bytes_per_application": vc["bytes"] / max(1, vc["launches"])},
                "top_level_spmv": {"kernel": f"{label}, A z in FGMRES ({p.n / 1e6:.2f}M rows)",
                                   "achieved": top_ach, "frac": (top_ach / peak) if top_ach else None,
                                   "launches": top["launches"],
                                   "avg_launch_us": 1e3 * top["ms"] / max(1, top["launches"]),
                                   "algorithmic_bytes_per_launch": top["bytes"] / max(1, top["launches"]),
                                   "traffic": (spmv_traffic(top_kernel) if args.mesh == 1024 else None),
                                   "traffic_note": "ncu capture of the same kernel on the 640x640 case scaled by "
                                                   "the algorithmic bytes"},
                "per_class_first_step": {"achieved": fam_bytes / max(fam_ms, 1e-9) / 1e6,
                                         "frac": fam_bytes / max(fam_ms, 1e-9) / 1e6 / peak,
                                         "note": "every solve-phase SpMV launch timed on its own (first warm-up "
                                                 "step; the events inside the graph slow it)"}}

    # the mixed-precision form on the same system: V-cycle in FP32 / bf16 values, FP64 outer loop
    forms = {}
    for name, prec in (("fp32", 1), ("bf16_values", 2)):
        par = airg.Params(precision=prec)
        Hw = airg.Hierarchy(rp, ci, v, par)
        Hw.solve(b, rtol=args.rtol, restart=args.restart)
        Hw.close()
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        su, so, its = [], [], []
        f0.record(stream)
        for _ in range(2):
            t0 = time.perf_counter()
            Hf = airg.Hierarchy(rp, ci, v, par)
            t1 = time.perf_counter()
            xf, inf = Hf.solve(b, rtol=args.rtol, restart=args.restart)
            t2 = time.perf_counter()
            Hf.close()
            su.append(1e3 * (t1 - t0))
            so.append(1e3 * (t2 - t1))
            its.append(inf["iters"])
        f1.record(stream)
        torch.cuda.synchronize(dev)
        ms = f0.elapsed_time(f1) / 2
        forms[name] = {"ms_per_step": round(ms, 2), "setup_ms": round(min(su), 2), "solve_ms": round(min(so), 2),
                       "iters": max(its), "relres": inf["relres"], "dofs_per_s": p.n / (ms / 1e3),
                       "solve_speedup_vs_fp64": round(min(solve_ms) / min(so), 3)}

    # parameter variants the paper sweeps: GMRES-polynomial order 1..6 with first-order fixed
    # sparsity (the paper's table of orders 1-6), orders 2, 3, 6 with second-order sparsity, orders 3
    # and 6 with every polynomial applied matrix-free, and order 6 with the approximate ideal
    # prolongator; same system, setup and solve to the same rtol
    poly_sweep = None
    if not args.no_forms:
        poly_sweep = {}
        variants = ([(d, 1, 0, 0) for d in range(1, 7)] + [(2, 2, 0, 0), (3, 2, 0, 0), (6, 2, 0, 0)] +
                    [(3, 1, 1, 0), (6, 1, 1, 0), (6, 1, 0, 1)])
        for d, so, mf, ip in variants:
            par = airg.Params(poly_order=d, sparsity_order=so, matrix_free=mf, ideal_prolong=ip)
            Hw = airg.Hierarchy(rp, ci, v, par)
            Hw.solve(b, rtol=args.rtol, restart=args.restart)
            Hw.close()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            Hd = airg.Hierarchy(rp, ci, v, par)
            t1 = time.perf_counter()
            xd, ind = Hd.solve(b, rtol=args.rtol, restart=args.restart)
            torch.cuda.synchronize(dev)
            t2 = time.perf_counter()
            Hd.close()
            key = (f"{d}_matrix_free" if mf else f"{d}_ideal_prolong" if ip else
                   str(d) if so == 1 else f"{d}_second_order_sparsity")
            poly_sweep[key] = {
                "setup_ms": round(1e3 * (t1 - t0), 2), "solve_ms": round(1e3 * (t2 - t1), 2),
                "iters": ind["iters"], "status": ind["status"]}

    # setup re-use: four energy groups of one 512x512 mesh and direction, and four directions of one
    # 512x512 unjittered mesh inside one 45-degree sector (same upwind pattern); members 1-3 set up
    # fresh and with member 0's splittings on every level, each then solved to the same rtol
    reuse = None
    if not args.no_forms:
        reuse = {"reused_levels": "all (the template member's splitting on every level)"}
        for name, members, wl in (
                ("energy_groups", P.groups_2d(512, ngroups=4),
                 "4 energy groups of a 512x512 P1 DG mesh (1,572,864 DOFs each), one direction; sigma block values "
                 "scaled by 0.1 * 4^g"),
                ("directions", P.directions_2d(512),
                 "4 directions (theta 0.15, 0.35, 0.55, 0.75) of one unjittered 512x512 P1 DG mesh (1,572,864 DOFs "
                 "each), same upwind pattern; sigma = 1")):
            gd = [tuple(torch.from_numpy(a).to(dev) for a in (g.rowptr, g.col, g.val, g.b)) for g in members]
            T = airg.Hierarchy(*gd[0][:3], params)
            rows = {"fresh": [], "reuse": []}
            for rep in range(2):  # the first pass warms up
                for q in range(1, 4):
                    for kind in ("fresh", "reuse"):
                        torch.cuda.synchronize(dev)
                        t0 = time.perf_counter()
                        Hq = airg.Hierarchy(*gd[q][:3], params, reuse=T if kind == "reuse" else None)
                        torch.cuda.synchronize(dev)
                        t1 = time.perf_counter()
                        _, iq = Hq.solve(gd[q][3], rtol=args.rtol, restart=args.restart)
                        torch.cuda.synchronize(dev)
                        t2 = time.perf_counter()
                        Hq.close()
                        if rep == 1:
                            rows[kind].append((1e3 * (t1 - t0), 1e3 * (t2 - t1), iq["iters"], iq["status"]))
            T.close()
            ent = {"workload": wl}
            for kind, r in rows.items():
                ent[kind] = {"setup_ms": [round(x[0], 2) for x in r], "solve_ms": [round(x[1], 2) for x in r],
                             "iters": [x[2] for x in r], "all_converged": all(x[3] == 0 for x in r)}
            ent["setup_speedup"] = round(sum(x[0] for x in rows["fresh"]) / sum(x[0] for x in rows["reuse"]), 3)
            ent["time_to_rtol_speedup"] = round(sum(x[0] + x[1] for x in rows["fresh"]) /
                                                sum(x[0] + x[1] for x in rows["reuse"]), 3)
            reuse[name] = ent

    # diagnostics of the splitting on every level of the 128x128 system: theta over the F-points
    # after PMISR alone and after DDC (airg_ddc_theta on the GPU; histogram on [0, 1.5)), and the
    # condition number of A_ff on levels small enough for a dense SVD on the host
    diag = None
    if not args.no_forms:
        pd = P.blocked_sigma_2d(128)
        Hd = airg.Hierarchy(*(torch.from_numpy(a).to(dev) for a in (pd.rowptr, pd.col, pd.val)),
                            airg.Params(keep_setup=1))
        diag = {"workload": "2D upwind P1 DG, 128x128 (98,304 DOFs), same generator as the main line",
                "levels": []}
        for l in range(Hd.num_levels - 1):
            lrp, lci, lv = Hd.export(l, "A")
            Ad = [torch.from_numpy(a).to(dev) for a in (lrp, lci, lv)]
            cf_after = torch.from_numpy(Hd.vectors(l)["cf"]).to(dev)
            cf_before = airg.cf_split(*Ad, airg.Params(ddc_fraction=0.0), level=l)
            row = {"level": l, "n": int(lrp.size - 1)}
            for tag, cf in (("pmisr", cf_before), ("pmisr_ddc", cf_after)):
                th = airg.ddc_theta(*Ad, cf).cpu().numpy()
                F = np.flatnonzero(cf.cpu().numpy() == 1)
                h, _ = np.histogram(th[F], bins=10, range=(0.0, 1.5))
                ent = {"n_f": int(F.size), "theta_max": round(float(th[F].max()), 4) if F.size else 0.0,
                       "theta_hist_0_1.5": h.tolist()}
                if 0 < F.size <= 4000:
                    M = np.zeros((lrp.size - 1, lrp.size - 1))
                    M[np.repeat(np.arange(lrp.size - 1), np.diff(lrp)), lci] = lv
                    sv = np.linalg.svd(M[np.ix_(F, F)], compute_uv=False)
                    ent["cond_aff"] = round(float(sv[0] / sv[-1]), 3)
                row[tag] = ent
            diag["levels"].append(row)
        Hd.close()

    # the mixed-precision form on its own configuration (3D P0, 128^3)
    forms3d = None
    if not args.no_forms:
        forms3d = mixed_forms_3d(args, airg, P, torch, dev, stream)

    # batched form (see batched_form); the adjoint form follows
    batched, adjoint = None, None
    if not args.no_forms:
        batched = batched_form(args, airg, P, torch, dev, stream, params, dist, world, rank)
        # adjoint form: J = w . u on 256 x 256 (393,216 DOFs) with per-element sigma; forward solve
        # and backward (A^T hierarchy + adjoint solve + SDDMM) through the autograd Function
        qa = P.adjoint_2d(256)
        val0, pos, coef, area = P.sigma_q_maps(qa)
        rpa, cia = (torch.from_numpy(a).to(dev) for a in (qa.rowptr, qa.col))
        pos_t, coef_t = torch.from_numpy(pos.ravel()).to(dev), torch.from_numpy(coef).to(dev)
        val0_t, area_t = torch.from_numpy(val0).to(dev), torch.from_numpy(area).to(dev)
        wq = torch.from_numpy(np.random.default_rng(240808266).standard_normal(qa.n)).to(dev)
        Fn = airg.solve_fn()

        def fwd_bwd():
            sg = torch.from_numpy(qa.meta["sigma_e"].copy()).to(dev).requires_grad_(True)
            qq = torch.ones(qa.meta["n_tri"], dtype=torch.float64, device=dev, requires_grad=True)
            val = val0_t.index_add(0, pos_t, (sg[:, None] * coef_t).reshape(-1))
            bb = torch.repeat_interleave(qq * area_t / 3.0, 3)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a2 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            xx = Fn.apply(rpa, cia, val, bb, params, args.rtol)
            J = (wq * xx).sum()
            a1.record(stream)
            J.backward()
            a2.record(stream)
            torch.cuda.synchronize(dev)
            return a0.elapsed_time(a1), a1.elapsed_time(a2)

        fwd_bwd()
        f_ms, b_ms = fwd_bwd()
        # re-use: the source q changes, the matrix does not (an optimisation over q); the cache keeps
        # the hierarchies of A and A^T, so forward and backward are solves only
        cache = airg.HierarchyCache()
        Fc = airg.solve_fn(cache)
        sg0 = torch.from_numpy(qa.meta["sigma_e"].copy()).to(dev)
        val_fixed = val0_t.index_add(0, pos_t, (sg0[:, None] * coef_t).reshape(-1))

        def fwd_bwd_q(qscale):
            qq = (qscale * torch.ones(qa.meta["n_tri"], dtype=torch.float64, device=dev)).requires_grad_(True)
            bb = torch.repeat_interleave(qq * area_t / 3.0, 3)
            a0, a1, a2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a0.record(stream)
            xx = Fc.apply(rpa, cia, val_fixed, bb, params, args.rtol)
            J = (wq * xx).sum()
            a1.record(stream)
            J.backward()
            a2.record(stream)
            torch.cuda.synchronize(dev)
            return a0.elapsed_time(a1), a1.elapsed_time(a2)

        fwd_bwd_q(1.0)  # builds the two hierarchies
        fq, bq = fwd_bwd_q(1.5)
        cache.clear()
        # plain FP64 AIRG on the same system: two setup + solve to the same rtol (what a forward and
        # a backward solve cost without the adjoint form)
        bpl = torch.repeat_interleave(torch.ones(qa.meta["n_tri"], dtype=torch.float64, device=dev) * area_t / 3.0, 3)
        Hp = airg.Hierarchy(rpa, cia, val_fixed, params)
        Hp.solve(bpl, rtol=args.rtol)
        Hp.close()
        torch.cuda.synchronize(dev)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(2):
            Hp = airg.Hierarchy(rpa, cia, val_fixed, params)
            _, ipl = Hp.solve(bpl, rtol=args.rtol)
            Hp.close()
        p1.record(stream)
        torch.cuda.synchronize(dev)
        plain2 = p0.elapsed_time(p1)
        adjoint = {"workload": "256x256 P1 DG (393,216 DOFs), theta 1.1, sigma_e ~ U[0,2], J = w.u; rtol "
                               f"{args.rtol:g}",
                   "forward_ms": round(f_ms, 2), "backward_ms": round(b_ms, 2),
                   "backward_over_forward": round(b_ms / f_ms, 3),
                   "cached_forward_ms": round(fq, 2), "cached_backward_ms": round(bq, 2),
                   "two_plain_fp64_setup_solve_ms": round(plain2, 2),
                   "fresh_forward_backward_vs_two_plain": round(plain2 / (f_ms + b_ms), 3),
                   "cached_forward_backward_vs_two_plain": round(plain2 / (fq + bq), 3),
                   "note": "fresh: both hierarchies set up inside the call (sigma changes); cached: the source q "
                           "changes, the hierarchies of A and A^T are re-used"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baselines(args, p)

    if rank == 0:
        med = lambda a: sorted(a)[len(a) // 2]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args.mesh), "n": p.n, "nnz": p.nnz,
                           "levels": lv0["levels"], "grid_complexity": round(lv0["grid"], 3),
                           "operator_complexity": round(lv0["operator"], 3), "iters": med(iters),
                           "setup_ms": round(med(setup_ms), 2), "solve_ms": round(med(solve_ms), 2),
                           "setup_phase_ms": {k: round(v, 2) for k, v in lv0["phase_ms"].items()},
                           "solve_kernels_first_step": {c: {"launches": kt0[c]["launches"], "ms": round(kt0[c]["ms"], 3),
                                                            "GBps": round(kt0[c]["bytes"] / max(kt0[c]["ms"], 1e-9) / 1e6, 1)}
                                                        for c in classes},
                           "solve_only_dofs_per_s": p.n / (med(solve_ms) / 1e3),
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                           "l2": "inputs larger than L2 (CSR alone %.0f MB)" % ((p.nnz * 12 + p.n * 4) / 1e6)},
                "roofline": roofline, "cpu_baseline": cpu, "mixed_precision_forms": forms,
                "mixed_precision_forms_3d": forms3d,
                "batched_form": batched, "adjoint_form": adjoint, "poly_order_sweep": poly_sweep,
                "setup_reuse_form": reuse, "splitting_diagnostics": diag,
                "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
