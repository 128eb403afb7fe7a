"""Benchmark of the Newton power-flow hot path on one GB300 (or N replicas).

A step is one converged Newton power-flow solve of the seeded 10,000-bus
synthetic transmission grid (average degree 2.7, 20% PV buses) with Newton-
Raphson, FP32 sparse-LU refactorisation and FP64 mismatch / refinement /
update, to a mismatch of 1e-8 pu.  Every step solves a different seeded load
scenario that is resident in HBM before the timed region; L2 is flushed
between timed steps (the working set of one solve fits in L2).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged solves/sec at 1e-8 pu mismatch"
WORKLOAD = "mesh10000 single-phase Newton-Raphson, FP32 LU + FP64 refinement"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes_per_iteration(st, refine=1, s_f=4):
    """Minimum bytes one mixed-precision NR iteration moves (single phase).

    mismatch: Ybus values + indices, row pointers, V, specified S, mismatch;
    assembly: Jacobian values written once; factor: L+U values read and
    written once; each triangular solve pass: L+U values + 3 vectors; each
    refinement: Ybus + V + step for J dx, L+U again, 4 FP64 vectors; update:
    |V|, angle, V.
    """
    n, nnz_y, N = st["n_bus"], st["nnz_y"], st["n_unknowns"]
    nnz_lu = st["nnz_lu"] * 4  # scalar values of the 2x2 blocks
    nnz_j = (nnz_y - n) * 4 + n * 4  # Jacobian values on the Ybus pattern
    a1 = nnz_y * (16 + 4) + 4 * (n + 1) + n * (16 + 16 + 16)
    a2 = nnz_j * s_f
    fac = nnz_lu * 2 * s_f
    solve = nnz_lu * s_f + 3 * N * s_f
    ref = nnz_y * (16 + 4) + n * 16 * 2 + nnz_lu * s_f + 4 * N * 8
    upd = n * (16 + 16 + 8)
    return a1 + a2 + fac + solve * (1 + refine) + ref * refine + upd


def make_workload(K):
    from paper_1711_10579_gb300 import cases

    case = cases.case_10000bus(0)
    pl, ql, pg = cases.scenario_loads(case, K, seed=2024, sigma=0.05)
    return case, pl, ql, pg


def run_reference(args, rank, world):
    """The FP64 CPU oracle, timed on host cores on the same workload."""
    if rank != 0:
        return
    from oracle import pf_oracle as O

    case, pl, ql, pg = make_workload(args.warmup + args.steps)
    Y = O.ybus_single(case)
    times, iters = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = O.newton_polar(case.with_loads(pl[k], ql[k], pg[k]), Y=Y)
        dt = time.perf_counter() - t0
        assert r["converged"]
        if k >= args.warmup:
            times.append(dt)
            iters.append(r["iterations"])
    tot = sum(times)
    val = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (oracle: FP64 polar NR, SuperLU/COLAMD)",
                   "n_bus": case.n_bus, "n_branch": case.n_branch},
        "ms_per_newton_iter": 1e3 * tot / sum(iters),
        "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} solves of the 10,000-bus grid, one thread"},
        "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(seconds=12.0):
    """The oracle as it stands on a bounded sample of the same workload."""
    from oracle import pf_oracle as O

    case, pl, ql, pg = make_workload(64)
    Y = O.ybus_single(case)
    t0 = time.perf_counter()
    k = 0
    while k < 64 and (time.perf_counter() - t0) < seconds:
        r = O.newton_polar(case.with_loads(pl[k], ql[k], pg[k]), Y=Y)
        assert r["converged"]
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} solves of the 10,000-bus grid in {dt:.1f} s, one thread"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    __graft_entry__.build()
    from paper_1711_10579_gb300 import pf

    K, W = args.steps, args.warmup
    case, pl, ql, pg = make_workload(W + K)
    ctx = pf.pf_ctx_create(local)
    c = pf.pf_create_case(ctx, case)
    st = pf.pf_case_get_stats(c)
    opts = pf.make_opts(precision=pf.PF_MIXED)
    n = case.n_bus
    d_pl = torch.tensor(pl, device=dev)
    d_ql = torch.tensor(ql, device=dev)
    d_pg = torch.tensor(pg, device=dev)
    d_vm = torch.zeros((W + K, n), dtype=torch.float64, device=dev)
    d_va = torch.zeros_like(d_vm)
    d_info = torch.zeros((W + K, pf.INFO_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(W + K)]

    def step(k):
        pf.pf_solve_batch_device(c, 1, d_pl[k], d_ql[k], d_pg[k], opts, d_vm[k], d_va[k],
                                 d_info[k], stream.cuda_stream)

    for k in range(W):
        flush.fill_(k & 255)
        step(k)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(W, W + K):
        flush.fill_(k & 255)
        ev[k][0].record(stream)
        step(k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    ms = np.array([ev[k][0].elapsed_time(ev[k][1]) for k in range(W, W + K)])
    info = np.frombuffer(d_info.cpu().numpy().tobytes(), dtype=pf.INFO_DTYPE)
    ok = info["status"][W:] == 0
    iters = info["iterations"][W:]
    total_ms = float(ms.sum())
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    converged = int(ok.sum())
    value = world * converged / (total_ms * 1e-3)

    # roofline of the (only) kernel: one persistent launch per solve
    bytes_iter = algorithmic_bytes_per_iteration(st)
    per_launch = bytes_iter * float(iters.mean())
    achieved = per_launch / (float(ms.mean()) * 1e-3) / 1e9
    peak, peak_kind = _peaks()

    # end to end through the host-buffer entry point
    e2e_t = []
    for k in range(min(K, 20)):
        t0 = time.perf_counter()
        pf.pf_solve_batch(c, pl[W + k:W + k + 1], ql[W + k:W + k + 1], pg[W + k:W + k + 1], opts)
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": len(e2e_t) / sum(e2e_t), "unit": "solves/s",
           "h2d_bytes_per_step": 3 * n * 8, "d2h_bytes_per_step": 2 * n * 8 + pf.INFO_DTYPE.itemsize}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": float(ms.mean()), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_bus": n, "n_branch": case.n_branch,
                   "nnz_lu_blocks": st["nnz_lu"], "levels": st["levels_factor"],
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "ms_per_newton_iter": float(ms.mean() / iters.mean()),
        "newton_iters_mean": float(iters.mean()),
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "converged": converged,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_source": peak_kind,
                     "note": "single 10,000-bus solve: L2-resident, level-latency bound"},
        "e2e": e2e, "gpu_launches": K, "clocks": clk, "wall_s": t_wall,
    }

    if rank == 0:
        prof, pinfo = pf.pf_profile_solve(c, opts)
        line["phase_us_one_solve"] = {k: round(v, 1) for k, v in prof.items()}
    if not args.no_variants and rank == 0:
        line["variants"] = variants(pf, ctx, torch, dev)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    pf.pf_destroy_case(c)
    pf.pf_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()


def _time_solves(pf, c, torch, dev, B, pl, ql, pg, opts, reps=5):
    d = [None if a is None else torch.tensor(a, device=dev) for a in (pl, ql, pg)]
    slots = pl.shape[1] if pl is not None else c.slots
    vm = torch.zeros((B, slots), dtype=torch.float64, device=dev)
    va = torch.zeros_like(vm)
    info = torch.zeros((B, pf.INFO_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream(dev)
    times = []
    for r in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        pf.pf_solve_batch_device(c, B, d[0], d[1], d[2], opts, vm, va, info, s.cuda_stream)
        e1.record(s)
        torch.cuda.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    inf = np.frombuffer(info.cpu().numpy().tobytes(), dtype=pf.INFO_DTYPE)
    ms = float(np.median(times))
    return {"solves_per_s": int((inf["status"] == 0).sum()) / (ms * 1e-3), "ms_per_launch": ms,
            "ms_per_newton_iter": ms / max(1.0, float(inf["iterations"].max())),
            "iterations": int(inf["iterations"].max()), "all_converged": bool((inf["status"] == 0).all())}


def variants(pf, ctx, torch, dev):
    from paper_1711_10579_gb300 import cases

    out = {}
    case = cases.case_10000bus(0)
    c = pf.pf_create_case(ctx, case)
    pl, ql, pg = cases.scenario_loads(case, 1, seed=7, sigma=0.05)
    out["mesh10000_nr_fp64"] = _time_solves(pf, c, torch, dev, 1, pl, ql, pg,
                                            pf.make_opts(precision=pf.PF_FP64))
    pf.pf_destroy_case(c)
    case = cases.case_2000bus(0)
    c = pf.pf_create_case(ctx, case)
    pl, ql, pg = cases.scenario_loads(case, 512, seed=11)
    out["mesh2000_x512_batched_mixed"] = _time_solves(pf, c, torch, dev, 512, pl, ql, pg,
                                                      pf.make_opts())
    pf.pf_destroy_case(c)
    case = cases.case_feeder8000(0)
    c = pf.pf_create_case(ctx, case)
    pl3, ql3 = cases.feeder_scenario_loads(case, 1, seed=3, sigma=0.05)
    for prec, nm in ((pf.PF_FP64, "fp64"), (pf.PF_MIXED, "mixed")):
        out[f"feeder8000_cim_{nm}"] = _time_solves(
            pf, c, torch, dev, 1, pl3.reshape(1, -1), ql3.reshape(1, -1), None,
            pf.make_opts(precision=prec))
    pf.pf_destroy_case(c)
    return out


if __name__ == "__main__":
    main()
