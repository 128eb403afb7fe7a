"""Benchmark of the Newton power-flow hot path on one GB300 (or N replicas).

A step solves one batch of B = 9,728 seeded load scenarios (64 per SM) of the
10,000-bus synthetic transmission grid (average degree 2.7, 20% PV buses;
every bus load x lognormal(0, 0.2), PV generation rescaled to match) to a
power mismatch of 1e-8 pu with Newton-Raphson: FP32 sparse-LU
refactorisation and sweeps, FP64 mismatch, refinement and update.  The batch
runs as phase kernels over the shared symbolic pattern inside one CUDA graph
whose loop the device ends (launch shapes autotuned).  Inputs are resident
in HBM before the timed region; each step has its own scenarios and L2 is
flushed between timed steps.  Batches of 608, 2,432 and 4,864 scenarios, single-
solve latency, the plain FP64 single-case solve, the Newton-Krylov solver,
the three-phase feeder, the 2,000-bus x 512 batch and a serving stream are
reported as variants.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload instead.
Under torchrun each rank is an independent replica (no data collective).
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
B_MAIN = 9728
ORACLE_SAMPLE = 16  # results of the timed step checked against the oracle
# DRAM traffic per scenario-unit of each phase kernel: ncu dram__bytes_read +
# dram__bytes_write of the first launch of each (every scenario running) in a
# batch of 4,864 scenarios of the 10,000-bus grid in the tuned shapes (one-pass
# capture at full size of `--profile-launches 1 --profile-batch 4864`), divided
# by the 4,864 scenarios (a launch's traffic is taken as these bytes per
# scenario times its scenarios).  Valid only for the kernel sources it was measured on
# (sha256 prefix of csrc/batch.cu + csrc/kernels.cuh); otherwise null.
NCU_SOURCES = "a6c0d90eac7da3ed"
NCU_TRAFFIC = {
    "k_factor": (8_101_610_496 + 5_945_336_320) / 4864,
    "k_solve": (6_198_040_832 + 843_860_224) / 4864,
    "k_mismatch": (3_846_259_968 + 3_717_613_824) / 4864,
    "k_update": (1_167_779_328 + 1_493_288_960) / 4864,
}
WORKLOAD = (f"mesh10000 x {B_MAIN} load scenarios per step, batched Newton-Raphson, "
            "FP32 LU + FP64 mismatch/refinement/update, one CUDA graph per batch")


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


def jacobian_nnz(case):
    """Scalar non-zeros of the polar Jacobian of Eq. 10 (J1..J4 blocks): one
    per Ybus entry (i, j) with i, j not the slack for dP/d delta, plus one
    for dP/d|V| where j is PQ, dQ/d delta where i is PQ, dQ/d|V| where both
    are PQ.  Counted from the branch list and bus types."""
    t = np.asarray(case.bus_type)
    f, g = np.asarray(case.br_from), np.asarray(case.br_to)
    pairs = np.unique(np.concatenate([np.stack([f, g], 1), np.stack([g, f], 1),
                                      np.stack([np.arange(case.n_bus)] * 2, 1)]), axis=0)
    i, j = pairs[:, 0], pairs[:, 1]
    ns = (t[i] != 0) & (t[j] != 0)
    pi, pj = t[i] == 2, t[j] == 2
    return int((ns * (1 + pj + pi + (pi & pj))).sum())


def scope_bytes(case, st, B):
    """Algorithmic bytes per unit of each phase kernel of a mixed-precision
    Newton-Raphson step, as the hot-path scope table counts them (Ybus and
    its indices are shared by the B scenarios):

    k_mismatch (a1 + a2), per scenario-iteration: Ybus values and column
      indices, row pointers; V, specified S and the mismatch per bus (16 B
      each); the Jacobian's scalar non-zeros written in FP32;
    k_factor, per scenario-factorisation: the factor's values read and
      written once (nnz_LU scalars of the 2x2 blocks, FP32);
    k_solve, per scenario-pass: the factor's values once and three FP32
      vectors of the N unknowns;
    k_update (a4), per scenario-iteration: 40 B per bus.
    """
    n, nnz_y, N = st["n_bus"], st["nnz_y"], st["n_unknowns"]
    nnz_lu = st["nnz_lu"] * 4
    a1 = nnz_y * (16 + 4) / B + 4 * (n + 1) / B + n * (16 + 16 + 16)
    a2 = jacobian_nnz(case) * 4
    return {"k_mismatch": a1 + a2, "k_factor": nnz_lu * 2 * 4,
            "k_solve": nnz_lu * 4 + 3 * N * 4, "k_update": n * (16 + 16 + 8)}


def _sources_sha():
    import hashlib

    h = hashlib.sha256()
    for f in ("batch.cu", "kernels.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1711_10579_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel, units):
    """Measured DRAM bytes of a launch of `kernel` over `units` scenario-units,
    if the sources are the ones profiled (else None)."""
    per = NCU_TRAFFIC.get(kernel)
    if per is None or _sources_sha() != NCU_SOURCES:
        return None
    return per * units


# phase of pf_profile_solve -> (kernel, unit counted per scenario)
PHASE_KERNELS = {"mismatch_jacobian": ("k_mismatch", "iterations+1"),
                 "factor": ("k_factor", "iterations"),
                 "triangular_solves": ("k_solve", "linear_iterations"),
                 "update": ("k_update", "iterations")}


def kernel_rooflines(case, st, B, phase_us, pinfo, peak):
    """Per-kernel roofline of one batch: algorithmic bytes of every unit the
    batch processed / the kernel's device time (CUDA events between the phase
    kernels), against the measured copy bandwidth."""
    per = scope_bytes(case, st, B)
    it = pinfo["iterations"].astype(float)
    units = {"iterations": float(it.sum()), "iterations+1": float((it + 1).sum()),
             "linear_iterations": float(pinfo["linear_iterations"].sum())}
    launches = {"iterations": float(it.max()), "iterations+1": float(it.max() + 1),
                "linear_iterations": float(it.max())}
    out = {}
    for ph, (kern, u) in PHASE_KERNELS.items():
        t = phase_us[ph] * 1e-6
        if t <= 0 or units[u] <= 0:
            continue
        ach = per[kern] * units[u] / t / 1e9
        out[kern] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "bytes_per_unit": per[kern], "unit_of_work":
                     "scenario-" + {"iterations": "iteration", "iterations+1": "iteration",
                                    "linear_iterations": "pass"}[u],
                     "units": units[u], "device_us": phase_us[ph],
                     "launch_us": phase_us[ph] / launches[u],
                     "share_of_phases": phase_us[ph] / sum(phase_us.values()),
                     "traffic": _ncu_traffic(kern, B),
                     "traffic_over_algorithmic": (NCU_TRAFFIC[kern] / per[kern]
                                                  if _ncu_traffic(kern, B) else None)}
    return out


def _case():
    from paper_1711_10579_gb300 import cases

    return cases.case_10000bus(0)


def _batch(case, B, seed):
    from paper_1711_10579_gb300 import cases

    return cases.scenario_loads(case, B, seed=seed, sigma=0.2)


# ----------------------------------------------------------------------------
# the reference arm: the FP64 CPU oracle
# ----------------------------------------------------------------------------

# The oracle runs in a pool of spawned processes, one per host core (a pool
# forked after CUDA initialisation can hang), each holding the grid and its
# Ybus; only the solves are timed.
_W = {}


def _oracle_init():
    from oracle import pf_oracle as O

    _W["O"] = O
    _W["case"] = _case()
    _W["Y"] = O.ybus_single(_W["case"])
    _W["named"] = {}


def _oracle_solve(loads):
    O, case = _W["O"], _W["case"]
    r = O.newton_polar(case.with_loads(*loads), Y=_W["Y"])
    assert r["converged"]
    return r["iterations"]


def named_case(key):
    """The seeded grids the benchmark and its variants solve, by name."""
    from paper_1711_10579_gb300 import cases

    name, seed = key
    return {"mesh14": cases.case_14bus, "mesh10000": cases.case_10000bus,
            "mesh2000": cases.case_2000bus, "feeder8000": cases.case_feeder8000,
            "mesh10000_heavy": heavy_case,
            "mesh10000_qlim": lambda s: cases.with_q_limits(cases.case_10000bus(s), 1),
            }[name](seed)


def heavy_case(seed=0):
    """The 10,000-bus grid loaded 5.3 times as heavily (DC angle target 1.6
    rad instead of 0.3; lowest |V| about 0.36 pu, near the nose of the
    loading curve), with 8 Newton steps instead of 5."""
    from paper_1711_10579_gb300 import cases

    return cases.transmission_case(10_000, 13_500, 2_000, seed, name="mesh10000_heavy",
                                   max_angle=HEAVY_ANGLE)


HEAVY_ANGLE = 1.6
HEAVY_SIGMA = 0.1  # lognormal spread of its scenarios' loads (0.2 puts some past the nose)


def _oracle_result(job):
    """FP64 oracle solution of one result to check: job = (case name and seed,
    or a case object; loads; reactive limits on).  Returns (|V|, angle) per
    bus (per node and phase for a feeder, absent phases 0)."""
    O = _W["O"]
    key, loads, qlim = job
    if isinstance(key, tuple):
        if key not in _W["named"]:
            _W["named"][key] = named_case(key)
        case = _W["named"][key]
    else:
        case = key
    if hasattr(case, "n_node"):
        r = O.newton_cim(case.with_loads(np.reshape(loads[0], (-1, 3)),
                                         np.reshape(loads[1], (-1, 3))))
        V = r["V"]
        return r["converged"], np.abs(V).reshape(-1), np.where(np.abs(V) > 0, np.angle(V), 0.0).reshape(-1)
    c = case.with_loads(*loads)
    r = O.newton_polar_qlim(c) if qlim else O.newton_polar(c)
    return r["converged"], r["vm"], r["va"]


def oracle_errors(pool, jobs, results):
    """Largest |dV| (pu) and |d theta| (rad) of GPU results against the FP64
    oracle's solutions of the same inputs, per result and overall."""
    refs = pool.map(_oracle_result, jobs, chunksize=1)
    per = []
    for (ok, rvm, rva), (vm, va) in zip(refs, results):
        vm, va = np.asarray(vm).reshape(-1), np.asarray(va).reshape(-1)
        dv = float(np.max(np.abs(vm - rvm)))
        dth = float(np.max(np.abs(np.angle(np.exp(1j * (va - rva))))))
        per.append([round(dv, 12), round(dth, 12), bool(ok)])
    return {"max_dv_pu": max(p[0] for p in per), "max_dtheta_rad": max(p[1] for p in per),
            "all_oracle_converged": all(p[2] for p in per), "per_result": per}


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_pool():
    import multiprocessing as mp

    cores = _host_cores()
    # one thread per process (the workers inherit the environment at spawn)
    saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                             "MKL_NUM_THREADS")}
    for v in saved:
        os.environ[v] = "1"
    try:
        pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_init)
    finally:
        for v, x in saved.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x
    pool.map(_oracle_warm, range(cores))  # every worker started and initialised
    return pool, cores


def _oracle_warm(_):
    return 0


def run_reference(args, rank, world):
    """The oracle as it stands, timed on the host cores on the same workload:
    each step solves one scenario per core of that step's batch."""
    if rank != 0:
        return
    case = _case()
    pool, cores = _oracle_pool()
    per_step = cores
    times, iters = [], []
    try:
        for k in range(args.warmup + args.steps):
            pl, ql, pg = _batch(case, per_step, seed=1000 + k)
            work = [(pl[b], ql[b], pg[b]) for b in range(per_step)]
            t0 = time.perf_counter()
            its = pool.map(_oracle_solve, work, chunksize=1)
            if k >= args.warmup:
                times.append(time.perf_counter() - t0)
                iters.extend(its)
    finally:
        pool.close()
        pool.join()
    tot = sum(times)
    val = args.steps * per_step / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + "; reference: FP64 CPU oracle (polar NR, "
                   f"SuperLU/COLAMD), one process per host core ({cores})",
                   "n_bus": case.n_bus, "n_branch": case.n_branch},
        "ms_per_newton_iter": 1e3 * tot * cores / sum(iters),
        "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} scenarios of each step's batch per step "
                                   f"(one per core), {args.steps} steps"},
        "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(pool, cores):
    """The oracle as it stands on a bounded sample of the same workload,
    one process per host core: 4 scenarios per core (about 0.3 s of one
    core each on this grid)."""
    case = _case()
    n = 4 * cores
    pl, ql, pg = _batch(case, n, seed=77)
    work = [(pl[b], ql[b], pg[b]) for b in range(n)]
    t0 = time.perf_counter()
    pool.map(_oracle_solve, work, chunksize=1)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} scenarios of the 10,000-bus grid in {dt:.2f} s on {cores} "
                      "processes (one per host core; start-up not timed)"}


# ----------------------------------------------------------------------------
# variants
# ----------------------------------------------------------------------------

def _device_solves(pf, c, torch, dev, B, pl, ql, pg, opts, reps=5, flush=None, check=None):
    """Times `reps` device-buffer batch solves; with check = (pool, case key)
    the FP64 oracle's error of up to 4 of the results (evenly spaced) is
    added as oracle_err."""
    d = [None if a is None else torch.tensor(a, device=dev) for a in (pl, ql, pg)]
    slots = pl.shape[1]
    vm = torch.zeros((B, slots), dtype=torch.float64, device=dev)
    va = torch.zeros_like(vm)
    info = torch.zeros((B, pf.INFO_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream(dev)
    times = []
    for r in range(reps + 2):
        if flush is not None:
            flush.fill_(r & 255)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        pf.pf_solve_batch_device(c, B, d[0], d[1], d[2], opts, vm, va, info, s.cuda_stream)
        e1.record(s)
        torch.cuda.synchronize()
        if r >= 2:
            times.append(e0.elapsed_time(e1))
    inf = np.frombuffer(info.cpu().numpy().tobytes(), dtype=pf.INFO_DTYPE)
    ms = float(np.median(times))
    ok = int((inf["status"] == 0).sum())
    its = float(inf["iterations"].mean())
    out = {"solves_per_s": ok / (ms * 1e-3), "ms_per_launch": ms,
           "latency_ms": {"p50": float(np.percentile(times, 50)),
                          "p99": float(np.percentile(times, 99))},
           "ms_per_newton_iter": ms / max(1.0, its), "newton_iters_mean": its,
           "linear_iters_mean": float(inf["linear_iterations"].mean()),
           "all_converged": bool(ok == B), "B": B}
    if check is not None:
        pool, key, qlim = check
        idx = np.unique(np.linspace(0, B - 1, min(B, 4)).astype(int))
        jobs = [(key, tuple(None if a is None else a[b] for a in (pl, ql, pg)), qlim)
                for b in idx]
        res = list(zip(vm[idx].cpu().numpy(), va[idx].cpu().numpy()))
        out["oracle_err"] = dict(oracle_errors(pool, jobs, res), scenarios=idx.tolist())
    return out


def variants(pf, ctx, torch, dev, flush, pool):
    from paper_1711_10579_gb300 import cases

    out = {}
    # the 14-bus mesh: one batch of B_MAIN load scenarios, and single solves
    case = named_case(("mesh14", 0))
    c = pf.pf_create_case(ctx, case)
    pl, ql, pg = _batch(case, B_MAIN, seed=5)
    pf.pf_autotune(c, B_MAIN, pf.make_opts())
    out[f"mesh14_x{B_MAIN}_batched_mixed"] = _device_solves(
        pf, c, torch, dev, B_MAIN, pl, ql, pg, pf.make_opts(), reps=10, flush=flush,
        check=(pool, ("mesh14", 0), False))
    for prec, nm in ((pf.PF_FP64, "fp64"), (pf.PF_MIXED, "mixed")):
        out[f"mesh14_single_nr_{nm}"] = _device_solves(
            pf, c, torch, dev, 1, pl[:1], ql[:1], pg[:1], pf.make_opts(precision=prec), reps=20,
            flush=flush, check=(pool, ("mesh14", 0), False))
    pf.pf_destroy_case(c)

    case = _case()
    key = ("mesh10000", 0)
    c = pf.pf_create_case(ctx, case)
    pl, ql, pg = _batch(case, 1, seed=7)
    out["mesh10000_single_nr_mixed"] = _device_solves(
        pf, c, torch, dev, 1, pl, ql, pg, pf.make_opts(precision=pf.PF_MIXED), reps=20, flush=flush,
        check=(pool, key, False))
    out["mesh10000_single_nr_mixed"]["launch"] = pf.pf_launch_config(c, pf.make_opts())
    prof, _ = pf.pf_profile_solve(c, pf.make_opts())
    out["mesh10000_single_nr_mixed"]["phase_us"] = {k: round(v, 1) for k, v in prof.items()}
    # branch flows and losses (post-step) of a solved 608-scenario batch
    plf, qlf, pgf = _batch(case, 608, seed=23)
    vmf, vaf, _ = pf.pf_solve_batch(c, plf, qlf, pgf)
    t0 = time.perf_counter()
    fl = pf.pf_branch_flows(c, vmf, vaf, case.n_branch)
    out["mesh10000_x608_branch_flows"] = {
        "ms_host_call": 1e3 * (time.perf_counter() - t0), "B": 608, "branches": case.n_branch,
        "mean_loss_p_pu": float(fl["loss"][:, 0].mean()),
        "note": "pf_branch_flows with host buffers (copies inside)"}
    out["mesh10000_single_nr_fp64"] = _device_solves(
        pf, c, torch, dev, 1, pl, ql, pg, pf.make_opts(precision=pf.PF_FP64), reps=20, flush=flush,
        check=(pool, key, False))
    for Bv, prec, nm in ((608, pf.PF_MIXED, "mixed"), (2432, pf.PF_MIXED, "mixed"),
                         (4864, pf.PF_MIXED, "mixed"), (B_MAIN, pf.PF_FP64, "fp64")):
        plb, qlb, pgb = _batch(case, Bv, seed=21)
        pf.pf_autotune(c, Bv, pf.make_opts(precision=prec))
        out[f"mesh10000_x{Bv}_batched_{nm}"] = _device_solves(
            pf, c, torch, dev, Bv, plb, qlb, pgb, pf.make_opts(precision=prec), reps=3,
            flush=flush, check=(pool, key, False))
    for prec, nm in ((pf.PF_MIXED, "mixed"), (pf.PF_FP64, "fp64")):
        out[f"mesh10000_single_nk_{nm}"] = _device_solves(
            pf, c, torch, dev, 1, pl, ql, pg, pf.make_opts(method=pf.PF_NK, precision=prec),
            reps=1, check=(pool, key, False))
        out[f"mesh10000_single_nk_bicgstab_{nm}"] = _device_solves(
            pf, c, torch, dev, 1, pl, ql, pg,
            pf.make_opts(method=pf.PF_NK, krylov=1, precision=prec, gmres_max_iter=2000), reps=1,
            check=(pool, key, False))
    pf.pf_destroy_case(c)

    # heavier loading: the mixed-precision steps slow down and the on-demand
    # FP64 refinement is taken
    case = named_case(("mesh10000_heavy", 0))
    c = pf.pf_create_case(ctx, case)
    plh, qlh, pgh = cases.scenario_loads(case, 2432, seed=31, sigma=HEAVY_SIGMA)
    pf.pf_autotune(c, 2432, pf.make_opts())
    r = _device_solves(pf, c, torch, dev, 2432, plh, qlh, pgh, pf.make_opts(), reps=3,
                       flush=flush, check=(pool, ("mesh10000_heavy", 0), False))
    r["max_angle_rad"] = HEAVY_ANGLE
    r["load_sigma"] = HEAVY_SIGMA
    r["load_scale"] = case.load_scale
    out["mesh10000_heavy_x2432_batched_mixed"] = r
    # the same with the FP64 refinement of every step below refine_below
    r = _device_solves(pf, c, torch, dev, 2432, plh, qlh, pgh, pf.make_opts(refine_stall=0.0),
                       reps=3, flush=flush, check=(pool, ("mesh10000_heavy", 0), False))
    r["refine_stall"] = 0.0
    out["mesh10000_heavy_x2432_batched_mixed_refine_always"] = r
    pf.pf_destroy_case(c)

    # reactive limits of PV buses enforced (rounds of PV -> PQ switching)
    qkey = ("mesh10000_qlim", 0)
    qcase = named_case(qkey)
    c = pf.pf_create_case(ctx, qcase)
    plq, qlq, pgq = _batch(qcase, 608, seed=21)
    r = _device_solves(pf, c, torch, dev, 608, plq, qlq, pgq, pf.make_opts(q_limits=1), reps=3,
                       flush=flush, check=(pool, qkey, True))
    _, _, iq = pf.pf_solve_batch(c, plq, qlq, pgq, pf.make_opts(q_limits=1))
    r["q_switched_mean"] = float(iq["q_switched"].mean())
    r["q_rounds_max"] = int(iq["q_rounds"].max())
    out["mesh10000_x608_batched_mixed_qlimits"] = r
    pf.pf_destroy_case(c)

    case = cases.case_2000bus(0)
    key = ("mesh2000", 0)
    c = pf.pf_create_case(ctx, case)
    pl, ql, pg = cases.scenario_loads(case, 512, seed=11)
    tuned = pf.pf_autotune(c, 512, pf.make_opts())
    out["mesh2000_x512_batched_mixed"] = _device_solves(pf, c, torch, dev, 512, pl, ql, pg,
                                                        pf.make_opts(), flush=flush,
                                                        check=(pool, key, False))
    out["mesh2000_x512_batched_mixed"]["tuned"] = {"scen_per_cta": tuned.scen_per_cta,
                                                   "block_threads": tuned.block_threads}
    # a batch of Newton-Krylov solves (one persistent launch)
    out["mesh2000_x64_batched_nk_mixed"] = _device_solves(
        pf, c, torch, dev, 64, pl[:64], ql[:64], pg[:64], pf.make_opts(method=pf.PF_NK), reps=1,
        flush=flush, check=(pool, key, False))
    pf.pf_destroy_case(c)

    case = cases.case_feeder8000(0)
    c = pf.pf_create_case(ctx, case)
    pl3, ql3 = cases.feeder_scenario_loads(case, 1, seed=3, sigma=0.05)
    for prec, nm in ((pf.PF_FP64, "fp64"), (pf.PF_MIXED, "mixed")):
        out[f"feeder8000_cim_{nm}"] = _device_solves(
            pf, c, torch, dev, 1, pl3.reshape(1, -1), ql3.reshape(1, -1), None,
            pf.make_opts(precision=prec), reps=10, flush=flush,
            check=(pool, ("feeder8000", 0), False))
    pf.pf_destroy_case(c)
    out["serving"] = serving_stream(pf, ctx, pool=pool)
    for grid, B in (("mesh2000", 512), ("mesh10000", 4864)):
        out[f"serving_burst_{grid}_x{B}"] = serving_burst(pf, ctx, pool, grid, B)
    return out


def serving_burst(pf, ctx, pool, grid, B, reps=2):
    """B requests of one grid queued together (pf_submit_batch), coalesced by
    the serving runtime into one batched solve: solves/s from the submit to
    the last result polled (host copies of every request's inputs and
    results included); the last of `reps` bursts is reported."""
    from paper_1711_10579_gb300 import cases

    case = named_case((grid, 0))
    h = pf.pf_create_case(ctx, case)
    pl, ql, pg = cases.scenario_loads(case, B, seed=23, sigma=0.2)
    st0 = pf.pf_serve_get_stats(ctx)
    res = None
    for _ in range(reps):
        t0 = time.perf_counter()
        ts = pf.pf_submit_batch(ctx, h, pl, ql, pg, pf.make_opts())
        pf.pf_drain(ctx, 600_000)
        res = [pf.pf_poll(ctx, t, h.slots) for t in ts]
        dt = time.perf_counter() - t0
    st = pf.pf_serve_get_stats(ctx)
    jobs = [((grid, 0), (pl[k], ql[k], pg[k]), False) for k in (0, B - 1)]
    err = oracle_errors(pool, jobs, [(res[k][0], res[k][1]) for k in (0, B - 1)])
    pf.pf_destroy_case(h)
    return {"B": B, "seconds": dt, "solves_per_s": B / dt,
            "converged": int(sum(r[2]["status"] == 0 for r in res)),
            "batch_launches": st["batch_launches"] - st0["batch_launches"],
            "max_batch": st["max_batch"], "oracle_err": err,
            "note": "end to end through pf_submit_batch / pf_poll; host copies included"}


def _pool_case(job):
    """One seeded topology of the serving pool (run in a worker process):
    the first of seeds seed, seed + 100,000, ... whose base case the FP64
    oracle solves from a flat start (some large generated meshes have no
    flat-start solution)."""
    from paper_1711_10579_gb300 import cases

    O = _W["O"]
    kind, n, seed = job
    for k in range(8):
        s = seed + 100_000 * k
        if kind == "transmission":
            c = cases.transmission_case(n, int(round(1.35 * n)), n // 5, s)
            ok = O.newton_polar(c)["converged"]
        else:
            c = cases.feeder_case(n, s)
            ok = O.newton_cim(c)["converged"]
        if ok:
            return c
    raise RuntimeError(f"no solvable {kind} topology of size {n} near seed {seed}")


def serving_pool(pool, count, seed):
    """`count` transmission grids (500-70,000 buses) and `count` feeders
    (1,000-20,000 nodes), sizes log-uniform, generated (and their base cases
    checked by the oracle) in the worker processes; returns
    {kind: [case, ...]}."""
    rng = np.random.default_rng(seed)
    jobs = [("transmission", int(s), seed * 1000 + i)
            for i, s in enumerate(np.exp(rng.uniform(np.log(500), np.log(70_000), count)))]
    jobs += [("feeder", int(s), seed * 1000 + 500 + i)
             for i, s in enumerate(np.exp(rng.uniform(np.log(1_000), np.log(20_000), count)))]
    made = pool.map(_pool_case, jobs, chunksize=1)
    return {"transmission": made[:count], "feeder": made[count:]}


def serving_stream(pf, ctx, pool, rate=2000.0, duration=60.0, seed=9, topologies=32,
                   check=8, warmup=2.0):
    """Poisson arrivals at `rate` for `duration` seconds, 70% transmission
    grids / 30% feeders drawn from resident pools of `topologies` each, every
    request with a fresh per-bus lognormal(0, 0.2) load multiplier (PV
    generation rescaled to 1.05 x the request's load), mixed precision, warm
    starts.  Latency = completion seen by the client - arrival time.  A
    `warmup`-second stream first (not reported) lets the runtime allocate
    its job slots."""
    from paper_1711_10579_gb300 import cases

    t_setup = time.perf_counter()
    pools = serving_pool(pool, topologies, seed)
    handles = {k: [pf.pf_create_case(ctx, c) for c in v] for k, v in pools.items()}
    pv_w = {}
    for i, c in enumerate(pools["transmission"]):
        pvm = c.bus_type == cases.PV
        w = np.where(pvm, c.p_gen, 0.0)
        pv_w[i] = (pvm, w / w.sum())
    setup_s = time.perf_counter() - t_setup
    opts = pf.make_opts(warm_start=1)
    rng = np.random.default_rng(seed + 1)
    # lognormal(0, 0.2) drawn by inverse-CDF lookup over 65,536 quantiles
    # (a uint16 draw per bus: the client keeps pace with the offered rate)
    from scipy.stats import norm

    quant = np.exp(0.2 * norm.ppf((np.arange(65536) + 0.5) / 65536))

    def loads(r):
        c = pools[r.kind][r.topo]
        n = c.n_bus if r.kind == "transmission" else c.n_node
        mult = quant[rng.integers(0, 65536, n, dtype=np.uint16)]
        if r.kind == "feeder":
            mult = mult[:, None]
        if r.kind == "feeder":
            return (c.p_load * mult).reshape(-1), (c.q_load * mult).reshape(-1), None
        pl, ql = c.p_load * mult, c.q_load * mult
        pvm, w = pv_w[r.topo]
        pg = np.where(pvm, 1.05 * pl.sum() * w, c.p_gen)
        return pl, ql, pg

    def run(reqs, dur, check):
        pending, lat, statuses, sample = [], [], [], []
        solve_us = {"transmission": [], "feeder": []}
        client_s, backlog = 0.0, 0
        t0 = time.perf_counter()
        k = 0
        while k < len(reqs) or pending:
            now = time.perf_counter() - t0
            while k < len(reqs) and reqs[k].t_arrive <= now:
                r = reqs[k]
                tc = time.perf_counter()
                pl, ql, pg = loads(r)
                h = handles[r.kind][r.topo]
                t = pf.pf_submit(ctx, h, pl, ql, pg, opts)
                client_s += time.perf_counter() - tc
                keep = check and k % max(1, len(reqs) // check) == 0
                pending.append((t, r.t_arrive, h.slots, r, (pl, ql, pg) if keep else None))
                k += 1
            backlog = max(backlog, len(pending))
            still = []
            for j, item in enumerate(pending):
                if j >= 128:  # completions come roughly in arrival order
                    still.extend(pending[j:])
                    break
                res = pf.pf_poll(ctx, item[0], item[2], values=item[4] is not None)
                if res is None:
                    still.append(item)
                    continue
                lat.append(time.perf_counter() - t0 - item[1])
                statuses.append(res[2]["status"])
                solve_us[item[3].kind].append(res[2]["solve_us"])
                if item[4] is not None and len(sample) < check:
                    r = item[3]
                    sample.append((pools[r.kind][r.topo], item[4], res[0], res[1]))
            pending = still
            if k < len(reqs) and not pending:
                time.sleep(max(0.0, min(0.0005, reqs[k].t_arrive - (time.perf_counter() - t0))))
        span = time.perf_counter() - t0
        lat_ms = np.array(lat) * 1e3
        ok = sum(1 for s_ in statuses if s_ == 0)
        stats = pf.pf_serve_get_stats(ctx)
        out = {"offered_req_per_s": rate, "duration_s": dur, "requests": len(reqs),
               "seconds": span, "solves_per_s": ok / span, "converged": ok,
               "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                              "p99": float(np.percentile(lat_ms, 99)),
                              "max": float(lat_ms.max())},
               "status_counts": {str(k): int(v) for k, v in zip(*np.unique(statuses,
                                                                             return_counts=True))},
               "device_ms_per_solve": {k: {"mean": float(np.mean(v)) * 1e-3,
                                           "p99": float(np.percentile(v, 99)) * 1e-3}
                                       for k, v in solve_us.items() if v},
               "max_pending": backlog, "client_ms_per_request": 1e3 * client_s / max(1, len(reqs)),
               "runtime": stats,
               "pool": {"transmission_buses": [c.n_bus for c in pools["transmission"]],
                        "feeder_nodes": [c.n_node for c in pools["feeder"]]},
               "setup_s": setup_s,
               "loads": "fresh per request: per-bus lognormal(0, 0.2) multipliers (inverse-CDF "
                        "lookup over 65,536 quantiles)"}
        return out, sample

    if warmup > 0:
        run(cases.serving_stream(seed + 7, rate=rate, duration=warmup, pool_size=topologies),
            warmup, 0)
    stats0 = pf.pf_serve_get_stats(ctx)
    reqs = cases.serving_stream(seed, rate=rate, duration=duration, pool_size=topologies)
    out, sample = run(reqs, duration, check)
    # counters of the timed stream (the largest group and peak include the warm-up)
    for key in ("requests", "group_launches"):
        out["runtime"][key] -= stats0[key]
    out["warmup_s"] = warmup
    jobs = [(c, ld, False) for c, ld, _, _ in sample]
    out["oracle_err"] = dict(oracle_errors(pool, jobs, [(vm, va) for _, _, vm, va in sample]),
                             sample=f"{len(sample)} served requests spread over the stream")
    for v in handles.values():
        for h in v:
            pf.pf_destroy_case(h)
    return out


def profile_launches(count, B=608, S=0, threads=0, grid="mesh10000"):
    """``count`` batched solves of B scenarios of a grid (default: the main
    step's), kernel by kernel (ncu does not look inside the CUDA graph of a
    batch), in the autotuned shapes of the factorisation and the sweeps (the
    timed step's), or in a fixed shape S scenarios per CTA x threads."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1711_10579_gb300 import pf

    dev = torch.device("cuda:0")
    ctx = pf.pf_ctx_create(0)
    case = named_case((grid, 0))
    c = pf.pf_create_case(ctx, case)
    pl, ql, pg = _batch(case, B, seed=1)
    d = [torch.tensor(a, device=dev) for a in (pl, ql, pg)]
    vm = torch.zeros((B, case.n_bus), dtype=torch.float64, device=dev)
    va = torch.zeros_like(vm)
    info = torch.zeros((B, pf.INFO_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    if S == 0:
        pf.pf_autotune(c, B, pf.make_opts())
    o = pf.make_opts(scen_per_cta=S, block_threads=threads, kernel_by_kernel=1)
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    # the profiled solves (ncu --nvtx --nvtx-include "pf_profiled/")
    torch.cuda.nvtx.range_push("pf_profiled")
    for _ in range(count):
        pf.pf_solve_batch_device(c, B, d[0], d[1], d[2], o, vm, va, info, s.cuda_stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    inf = np.frombuffer(info.cpu().numpy().tobytes(), dtype=pf.INFO_DTYPE)
    print(json.dumps({"solves": count, "B": B, "launch": pf.pf_launch_config(c, o, B),
                      "all_converged": bool((inf["status"] == 0).all())}))
    pf.pf_destroy_case(c)
    pf.pf_ctx_destroy(ctx)


def profile_single(count, precision="mixed", method="nr", grid="mesh10000"):
    """``count`` single solves of a grid (default: the main step's) in the
    persistent single-solve kernel, for ncu."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_1711_10579_gb300 import pf

    ctx = pf.pf_ctx_create(0)
    case = named_case((grid, 0))
    c = pf.pf_create_case(ctx, case)
    o = pf.make_opts(precision=pf.PF_MIXED if precision == "mixed" else pf.PF_FP64,
                     method=pf.PF_NK if method == "nk" else pf.PF_NR)
    infos = [pf.pf_solve(c, o)[2] for _ in range(count)]
    print(json.dumps({"solves": count, "status": [i["status"] for i in infos],
                      "iterations": [i["iterations"] for i in infos],
                      "solve_us": [i["solve_us"] for i in infos]}))
    pf.pf_destroy_case(c)
    pf.pf_ctx_destroy(ctx)


def profile_serve(count):
    """``count`` served requests submitted at once, over a 500-, a 2,000-, a
    10,000-bus grid and a 2,000-node feeder (group launches), for ncu."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_1711_10579_gb300 import cases, pf

    ctx = pf.pf_ctx_create(0)
    pool = [cases.transmission_case(500, 675, 100, 3), cases.case_2000bus(0), _case(),
            cases.feeder_case(2000, 4)]
    hs = [pf.pf_create_case(ctx, c) for c in pool]
    tickets = [(pf.pf_submit(ctx, hs[k % 4]), hs[k % 4].slots) for k in range(count)]
    pf.pf_drain(ctx, 120_000)
    st = [pf.pf_poll(ctx, t, n, values=False)[2]["status"] for t, n in tickets]
    print(json.dumps({"requests": count, "status": st, "runtime": pf.pf_serve_get_stats(ctx)}))
    for h in hs:
        pf.pf_destroy_case(h)
    pf.pf_ctx_destroy(ctx)


# ----------------------------------------------------------------------------
# main
# ----------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile-launches", type=int, default=0,
                    help="only run the batched solve this many times (for ncu)")
    ap.add_argument("--profile-batch", type=int, default=608,
                    help="scenarios of the --profile-launches batch")
    ap.add_argument("--profile-shape", default="0,0",
                    help="scenarios per CTA and threads of the --profile-launches batch "
                         "(0,0: the autotuned shapes)")
    ap.add_argument("--profile-grid", default="mesh10000",
                    help="grid of --profile-launches / --profile-single (mesh10000, mesh2000, "
                         "feeder8000, ...)")
    ap.add_argument("--profile-single", type=int, default=0,
                    help="only run this many single solves of the main grid (for ncu)")
    ap.add_argument("--profile-precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--profile-method", default="nr", choices=["nr", "nk"])
    ap.add_argument("--profile-serve", type=int, default=0,
                    help="only submit this many served requests at once (for ncu)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_single:
        profile_single(args.profile_single, args.profile_precision, args.profile_method,
                       args.profile_grid)
        return
    if args.profile_serve:
        profile_serve(args.profile_serve)
        return
    if args.profile_launches:
        S, T = (int(x) for x in args.profile_shape.split(","))
        profile_launches(args.profile_launches, args.profile_batch, S, T, args.profile_grid)
        return

    # the oracle's worker processes (spawned), for the error check of the
    # results and the CPU baseline
    pool, cores = _oracle_pool() if rank == 0 else (None, 0)

    import torch

    from paper_1711_10579_gb300 import replicas

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    __graft_entry__.build()
    from paper_1711_10579_gb300 import pf

    K, W, B = args.steps, args.warmup, B_MAIN
    case = _case()
    n = case.n_bus
    ctx = pf.pf_ctx_create(local)
    c = pf.pf_create_case(ctx, case)
    st = pf.pf_case_get_stats(c)
    tuned = pf.pf_autotune(c, B, pf.make_opts(precision=pf.PF_MIXED))
    opts = pf.make_opts(precision=pf.PF_MIXED)  # zeros: the tuned shapes of each phase
    batches = [_batch(case, B, replicas.scenario_seed(1000 + k, rank)) for k in range(W + K)]
    d_in = [[torch.tensor(a, device=dev) for a in bt] for bt in batches]
    d_vm = torch.zeros((B, n), dtype=torch.float64, device=dev)
    d_va = torch.zeros_like(d_vm)
    d_info = torch.zeros((W + K, B, pf.INFO_DTYPE.itemsize), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(W + K)]

    def step(k):
        pf.pf_solve_batch_device(c, B, d_in[k][0], d_in[k][1], d_in[k][2], opts, d_vm, d_va,
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
    info = np.frombuffer(d_info[W:].cpu().numpy().tobytes(), dtype=pf.INFO_DTYPE)
    converged = int((info["status"] == 0).sum())
    value, max_ms, total = replicas.aggregate(float(ms.sum()), converged, dist)

    # per-kernel device times of the same batch (events between the phase
    # kernels, launched one by one, on the library's stream), for the
    # roofline of every phase kernel; the dominant one heads the line
    phases, pinfo = [], None
    for _ in range(3):
        ph, pinfo = pf.pf_profile_solve(c, opts, B)
        phases.append(ph)
    phase_us = {k: float(np.median([p[k] for p in phases])) for k in phases[0]}
    peak, peak_kind = _peaks()
    kr = kernel_rooflines(case, st, B, phase_us, pinfo, peak)
    dom = max(kr, key=lambda k: kr[k]["device_us"])
    # algorithmic bytes of the timed steps: every phase kernel's units, plus
    # the FP64 residuals of the refinements taken (on demand)
    per = scope_bytes(case, st, B)
    its = info["iterations"].astype(float)
    nref = float((info["linear_iterations"] - info["iterations"]).sum())
    step_bytes = (per["k_mismatch"] * (its + 1).sum() + (per["k_factor"] + per["k_update"]) * its.sum()
                  + per["k_solve"] * float(info["linear_iterations"].sum())
                  + nref * (st["nnz_y"] * 20 / B + n * 32 + 4 * st["n_unknowns"] * 8)) / K
    # kernels per step: the call record, the graph's prologue (set-up,
    # mismatch, stop test), one loop body per Newton step of the slowest
    # scenario (refinement flag, factor, sweeps, update, mismatch, stop
    # test), the refinement launches (voltage change, residual, sweeps) of
    # the steps where a scenario refines (at least the most any scenario
    # took), the results
    refine = pf.make_opts().refine_steps
    loops = info["iterations"].reshape(K, B).max(1)
    refs = (info["linear_iterations"] - info["iterations"]).reshape(K, B).max(1)
    launches = int(sum(5 + int(L) * 6 + 3 * refine * int(R) for L, R in zip(loops, refs)))
    # end to end through the host-buffer entry point: inputs and results in
    # pinned host memory, their copies inside the timed call
    def pinned(shape, dtype=torch.float64):
        return torch.empty(shape, dtype=dtype, pin_memory=True).numpy()

    h_in = [pinned((B, n)) for _ in range(3)]
    h_vm, h_va = pinned((B, n)), pinned((B, n))
    h_info = pinned((B * pf.INFO_DTYPE.itemsize,), torch.uint8).view(pf.INFO_DTYPE)
    e2e_t = []
    for k in range(W, min(W + 5, W + K)):
        for a, src in zip(h_in, batches[k]):
            a[...] = src  # the step's inputs, staged outside the timed call
        t0 = time.perf_counter()
        pf.pf_solve_batch(c, h_in[0], h_in[1], h_in[2], opts, out=(h_vm, h_va, h_info))
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": B * len(e2e_t) / sum(e2e_t), "unit": "solves/s",
           "h2d_bytes_per_step": 3 * B * n * 8,
           "d2h_bytes_per_step": 2 * B * n * 8 + B * pf.INFO_DTYPE.itemsize,
           "host_buffers": "pinned"}

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": float(ms.mean()), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_bus": n, "n_branch": case.n_branch,
                   "scenarios_per_step": B, "nnz_lu_blocks": st["nnz_lu"],
                   "levels": st["levels_factor"],
                   "launch": pf.pf_launch_config(c, opts, B),
                   "tuned_factor_shape": {"scen_per_cta": tuned.scen_per_cta,
                                          "block_threads": tuned.block_threads},
                   "l2": "flushed between timed steps (256 MB write); inputs exceed L2",
                   "parallelism": f"replicas x{world}"},
        "ms_per_newton_iter": float(ms.mean() / info["iterations"].reshape(K, B).max(1).mean()),
        "newton_iters_mean": float(info["iterations"].mean()),
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                       "note": "per batch step; single-solve latency in variants"},
        "converged": total, "solves": world * B * K,
        "roofline": dict(kr[dom], kernel=dom, peak_source=peak_kind,
                         traffic=_ncu_traffic(dom, B),
                         note="achieved = algorithmic bytes per scenario-unit (hot-path scope "
                              "table) x units the batch processed / device time of the "
                              "kernel's launches (CUDA events between the phase kernels of a "
                              "batch of the same size, right after the timed region); traffic "
                              "= ncu DRAM bytes per launch of B scenarios"),
        "kernel_rooflines": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv)
                                 for kk, vv in v.items()} for k, v in kr.items()},
        "phase_us": {k: round(v, 1) for k, v in phase_us.items()},
        "step_algorithmic_gb": step_bytes / 1e9,
        "e2e": e2e, "gpu_launches": launches, "clocks": clk, "wall_s": t_wall,
    }
    if rank == 0:
        # the FP64 oracle's error of a sample of the last timed step's results
        idx = np.unique(np.linspace(0, B - 1, ORACLE_SAMPLE).astype(int))
        last = batches[W + K - 1]
        jobs = [(("mesh10000", 0), tuple(a[b] for a in last), False) for b in idx]
        res = list(zip(d_vm[idx].cpu().numpy(), d_va[idx].cpu().numpy()))
        line["oracle_err"] = dict(oracle_errors(pool, jobs, res), scenarios=idx.tolist(),
                                  sample=f"{len(idx)} of the {B} scenarios of the last timed "
                                         "step, evenly spaced")
    if rank == 0 and not args.no_variants:
        line["variants"] = variants(pf, ctx, torch, dev, flush, pool)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(pool, cores)
    if pool is not None:
        pool.close()
        pool.join()
    if rank == 0:
        print(json.dumps(line), flush=True)
    pf.pf_destroy_case(c)
    pf.pf_ctx_destroy(ctx)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
