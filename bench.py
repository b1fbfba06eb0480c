#!/usr/bin/env python
"""Benchmark of the Holstein HMC hot path on GB300.

Workload (one "step"): L=32 (N=1024), Ltau=200, beta=20, omega0=0.5,
alpha=1, t=1, mu=0, dtau=0.1, x ~ N(0, 1/omega0^2) i.i.d., 16 Gaussian
pseudofermion draws R_k. One step runs the whole single-chain hot path on
that batch: field set-up (expV, dbar, spectral bounds), b_k = M^T R_k, the
mixed-precision CG solve of M^T M v_k = b_k for all 16 right-hand sides to a
certified FP64 residual 1e-8 (FP32 operator and iterations, FP64 dot
products, FP64 reliable updates every 50 iterations), and the phonon force
summed over the 16 solutions.

Metric: CG solves/s (whole job, all ranks); the JSON line also carries
matvecs/s, the roofline of the dominant kernel (the fused FP32 M^T M of the
CG iteration, timed live with CUDA events on its stream during the timed
region), the FP64-only solve rate on the same inputs, the end-to-end rate
through the public API with host buffers, the clocks seen during the timed
region, and the oracle timed on the host cores (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --mode matvec --rhs 64      # fused M^T M alone, cold L2
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import holstein_inputs as hi  # noqa: E402

METRIC = "CG solves/s (M^T M v = b, certified FP64 residual 1e-8) at L=32, Ltau=200"
WORKLOAD = hi.WORKLOADS["big32"]
TOL = 1e-8
RELIABLE_EVERY = 50
# CUDA events around one in every TIMER_STRIDE launches of each kernel class
# during the timed region: about 200 samples of the CG kernels over 20 steps,
# while the bracketed launches (which lose their programmatic-launch overlap
# with the neighbours) stay below 0.5 % of the launches, so ms_per_step is
# not perturbed measurably
TIMER_STRIDE = 256
LEG_TIMER_STRIDE = 32     # the same inside the secondary rows (fewer launches)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["step", "matvec", "precond", "leg"], default="step")
    ap.add_argument("--leg", choices=["trajectory", "trajectory64", "measurement",
                                      "measurement32", "global",
                                      "chains", "prior", "split"],
                    default="trajectory", help="with --mode leg: run one of the other rows alone")
    ap.add_argument("--rhs", type=int, default=16)
    ap.add_argument("--lattice", default=None,
                    help="--mode precond: LxLtau of a chain lattice of the batching workload "
                         "(omega0=1, alpha=1, x ~ N(0, 1)) instead of the L=32, Ltau=200 one")
    ap.add_argument("--prec", choices=["f32", "f64"], default="f32",
                    help="--mode matvec: the fused FP32 M^T M (f32) or FP64 M and M^T (f64)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape")
    ap.add_argument("--option", action="append", default=[],
                    help="NAME=VALUE launch option applied after tuning (hol_set_option)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the trajectory and measurement legs")
    ap.add_argument("--field", choices=["iid", "ar1"], default="iid",
                    help="phonon field: i.i.d. Gaussian (default) or tau-correlated AR(1)")
    ap.add_argument("--precond", action="store_true",
                    help="time the adiabatic-preconditioned solve as the main step")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (one process per GPU; independent replicas)
# ----------------------------------------------------------------------------
def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(world, val, device="cuda"):
    """Maximum of a per-rank scalar over the ranks (the job's time)."""
    if world == 1:
        return val
    import torch
    import torch.distributed as dist
    t = torch.tensor([val], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(world, val, device="cuda"):
    """Sum of a per-rank scalar over the ranks (the job's work)."""
    if world == 1:
        return val
    import torch
    import torch.distributed as dist
    t = torch.tensor([val], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(world, units, ms, device="cuda"):
    """Whole-job throughput of independent replicas: the units all ranks
    processed over the slowest rank's time (units per second)."""
    return reduce_sum(world, units, device) / (reduce_max(world, ms, device) / 1e3)


def replica_inputs(w, n_rhs, rank, field="iid"):
    """The seeded inputs of one rank's replica (phonon field and pseudofermion
    draws); every rank draws its own."""
    if field == "ar1":
        x = hi.phonon_field_ar1(w, corr=1.0 / w.omega0, seed=w.seed + 100 * rank)
    else:
        x = hi.phonon_field(w, seed=w.seed + 100 * rank)
    return x, hi.gaussian_vectors(w, n_rhs, seed=2 + 100 * rank)


class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# CPU baseline: the oracle as it stands (matrix-free C, FP64, OpenMP)
# ----------------------------------------------------------------------------
def cpu_oracle_solves(n_solves, seed_offset=0, with_force=True):
    """Time n_solves single-rhs oracle CG solves (+ force) of the benchmark
    workload. Returns (seconds, iterations list, threads)."""
    from oracle import matfree as MF
    w = WORKLOAD
    x = hi.phonon_field(w, seed=w.seed + seed_offset)
    R = hi.gaussian_vectors(w, n_solves, seed=2 + seed_offset)
    t0 = time.perf_counter()
    its = []
    for k in range(n_solves):
        b = MF.MT_apply(w, x, R[k])
        v, it, res = MF.cg(w, x, b, tol=TOL, max_iter=100000)
        its.append(it)
        if with_force:
            MF.force_fermion(w, x, v, b)
    return time.perf_counter() - t0, its, MF.num_threads()


def cpu_baseline_block(target_s=15.0):
    one, its, thr = cpu_oracle_solves(1)
    n = max(1, min(16, int(target_s / max(one, 1e-3))))
    if n > 1:
        tt, its2, thr = cpu_oracle_solves(n, seed_offset=0)
    else:
        tt, its2 = one, its
    return {"value": n / tt, "unit": "CG solves/s", "cores": thr, "kind": "oracle",
            "sample": f"{n} single-rhs FP64 textbook CG solves (+ force) of the L=32 Ltau=200 "
                      f"workload to residual 1e-8 (matrix-free C oracle, OpenMP), mean "
                      f"{float(np.mean(its2)):.0f} iterations"}


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(a):
    import torch
    import paper_2203_01291_gb300 as hg
    from paper_2203_01291_gb300 import build as hb
    world, rank, local = dist_setup(a.gpus)
    if rank == 0 or world > 1:
        hb.build()
    barrier(world)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = WORKLOAD
    nr = w.n_rhs
    x, R = replica_inputs(w, nr, rank, a.field)
    ctx = hg.Context.from_workload(w, max_rhs=nr)
    xd = torch.tensor(x, device=dev)
    Rd = torch.tensor(R, device=dev)
    bd = torch.empty_like(Rd)
    vd = torch.empty_like(Rd)
    Fd = torch.empty_like(xd)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stats = {"iters": [], "resid": []}

    v0_arn = torch.tensor(hi.site_vector(w, seed=11), device=dev)   # Arnoldi start vector

    def step(xin, Rin, prec=hg.HOL_F32, precond=a.precond, arnoldi=None):
        ctx.set_field(xin)
        if arnoldi is not None:   # Arnoldi bounds (20 steps, 5 % margin) for the preconditioner
            arnoldi.update(ctx.arnoldi_bounds(v0_arn, 20, 0.05, install=True))
        ctx.fermion_matvec(hg.HOL_OP_MT, Rin, bd)
        it, res = ctx.cg_solve(bd, vd, tol=TOL, prec=prec, reliable_every=RELIABLE_EVERY,
                               check_every=10, max_iter=50000, precond=precond)
        ctx.force(vd, bd, Fd, with_bosonic=True)
        return it, res

    ctx.set_field(xd)
    apply_options(ctx, a.option)      # before tuning: the tuner times what the solver runs
    tuned = ctx.tune(nr) if not a.no_tune else None
    apply_options(ctx, a.option)      # explicit shapes win over the tuned ones
    for _ in range(a.warmup):
        flush_l2(flush)
        step(xd, Rd)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ctx.timer_enable(TIMER_STRIDE)
    l0 = hg.hol_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        flush_l2(flush)
        it, res = step(xd, Rd)
        stats["iters"].append(it)
        stats["resid"].append(res)
    e1.record()
    torch.cuda.synchronize()
    launches = hg.hol_launch_count() - l0
    ms_total = e0.elapsed_time(e1)
    op_cnt, op_ms, op_units = ctx.timer_read(hg.TIMER_OPERATOR)
    up_cnt, up_ms, up_units = ctx.timer_read(hg.TIMER_UPDATE)
    fo_cnt, fo_ms, _ = ctx.timer_read(hg.TIMER_FORCE)
    pc_cnt, pc_ms, _ = ctx.timer_read(hg.TIMER_PRECOND)
    if ctx.get_option("fused_cg") and not a.precond:
        ctx_kernel_name = ("k_cg_fused<32> (one kernel per CG iteration: r' = r - alpha q, "
                           "p' = r' + beta p, x += alpha p, q' = M^T M p', partials of "
                           "r'.r', p'.q', r'.q', q'.q')")
    elif ctx.get_option("merged_cg") and not a.precond:
        ctx_kernel_name = ("k_cg_merged (one kernel per CG iteration: p = r + beta p, "
                           "s = w + beta s, x += alpha p every other iteration, "
                           "r' = r - alpha s, w' = M^T M r', r'.r' and |M r'|^2)")
    elif op_avg_ms_hint(op_ms, op_cnt, up_cnt):
        ctx_kernel_name = ("k_cg_persist (fused CG chunk: p = r + beta p, q = M^T M p in shared "
                           "memory, e += alpha p, r -= alpha q; per iteration r, p, e read and "
                           "written once)")
    else:
        kname = {0: "k_cg_mtm32<32>", 1: "k_cg_mtm32_v4<32>", 2: "k_cg_mtm32_v4a<32,2>",
                 3: "k_cg_mtm32_v4s<32,3>", 4: "k_cg_mtm32_split<32,2>",
                 5: "k_cg_mtm32_split<32,4>", 6: "k_cg_mtm32_v4a<32,3>",
                 7: "k_cg_mtm32_tp<32>"}[ctx.get_option("layout")]
        ctx_kernel_name = kname + " (fused p = r + beta p, q = M^T M p, |Mp|^2)"
    ctx.timer_enable(0)
    clk = clocks.stop()
    barrier(world)
    ms_max = reduce_max(world, ms_total)

    iters = np.array(stats["iters"])          # [steps][rhs]
    assert np.all(np.array(stats["resid"]) < TOL)
    solves = a.steps * nr
    value = job_rate(world, solves, ms_total)
    # matvec count: 2 per CG iteration per rhs, M^T for b, 2 per reliable update
    # (counted as one per 50 iterations plus the final certification), 1 in the force
    rel = np.ceil(iters / RELIABLE_EVERY) + 1
    mv = float(np.sum(2 * iters + 1 + 2 * rel + 1))
    total_mv = reduce_sum(world, mv)

    # roofline of the dominant kernel (the CG operator: the merged CG
    # iteration, the persistent fused CG chunk, or the fused M^T M). The
    # library records CUDA events around one in every TIMER_STRIDE launches
    # on the launching stream during the timed region, with each launch's
    # algorithmic bytes (every array read once and written once, plus expV;
    # the tau halo re-reads are not counted).
    op_avg_ms = op_ms / max(op_cnt, 1)
    alg_bytes = op_units / max(op_cnt, 1)
    achieved = op_units / max(op_ms / 1e3, 1e-12) / 1e9
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    traffic = traffic_from_profiles(ctx_kernel_name.split()[0], op_cnt and alg_bytes)

    # The whole CG iteration against the same peak: its algorithmic bytes
    # (operator + vector update, every array once) over the wall time per
    # iteration of the timed steps, which also carries the reliable updates,
    # the polling, the set-up, b = M^T R and the force.
    it_bytes = alg_bytes + (up_units / up_cnt if up_cnt else 0.0)
    it_count = float(np.sum(np.max(iters, axis=1)))   # iterations the loop ran, per step
    it_us = ms_total * 1e3 / it_count
    cg_iteration = {"alg_bytes": it_bytes, "us_per_iteration": it_us,
                    "achieved_gbs": it_bytes / (it_us * 1e-6) / 1e9,
                    "frac": it_bytes / (it_us * 1e-6) / 1e9 / hbm,
                    "note": "operator + update bytes per iteration over the step's wall time per "
                            "iteration (reliable updates, polling, set-up and force included)"}

    # FP64-only path on the same inputs (mixed vs FP64 at equal residual)
    fp64 = None
    if not a.no_fp64:
        step(xd, Rd, prec=hg.HOL_F64)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        ksteps = 2
        f0.record()
        its64 = []
        for _ in range(ksteps):
            flush_l2(flush)
            it64, res64 = step(xd, Rd, prec=hg.HOL_F64)
            its64.append(it64)
            assert np.all(res64 < TOL)
        f1.record()
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / ksteps
        fp64 = {"solves_per_s": nr / (ms64 / 1e3), "ms_per_step": ms64,
                "mean_iters": float(np.mean(its64)),
                "mixed_over_fp64": (solves / (ms_total / 1e3)) / (nr / (ms64 / 1e3))}

    # the dominant kernel cold: one fused M^T M launch after an L2 flush
    cold = cold_operator_block(ctx, xd, nr, flush, hbm)
    rates = unit_rates_block(ctx, xd, vd, bd, Fd, nr, flush, cold)

    # precision of the mixed path against the FP64 path on the same inputs
    prec_err = None if a.no_fp64 else precision_error_block(ctx, xd, Rd, nr)

    # the other solver variant on the same inputs (plain CG <-> preconditioned)
    alt = None
    if not a.no_fp64:
        step(xd, Rd, precond=not a.precond)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        itsa = []
        for _ in range(2):
            flush_l2(flush)
            ita, resa = step(xd, Rd, precond=not a.precond)
            itsa.append(ita)
            assert np.all(resa < TOL)
        f1.record()
        torch.cuda.synchronize()
        msa = f0.elapsed_time(f1) / 2
        alt = {"precond": not a.precond, "solves_per_s": nr / (msa / 1e3), "ms_per_step": msa,
               "mean_iters": float(np.mean(itsa))}
        # the preconditioned solve with the paper's Arnoldi bounds (App. C D)
        # instead of the deterministic norm bounds
        arn = {}
        step(xd, Rd, precond=True, arnoldi=arn)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        itsb = []
        for _ in range(2):
            flush_l2(flush)
            itb, resb = step(xd, Rd, precond=True, arnoldi=arn)
            itsb.append(itb)
            assert np.all(resb < TOL)
        f1.record()
        torch.cuda.synchronize()
        msb = f0.elapsed_time(f1) / 2
        ctx.set_field(xd)
        det = ctx.arnoldi_bounds(v0_arn, 20, 0.0)   # (only to report; not installed)
        alt["arnoldi_bounds"] = {
            "bmin": arn["bmin"], "bmax": arn["bmax"], "steps": arn["steps"],
            "ritz_extremes": [det["bmin"], det["bmax"]],
            "norm_bounds": list(ctx.bounds()),
            "solves_per_s": nr / (msb / 1e3), "ms_per_step": msb,
            "mean_iters": float(np.mean(itsb))}
        # shorter Chebyshev series (a1 < 1 in Eq. (NP_heuristic)), same inputs
        ctx.set_field(xd)
        bs = torch.empty_like(Rd)
        ctx.fermion_matvec(hg.HOL_OP_MT, Rd, bs)
        alt["pcg_short_series"] = short_series_rows(ctx, xd, bs, torch.empty_like(Rd))
        apply_options(ctx, a.option)   # an explicit kpm_a1_percent stays in force

    # end to end through the public API: host (pinned) inputs -> device,
    # solve + force, solutions and force back to host, every step
    xh = torch.tensor(x).pin_memory()
    Rh = torch.tensor(R).pin_memory()
    vh = torch.empty(vd.shape, dtype=torch.float64).pin_memory()
    Fh = torch.empty(Fd.shape, dtype=torch.float64).pin_memory()
    ke = max(1, min(a.steps, 5))
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record()
    for _ in range(ke):
        flush_l2(flush)
        xd.copy_(xh, non_blocking=True)
        Rd.copy_(Rh, non_blocking=True)
        step(xd, Rd)
        vh.copy_(vd, non_blocking=True)
        Fh.copy_(Fd, non_blocking=True)
    g1.record()
    torch.cuda.synchronize()
    ms_e2e = reduce_max(world, g0.elapsed_time(g1) / ke)
    e2e = {"value": reduce_sum(world, nr) / (ms_e2e / 1e3), "unit": "CG solves/s",
           "h2d_bytes_per_step": int(xh.numel() * 8 + Rh.numel() * 8),
           "d2h_bytes_per_step": int(vh.numel() * 8 + Fh.numel() * 8)}

    extra = None
    if not a.no_extra:
        # the other rows are reported beside the headline; a row that fails
        # reports its error instead of taking the headline line down with it
        extra = {}
        for name, leg in (("trajectory", trajectory_pair), ("measurement", measurement_leg),
                          ("global_updates", global_update_leg), ("chains", chains_leg),
                          ("prior_field", prior_field_leg), ("split_sweep", split_sweep_leg)):
            try:
                extra[name] = leg(dev)
            except Exception as e:   # noqa: BLE001
                extra[name] = {"error": f"{type(e).__name__}: {e}"}

    alu = {"fp64_fma_gflops": hg.hol_fma_peak(hg.HOL_F64),
           "fp32_fma_gflops": hg.hol_fma_peak(hg.HOL_F32),
           "how": "project FMA microbenchmark (hol_fma_peak), 2 flops per FMA"}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        cpu = cpu_baseline_block()

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "CG solves/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64",
            "precision": "FP32 operator and CG iterations; FP64 dot products, solution and "
                         "reliable updates; convergence certified by an FP64 true residual",
            "data": "synthetic (seeded i.i.d. Gaussian phonon field and pseudofermion draws)",
            "config": {"workload": "L=32 N=1024 Ltau=200 beta=20 dtau=0.1 t=1 mu=0 omega0=0.5 "
                                   "alpha=1 x~N(0,4), 16 rhs b=M^T R, mixed CG to 1e-8 "
                                   "(reliable update every 50) + force",
                       "field": a.field,
                       "l2": "flushed between steps (256 MB write + read inside the timed loop)",
                       "per_rank": "independent replica, own seeds"},
            "matvecs_per_s": total_mv / (ms_max / 1e3),
            "mean_cg_iters": float(np.mean(iters)),
            "tuned_launch": tuned,
            "options": a.option,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": ctx_kernel_name,
                         "alg_bytes_per_launch": alg_bytes,
                         "avg_launch_ms": op_avg_ms, "launches": op_cnt,
                         "sampling": f"CUDA events around one launch in {TIMER_STRIDE} of the "
                                     f"timed region, on the launching stream (warm: the CG "
                                     f"vectors stay in L2 between launches)",
                         "peak_src": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                         "cold": cold},
            "cg_iteration": cg_iteration,
            "unit_rates": rates,
            "kernel_ms": {"cg_operator": op_ms, "cg_update": up_ms, "force": fo_ms,
                          "precond": pc_ms, "timed_total": ms_total,
                          "timer_stride": TIMER_STRIDE,
                          "recorded_launches": {"cg_operator": op_cnt, "cg_update": up_cnt,
                                                "force": fo_cnt, "precond": pc_cnt}},
            "fp64_compare": fp64,
            "precision_error": prec_err,
            "solver": "preconditioned CG (adiabatic P, FP32)" if a.precond else "plain CG",
            "other_solver": alt,
            "e2e": e2e,
            "other_rows": extra,
            "alu_peaks": alu,
            "gpu_launches": int(launches),
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(strict_json(out)))
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def event_times(fn, flush, launches):
    """Device times (ms) of `fn`, each call alone between two CUDA events on
    the current stream, after an L2 flush (flush=None: no flush, warm)."""
    import torch
    times = []
    for _ in range(launches):
        if flush is not None:
            flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times


def unit_rates_block(ctx, xd, vd, bd, Fd, nr, flush, cold, launches=10):
    """The per-unit rates asked beside the solve rate, each launch timed alone
    after an L2 flush: fermion matvecs/s (one M or M^T on one right-hand
    side; the fused FP32 M^T M counts two) in FP32 and FP64, and forces/s
    (the force of one pseudofermion; one call computes nr of them plus the
    bosonic term, with the solutions of the last benchmark step)."""
    import torch
    import paper_2203_01291_gb300 as hg
    ctx.set_field(xd)
    v64 = torch.tensor(hi.gaussian_vectors(WORKLOAD, nr, seed=5), device="cuda")
    o64 = torch.empty_like(v64)
    out = {"fp32_fused_mtm_matvecs_per_s": 2 * nr / (cold["median_us"] / 1e6),
           "fp32_fused_mtm_matvecs_per_s_streaming": 2 * nr / (cold["stream_us"] / 1e6)}
    fp64_peak = hg.hol_fma_peak(hg.HOL_F64)   # GFLOP/s, the FP64 roofline of these kernels
    for name, op in (("fp64_M", hg.HOL_OP_M), ("fp64_MT", hg.HOL_OP_MT)):
        ctx.fermion_matvec(op, v64, o64)
        ms = statistics.median(event_times(lambda: ctx.fermion_matvec(op, v64, o64), flush,
                                           launches))
        out[name + "_us"] = ms * 1e3
        out[name + "_matvecs_per_s"] = nr / (ms / 1e3)
        # 10 algorithmic flops per element (4 checkerboard colours, one FMA per
        # site each; the D term's multiply and add)
        out[name + "_frac_of_fp64_fma"] = 10.0 * nr * ctx.n / (ms / 1e3) / 1e9 / fp64_peak
    ctx.force(vd, bd, Fd, with_bosonic=True)
    ms = statistics.median(event_times(lambda: ctx.force(vd, bd, Fd, with_bosonic=True),
                                       flush, launches))
    out["force_us"] = ms * 1e3
    out["forces_per_s"] = nr / (ms / 1e3)
    out["fp64_fma_gflops"] = fp64_peak
    out["note"] = ("cold single launches (L2 flushed before each); the FP32 figures are the "
                   "cold operator block's, single and streaming; the FP64 fractions count 10 "
                   "flops per element against the measured FP64 FMA rate")
    return out


def cold_operator_block(ctx, xd, nr, flush, hbm, launches=20):
    """The fused FP32 M^T M (the CG operator kernel, here without the
    direction update) on nr right-hand sides, each launch timed alone with
    CUDA events after an L2 flush (cold). Two units of algorithmic bytes:
    the operator's own (v in, q out, expV: nr n 8 B + n 4 B, which is also
    the matvec unit of one M apply on nr rhs), and the bytes the CG
    iteration's launch moves (r and p_old in, p_new and q out: nr n 16 B +
    n 4 B). Beside it: the floor of such a measurement (the same kernel on
    64 sites after the same flush, the same without the flush, and a
    128-element torch kernel after the flush) and the same operator on 64
    right-hand sides (launch shapes tuned for 64), where the floor weighs
    four times less."""
    import torch
    import paper_2203_01291_gb300 as hg
    n = ctx.n
    v = torch.tensor(hi.gaussian_vectors(WORKLOAD, nr, seed=5), device="cuda",
                     dtype=torch.float32)
    q = torch.empty_like(v)
    for _ in range(3):
        ctx.fermion_matvec(hg.HOL_OP_MTM, v, q)
    times = event_times(lambda: ctx.fermion_matvec(hg.HOL_OP_MTM, v, q), flush, launches)
    ms = statistics.median(times)
    # two launches on different inputs after the flush: the second one meets
    # cold data (its own v, q and the evicted expV rows are not in L2) but
    # not the cold start of the first (kernel code, parameters, TLB)
    v2 = torch.tensor(hi.gaussian_vectors(WORKLOAD, nr, seed=7), device="cuda",
                      dtype=torch.float32)
    q2 = torch.empty_like(v2)

    def pair():
        ctx.fermion_matvec(hg.HOL_OP_MTM, v, q)
        ctx.fermion_matvec(hg.HOL_OP_MTM, v2, q2)

    ms_pair = statistics.median(event_times(pair, flush, launches))
    # a run of launches over eight different input sets after the flush
    # (216 MB of inputs and outputs, more than L2): every launch streams cold
    # data; the run's time over its launches is not limited by the event
    # resolution (about 0.5 us) as a single short launch is
    n_set = 8
    vs = [torch.tensor(hi.gaussian_vectors(WORKLOAD, nr, seed=20 + j), device="cuda",
                       dtype=torch.float32) for j in range(n_set)]
    qs = [torch.empty_like(vj) for vj in vs]

    def run():
        for vj, qj in zip(vs, qs):
            ctx.fermion_matvec(hg.HOL_OP_MTM, vj, qj)

    ms_run = statistics.median(event_times(run, flush, max(5, launches // 4))) / n_set
    del vs, qs
    unit = nr * n * 8.0 + n * 4.0
    cg_bytes = nr * n * 16.0 + n * 4.0
    # the floor of one event-bracketed launch of the same kernel: the fused
    # M^T M on a 1-rhs L=8, Ltau=2 lattice (64 sites)
    tiny = hg.Context(L=8, Ltau=2, max_rhs=1)
    try:
        tiny.set_field(torch.zeros(2, 64, dtype=torch.float64, device="cuda"))
        tv = torch.ones(1, 2, 64, dtype=torch.float32, device="cuda")
        tq = torch.empty_like(tv)
        for _ in range(3):
            tiny.fermion_matvec(hg.HOL_OP_MTM, tv, tq)
        floor = event_times(lambda: tiny.fermion_matvec(hg.HOL_OP_MTM, tv, tq), flush, launches)
        floor_warm = event_times(lambda: tiny.fermion_matvec(hg.HOL_OP_MTM, tv, tq), None,
                                 launches)
    finally:
        tiny.close()
    small = torch.zeros(128, dtype=torch.float32, device="cuda")
    floor_torch = event_times(lambda: small.add_(1.0), flush, launches)
    floor_ms = statistics.median(floor)

    def ceiling(unit_bytes):
        return unit_bytes / (floor_ms / 1e3 + unit_bytes / (hbm * 1e9)) / 1e9 / hbm

    rhs64 = None
    if nr < 64:
        nr64 = 64
        v64 = torch.tensor(hi.gaussian_vectors(WORKLOAD, nr64, seed=6), device="cuda",
                           dtype=torch.float32)
        q64 = torch.empty_like(v64)
        with hg.Context.from_workload(WORKLOAD, max_rhs=nr64) as c64:
            c64.set_field(xd)
            tuned64 = c64.tune(nr64)
            for _ in range(3):
                c64.fermion_matvec(hg.HOL_OP_MTM, v64, q64)
            t64 = event_times(lambda: c64.fermion_matvec(hg.HOL_OP_MTM, v64, q64), flush,
                              launches)
        ms64 = statistics.median(t64)
        unit64 = nr64 * n * 8.0 + n * 4.0
        rhs64 = {"rhs": nr64, "median_us": ms64 * 1e3, "unit_bytes": unit64,
                 "achieved_gbs": unit64 / (ms64 / 1e3) / 1e9,
                 "frac": unit64 / (ms64 / 1e3) / 1e9 / hbm, "frac_ceiling": ceiling(unit64),
                 "frac_beyond_floor": (unit64 / ((ms64 - floor_ms) / 1e3) / 1e9 / hbm
                                       if ms64 > floor_ms else None),
                 "tuned_launch": tuned64}
        del v64, q64
    return {"rhs": nr, "median_us": ms * 1e3, "min_us": min(times) * 1e3,
            "unit_bytes": unit, "achieved_gbs": unit / (ms / 1e3) / 1e9,
            "frac": unit / (ms / 1e3) / 1e9 / hbm,
            "cg_launch_bytes": cg_bytes,
            "launch_floor_us": floor_ms * 1e3,
            "launch_floor_warm_us": statistics.median(floor_warm) * 1e3,
            "torch_kernel_floor_us": statistics.median(floor_torch) * 1e3,
            "frac_ceiling": ceiling(unit),
            "frac_beyond_floor": (unit / ((ms - floor_ms) / 1e3) / 1e9 / hbm
                                  if ms > floor_ms else None),
            "stream_us": ms_run * 1e3, "stream_frac": unit / (ms_run / 1e3) / 1e9 / hbm,
            "second_launch_us": (ms_pair - ms) * 1e3,
            "second_launch_frac": (unit / ((ms_pair - ms) / 1e3) / 1e9 / hbm
                                   if ms_pair > ms else None),
            "rhs64": rhs64,
            "note": "median of single launches after a 256 MB L2 flush; frac by the operator's "
                    "algorithmic bytes (v in, q out, expV), of measured HBM; launch_floor_us: "
                    "the same kernel on 64 sites, timed the same way; torch_kernel_floor_us: a "
                    "128-element torch add after the same flush (the floor is the platform's, "
                    "not the kernel's); launch_floor_warm_us: the 64-site kernel without the "
                    "flush, where the GPU is idle when the first event is recorded and waits "
                    "for the host's launch call (so it measures the host path; with the flush "
                    "queued first the kernel is already queued when the event fires); "
                    "frac_ceiling: the fraction a launch with that floor would reach moving "
                    "the bytes at peak; frac_beyond_floor: the bytes over the launch's time "
                    "beyond the floor; second_launch_*: a second launch on other inputs right "
                    "after the first, from the same flush (cold data, warm start), timed as "
                    "the difference of the pair and the single launch; stream_*: eight "
                    "launches on eight different input sets after the flush (216 MB, more "
                    "than L2), per launch: every launch streams cold data"}


def precision_error_block(ctx, xd, Rd, nr):
    """Error of the mixed path against the FP64 path (itself compared with
    the FP64 oracle element by element in the tests) on the benchmark's own
    inputs: the solution and the force at the benchmark's residual 1e-8, and
    the force after refining the mixed solve to 1e-11 (max norm, relative to
    the FP64 result at 1e-12)."""
    import torch
    import paper_2203_01291_gb300 as hg
    b = torch.empty_like(Rd)
    ctx.set_field(xd)
    ctx.fermion_matvec(hg.HOL_OP_MT, Rd, b)
    out = {}

    def solve(prec, tol):
        v = torch.empty_like(b)
        F = torch.empty(xd.shape, dtype=torch.float64, device=xd.device)
        _, res = ctx.cg_solve(b, v, tol=tol, prec=prec, reliable_every=RELIABLE_EVERY,
                              check_every=10, max_iter=200000)
        ctx.force(v, b, F, with_bosonic=False)
        return v, F, float(np.max(res))

    def rel(a, r):
        return float((a - r).abs().max() / r.abs().max())

    v64, F64, r64 = solve(hg.HOL_F64, 1e-8)
    v32, F32, r32 = solve(hg.HOL_F32, 1e-8)
    out["at_1e-8"] = {"solution_rel": rel(v32, v64), "force_rel": rel(F32, F64),
                      "true_residual_mixed": r32, "true_residual_fp64": r64}
    v64t, F64t, _ = solve(hg.HOL_F64, 1e-12)
    v32t, F32t, r32t = solve(hg.HOL_F32, 1e-11)
    out["refined"] = {"mixed_tol": 1e-11, "fp64_tol": 1e-12, "force_rel": rel(F32t, F64t),
                      "solution_rel": rel(v32t, v64t), "true_residual_mixed": r32t,
                      "target_force_rel": 1e-7}
    out["note"] = ("max-norm relative differences from the FP64 path on the same inputs; the "
                   "FP64 path matches the FP64 oracle to 1e-12 in the tests")
    return out


def trajectory_leg(dev, n_traj=5, options=(), prec=None):
    """Algorithm 1 on the hmc16 workload: L=16, Ltau=160, alpha=1.5, omega0=1,
    x ~ N(0.5, 1), two pseudofermions, N_t=20, n_t=4, dt=0.01, m_reg=omega0,
    adiabatic preconditioner, force solves to 1e-5 and the action solve to
    1e-10 (Sec. VI B), in mixed precision (prec HOL_F32) or all FP64 (HOL_F64,
    the precision the workload states). One untimed trajectory, then n_traj
    trajectories each timed with CUDA events on the stream (mean and spread
    over them). Every trajectory's final action solve is certified to 1e-10
    by the FP64 true residual, so both precisions end at the same residual."""
    import torch
    import paper_2203_01291_gb300 as hg
    prec = hg.HOL_F32 if prec is None else prec
    w = hi.WORKLOADS["hmc16"]
    o = hg.md_opts(0.01, 20, 4, w.omega0, force_tol=1e-5, action_tol=1e-10,
                   prec=prec, precond=True)
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        x = torch.tensor(hi.phonon_field(w), device=dev)
        ctx.set_field(x)
        ctx.tune(2)                   # launch shapes for 2 rhs (outside the timed region)
        apply_options(ctx, options)
        u = hi.uniforms(n_traj + 2, seed=77)
        acc, dhs, times = [], [], []
        # trajectory 0 warms up, 1..n_traj are timed, the last one (untimed)
        # samples per-launch durations of the kernel classes
        for k in range(n_traj + 2):
            R = torch.tensor(hi.gaussian_vectors(w, 2, seed=300 + k), device=dev)
            Rp = torch.tensor(hi.gaussian_vectors(w, 1, seed=400 + k)[0], device=dev)
            if k == n_traj + 1:
                torch.cuda.synchronize()
                ctx.timer_enable(LEG_TIMER_STRIDE)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            a_, dh, _ = ctx.fourier_accel_leapfrog(x, R, Rp, o, float(u[k]))
            e1.record()
            torch.cuda.synchronize()
            if 1 <= k <= n_traj:
                acc.append(a_)
                dhs.append(dh)
                times.append(e0.elapsed_time(e1))
        # average launch durations of the solver's kernel classes (one launch in
        # LEG_TIMER_STRIDE is bracketed by CUDA events on the launching stream)
        avg_us = {}
        for name, klass in (("cg_operator", hg.TIMER_OPERATOR), ("cg_update", hg.TIMER_UPDATE),
                            ("precond", hg.TIMER_PRECOND), ("force", hg.TIMER_FORCE)):
            cnt, tot, _ = ctx.timer_read(klass)
            avg_us[name] = 1e3 * tot / cnt if cnt else None
        ctx.timer_enable(0)
    ms = float(np.mean(times))
    return {"workload": "hmc16 L=16 Ltau=160, N_t=20 n_t=4 dt=0.01, PCG "
                        + ("mixed" if prec == hg.HOL_F32 else "FP64")
                        + ", forces to 1e-5, action to 1e-10",
            "precision": "mixed" if prec == hg.HOL_F32 else "fp64",
            "trajectories_per_s": 1e3 / ms, "ms_per_trajectory": ms,
            "ms_min": float(np.min(times)), "ms_max": float(np.max(times)),
            "ms_std": float(np.std(times)), "repeats": n_traj,
            "accepted": int(sum(acc)), "of": n_traj, "mean_abs_dH": float(np.mean(np.abs(dhs))),
            "dH": [float(d) for d in dhs],
            "avg_launch_us": avg_us}


def trajectory_pair(dev, n_traj=5):
    """The hmc16 trajectory row in both precisions at equal final residual,
    and their rate ratio (mixed over FP64); beside them the mixed trajectory
    with the first Chebyshev order constant a1 = 0.5 instead of the paper's
    1 (Eq. (NP_heuristic): a shorter series, a cheaper P^-1)."""
    import paper_2203_01291_gb300 as hg
    mixed = trajectory_leg(dev, n_traj, prec=hg.HOL_F32)
    fp64 = trajectory_leg(dev, n_traj, prec=hg.HOL_F64)
    short = trajectory_leg(dev, n_traj, options=("kpm_a1_percent=50",), prec=hg.HOL_F32)
    return {"mixed": mixed, "fp64": fp64,
            "mixed_over_fp64": mixed["trajectories_per_s"] / fp64["trajectories_per_s"],
            "mixed_a1_0.5": {k: short[k] for k in ("trajectories_per_s", "ms_per_trajectory",
                                                   "ms_min", "ms_max", "accepted", "of",
                                                   "mean_abs_dH", "avg_launch_us")}}


def measurement_leg(dev, n_rv=128, repeats=3):
    """Stochastic Green's function (2-point and the type-2 Wick product) of one
    L=28, Ltau=120 chain (beta=12, omega0=1, alpha=1, x ~ N(0, 1)) with 128
    Z2 probes solved in mixed precision to 1e-8 (`repeats` timed measurements
    of the same probes, mean and spread)."""
    import torch
    import paper_2203_01291_gb300 as hg
    w = hi.Workload("chain28", L=28, Ltau=120, omega0=1.0, alpha=1.0, seed=1047)
    # all probes in one block solve (127 ms against 244 ms in blocks of 16)
    with hg.Context.from_workload(w, max_rhs=n_rv) as ctx:
        ctx.set_field(torch.tensor(hi.phonon_field(w), device=dev))
        tuned = ctx.tune(n_rv)        # launch shapes for the probe block (outside the timing)
        xi = torch.tensor(hi.z2_vectors(w, n_rv, seed=5), device=dev)
        Gxi = torch.empty_like(xi)
        G2 = torch.empty(2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=dev)
        G4 = torch.empty(3, 2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=dev)
        ctx.stochastic_measure(xi[:16].contiguous(), Gxi[:16], G2, G4, 2, tol=1e-8,
                               prec=hg.HOL_F32)
        torch.cuda.synchronize()
        times = []
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            its = ctx.stochastic_measure(xi, Gxi, G2, G4, 2, tol=1e-8, prec=hg.HOL_F32)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.mean(times))
    return {"workload": f"L=28 Ltau=120 chain, {n_rv} Z2 probes, 2-point + type-2 Wick",
            "probes": n_rv, "measurements_per_s": 1e3 / ms, "ms_per_measurement": ms,
            "ms_min": float(np.min(times)), "ms_max": float(np.max(times)), "repeats": repeats,
            "mean_cg_iters": float(np.mean(its)), "tuned_launch": tuned}


def chains_leg(dev, n_rv=128, precs=None, repeats=3):
    """The batching configuration: 48 independent chains of uneven size
    (L in {8, 12, 16, 20, 24, 28}, 8 each, Ltau=120, beta=12, omega0=1,
    alpha=1, x ~ N(0, 1) per chain seed). One HMC trajectory per chain
    (Algorithm 1: N_t=20, n_t=4, dt=0.01, adiabatic PCG, forces to 1e-5,
    action to 1e-10 certified by the FP64 true residual) in mixed precision
    and in FP64 (each `repeats` times from the same start, mean and spread),
    and one stochastic measurement per chain (128 Z2 probes, 2-point
    function, mixed CG to 1e-8), each chain on its own stream, all chains
    concurrent (hmc_batch / measure_batch)."""
    import torch
    import paper_2203_01291_gb300 as hg
    precs = (hg.HOL_F32, hg.HOL_F64) if precs is None else precs
    ws = hi.chain_workloads(8, 120)
    # all 128 probes of a chain in one block solve (23.8 against 22.8
    # measurements/s in blocks of 64, 19.1 in blocks of 16)
    ctxs = [hg.Context.from_workload(w, max_rhs=n_rv) for w in ws]
    out = {"workload": "48 chains, L in {8..28} x 8, Ltau=120; one trajectory (N_t=20, n_t=4, "
                       "PCG, forces 1e-5, action 1e-10) per chain in each precision (graph "
                       "path; the host-thread path for comparison), and one 128-probe "
                       "measurement per chain (mixed, 1e-8; graph path and host-thread path)"}
    try:
        x0 = [hi.phonon_field(w) for w in ws]
        xs = [torch.tensor(x, device=dev) for x in x0]
        for c, x in zip(ctxs, xs):    # launch shapes per lattice (outside the timed region)
            c.set_field(x)
            c.tune(2)
        Rs = [torch.tensor(hi.gaussian_vectors(w, 2, seed=w.seed + 1), device=dev) for w in ws]
        Rps = [torch.tensor(hi.gaussian_vectors(w, 1, seed=w.seed + 2)[0], device=dev)
               for w in ws]
        u = hi.uniforms(len(ws), seed=903)
        runs = [("graph", p) for p in precs] + [("threads", hg.HOL_F32)]
        for path, prec in runs:
            o = hg.md_opts(0.01, 20, 4, 1.0, force_tol=1e-5, action_tol=1e-10, prec=prec,
                           precond=True)
            times, accs = [], []
            for rep in range(repeats + 1):          # the first pass warms up
                for x, xh in zip(xs, x0):
                    x.copy_(torch.from_numpy(xh))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if path == "graph":
                    acc, dh = hg.hmc_batch_graph(ctxs, xs, Rs, Rps, o, u)
                else:
                    acc, dh = hg.hmc_batch(ctxs, xs, Rs, Rps, o, u, n_threads=8)
                torch.cuda.synchronize()
                if rep:
                    times.append(time.perf_counter() - t0)
                    accs.append(int(np.sum(acc)))
            key = ("mixed" if prec == hg.HOL_F32 else "fp64") + \
                ("" if path == "graph" else "_host_threads")
            t = float(np.mean(times))
            out[key] = {"trajectories_per_s": len(ws) / t, "ms_all_trajectories": t * 1e3,
                        "ms_min": float(np.min(times)) * 1e3, "ms_max": float(np.max(times)) * 1e3,
                        "repeats": repeats, "accepted": accs[-1], "of": len(ws),
                        "mean_abs_dH": float(np.mean(np.abs(dh))),
                        "path": "one captured CUDA graph per leapfrog step over all 48 chains, "
                                "solves device-driven (hmc_batch_graph)" if path == "graph" else
                                "one stream per chain, driven by 8 host threads (hmc_batch)"}
        if "mixed" in out and "fp64" in out:
            out["mixed_over_fp64"] = out["mixed"]["trajectories_per_s"] / \
                out["fp64"]["trajectories_per_s"]
        for c, x in zip(ctxs, xs):
            c.set_field(x)
            c.tune(n_rv)              # shapes for the probe block (outside the timed region)
        xis = [torch.tensor(hi.z2_vectors(w, n_rv, seed=w.seed + 3), device=dev) for w in ws]
        Gxis = [torch.empty_like(xi) for xi in xis]
        G2s = [torch.empty(2 * w.Ltau, w.L, w.L, dtype=torch.float64, device=dev) for w in ws]
        mo = hg.hol_cg_opts(1e-8, 100000, 0, hg.HOL_F32, 50, 10)
        meas = {}
        for path in ("graph", "graph8", "threads"):
            times = []
            for rep in range(2):                    # the first pass warms up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if path == "graph":
                    hg.measure_batch_graph(ctxs, xis, Gxis, G2s, mo)
                elif path == "graph8":   # at most 8 chains in flight
                    hg.measure_batch_graph(ctxs, xis, Gxis, G2s, mo, concurrency=8)
                else:
                    hg.measure_batch(ctxs, xis, Gxis, G2s, mo, n_threads=8)
                torch.cuda.synchronize()
                if rep:
                    times.append(time.perf_counter() - t0)
            meas[path] = float(np.mean(times))
    finally:
        for c in ctxs:
            c.close()
    out.update({"measurements_per_s": len(ws) / meas["graph"],
                "ms_all_measurements": meas["graph"] * 1e3,
                "measurement_path": "all 48 chains' measurements (probe solves device-driven, "
                                    "FFT accumulation) in one captured graph "
                                    "(measure_batch_graph)",
                "measurements_per_s_graph_8_in_flight": len(ws) / meas["graph8"],
                "measurements_per_s_host_threads": len(ws) / meas["threads"]})
    return out


def prior_field_leg(dev, n_rhs=16, repeats=3):
    """The L=32, Ltau=200 workload (omega0=0.5, alpha=1, 16 rhs, mixed CG to
    a certified 1e-8) on a tau-smooth field drawn from the free-phonon law
    exp(-S_B) (holstein_inputs.phonon_field_prior) instead of the i.i.d.
    one: iterations and solves/s with and without the adiabatic
    preconditioner (Sec. VI B; i.i.d. fields are its worst case)."""
    import torch
    import paper_2203_01291_gb300 as hg
    w = WORKLOAD
    x = hi.phonon_field_prior(w, seed=w.seed + 7)
    R = torch.tensor(hi.gaussian_vectors(w, n_rhs, seed=8), device=dev)
    out = {"workload": "L=32 Ltau=200 omega0=0.5 alpha=1, x from exp(-S_B) (tau-smooth), "
                       "16 rhs b = M^T R, mixed CG to 1e-8",
           "x_std": float(np.std(x))}
    with hg.Context.from_workload(w, max_rhs=n_rhs) as ctx:
        xd = torch.tensor(x, device=dev)
        ctx.set_field(xd)
        ctx.tune(n_rhs)
        b = torch.empty_like(R)
        v = torch.empty_like(R)
        ctx.fermion_matvec(hg.HOL_OP_MT, R, b)
        for pc in (False, True):
            ctx.cg_solve(b, v, tol=TOL, prec=hg.HOL_F32, reliable_every=RELIABLE_EVERY,
                         max_iter=50000, precond=pc)
            torch.cuda.synchronize()
            times = []
            for _ in range(repeats):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                its, res = ctx.cg_solve(b, v, tol=TOL, prec=hg.HOL_F32,
                                        reliable_every=RELIABLE_EVERY, max_iter=50000,
                                        precond=pc)
                e1.record()
                torch.cuda.synchronize()
                assert np.all(res < TOL)
                times.append(e0.elapsed_time(e1))
            ms = float(np.mean(times))
            out["pcg" if pc else "cg"] = {"solves_per_s": n_rhs / (ms / 1e3), "ms": ms,
                                          "ms_min": float(np.min(times)),
                                          "ms_max": float(np.max(times)), "repeats": repeats,
                                          "mean_iters": float(np.mean(its))}
        out["pcg_short_series"] = short_series_rows(ctx, xd, b, v)
    out["iteration_ratio"] = out["cg"]["mean_iters"] / out["pcg"]["mean_iters"]
    out["speedup"] = out["pcg"]["solves_per_s"] / out["cg"]["solves_per_s"]
    return out


def short_series_rows(ctx, x, b, v, a1_percents=(50, 25)):
    """The preconditioned solve with the first Chebyshev order constant of
    Eq. (NP_heuristic) below the paper's a1 = 1 (a2 = 1 kept): a shorter
    series is a cheaper P^-1 and, on these fields, also the better
    preconditioner. The constants take effect at the next set_field (which
    recomputes the Chebyshev plan for x). Each row: one warm solve, then one
    timed; the context's a1 is put back to 1 afterwards."""
    import torch
    import paper_2203_01291_gb300 as hg
    rows = {}
    n_rhs = b.shape[0]
    try:
        for a1 in a1_percents:
            ctx.set_option("kpm_a1_percent", a1)
            ctx.set_field(x)
            ctx.cg_solve(b, v, tol=TOL, prec=hg.HOL_F32, reliable_every=RELIABLE_EVERY,
                         max_iter=50000, precond=True)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            its, res = ctx.cg_solve(b, v, tol=TOL, prec=hg.HOL_F32,
                                    reliable_every=RELIABLE_EVERY, max_iter=50000, precond=True)
            e1.record()
            torch.cuda.synchronize()
            assert np.all(res < TOL)
            ms = e0.elapsed_time(e1)
            rows[f"a1={a1 / 100:g}"] = {"solves_per_s": n_rhs / (ms / 1e3), "ms": ms,
                                        "mean_iters": float(np.mean(its))}
    finally:
        ctx.set_option("kpm_a1_percent", 100)
        ctx.set_field(x)
    return rows


def split_sweep_leg(dev, n_traj=4, dts=(0.01, 0.1, 0.2, 0.35)):
    """Acceptance against the number n_t of bosonic sub-steps (Sec. III B,
    time-step splitting): omega0=1, lambda = alpha^2/(omega0^2 W) = 0.25
    (W = 8 t, so alpha = sqrt(2)), beta=4 (Ltau=40), L=16, Fourier
    acceleration off (m_reg = infinity, constant mass dtau), N_t=100 steps,
    two pseudofermions, PCG mixed (forces 1e-5, action 1e-10), fields drawn
    from exp(-S_B) (a fresh one per trajectory). The paper's dt for this
    sweep is not stated: dt = 0.01 is its default; with the constant mass
    the fastest bosonic mode has frequency sqrt(omega0^2 + 4/dtau^2) ~ 20,
    so the leapfrog sub-step dt/n_t is stable for dt/n_t < 0.1: dt = 0.1
    and 0.2 put that edge at n_t = 1 and 2, dt = 0.35 between n_t = 3 and 4
    where the paper sees it. The acceptance estimate is the mean of
    min(1, exp(-dH)); a trajectory whose solves fail counts as rejected."""
    import torch
    import paper_2203_01291_gb300 as hg
    w = hi.Workload("split16", L=16, Ltau=40, omega0=1.0, alpha=float(np.sqrt(2.0)), seed=511)
    res = {"workload": "L=16 Ltau=40 beta=4 omega0=1 lambda=0.25, m_reg=inf, N_t=100, "
                       "fields from exp(-S_B)", "trajectories_per_point": n_traj}
    t0 = time.perf_counter()
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        ctx.set_field(torch.tensor(hi.phonon_field_prior(w), device=dev))
        ctx.tune(2)
        for dt in dts:
            rows = []
            for n_t in range(1, 9):
                # a bounded iteration cap: an unstable trajectory drives the
                # field to extreme values where the solves stop converging
                o = hg.hol_md_opts(dt, 100, n_t, float("inf"),
                                   hg.hol_cg_opts(1e-5, 3000, 1, hg.HOL_F32, 50, 10),
                                   hg.hol_cg_opts(1e-10, 6000, 1, hg.HOL_F32, 50, 10))
                pacc, dhs = [], []
                for k in range(n_traj):
                    x = torch.tensor(hi.phonon_field_prior(w, seed=600 + k), device=dev)
                    R = torch.tensor(hi.gaussian_vectors(w, 2, seed=700 + k), device=dev)
                    Rp = torch.tensor(hi.gaussian_vectors(w, 1, seed=800 + k)[0], device=dev)
                    try:
                        _, dh, _ = ctx.fourier_accel_leapfrog(x, R, Rp, o, 1.0)
                    except hg.HolError:          # an unstable trajectory can blow up the field
                        dh = float("inf")
                    dhs.append(dh)
                    pacc.append(float(min(1.0, np.exp(-dh))) if np.isfinite(dh) else 0.0)
                med = float(np.median(np.abs(dhs)))
                # failed trajectories count as dH = infinity; strict JSON has
                # no infinity, so an infinite median is reported as null
                rows.append({"n_t": n_t, "acceptance": float(np.mean(pacc)),
                             "median_abs_dH": med if np.isfinite(med) else None,
                             "failed": int(sum(not np.isfinite(d) for d in dhs))})
            res[f"dt={dt:g}"] = rows
    res["seconds"] = time.perf_counter() - t0
    return res


def global_update_leg(dev, n_moves=16):
    """Reflection and swap updates (Sec. IV) on the hmc16 workload: L=16,
    Ltau=160, alpha=1.5, x ~ N(0.5, 1), two pseudofermion fields, alternating
    single-site reflections and nearest-neighbour swaps at random sites, each
    with one tight action solve (mixed precision, certified 1e-10)."""
    import torch
    import paper_2203_01291_gb300 as hg
    w = hi.WORKLOADS["hmc16"]
    rng = np.random.default_rng(901)
    with hg.Context.from_workload(w, max_rhs=2) as ctx:
        x = torch.tensor(hi.phonon_field(w), device=dev)
        R = torch.tensor(hi.gaussian_vectors(w, 2, seed=902), device=dev)
        Phi = torch.empty_like(R)
        ctx.set_field(x)
        ctx.tune(2)                   # launch shapes for 2 rhs (outside the timed region)
        ctx.pseudofermion_phi(R, Phi)
        moves = [(k % 2, int(rng.integers(0, w.N)), float(rng.random())) for k in range(n_moves)]
        acc, dS, S = ctx.global_update(x, Phi, 0, 0, -1, u=0.0, tol=1e-10, prec=hg.HOL_F32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_acc = 0
        for kind, i, u in moves:
            j = (i + 1) % w.L + (i // w.L) * w.L    # x-neighbour
            acc, dS, S = ctx.global_update(x, Phi, kind, i, j, u=u, tol=1e-10, prec=hg.HOL_F32,
                                           S_cur=S)
            n_acc += int(acc)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    return {"workload": "hmc16 L=16 Ltau=160, 2 pseudofermions, alternating reflections and "
                        "neighbour swaps, action solve mixed to 1e-10",
            "updates_per_s": n_moves / dt, "ms_per_update": dt / n_moves * 1e3,
            "accepted": n_acc, "of": n_moves}


KERNEL_HEADERS = ("cb.cuh", "cb4.cuh")   # device helpers of the operator kernels


def kernel_source_digest(kernel):
    """Digest of a kernel's own source text (its __global__ definition in
    csrc/) and of the device helper headers it uses: a profile taken on other
    sources no longer describes the running kernel."""
    import glob
    import hashlib
    import re
    name = kernel.split("<")[0]
    # (launch bounds may hold one level of parentheses: sizeof(R) == 4 ? 4 : 2)
    pat = re.compile(r"__global__ void(?: __launch_bounds__\((?:[^()]|\([^()]*\))*\))? "
                     + re.escape(name) + r"\(")
    csrc = os.path.join(ROOT, "paper_2203_01291_gb300", "csrc")
    h = hashlib.sha256()
    for hname in KERNEL_HEADERS:
        with open(os.path.join(csrc, hname), "rb") as f:
            h.update(f.read())
    for path in sorted(glob.glob(os.path.join(csrc, "*.cu"))):
        src = open(path).read()
        m = pat.search(src)
        if not m:
            continue
        start = src.rfind("template <", 0, m.start())
        if start < 0 or src.find(";", start, m.start()) >= 0:
            start = m.start()
        depth, k = 0, src.index("{", m.end())
        while True:
            if src[k] == "{":
                depth += 1
            elif src[k] == "}":
                depth -= 1
                if depth == 0:
                    break
            k += 1
        h.update(src[start:k + 1].encode())
        return h.hexdigest()[:12]
    return None


def traffic_from_profiles(kernel, alg_bytes):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    of `kernel` from a committed ncu summary: a line
    `traffic_per_launch: <kernel> <source digest> <bytes> <alg bytes>` in
    profiles/*.md, scaled to this run's algorithmic bytes per launch. None
    when no summary matches the current kernel sources."""
    import glob
    digest = kernel_source_digest(kernel)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            if not line.startswith("traffic_per_launch:"):
                continue
            parts = line.split()
            if len(parts) < 5 or parts[1] != kernel or parts[2] != digest:
                continue
            traffic, prof_alg = float(parts[3]), float(parts[4])
            return traffic * (alg_bytes / prof_alg) if alg_bytes else traffic
    return None


def strict_json(obj):
    """A copy of obj with every non-finite float replaced by None: the line
    must parse as strict JSON, which has no NaN or infinity."""
    if isinstance(obj, float):
        return obj if np.isfinite(obj) else None
    if isinstance(obj, dict):
        return {k: strict_json(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [strict_json(v) for v in obj]
    return obj


def flush_l2(buf):
    """Evict the working set from L2: write a buffer larger than L2, then
    read it back, so that L2 ends up holding clean lines of the buffer (the
    next kernel then pays no write-back of the flush's dirty lines)."""
    buf.zero_()
    buf.sum()


def apply_options(ctx, options):
    """NAME=VALUE launch options (hol_set_option)."""
    for opt in options:
        name, val = opt.split("=")
        ctx.set_option(name, int(val))


def op_avg_ms_hint(op_ms, op_cnt, up_cnt):
    """The persistent path records no separate update launches."""
    return op_cnt > 0 and up_cnt == 0


def run_matvec(a):
    """Fused FP32 M^T M alone on `rhs` right-hand sides, cold L2 per launch."""
    import torch
    import paper_2203_01291_gb300 as hg
    from paper_2203_01291_gb300 import build as hb
    hb.build()
    torch.cuda.set_device(0)
    w = WORKLOAD
    nr = a.rhs
    ctx = hg.Context.from_workload(w, max_rhs=nr)
    ctx.set_field(torch.tensor(hi.phonon_field(w), device="cuda"))
    apply_options(ctx, a.option)
    tuned = ctx.tune(nr) if not a.no_tune else None
    apply_options(ctx, a.option)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    if a.prec == "f64":
        run_matvec64(a, ctx, w, nr, flush, tuned)
        return
    v = torch.tensor(hi.gaussian_vectors(w, nr, seed=5), device="cuda", dtype=torch.float32)
    q = torch.empty_like(v)
    for _ in range(a.warmup):
        ctx.fermion_matvec(hg.HOL_OP_MTM, v, q)
    times = []
    for _ in range(a.steps):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.fermion_matvec(hg.HOL_OP_MTM, v, q)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    alg = nr * w.n * 4 * 2 + w.n * 4          # v in, q out, expV
    hbm = peaks().get("hbm_gbs", 6800.0)
    print(json.dumps({"mode": "matvec", "rhs": nr, "median_ms": ms, "tuned_launch": tuned,
                      "options": a.option,
                      "alg_bytes": alg, "achieved_gbs": alg / (ms / 1e3) / 1e9,
                      "frac_of_measured_hbm": alg / (ms / 1e3) / 1e9 / hbm,
                      "matvecs_per_s": 2 * nr / (ms / 1e3)}))
    ctx.close()


def run_matvec64(a, ctx, w, nr, flush, tuned):
    """FP64 M and M^T alone on nr right-hand sides (the operators of the FP64
    solver and of the mixed solver's reliable updates), each launch timed
    alone after an L2 flush. ALU-bound on this part: algorithmic flops per
    element 10 for either (C: 4 colours x one FMA per site; D and the sign
    term: one multiply and one add), against the measured FP64 FMA rate."""
    import torch
    import paper_2203_01291_gb300 as hg
    v = torch.tensor(hi.gaussian_vectors(w, nr, seed=5), device="cuda")
    out = torch.empty_like(v)
    peak = hg.hol_fma_peak(hg.HOL_F64)
    res = {"mode": "matvec", "prec": "f64", "rhs": nr, "tuned_launch": tuned,
           "options": a.option, "flops_per_element": 10, "fp64_fma_gflops": peak}
    for name, op in (("M", hg.HOL_OP_M), ("MT", hg.HOL_OP_MT)):
        for _ in range(a.warmup):
            ctx.fermion_matvec(op, v, out)
        ms = statistics.median(event_times(lambda: ctx.fermion_matvec(op, v, out), flush,
                                           a.steps))
        gf = 10.0 * nr * w.n / (ms / 1e3) / 1e9
        res[name] = {"median_us": ms * 1e3, "gflops": gf, "frac_of_fp64_fma": gf / peak}
    print(json.dumps(strict_json(res)))
    ctx.close()


def run_precond(a):
    """z = P^{-1} P^{-T} r (FP32 and FP64) on `rhs` right-hand sides, cold L2."""
    import torch
    import paper_2203_01291_gb300 as hg
    from paper_2203_01291_gb300 import build as hb
    hb.build()
    torch.cuda.set_device(0)
    w = WORKLOAD
    if a.lattice:
        L, T = (int(t) for t in a.lattice.lower().split("x"))
        w = hi.Workload(f"chain{L}", L=L, Ltau=T, omega0=1.0, alpha=1.0, x_std=1.0, seed=1000 + L)
    nr = a.rhs
    ctx = hg.Context.from_workload(w, max_rhs=nr)
    ctx.set_field(torch.tensor(hi.phonon_field(w), device="cuda"))
    apply_options(ctx, a.option)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    res = {"mode": "precond", "lattice": f"L={w.L} Ltau={w.Ltau}", "rhs": nr,
           "options": list(a.option), "kpm_registers": ctx.get_option("kpm_registers")}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        v = torch.tensor(hi.gaussian_vectors(w, nr, seed=5), device="cuda", dtype=dt)
        z = torch.empty_like(v)
        for _ in range(a.warmup):
            ctx.precond_apply(hg.HOL_PINV_PINVT, v, z)
        times = []
        for _ in range(a.steps):
            flush_l2(flush)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.precond_apply(hg.HOL_PINV_PINVT, v, z)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        res[name + "_median_ms"] = statistics.median(times)
    print(json.dumps(strict_json(res)))
    ctx.close()


# ----------------------------------------------------------------------------
# reference arm: the oracle as it stands, timed on the host cores
# ----------------------------------------------------------------------------
def run_reference(a):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import matfree as MF
    MF.build()
    for k in range(a.warmup):
        cpu_oracle_solves(1, seed_offset=1000 + k)
    t0 = time.perf_counter()
    its = []
    for k in range(a.steps):
        _, it, thr = cpu_oracle_solves(1, seed_offset=k)
        its += it
    dt = time.perf_counter() - t0
    value = a.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "CG solves/s",
           "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "L=32 N=1024 Ltau=200 beta=20 omega0=0.5 alpha=1, "
                                  "one rhs per step, FP64 CG to 1e-8 + force"},
           "cpu_baseline": {"value": value, "unit": "CG solves/s", "cores": MF.num_threads(),
                            "kind": "oracle",
                            "sample": f"{a.steps} single-rhs solves, mean "
                                      f"{float(np.mean(its)):.0f} iterations"},
           "e2e": {"value": value, "unit": "CG solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(strict_json(out)))


def run_leg(a):
    """One of the other rows of the JSON line alone (for profiling)."""
    import torch
    from paper_2203_01291_gb300 import build as hb
    hb.build()
    torch.cuda.set_device(0)
    legs = {"trajectory": lambda: trajectory_leg("cuda", n_traj=1, options=a.option),
            "trajectory64": lambda: trajectory_leg("cuda", n_traj=1, options=a.option,
                                                   prec=0),
            "measurement": lambda: measurement_leg("cuda"),
            "measurement32": lambda: measurement_leg("cuda", n_rv=32),
            "global": lambda: global_update_leg("cuda"),
            "chains": lambda: chains_leg("cuda", repeats=1),
            "prior": lambda: prior_field_leg("cuda"),
            "split": lambda: split_sweep_leg("cuda")}
    print(json.dumps(strict_json({"mode": "leg", "leg": a.leg, **legs[a.leg]()})))


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "matvec":
        run_matvec(a)
    elif a.mode == "precond":
        run_precond(a)
    elif a.mode == "leg":
        run_leg(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
