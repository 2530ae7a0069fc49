"""Benchmark: particle-forces/s of the momentum-conserving FMM + HHS step on one GB300.

Workload (default, the largest single-GPU FMM + HHS configuration): an isolated disk galaxy,
N = 2^22 -- exponential disk (R_d = 3, z0 = 0.3, 10 %, velocities from Jeans moments with Toomre
Q = 1.5), Hernquist bulge (5 %), NFW halo (c = 10, 85 %) -- Wendland C2 softening eps = 0.02, p = 6,
theta = 0.6, kappa = 1, float32 P2P/M2L, HHS with eta = 0.025, dt_max = 2 and k_max = 14 (the
initial galaxy then spans rungs 0-6).  `--workload collapse` selects the cold collapse of a uniform
sphere (N = 2^20, eps = 0.005, p = 6, theta = 0.5, dt_max = 1/16, k_max = 10), whose t = 0 step is
also reported beside the headline.

One step = one rung-0 step of EVOLVE_HOLD (every stage of the hot path: keys, sort, octree,
P2M/M2M, walk, M2L, P2P, L2L/L2P, timestep split, kicks, drifts), starting each time from the
same initial state.  A particle-force is one sink's acceleration from one FMM evaluation.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-forces/s (FMM+HHS, 1 GB300) at median force err <=1e-4; |sum m v| drift"
FP32_LANES_PER_SM = 128

WORKLOADS = {
    "disk": dict(
        n=1 << 22, seed=1003,
        desc="isolated disk galaxy N={n}: exponential disk (Rd=3, z0=0.3, 10%, Jeans velocities, Toomre Q=1.5) + "
             "Hernquist bulge (5%) + NFW halo (c=10, 85%), eps=0.02 Wendland C2, p=6, theta=0.6, fp32 P2P/M2L, "
             "HHS k_max=14 dt_max=2 eta=0.025 (one rung-0 step from t=0)",
        params=dict(p=6, theta=0.6, eps=0.02, kernel=0, n_crit=96, kappa=1.0, eta=0.025, dt_max=2.0, k_max=14)),
    "collapse": dict(
        n=1 << 20, seed=1002,
        desc="cold-collapse uniform sphere N={n}, eps=0.005 Wendland C2, p=6, theta=0.5, fp32 P2P/M2L, "
             "HHS k_max=10 dt_max=1/16 eta=0.025 (one rung-0 step from t=0)",
        params=dict(p=6, theta=0.5, eps=0.005, kernel=0, n_crit=96, kappa=1.0, eta=0.025, dt_max=1.0 / 16, k_max=10)),
}
# the default workload's parameters (the θ/p sweeps and momentum runs keep their own)
PARAMS = WORKLOADS["disk"]["params"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="disk", choices=sorted(WORKLOADS))
    ap.add_argument("--n", type=int, default=0, help="particle count (0: the workload's own)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the cold-collapse t = 0 figures beside the headline")
    ap.add_argument("--evolved", action="store_true",
                    help="also time the cold collapse from an evolved state (untimed evolution to t = 1 first)")
    ap.add_argument("--momentum-contrast", action="store_true",
                    help="run HHS and the traditional integrator to t = --contrast-t on the unit-cube collapse "
                         "and print |sum m v| for both")
    ap.add_argument("--sweep-grid", default="",
                    help="with --sweep: comma-separated theta:p points instead of the default grid")
    ap.add_argument("--sweep", action="store_true",
                    help="theta / p sweep of the unit-cube collapse with HHS and the traditional integrator")
    ap.add_argument("--contrast-n", type=int, default=10000)
    ap.add_argument("--contrast-t", type=float, default=1.0)
    ap.add_argument("--mac", default="side", choices=["side", "sphere"],
                    help="multipole acceptance: the paper's R = kappa*side, or enclosing-sphere radii")
    ap.add_argument("--theta", type=float, default=0.0, help="opening angle (0: the workload's own)")
    ap.add_argument("--eta-tot", type=float, default=0.0,
                    help="eta_1 of the Eq. (9) minimum timestep from the total acceleration (0 = off)")
    ap.add_argument("--no-fp64-plain", action="store_true",
                    help="skip the timing of the plain float64 GPU path beside the float32 one")
    ap.add_argument("--cpu-sample", type=int, default=1024)
    ap.add_argument("--n-crit", type=int, default=0, help="leaf size (0: the workload's own)")
    ap.add_argument("--batched", type=int, default=1, choices=[0, 1],
                    help="1: HOLD steps as one CUDA graph with a device-side work queue (tg_params.batched); "
                         "0: the plain host-driven step")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the workload's leaf size and the default launch shapes (no tg_autotune)")
    ap.add_argument("--eval-only", action="store_true",
                    help="run warmup + steps single FMM evaluations of the workload (for profiler captures)")
    ap.add_argument("--masked", action="store_true", help="with --eval-only: 30%% of the particles in the fast set")
    ap.add_argument("--m2l-form", type=int, default=-1, choices=[-1, 0, 1],
                    help="with --eval-only: float32 harmonic M2L form (0 mutual, 1 directed; -1 the default)")
    return ap.parse_args()


def workload(name, n, seed=None):
    """(pos, vel, mass) of a workload: seeded synthetic inputs (CPU, float64)."""
    from paper_1712_10116_gb300 import ics
    w = WORKLOADS[name]
    seed = w["seed"] if seed is None else seed
    if name == "disk":
        return ics.disk_galaxy(n, seed, velocities=True)
    return ics.uniform_sphere(n, seed)


def run_params(args, name):
    prm = dict(WORKLOADS[name]["params"])
    if args.n_crit:
        prm["n_crit"] = args.n_crit
    if args.theta:
        prm["theta"] = args.theta
    prm["eta_tot"] = args.eta_tot
    prm["mac"] = 1 if args.mac == "sphere" else 0
    prm["batched"] = int(args.batched) if prm["mac"] == 0 and 4 <= prm["p"] <= 6 else 0
    return prm


def combine_ranks(t_dev, sinks, device, world):
    """Whole-job figures of the replicas: the slowest rank's timed seconds and the particle-forces of
    all ranks (every rank integrates its own system)."""
    if world <= 1:
        return t_dev, sinks
    import torch
    import torch.distributed as dist
    mx = torch.tensor([t_dev], dtype=torch.float64, device=device)
    sm = torch.tensor([sinks], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[0])


# ---------------------------------------------------------------- clocks sampler
class Clocks:
    def __init__(self):
        self.samples = []
        self._stop = threading.Event()
        self._th = None

    def start(self):
        def run():
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", os.environ.get("LOCAL_RANK", "0")],
                                         capture_output=True, text=True, timeout=5).stdout.strip()
                    if out:
                        self.samples.append([x.strip() for x in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._th = threading.Thread(target=run, daemon=True)
        self._th.start()

    def stop(self):
        self._stop.set()
        if self._th:
            self._th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------- reference arm: the CPU oracle
def cpu_oracle_rate(name, n, n_sample, args, seed=7):
    import oracle
    pos, _, mass = workload(name, n)
    prm_d = run_params(args, name)
    prm = oracle.params(p=prm_d["p"], theta=prm_d["theta"], eps=prm_d["eps"], kernel=prm_d["kernel"],
                        n_crit=prm_d["n_crit"], kappa=prm_d["kappa"], mac=prm_d["mac"])
    sample = np.random.default_rng(seed).choice(n, n_sample, replace=False)
    t0 = time.perf_counter()
    oracle.fmm_sample(pos, mass, prm, sample)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt, oracle.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload
    n = args.n or WORKLOADS[name]["n"]
    n_sample = max(16, args.cpu_sample // 4)
    times = []
    for i in range(args.warmup + args.steps):
        rate, dt, cores = cpu_oracle_rate(name, n, n_sample, args, seed=100 + i)
        if i >= args.warmup:
            times.append(dt)
    value = n_sample * len(times) / sum(times)
    sample_desc = f"oracle FMM (FP64, C, OpenMP) for {n_sample} random sinks of the N={n} {name} workload per " \
                  f"step, tree + moments of all N included"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-forces/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[name]["desc"].format(n=n), "n": n, "l2": "cpu"},
            "cpu_baseline": {"value": value, "unit": "particle-forces/s", "cores": cores, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": value, "unit": "particle-forces/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
class HHSRun:
    """One bound HHS system on the GPU that can be reset to its initial state between timed steps."""

    def __init__(self, tg, prm, pos0, vel0, mass0, dev, stream):
        import torch
        self.tg = tg
        self.solver = tg.Solver(prm, stream)
        self.P0 = torch.tensor(pos0, device=dev)
        self.V0 = torch.tensor(vel0, device=dev)
        self.M = torch.tensor(mass0, device=dev)
        self.P = self.P0.clone()
        self.V = self.V0.clone()
        self.solver.hhs_init(self.P, self.V, self.M)
        n = self.M.shape[0]
        _, self.aold0, self.acur0, self.atot0 = tg.tg_hhs_state(self.solver.ctx, n, dev, with_total=True)

    def reset(self):
        self.P.copy_(self.P0)
        self.V.copy_(self.V0)
        self.tg.tg_hhs_set_accel(self.solver.ctx, self.aold0, self.acur0, self.atot0)

    def close(self):
        self.solver.close()


def time_hhs_steps(run, steps, warmup, stream, flush, prof_level=1, clocks=None, barrier=None):
    """Warm-up steps, then `steps` timed rung-0 steps (each from the initial state, L2 flushed before
    each); returns (per-step ms list, stats, profile)."""
    import torch
    tg = run.tg
    for _ in range(warmup):
        run.reset()
        run.solver.hhs_step()
    torch.cuda.synchronize()
    tg.tg_set_profiling(run.solver.ctx, prof_level)
    tg.tg_reset_stats(run.solver.ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if barrier:
        barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    for k in range(steps):
        run.reset()
        flush.zero_()
        ev[k][0].record(stream)
        run.solver.hhs_step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if clocks:
        clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    stats = run.solver.stats()
    prof = tg.tg_get_profile(run.solver.ctx)
    tg.tg_set_profiling(run.solver.ctx, 0)
    return step_ms, stats, prof


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1712_10116_gb300 import binding as tg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count

    name = args.workload
    n = args.n or WORKLOADS[name]["n"]
    # replicas only: each rank integrates its own independent system (seed per rank)
    pos0, vel0, mass0 = workload(name, n, seed=WORKLOADS[name]["seed"] + rank)
    prec = tg.TG_PREC_FP32 if args.precision == "fp32" else tg.TG_PREC_FP64
    rp = run_params(args, name)
    prm = tg.Params(precision=prec, **rp)
    run = HHSRun(tg, prm, pos0, vel0, mass0, dev, stream)
    solver = run.solver
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > 129 MB L2
    tuning = None
    if not args.no_autotune and not args.n_crit:
        # step objective: rung-0 steps of the bound system itself (the state is put back after each)
        w0 = time.perf_counter()
        tuning = solver.autotune()
        tuning["wall_s"] = time.perf_counter() - w0
        tuning["objective"] = "one rung-0 HOLD step of the bound system, after one untimed step per setting"

    d_start = solver.diagnostics()
    clocks = Clocks()
    barrier = dist.barrier if world > 1 else None
    wall0 = time.perf_counter()
    step_ms, stats, prof = time_hhs_steps(run, args.steps, args.warmup, stream, flush, 1, clocks, barrier)
    wall = time.perf_counter() - wall0
    d_end = solver.diagnostics()   # the state after the last timed step (one rung-0 step from t = 0)
    # Kernel times: a graph hides its launches from per-launch events, so with the batched step they come
    # from a twin context running the plain host-driven step on the same state with the same tuning (the
    # same kernels, launched one by one): one step timing the M2L and P2P launches, one timing every launch
    timing_source = "timed steps"
    prof_k, stats_k = prof, stats
    twin = None
    if rp.get("batched"):
        twin = HHSRun(tg, tg.Params(precision=prec, **dict(rp, batched=0)), pos0, vel0, mass0, dev, stream)
        tg.tg_set_tuning(twin.solver.ctx, tg.tg_get_tuning(solver.ctx))
        _, stats_k, prof_k = time_hhs_steps(twin, 1, 1, stream, flush, 1)
        timing_source = ("CUDA events around each launch of one untimed plain-path step of the same state, "
                         "tuning and kernels (the batched step runs them inside one graph)")
    prof_run = twin if twin else run
    tg.tg_reset_stats(prof_run.solver.ctx)
    tg.tg_set_profiling(prof_run.solver.ctx, 2)
    prof_run.reset()
    prof_run.solver.hhs_step()
    breakdown = {k: v["ms"] for k, v in tg.tg_get_profile(prof_run.solver.ctx).items() if k != "_all"}
    tg.tg_set_profiling(prof_run.solver.ctx, 0)
    if twin:
        twin.close()
    t_dev = sum(step_ms) / 1e3
    sinks = stats["sink_forces"]
    t_max, sinks_all = combine_ranks(t_dev, float(sinks), dev, world)
    value = sinks_all / t_max

    # accuracy gate: one float32 evaluation of the initial state vs float64 direct summation
    acc, _ = solver.fmm_forces(run.P0, run.M, want_pot=False)
    sample = torch.tensor(np.random.default_rng(3).choice(n, 4096, replace=False), device=dev)
    ad, _ = solver.direct_forces(run.P0, run.M, None, sample)
    a = acc[:, sample]
    err = (torch.linalg.norm(a - ad, dim=0) / torch.linalg.norm(ad, dim=0)).cpu().numpy()

    # end to end through the C ABI with host buffers: pinned H2D of the state, the step, D2H
    hP = run.P0.cpu().pin_memory()
    hV = run.V0.cpu().pin_memory()
    oP = torch.empty_like(hP).pin_memory()
    oV = torch.empty_like(hV).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    tg.tg_reset_stats(solver.ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        run.P.copy_(hP, non_blocking=True)
        run.V.copy_(hV, non_blocking=True)
        tg.tg_hhs_set_accel(solver.ctx, run.aold0, run.acur0, run.atot0)
        solver.hhs_step()
        oP.copy_(run.P, non_blocking=True)
        oV.copy_(run.V, non_blocking=True)
        torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    e2e_sinks = solver.stats()["sink_forces"]
    h2d = 2 * 3 * n * 8
    d2h = 2 * 3 * n * 8

    # the plain float64 path against the float32 path on one evaluation of the whole initial state
    # (same tree and walk; float64 P2P tiles, generic float64 M2L with the potential)
    fp64 = None
    if rank == 0 and prec == tg.TG_PREC_FP32 and not args.no_fp64_plain:
        fp64 = compare_fp64_plain(tg, rp, run, stream, flush)

    extra = {}
    if rank == 0 and not args.no_extra and name != "collapse":
        extra["cold_collapse_t0"] = measure_other(tg, args, "collapse", dev, stream, flush, evolved=False)
    if rank == 0 and not args.no_extra:
        extra["ensemble_64"] = measure_ensemble(tg, dev, stream, flush)
        extra["plummer_4096_fp64"] = measure_plummer(tg, dev, stream)
        extra["clustered_box_fp32_vs_fp64"] = measure_box(tg, dev, stream, flush)
    if rank == 0 and args.evolved:
        extra["cold_collapse_evolved_t1"] = measure_other(tg, args, "collapse", dev, stream, flush, evolved=True)

    if rank != 0:
        run.close()
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    clk = clocks.summary()
    roof = roofline(prof_k, stats_k, rp["p"], sm_count)
    if roof:
        roof["timing"] = timing_source
    cpu = None
    if not args.no_cpu_baseline and (world == 1 or args.gpus == 1):
        rate, dt, cores = cpu_oracle_rate(name, n, args.cpu_sample, args)
        cpu = {"value": rate, "unit": "particle-forces/s", "cores": cores, "kind": "oracle",
               "sample": f"oracle FMM (FP64) of {args.cpu_sample} random sinks of the same N={n} {name} workload, "
                         f"tree + moments of all N included, {dt:.1f} s"}
    mom_scale = float((run.M * run.V0.abs().sum(0)).sum()) or 1.0
    launches = int(prof.get("_all", {}).get("launches", 0))
    line = {
        "metric": METRIC, "value": value, "unit": "particle-forces/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == tg.TG_PREC_FP32 else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[name]["desc"].format(n=n), "n": n,
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{world}", "kappa": rp["kappa"], "n_crit": rp["n_crit"],
                   "eta_tot": rp["eta_tot"], "theta": rp["theta"], "mac": args.mac, "dt_max": rp["dt_max"],
                   "k_max": rp["k_max"], "autotune": tuning,
                   "n_crit_used": tg.tg_get_tuning(solver.ctx)["n_crit"]},
        "accuracy": {"median_force_err_vs_fp64_direct": float(np.median(err)),
                     "p99_force_err": float(np.percentile(err, 99)), "sample_sinks": int(sample.numel()),
                     "momentum_drift_one_step": float(np.abs(d_end[:3] - d_start[:3]).max()),
                     "momentum_scale": mom_scale},
        "work": per_step_work(stats, launches, args.steps),
        "kernels_ms_per_step": {k: v["ms"] / (args.steps if prof_k is prof else 1) for k, v in prof_k.items()
                                if k != "_all" and v["launches"] > 0 and v["ms"] > 0},
        "stage_ms_one_step_all_timed": breakdown,
        "roofline": roof,
        "fp64_plain_gpu": fp64,
        "extra": extra,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_sinks / e2e_t, "unit": "particle-forces/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    print(json.dumps(line), flush=True)
    run.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def per_step_work(stats, launches, steps):
    return {"sink_forces_per_step": stats["sink_forces"] / steps,
            "evaluations_per_step": stats["evaluations"] / steps,
            "kdk_frames_per_step": stats["kdk_frames"] / steps,
            "kernel_launches_per_step": launches / steps,
            "host_syncs_per_step": stats["host_syncs"] / steps,
            "p2p_pairs_per_step": stats["p2p_pairs"] / steps,
            "m2l_pairs_per_step": stats["m2l_pairs"] / steps, "max_rung": stats["max_rung"]}


def roofline(prof, stats, p, sm_count):
    """Roofline of the dominant kernel class (by live CUDA-event time over the timed steps)."""
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    sm_max = 2070.0
    if os.path.exists(peaks_path):
        try:
            sm_max = float(json.load(open(peaks_path)).get("sm_max_mhz", 2070.0))
        except Exception:
            pass
    fp32_peak_tflops = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    kernels = {k: v for k, v in prof.items() if v["launches"] > 0 and k != "_all"}
    traffic = captured_traffic()
    dom = max(kernels.items(), key=lambda kv: kv[1]["ms"])[0] if kernels else None
    if dom == "p2p":
        flops = float(P2P_FLOPS_PER_PAIR) * stats["p2p_pairs"]
        units = stats["p2p_pairs"] / kernels["p2p"]["launches"]
        kname = "p2p_mutual"
    elif dom == "m2l":
        flops = m2l_flops(p, stats["m2l_pairs"], stats)
        units = stats["m2l_pairs"] / kernels["m2l"]["launches"]
        kname = "m2l_mutual"
    else:
        return None
    achieved = flops / (kernels[dom]["ms"] / 1e3) / 1e12
    return {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak_tflops, "traffic": scaled_traffic(traffic, dom, units),
            "peak_note": f"float32 SIMT peak = {sm_count} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock)",
            "per_launch": {"flops": flops / kernels[dom]["launches"], "ms": kernels[dom]["ms"] / kernels[dom]["launches"]}}


def compare_fp64_plain(tg, rp, run, stream, flush):
    """One evaluation of the whole initial state in the plain float64 path and in the float32 path."""
    import torch
    out = {}
    for key, prec in (("fp64", tg.TG_PREC_FP64), ("fp32", tg.TG_PREC_FP32)):
        s = tg.Solver(tg.Params(precision=prec, **rp), stream)
        s.fmm_forces(run.P0, run.M, want_pot=False)   # warm-up (buffers)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        s.fmm_forces(run.P0, run.M, want_pot=False)
        e1.record(stream)
        torch.cuda.synchronize()
        out[key] = e0.elapsed_time(e1)
        s.close()
    n = run.M.shape[0]
    return {"eval_ms_fp64": out["fp64"], "eval_ms_fp32": out["fp32"],
            "value_fp64": n / (out["fp64"] / 1e3), "unit": "particle-forces/s",
            "speedup_of_fp32_path": out["fp64"] / out["fp32"],
            "note": "one all-from-all evaluation of the initial state: plain float64 path (float64 P2P block per "
                    "leaf pair, generic float64 M2L, potentials) vs the float32 path (accelerations only)"}


BOX_PARAMS = dict(p=6, theta=0.5, eps=1e-3, kernel=0, n_crit=96, kappa=1.0)


def measure_box(tg, dev, stream, flush, n_sinks=10000):
    """The clustered box (N = 2^24): one all-from-all evaluation in the float32 path and in the float64
    path, each timed with CUDA events (after a warm-up evaluation, L2 flushed), and the force error of
    both against float64 direct summation on n_sinks random sinks (the direct sum runs on the GPU)."""
    import torch
    from paper_1712_10116_gb300 import ics
    pos, mass = ics.clustered_box(256)
    P, M = torch.tensor(pos, device=dev), torch.tensor(mass, device=dev)
    n = M.shape[0]
    sinks = torch.tensor(np.random.default_rng(11).choice(n, n_sinks, replace=False), device=dev)
    ref = tg.Solver(tg.Params(precision=tg.TG_PREC_FP64, **BOX_PARAMS), stream)
    ad, _ = ref.direct_forces(P, M, sinks=sinks)
    ref.close()
    nd = torch.linalg.norm(ad, dim=0)
    out = {"workload": "clustered box N=16777216: Zel'dovich-displaced 256^3 lattice (P(k)~k^-2, 0.5 cell rms) + "
                       "1000 NFW clumps (c=10, log-uniform 1e-5..1e-2), eps=1e-3 Wendland C2, p=6, theta=0.5, "
                       "n_crit=96; one all-from-all evaluation",
           "n": n, "error_sinks": n_sinks, "reference": "float64 direct summation on the GPU"}
    accs = {}
    for key, prec in (("fp32", tg.TG_PREC_FP32), ("fp64", tg.TG_PREC_FP64)):
        s = tg.Solver(tg.Params(precision=prec, **BOX_PARAMS), stream)
        s.fmm_forces(P, M, want_pot=False)   # warm-up (buffers)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        acc, _ = s.fmm_forces(P, M, want_pot=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        a = acc[:, sinks]
        err = (torch.linalg.norm(a - ad, dim=0) / nd).cpu().numpy()
        accs[key] = a
        out[key] = {"eval_ms": ms, "value": n / (ms / 1e3), "unit": "particle-forces/s",
                    "median_force_err": float(np.median(err)), "p99_force_err": float(np.quantile(err, 0.99))}
        s.close()
    d = (torch.linalg.norm(accs["fp32"] - accs["fp64"], dim=0) / torch.linalg.norm(accs["fp64"], dim=0)).cpu().numpy()
    out["fp32_vs_fp64_median"] = float(np.median(d))
    out["speedup_of_fp32"] = out["fp64"]["eval_ms"] / out["fp32"]["eval_ms"]
    return out


PLUMMER_PARAMS = dict(p=4, theta=0.5, eps=0.01, kernel=1, n_crit=64, kappa=1.0, eta=0.025, dt_max=1.0 / 64, k_max=10)


def measure_plummer(tg, dev, stream, steps=16):
    """The Plummer sphere (N = 4096, Plummer softening 0.01, p = 4, theta = 0.5, float64): the initial
    evaluation and 16 rung-0 HOLD steps (batched), timed with CUDA events; momentum and energy drift."""
    import torch
    from paper_1712_10116_gb300 import ics
    pos, vel, mass = ics.plummer(4096, 1001)
    P, V, M = (torch.tensor(a, device=dev) for a in (pos, vel, mass))
    s = tg.Solver(tg.Params(precision=tg.TG_PREC_FP64, batched=1, **PLUMMER_PARAMS), stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    s.hhs_init(P, V, M)
    ev[1].record(stream)
    d0 = s.diagnostics()   # untimed: the energy takes a fresh evaluation with potentials
    ev[2].record(stream)
    for _ in range(steps):
        s.hhs_step()
    ev[3].record(stream)
    torch.cuda.synchronize()
    d1 = s.diagnostics()
    st = s.stats()
    s.close()
    ms = ev[0].elapsed_time(ev[1]) + ev[2].elapsed_time(ev[3])
    pscale = float(np.sum(np.abs(mass * vel)))
    return {"workload": "Plummer sphere N=4096 (a=1, distribution-function velocities), Plummer eps=0.01, p=4, "
                        "theta=0.5, fp64, batched HHS k_max=10 dt_max=1/64 eta=0.025: initial evaluation + 16 steps",
            "ms_total": ms, "value": st["sink_forces"] / (ms / 1e3), "unit": "particle-forces/s",
            "evaluations": st["evaluations"], "max_rung": st["max_rung"],
            "momentum_drift": float(np.linalg.norm(d1[:3] - d0[:3])) / pscale,
            "energy_drift": float(abs((d1[6] - d0[6]) / d0[6]))}


ENSEMBLE_PARAMS = dict(p=4, theta=0.5, eps=0.01, kernel=1, n_crit=64, kappa=1.0, eta=0.025, dt_max=1.0 / 64, k_max=10)


def measure_ensemble(tg, dev, stream, flush, steps=3, warmup=2):
    """The 64-system ensemble (Plummer and King W0 = 6 spheres, N = round(2^U(10, 17)), each with its own
    HHS rungs), float32: one rung-0 step of every system, (a) as 64 plain host-driven steps one after
    another, (b) as one graph launch holding every system's work-queue loop (tg_ensemble_step)."""
    import torch
    from paper_1712_10116_gb300 import ics
    systems = ics.ensemble(velocities=True)
    out = {"workload": "64 systems: even Plummer (a=1), odd King W0=6 (r_half 1.305), N=round(2^U(10,17)), "
                       "Plummer eps=0.01, p=4, theta=0.5, n_crit=64, fp32, HHS k_max=10 dt_max=1/64 eta=0.025",
           "particles": int(sum(s[2].shape[0] for s in systems))}
    for mode in ("plain", "ensemble"):
        runs = [HHSRun(tg, tg.Params(precision=tg.TG_PREC_FP32, batched=int(mode == "ensemble"), **ENSEMBLE_PARAMS),
                       pos, vel, mass, dev, stream) for pos, vel, mass in systems]
        ctxs = [r.solver.ctx for r in runs]

        def step():
            if mode == "plain":
                for r in runs:
                    r.solver.hhs_step()
            else:
                tg.tg_ensemble_step(ctxs)

        for _ in range(warmup):
            for r in runs:
                r.reset()
            step()
        torch.cuda.synchronize()
        for r in runs:
            tg.tg_reset_stats(r.solver.ctx)
        ms = []
        for _ in range(steps):
            for r in runs:
                r.reset()
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = [r.solver.stats() for r in runs]
        sinks = sum(x["sink_forces"] for x in st)
        out[mode] = {"ms_per_step": sum(ms) / steps, "value": sinks / (sum(ms) / 1e3), "unit": "particle-forces/s",
                     "evaluations_per_step": sum(x["evaluations"] for x in st) / steps,
                     "host_syncs_per_step": sum(x["host_syncs"] for x in st) / steps,
                     "max_rung": max(x["max_rung"] for x in st)}
        for r in runs:
            r.close()
    out["speedup_of_ensemble"] = out["plain"]["ms_per_step"] / out["ensemble"]["ms_per_step"]
    return out


def measure_other(tg, args, name, dev, stream, flush, evolved):
    """Figures of a second workload: a few timed rung-0 steps (after an untimed evolution to t = 1
    when `evolved`)."""
    w = WORKLOADS[name]
    n = w["n"]
    pos0, vel0, mass0 = workload(name, n)
    rp = dict(w["params"], eta_tot=0.0, mac=0, batched=int(args.batched))
    run = HHSRun(tg, tg.Params(precision=tg.TG_PREC_FP32, **rp), pos0, vel0, mass0, dev, stream)
    t_evolve = 0.0
    if evolved:
        import torch
        nsteps = int(round(1.0 / rp["dt_max"]))
        w0 = time.perf_counter()
        for _ in range(nsteps):
            run.solver.hhs_step()
        torch.cuda.synchronize()
        t_evolve = time.perf_counter() - w0
        # the evolved state becomes the state each timed step starts from
        run.P0.copy_(run.P)
        run.V0.copy_(run.V)
        _, run.aold0, run.acur0, run.atot0 = tg.tg_hhs_state(run.solver.ctx, n, dev, with_total=True)
    steps = 2 if evolved else 3
    step_ms, stats, prof = time_hhs_steps(run, steps, 1 if evolved else 2, stream, flush)
    t = sum(step_ms) / 1e3
    out = {"workload": w["desc"].format(n=n).replace("from t=0", "from t=1" if evolved else "from t=0"),
           "value": stats["sink_forces"] / t, "unit": "particle-forces/s", "ms_per_step": 1e3 * t / steps,
           "steps": steps, "work": per_step_work(stats, int(prof.get("_all", {}).get("launches", 0)), steps)}
    if evolved:
        out["untimed_evolution_s"] = t_evolve
    run.close()
    return out


def captured_traffic():
    """DRAM bytes per launch from the committed ncu captures, kept only while the kernel source
    hash recorded with them still matches the source being run."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(path):
        return {}
    data = json.load(open(path))
    out = {}
    for key, rec in data.items():
        if not isinstance(rec, dict) or "source" not in rec:
            continue
        h = hashlib.sha256()
        for part in rec["source"].split("+"):
            f = part if os.path.isabs(part) else os.path.join(ROOT, part) if "/" in part else \
                os.path.join(ROOT, "paper_1712_10116_gb300", "csrc", part)
            h.update(open(f, "rb").read())
        if h.hexdigest()[:16] == rec["source_sha256_16"]:
            out[key] = rec
    return out


def scaled_traffic(traffic, key, units_per_launch):
    """Captured bytes per launch scaled to the bench's average launch by the units it processes."""
    rec = traffic.get(key)
    if not rec:
        return None
    return rec["bytes_per_launch"] * units_per_launch / rec["units_per_launch"]


def m2l_flops(p, pairs, stats):
    # per unordered cell pair: the D recurrence, ~3 C(p+4,4) flops; per direction and local-expansion
    # class (one, or two in a kick pair) the contraction for the accelerations, i.e. the C(p+6,6)
    # terms with |n| + |j| <= p less the C(p+3,3) terms of L^0 (the potential), 2 flops each.  The
    # timed HHS evaluations request accelerations only.
    from math import comb
    d = 3 * comb(p + 4, 4)
    contr = 2 * 2 * (comb(p + 6, 6) - comb(p + 3, 3))
    return pairs * d + stats.get("m2l_class_pairs", pairs) * contr


# P2P flops per unordered particle pair for the accelerations of both particles: 3 differences,
# 5 for r^2, 1 rsqrt, 2 for r^-3, 2 mass products, 6 fused multiply-adds (12)
P2P_FLOPS_PER_PAIR = 25


def run_eval_only(args):
    """Plain FMM evaluations of the workload (no HHS), for kernel captures with a profiler."""
    import torch

    from paper_1712_10116_gb300 import binding as tg
    from paper_1712_10116_gb300 import ics

    dev = torch.device("cuda", 0)
    n = args.n or WORKLOADS[args.workload]["n"]
    pos, _, mass = workload(args.workload, n)
    prec = tg.TG_PREC_FP32 if args.precision == "fp32" else tg.TG_PREC_FP64
    solver = tg.Solver(tg.Params(precision=prec, **run_params(args, args.workload)))
    P = torch.tensor(pos, device=dev)
    M = torch.tensor(mass, device=dev)
    F = torch.tensor(ics.random_fast_mask(n, 17), device=dev) if args.masked else None
    if args.m2l_form >= 0:
        t = tg.tg_get_tuning(solver.ctx)
        t["m2l_form"] = args.m2l_form
        tg.tg_set_tuning(solver.ctx, t)
    for _ in range(args.warmup):
        solver.fmm_forces(P, M, F, want_pot=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.fmm_forces(P, M, F, want_pot=False)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    # one more evaluation with every launch timed, for the per-stage breakdown
    tg.tg_reset_stats(solver.ctx)
    tg.tg_set_profiling(solver.ctx, 2)
    solver.fmm_forces(P, M, F, want_pot=False)
    stages = {k: round(v["ms"], 3) for k, v in tg.tg_get_profile(solver.ctx).items()}
    tg.tg_set_profiling(solver.ctx, 0)
    print(json.dumps({"mode": "eval-only", "workload": args.workload, "n": n, "masked": bool(args.masked),
                      "ms_per_eval": 1e3 * dt, "stage_ms": stages, "stats": solver.stats()}), flush=True)
    solver.close()


def run_momentum_contrast(args):
    """|sum m v| after a cold collapse to t = 1 with HHS and with the traditional individual-timestep
    integrator (Sec. 3.2.1, the paper's momentum test): unit cube, N = 10^4, eps = 0.01
    (eps = 0.01 (N/10^4)^(-1/3)), Wendland C2, theta = 0.45, p = 5, float64 on the GPU."""
    import torch
    from paper_1712_10116_gb300 import binding as tg
    from paper_1712_10116_gb300 import ics
    n = args.contrast_n
    eps = 0.01 * (n / 1e4) ** (-1.0 / 3.0)
    pos, vel, mass = ics.uniform_cube(n, 1006)
    dt_max = 1.0 / 64
    steps = int(round(args.contrast_t / dt_max))
    prm = tg.Params(p=5, theta=0.45, eps=eps, kernel=0, precision=tg.TG_PREC_FP64, n_crit=64, eta=0.02,
                    dt_max=dt_max, k_max=10, eta_tot=args.eta_tot, mac=1 if args.mac == "sphere" else 0)
    out = {"mode": "momentum-contrast", "eta_tot": args.eta_tot, "mac": args.mac,
           "workload": f"cold collapse of a unit cube at rest, N={n}, eps={eps:.4g} "
           f"Wendland C2, theta=0.45 ({args.mac} criterion), p=5, float64, eta=0.02, dt_max=1/64, k_max=10, "
           f"t=0..{args.contrast_t}",
           "data": "synthetic"}
    for name in ("hhs", "traditional"):
        s = tg.Solver(prm)
        P = torch.tensor(pos, device="cuda")
        V = torch.tensor(vel, device="cuda")
        M = torch.tensor(mass, device="cuda")
        (s.hhs_init if name == "hhs" else s.trad_init)(P, V, M)
        e0 = float(s.diagnostics()[6])
        tg.tg_reset_stats(s.ctx)
        step = s.hhs_step if name == "hhs" else s.trad_step
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        d = s.diagnostics()
        st = s.stats()
        pmag = float(np.linalg.norm(d[:3]))
        out[name] = {"t": float(d[7]), "abs_P": pmag, "log10_abs_P": float(np.log10(max(pmag, 1e-300))),
                     "rel_dE": float(abs((d[6] - e0) / e0)),
                     "evaluations": st["evaluations"], "sink_forces": st["sink_forces"], "max_rung": st["max_rung"],
                     "wall_s": wall, "particle_forces_per_s": st["sink_forces"] / wall}
        s.close()
    print(json.dumps(out), flush=True)


def run_sweep(args):
    """The theta / p sweeps of the cold-collapse tests (Sec. 3.2, Figs. 4-7 analogues) on the unit cube:
    for each (theta, p), HHS and the traditional integrator from the same state to t = --contrast-t,
    float64 on the GPU; |sum m v|, |sum m x cross v|, the relative energy error and the cost."""
    import torch
    from paper_1712_10116_gb300 import binding as tg
    from paper_1712_10116_gb300 import ics
    n = args.contrast_n
    eps = 0.01 * (n / 1e4) ** (-1.0 / 3.0)
    pos, vel, mass = ics.uniform_cube(n, 1006)
    dt_max = 1.0 / 64
    steps = int(round(args.contrast_t / dt_max))
    if args.sweep_grid:
        grid = [(float(a), int(b)) for a, b in (item.split(":") for item in args.sweep_grid.split(","))]
    else:
        grid = [(th, 5) for th in (0.7, 0.45, 0.3, 0.2, 0.1, 0.05)] + \
               [(0.45, p) for p in (3, 4, 6, 7, 8, 10, 12, 16, 20)]
    rows = []
    for theta, p in grid:
        row = {"theta": theta, "p": p}
        for name in ("hhs", "traditional"):
            prm = tg.Params(p=p, theta=theta, eps=eps, kernel=0, precision=tg.TG_PREC_FP64, n_crit=64, eta=0.02,
                            dt_max=dt_max, k_max=10)
            s = tg.Solver(prm)
            P = torch.tensor(pos, device="cuda")
            V = torch.tensor(vel, device="cuda")
            M = torch.tensor(mass, device="cuda")
            (s.hhs_init if name == "hhs" else s.trad_init)(P, V, M)
            d0 = s.diagnostics()
            tg.tg_reset_stats(s.ctx)
            step = s.hhs_step if name == "hhs" else s.trad_step
            t0 = time.perf_counter()
            for _ in range(steps):
                step()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            d = s.diagnostics()
            st = s.stats()
            row[name] = {"abs_P": float(np.linalg.norm(d[:3])), "abs_L": float(np.linalg.norm(d[3:6])),
                         "rel_dE": float(abs((d[6] - d0[6]) / d0[6])), "evaluations": st["evaluations"],
                         "p2p_pairs": st["p2p_pairs"], "m2l_pairs": st["m2l_pairs"], "wall_s": wall}
            s.close()
        rows.append(row)
        print(json.dumps({"mode": "sweep-point", **row}), flush=True)
    print(json.dumps({"mode": "sweep", "workload": f"cold collapse of a unit cube at rest, N={n}, eps={eps:.4g} "
                      f"Wendland C2, float64, eta=0.02, dt_max=1/64, k_max=10, t=0..{args.contrast_t}",
                      "data": "synthetic", "points": rows}), flush=True)


def main():
    args = parse()
    if args.sweep:
        run_sweep(args)
        return
    if args.eval_only:
        run_eval_only(args)
        return
    if args.momentum_contrast:
        run_momentum_contrast(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
