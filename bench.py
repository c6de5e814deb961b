#!/usr/bin/env python
"""Benchmark of the SPaSM hot path on GB300: 10-block tower solves (both stages).

One step = one full solve of a seeded 10-block tower in clutter (64 cuboids, 16384 ->
4096 placement particles, 4096 trajectory particles, 20 segments x 32 waypoints):
stage-1 sampling, selection and descent, lift, fused trajectory optimisation, ranking
and the FP64 check, all on the device.  Inputs (the problem tables) are resident in HBM
before the timed region; L2 is flushed (256 MB write) between steps, outside the
per-step CUDA events.

Prints ONE JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle instead
(on the host cores, a bounded sample of the same workload per step, extrapolated to a
solve).  Multi-GPU (torchrun): every rank solves its own problems (replicas, weak
scaling); there is no data-path collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "10-block solve ms p50/p99; particle-iters/s; served solves/s vs plain form"
WORKLOAD = "tower10"
WORKLOAD_DESC = ("10-block tower in clutter: 64 random cuboids (sides 0.05-0.3 m) + table, 7-R arm with 52 spheres, "
                 "N=16384 -> M=4096 placement particles, Q=4096 trajectory particles, 20 segments x 32 waypoints, "
                 "FP32, Philox seeded; seed s = scene + Philox seed")
# nominal FP32 peak (context only; the roofline uses the measured FMA throughput of
# spasm_fp32_fma_peak): 152 SMs x 128 FP32 lanes x 2 flop (FMA) x max SM clock
SM_COUNT, FP32_LANES = 152, 128
# algorithmic FP32 work per unit (the per-unit figures of the hot-path analysis): one
# sphere-cuboid test with its gradient, about 32 instructions = 40 flop (FMA counted as 2)
FLOP_PER_TEST = 40
# forward kinematics of one configuration (about 0.9 kflop), run where its chunk is culled
FLOP_PER_CONFIG_FK = 900
# exact box cull of one (configuration, obstacle) pair: 6 comparisons
FLOP_PER_CULL = 6
# sphere centres and the backward chain of a configuration with a candidate (about 3.3 kflop)
FLOP_PER_CONFIG_CAND = 3300
# every configuration, every evaluation: the descent update with its motion bound, and the
# path, joint-limit and gradient assembly terms (about 120 flop)
FLOP_PER_CONFIG_STEP = 120
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_traj_tower10.md")
KERNEL_SOURCES = ["paper_2510_07674_gb300/csrc/kernels_s2.cu", "paper_2510_07674_gb300/csrc/stage2.cuh",
                  "paper_2510_07674_gb300/csrc/common.cuh", "paper_2510_07674_gb300/csrc/stage1.cuh"]


def code_text(src: str) -> str:
    """Source text without comments, blank lines and layout whitespace: what the compiler sees
    of a kernel file, so that editing a comment does not make a profile summary of the same
    code stale."""
    out, i, n = [], 0, len(src)
    while i < n:
        if src.startswith("//", i):
            i = src.find("\n", i)
            i = n if i < 0 else i
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif src[i] == '"':   # string literal: copied as is
            j = i + 1
            while j < n and src[j] != '"':
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(src[i])
            i += 1
    return "\n".join(" ".join(line.split()) for line in "".join(out).splitlines() if line.strip())


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(code_text(fh.read()).encode())
    return h.hexdigest()[:16]


def profile_values() -> dict:
    """Entries of the committed ncu summary of k_traj, if it was taken on the current kernel
    sources (else {})."""
    if not os.path.exists(PROFILE_SUMMARY):
        return {}
    vals = {}
    for line in open(PROFILE_SUMMARY):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    recorded = (vals.get("kernel_sources_sha256_16") or "").split()
    return vals if recorded and recorded[0] == kernel_hash() else {}


def traffic_from_profile():
    """DRAM bytes per k_traj launch recorded by the committed ncu summary (None if stale)."""
    try:
        return float(profile_values()["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


def issue_from_profile() -> dict:
    """Issue activity and top stall of k_traj from the committed ncu summary ({} if stale):
    the kernel is bound by instruction issue and latency, which the ALU fraction does not show."""
    vals = profile_values()
    out = {}
    try:
        out["issue_active_pct"] = float(vals["issue_active_pct"])
    except (KeyError, ValueError):
        pass
    if "top stalls per issued instruction" in vals:
        out["top_stalls_per_issue"] = vals["top stalls per issued instruction"]
    try:   # FADD + FMUL + 2 FFMA thread instructions counted by the hardware, per launch
        out["fp32_flop_counted_per_launch"] = float(vals["fp32_flop_counted"].split()[0])
    except (KeyError, ValueError, IndexError):
        pass
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        power = [num(r[3]) for r in rows]
        pmax = max(p for p in power if p == p) if any(p == p for p in power) else 0.0
        loaded = [s for s, p in zip(sm, power) if p == p and p >= 0.5 * pmax] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(num(r[2]) for r in rows), "reasons": reasons,
                "samples": len(rows), "power_w_max": pmax}


def measured_fp32_peak(local: int, target_ms: float = 300.0) -> dict:
    """FP32 FMA throughput measured on this GPU by the library's FMA-chain kernel (CUDA
    events), with the SM clock sampled while it runs."""
    import torch

    from paper_2510_07674_gb300 import spasm as S
    S.spasm_fp32_fma_peak(20.0)   # warm-up (module load, clocks up)
    sampler = ClockSampler(local)
    sampler.start()
    runs = [S.spasm_fp32_fma_peak(target_ms) for _ in range(3)]
    torch.cuda.synchronize()
    clk = sampler.stop()
    best = max(runs, key=lambda r: r["tflops"])
    return {"tflops": best["tflops"], "ms": best["ms"], "runs_tflops": [r["tflops"] for r in runs],
            "sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"), "reasons": clk.get("reasons")}


def tail_leg(args, rank, overrides, flush) -> dict:
    """p50 / p99 of the 10-block solve over `tail_seeds` seeds (scene and Philox seed s =
    0, 1, ...): each seed's problem is created (and its stage graphs built) before its timed
    region; CUDA events on the problem's stream bracket spasm_optimize, L2 flushed before."""
    import torch

    from paper_2510_07674_gb300 import scenes
    from paper_2510_07674_gb300 import spasm as S
    times, ok, att1, att2 = [], 0, [], []
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for i in range(args.tail_seeds):
        wl = scenes.make_problem(WORKLOAD, seed=rank * 100000 + i,
                                 **{k: v for k, v in overrides.items() if k != "max_steps"})
        pr = S.Problem(wl, max_steps=overrides["max_steps"])
        try:
            flush.fill_(float(i))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            S.spasm_optimize(pr)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
            r = S.spasm_result(pr, allow_empty=True)
            st = S.spasm_get_stats(pr)
            ok += int(r["success"].sum() > 0)
            att1.append(st["place_attempts"])
            att2.append(st["traj_attempts"])
        finally:
            pr.close()
    clocks = sampler.stop()
    return {"seeds": len(times), "p50_ms": _percentile(times, 0.5), "p99_ms": _percentile(times, 0.99),
            "max_ms": max(times), "mean_ms": statistics.mean(times), "success_rate": ok / len(times),
            "stage1_attempts_mean": statistics.mean(att1), "stage2_attempts_mean": statistics.mean(att2),
            "timed": "CUDA events around spasm_optimize (both stages, graphs with device-side attempt loops), "
                     "L2 flushed before each solve",
            "clocks": clocks}


def count_tests(wl) -> dict:
    """Sphere-cuboid (and sphere-sphere) tests of one stage-2 particle-iteration."""
    B = len(wl.scene.half)
    S = wl.params.W - 1
    C = 2 * B * S + 1
    n_obs = len(wl.scene.cuboid) + len(wl.scene.sphere) + (B - 1)
    n_rsph = len(wl.robot.sphere)
    held_cfgs = B * (S - 1)
    tests = (C - 1) * n_rsph * n_obs + held_cfgs * 8 * n_obs
    return {"C": C, "tests": tests, "n_obs": n_obs}


def rank_seeds(rank: int, n: int) -> list:
    """Scene/Philox seeds of one rank's solves: replicas solve different problems."""
    return [rank * 100000 + i for i in range(n)]


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """The timed region's duration is the slowest rank's (MAX over ranks)."""
    if ws <= 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_throughput(units_per_rank: int, ws: int, max_ms: float) -> float:
    """Units processed by all ranks / the slowest rank's time (weak scaling)."""
    return ws * units_per_rank / (max_ms / 1000.0)


# ------------------------------------------------------------------------------- native
def run_native(args, ws, rank, local):
    import torch

    from paper_2510_07674_gb300 import build as B
    from paper_2510_07674_gb300 import scenes
    from paper_2510_07674_gb300 import spasm as S

    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    overrides = {"max_steps": args.max_steps}
    for kv in args.override:
        k, v = kv.split("=", 1)
        overrides[k] = float(v) if any(ch in v for ch in ".e") else int(v)
    n_total = args.warmup + args.steps
    seeds = rank_seeds(rank, n_total)
    wls = [scenes.make_problem(WORKLOAD, seed=s, **{k: v for k, v in overrides.items() if k != "max_steps"})
           for s in seeds]
    probs = [S.Problem(w, **overrides) for w in wls]
    for p in probs:
        S.spasm_set_timing(p, True)
        if args.launch_mode == "eager":   # kernel by kernel, for profilers that cannot enter the graphs
            S.spasm_set_launch_mode(p, S.SPASM_LAUNCH_EAGER)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    fp32_peak = measured_fp32_peak(local)

    def solve(p):
        S.spasm_reset_stats(p)
        try:
            S.spasm_optimize(p)
        except S.SpasmError as e:   # no solution within max_steps: counted as a failure
            if e.status != -4:
                raise

    for i in range(args.warmup):
        solve(probs[i])
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    times, stats = [], []
    for i in range(args.warmup, n_total):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        solve(probs[i])
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(S.spasm_get_stats(probs[i]))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()

    total_ms = max_over_ranks(sum(times), ws, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_throughput(args.steps, ws, total_ms)

    tc = count_tests(wls[0])
    traj_ms = sum(s["ms_traj"] for s in stats)
    traj_launches = sum(s["traj_launches"] for s in stats)
    pits = sum(s["particle_iters"] for s in stats)
    K = wls[0].params.K_traj
    Q = wls[0].params.Q
    # one launch runs K descent iterations plus the final evaluation pass.  Work actually
    # required: the tests that survive the exact box cull (counted by the kernel), the cull
    # itself and the forward kinematics; the all-pairs count is reported as effective tests/s.
    evals = Q * (K + 1) * max(traj_launches, 1)
    tests_exec = sum(s["tests_executed"] for s in stats)
    cull_cfg = sum(s["cull_configs"] for s in stats)
    cand_cfg = sum(s["cand_configs"] for s in stats)
    flop_total = traj_flop(tc, evals, tests_exec, cull_cfg, cand_cfg)
    flop_per_launch = flop_total / max(traj_launches, 1)
    avg_launch_s = traj_ms / max(traj_launches, 1) / 1000.0
    achieved = flop_per_launch / avg_launch_s / 1e12 if avg_launch_s > 0 else None
    clk = clocks.get("sm_max_mhz") or 2070.0
    nominal = SM_COUNT * FP32_LANES * 2 * clk * 1e6 / 1e12
    peak = fp32_peak["tflops"]
    traffic = traffic_from_profile()
    roofline = {"bound": "alu", "kernel": "k_traj (fused stage-2 descent, one CTA per particle)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": traffic,
                "peak_basis": (f"measured: FP32 FMA chains on every SM (spasm_fp32_fma_peak), "
                               f"{fp32_peak['tflops']:.1f} TFLOP/s at a median SM clock of {fp32_peak['sm_mhz']} MHz; "
                               f"nominal 152 SMs x 128 lanes x 2 x {clk:.0f} MHz = {nominal:.1f} TFLOP/s"),
                "fp32_probe": fp32_peak,
                "flop_per_launch": flop_per_launch, "avg_launch_ms": avg_launch_s * 1e3,
                "tests_per_particle_iter_all_pairs": tc["tests"],
                "tests_per_particle_iter_executed": tests_exec / max(evals, 1),
                "culled_configs_per_particle_iter": cull_cfg / max(evals, 1),
                "candidate_configs_per_particle_iter": cand_cfg / max(evals, 1),
                "effective_pair_tests_per_s": tc["tests"] * evals / max(traj_ms / 1000.0, 1e-9),
                "ncu": issue_from_profile()}
    succ = [s["n_success"] > 0 for s in stats]

    # ---- end to end through the public API with host buffers
    e2e_times, h2d, d2h = [], [], []
    n_e2e = min(args.steps, args.e2e_steps)
    for i in range(n_e2e):
        wl = wls[args.warmup + i]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p = S.Problem(wl, **overrides)
        try:
            S.spasm_optimize(p)
        except S.SpasmError as e:
            if e.status != -4:
                raise
        res = S.spasm_result(p, allow_empty=True)
        st = S.spasm_get_stats(p)
        p.close()
        t1 = time.perf_counter()
        e2e_times.append(t1 - t0)
        h2d.append(st["h2d_bytes"])
        d2h.append(st["d2h_bytes"])
        del res
    e2e_value = ws * len(e2e_times) / sum(e2e_times) if e2e_times else None

    tail = tail_leg(args, rank, overrides, flush) if args.tail_seeds > 0 else None
    batched = served = None
    if args.serve_problems > 0:
        batched, served = run_forms(args, rank, overrides, peak)
    packing = run_packing(args, rank) if args.pack_seeds > 0 else None
    sweep = sweep_leg(args, rank) if args.sweep_seconds > 0 else None
    p2p = run_p2p(args, rank) if args.p2p_seeds > 0 else None
    ik_modes = run_ik_modes(args, rank) if args.ik_seeds > 0 else None

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (FP64 final check)", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "parallelism": f"replicas x{ws}", "l2": "flushed between steps "
                   "(256 MB write outside the per-step events)", "max_steps": args.max_steps,
                   "overrides": {k: v for k, v in overrides.items() if k != "max_steps"},
                   "launch_mode": args.launch_mode},
        # p50 / p99 over the tail leg's seeds when it ran (the metric's distribution), else over the
        # timed steps
        "solve_ms_p50": tail["p50_ms"] if tail else float(statistics.median(times)),
        "solve_ms_p99": tail["p99_ms"] if tail else _percentile(times, 0.99),
        "solve_ms_steps": {"p50": float(statistics.median(times)), "max": max(times), "n": len(times)},
        "solve_ms_seeds": tail,
        "particle_iters_per_s": pits / (total_ms / 1000.0) * ws,
        "success_rate": sum(succ) / len(succ),
        "attempts": {"stage1_mean": statistics.mean(s["place_attempts"] for s in stats),
                     "stage2_mean": statistics.mean(s["traj_attempts"] for s in stats)},
        "phase_ms_mean": {"stage1": statistics.mean(s["ms_place"] for s in stats),
                          "lift": statistics.mean(s["ms_lift"] for s in stats),
                          "traj": statistics.mean(s["ms_traj"] for s in stats),
                          "retry": statistics.mean(s["ms_retry"] for s in stats),
                          "finish": statistics.mean(s["ms_finish"] for s in stats)},
        "host_waits_per_solve": statistics.mean(s["host_waits"] for s in stats),
        "wall_s": wall,
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": statistics.mean(h2d) if h2d else 0,
                "d2h_bytes_per_step": statistics.mean(d2h) if d2h else 0, "steps": len(e2e_times),
                "path": "spasm_create_problem (host arrays) + spasm_optimize + spasm_result + destroy"},
        "batched": batched,
        "served": served,
        "packing": packing,
        "sweep": sweep,
        "p2p": p2p,
        "ik_modes": ik_modes,
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "clocks": clocks,
        "kernel_sources_sha256_16": kernel_hash(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wls[0], args.cpu_budget_s)
    return out


def _percentile(xs, q):
    xs = sorted(xs)
    return float(xs[min(len(xs) - 1, max(0, math.ceil(q * len(xs)) - 1))])


def traj_flop(tc, evals, tests, cull_configs, cand_configs) -> float:
    """FP32 work the trajectory kernel executes: the sphere-obstacle tests left by the exact
    cull, the kinematics and cull of the configurations whose chunk was culled (the others
    kept an earlier cull, valid by their clearance), sphere centres and gradient chain where a
    configuration has a candidate, and the per-configuration step terms of every evaluation."""
    return (FLOP_PER_TEST * tests + (FLOP_PER_CONFIG_FK + FLOP_PER_CULL * tc["n_obs"]) * cull_configs
            + FLOP_PER_CONFIG_CAND * cand_configs + FLOP_PER_CONFIG_STEP * evals * (tc["C"] - 1))


def solve_flop(wl, st) -> float:
    """Executed trajectory work of one finished solve (the headline roofline's count)."""
    tc = count_tests(wl)
    evals = wl.params.Q * (wl.params.K_traj + 1) * max(st["traj_launches"], 1)
    return traj_flop(tc, evals, st["tests_executed"], st["cull_configs"], st["cand_configs"])


def run_forms(args, rank, overrides, peak):
    """The same heterogeneous problems (1-10 blocks, 8-64 cuboids, 1024-4096 trajectory
    particles, 32 waypoints per segment) solved (a) one after another through the plain API,
    (b) as one batch (spasm_optimize_batch: one CUDA graph, one persistent trajectory
    launch; schedule from spasm_batch_autotune on a separate copy of the problems), (c) all
    submitted at once to the continuous-batching service (epochs: one batched trajectory
    attempt of every request in flight); then (d) Poisson arrivals at each rate to the
    service, latency from arrival to completion.  Problem creation and the
    result read-back are inside every timed region."""
    import random

    import torch

    from paper_2510_07674_gb300 import scenes
    from paper_2510_07674_gb300 import spasm as S
    n = args.serve_problems
    wls = scenes.heterogeneous_batch(n, seed=1000 + rank)
    ov = {"max_steps": overrides.get("max_steps", 1000)}

    def form(t, ok, flop, **extra):
        ach = flop / t / 1e12
        return dict(solves_per_s=n / t, success=ok / n, achieved_tflops=ach, frac_of_alu_peak=ach / peak, **extra)

    # (a) plain form
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ok = flop = 0
    for wl in wls:
        p = S.Problem(wl, **ov)
        try:
            S.spasm_optimize(p)
        except S.SpasmError as e:
            if e.status != -4:
                raise
        r = S.spasm_result(p, allow_empty=True)
        ok += int(r["success"].sum() > 0)
        flop += solve_flop(wl, S.spasm_get_stats(p))
        p.close()
    torch.cuda.synchronize()
    plain = form(time.perf_counter() - t0, ok, flop)
    plain_flop = flop   # every form solves the same problems to the same bits: the same executed work

    # (b) batched form
    stream = torch.cuda.Stream()
    tune = [S.Problem(wl, stream=stream.cuda_stream, **ov) for wl in wls]
    sched = S.spasm_batch_autotune(tune, stream=stream.cuda_stream)
    for p in tune:
        p.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prs = [S.Problem(wl, stream=stream.cuda_stream, **ov) for wl in wls]
    S.spasm_optimize_batch(prs, stream=stream.cuda_stream, config=sched)
    ok = flop = 0
    for wl, p in zip(wls, prs):
        r = S.spasm_result(p, allow_empty=True)
        ok += int(r["success"].sum() > 0)
        flop += solve_flop(wl, S.spasm_get_stats(p))
        p.close()
    torch.cuda.synchronize()
    batched = form(time.perf_counter() - t0, ok, flop, schedule=sched,
                   form="spasm_optimize_batch: stage-1 graph + stage-2 graph with one persistent trajectory launch")
    batched["speedup_vs_plain"] = batched["solves_per_s"] / plain["solves_per_s"]

    def epoch_stats(before, after):
        e = max(after["epochs"] - before["epochs"], 1)
        return {"epochs": after["epochs"] - before["epochs"],
                "requests_per_epoch": (after["requests_in_epochs"] - before["requests_in_epochs"]) / e,
                "particles_per_epoch": (after["particles_in_epochs"] - before["particles_in_epochs"]) / e}

    # (c) the service, everything submitted at once
    sv = S.Server(budget_bytes=150 << 30, max_inflight=args.serve_slots)
    st0 = S.spasm_server_get_stats(sv)
    t0 = time.perf_counter()
    tickets = [S.spasm_server_submit(sv, wl, **ov) for wl in wls]
    for t in tickets:
        S.spasm_server_wait(sv, t, 600.0)
    t_all = time.perf_counter() - t0
    res = [S.spasm_server_result(sv, t) for t in tickets]
    for t in tickets:
        S.spasm_server_release(sv, t)
    service = form(t_all, sum(int(r["success"].sum() > 0) for r in res), plain_flop,
                   slots=args.serve_slots, budget_gb=150, **epoch_stats(st0, S.spasm_server_get_stats(sv)))
    service["speedup_vs_plain"] = service["solves_per_s"] / plain["solves_per_s"]

    # (d) served: Poisson arrivals
    served = []
    rng = random.Random(7 + rank)
    for rate in args.serve_rates:
        arrivals, tcur = [], 0.0
        for _ in range(n):
            tcur += rng.expovariate(rate)
            arrivals.append(tcur)
        st0 = S.spasm_server_get_stats(sv)
        start = time.perf_counter()
        tickets = []
        for i, wl in enumerate(wls):
            delay = arrivals[i] - (time.perf_counter() - start)
            if delay > 0:
                time.sleep(delay)
            tickets.append(S.spasm_server_submit(sv, wl, **ov))
        for t in tickets:
            S.spasm_server_wait(sv, t, 600.0)
        end = time.perf_counter() - start
        rs = [S.spasm_server_result(sv, t) for t in tickets]
        lat = [r["latency_ms"] for r in rs]
        for t in tickets:
            S.spasm_server_release(sv, t)
        served.append({"rate_per_s": rate, "requests": n, "solves_per_s": n / end,
                       "speedup_vs_plain": n / end / plain["solves_per_s"],
                       "frac_of_alu_peak": plain_flop / end / 1e12 / peak,
                       "success": sum(int(r["success"].sum() > 0) for r in rs) / n,
                       "latency_ms_p50": _percentile(lat, 0.5), "latency_ms_p99": _percentile(lat, 0.99),
                       **epoch_stats(st0, S.spasm_server_get_stats(sv))})
    sv.close()
    forms = {"problems": n, "workload": "heterogeneous: B~U{1..10}, O~U{8..64}, Q~U{1024..4096}, N=4096->M=1024, "
             "32 waypoints per segment", "plain": plain, "batched": batched, "service_all_at_once": service}
    return forms, served


def stage1_first_solution(wl):
    """(solved, ms, attempts) of one stage-1 solve: CUDA events around spasm_place."""
    import torch

    from paper_2510_07674_gb300 import spasm as S
    pr = S.Problem(wl)
    try:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        try:
            S.spasm_place(pr)
        except S.SpasmError as e:
            if e.status != -4:
                raise
        e1.record()
        torch.cuda.synchronize()
        st = S.spasm_get_stats(pr)
        n = S.spasm_placements(pr, allow_empty=True)["n_place"]
        return n > 0, e0.elapsed_time(e1), st["place_attempts"]
    finally:
        pr.close()


def _summary(times, ok, att):
    import numpy as np
    t = np.array(times)
    ci = 1.96 * t.std(ddof=1) / math.sqrt(len(t)) if len(t) > 1 else 0.0
    return {"seeds": len(t), "success": ok / len(t), "ms_mean": float(t.mean()), "ms_ci95": float(ci),
            "ms_p50": float(np.median(t)), "attempts_mean": float(np.mean(att))}


def run_packing(args, rank):
    """Stage 1 (Alg. 1) on the packing workloads (the appendix's Tetris problem): time to
    first solution per seed, capped at 30 000 gradient steps as in the paper's runs."""
    from paper_2510_07674_gb300 import scenes
    out = {}
    for name, n in (("tetris5", args.pack_seeds), ("tetris8", args.pack8_seeds)):
        times, ok, att = [], 0, []
        for i in range(n):
            solved, ms, a = stage1_first_solution(scenes.make_packing(name, seed=rank * 1000 + i, max_steps=30000))
            ok += solved
            times.append(ms)
            att.append(a)
        out[name] = _summary(times, ok, att)
    out["workload"] = ("seeded tetromino tilings of a 5x4 (5 blocks) and 8x4 (8 blocks) cell region, cell units, "
                       "stage 1 only; see scenes.PACKINGS for N, M, steps")
    return out


def run_p2p(args, rank):
    """Point-to-point trajectory optimisation (stage 2 on one segment, Sec. IV's motion
    planning use): solve time per seed (CUDA events around spasm_optimize) and success."""
    import torch

    from paper_2510_07674_gb300 import scenes
    from paper_2510_07674_gb300 import spasm as S
    times, ok, att = [], 0, []
    for i in range(args.p2p_seeds):
        wl = scenes.make_p2p("p2p", seed=rank * 1000 + i, max_steps=30000)
        pr = S.Problem(wl)
        try:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            try:
                S.spasm_optimize(pr)
            except S.SpasmError as e:
                if e.status != -4:
                    raise
            e1.record()
            torch.cuda.synchronize()
            r = S.spasm_result(pr, allow_empty=True)
            ok += int(r["success"].sum() > 0)
            times.append(e0.elapsed_time(e1))
            att.append(S.spasm_get_stats(pr)["traj_attempts"])
        finally:
            pr.close()
    out = _summary(times, ok, att)
    out["workload"] = ("q_home to a top-down tool target over the table, 48 cuboids (half between robot and target), "
                       "Q=1024 trajectory particles, 32 waypoints, 50 iterations")
    return out


def run_sweep(args):
    """Hyper-parameter sweep (Sec. IV, Fig. 5 analogue): time to first solution of stage 1
    over a grid of sampling batch N and optimisation batch M, per workload."""
    from paper_2510_07674_gb300 import scenes
    rows = []
    for name in args.sweep_workloads:
        for N in [2 ** k for k in range(9, 16)]:
            for M in [2 ** k for k in range(8, 14)]:
                if M > N:
                    continue
                times, ok, att = [], 0, []
                for t in range(args.sweep_trials):
                    kw = dict(seed=t, N=N, M=M, P=min(8, M), max_steps=30000)
                    wl = scenes.make_packing(name, **kw) if name in scenes.PACKINGS else scenes.make_problem(name, **kw)
                    solved, ms, a = stage1_first_solution(wl)
                    ok += solved
                    times.append(ms)
                    att.append(a)
                rows.append(dict(workload=name, N=N, M=M, **_summary(times, ok, att)))
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"sweep": rows, "trials": args.sweep_trials,
                      "metric": "stage-1 time to first solution (ms), mean over seeds"}))


SWEEP_LEG_GRID = {
    # workload: (N values, M values, seeds per cell)
    "tetris5": ([512, 2048, 8192, 32768], [256, 1024, 4096], 5),
    "tetris8": ([8192, 16384], [512, 1024, 2048, 4096], 10),
    "tower10": ([1024, 8192, 32768], [256, 1024, 4096], 5),
}


def sweep_leg(args, rank) -> dict:
    """The N x M stage-1 sweep (Sec. IV, Fig. 5 analogue) on a reduced grid, inside the
    benchmark's JSON line: time to first solution (CUDA events around spasm_place) per cell, the
    success fraction within the 30 000-step cap and the attempts; cells are run in order until
    the leg's time budget is spent (the rest are listed as skipped)."""
    from paper_2510_07674_gb300 import scenes
    t_start = time.perf_counter()
    rows, skipped = [], []
    for name, (Ns, Ms, seeds) in SWEEP_LEG_GRID.items():
        for N in Ns:
            for M in Ms:
                if M > N:
                    continue
                if time.perf_counter() - t_start > args.sweep_seconds:
                    skipped.append(f"{name} N={N} M={M}")
                    continue
                times, ok, att = [], 0, []
                for t in range(seeds):
                    kw = dict(seed=rank * 1000 + t, N=N, M=M, P=min(8, M), max_steps=30000)
                    wl = scenes.make_packing(name, **kw) if name in scenes.PACKINGS else scenes.make_problem(name, **kw)
                    solved, ms, a = stage1_first_solution(wl)
                    ok += solved
                    times.append(ms)
                    att.append(a)
                rows.append(dict(workload=name, N=N, M=M, **_summary(times, ok, att)))
    return {"metric": "stage-1 time to first solution (ms), 30 000-step cap", "cells": rows, "skipped": skipped,
            "seconds": time.perf_counter() - t_start}


# ------------------------------------------------------------------------------- oracle
def cpu_baseline(wl, budget_s: float) -> dict:
    """The FP64 oracle, as it stands, on a bounded sample of the same workload: a stage-1
    sample (cost of n particles, descent of m) and a stage-2 sample (descent steps of a
    few lifted particles), extrapolated to one solve (N costs, M x (K_lin + K_quad)
    descent steps, Q x K_traj trajectory particle-iterations)."""
    import numpy as np

    from oracle import oracle as O
    cores = os.cpu_count() or 1
    orc = O.Oracle(wl, n_threads=cores)
    p = wl.params
    t0 = time.perf_counter()
    n1 = 256
    x = orc.place_sample(n1)
    ta = time.perf_counter()
    for xi in x:
        orc.place_cost(xi, grad=False)
    t_cost = (time.perf_counter() - ta) / n1
    m1 = 64
    ta = time.perf_counter()
    orc.place_descend(x[:m1])
    t_desc = (time.perf_counter() - ta) / m1          # per particle, K_lin + K_quad steps
    # stage 2: lift from a cheap placement (the stage-1 sample's best particle) and time
    # descent steps of n2 particles
    place = x[0]
    n2 = max(cores, 4)
    qs = np.stack([orc.lift(place, i) for i in range(n2)])
    ta = time.perf_counter()
    orc.traj_descend(qs, k_steps=1)
    probe = time.perf_counter() - ta
    # fill the rest of the budget with more descent steps of the same particles
    k2 = max(1, int((0.6 * budget_s) / max(probe, 1e-3)))
    ta = time.perf_counter()
    orc.traj_descend(qs, k_steps=k2)
    t_pi_wall = (time.perf_counter() - ta) / (n2 * k2)   # wall seconds per particle-iteration
    spent = time.perf_counter() - t0
    t_solve = p.N * t_cost / cores + p.M * t_desc + p.Q * p.K_traj * t_pi_wall
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": (f"stage 1: cost of {n1} particles (serial) and descent of {m1} particles ({cores} threads); "
                       f"stage 2: {k2} descent step(s) of {n2} lifted particles ({cores} threads); "
                       f"extrapolated to N={p.N} costs, M={p.M} descents, Q x K_traj={p.Q}x{p.K_traj} "
                       f"particle-iterations; {spent:.1f} s of CPU work"),
            "particle_iters_per_s": 1.0 / t_pi_wall, "seconds_per_solve": t_solve}


def run_reference(args, ws, rank, local):
    from paper_2510_07674_gb300 import scenes
    times = []
    last = None
    for i in range(args.warmup + args.steps):
        wl = scenes.make_problem(WORKLOAD, seed=i)
        cb = cpu_baseline(wl, args.cpu_budget_s)
        if i >= args.warmup:
            times.append(cb["seconds_per_solve"] * 1000.0)
        last = cb
    ms = statistics.mean(times)
    value = 1000.0 / ms
    return {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_DESC, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": last["cores"], "kind": "oracle",
                             "sample": "per step: " + last["sample"]},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_ik_modes(args, rank):
    """The lift's two IK forms on the 10-block tower: the lift alone (spasm_lift of the Q
    trajectory particles, CUDA events, median of repeats) and whole solves (spasm_optimize)
    with the analytic IK, per seed, with success and stage-2 attempts."""
    import torch

    from paper_2510_07674_gb300 import scenes
    from paper_2510_07674_gb300 import spasm as S
    out = {}
    for mode in (0, 1):
        wl = scenes.make_problem(WORKLOAD, seed=rank * 1000, ik_mode=mode)
        pr = S.Problem(wl)
        try:
            place = torch.from_numpy(wl.scene.init.reshape(1, -1)).float().cuda().contiguous()
            q = torch.zeros(wl.params.Q, pr.C, 8, device="cuda")
            ms = []
            for r in range(6):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record()
                S.spasm_lift(pr, wl.params.Q, place, 1, r, q)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            out[f"lift_ms_ik_mode{mode}"] = float(statistics.median(ms[1:]))
        finally:
            pr.close()
    times, ok, att, lift = [], 0, [], []
    for i in range(args.ik_seeds):
        wl = scenes.make_problem(WORKLOAD, seed=rank * 1000 + i, ik_mode=1)
        pr = S.Problem(wl, max_steps=args.max_steps)
        try:
            S.spasm_set_timing(pr, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            try:
                S.spasm_optimize(pr)
            except S.SpasmError as e:
                if e.status != -4:
                    raise
            e1.record()
            torch.cuda.synchronize()
            st = S.spasm_get_stats(pr)
            ok += int(st["n_success"] > 0)
            times.append(e0.elapsed_time(e1))
            att.append(st["traj_attempts"])
            lift.append(st["ms_lift"])
        finally:
            pr.close()
    out["analytic_solve"] = _summary(times, ok, att)
    out["analytic_solve"]["lift_ms_mean"] = statistics.mean(lift) if lift else None
    out["workload"] = WORKLOAD_DESC + "; lift with ik_mode 1 (analytic, Franka joint layout) vs 0 (damped least squares)"
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--max-steps", type=int, default=1000,
                    help="cap on gradient steps per stage (re-initialisation budget)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--launch-mode", choices=["graph", "eager"], default="graph",
                    help="graph: each stage one CUDA graph with a device-side attempt loop; eager: the same kernels "
                         "launched one at a time with the loop on the host (for kernel profilers)")
    ap.add_argument("--tail-seeds", type=int, default=100,
                    help="10-block solves (one per seed, 0..n-1) for the p50 / p99 of the metric (0 = skip)")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-problems", type=int, default=64,
                    help="heterogeneous problems for the batched / served measurements (0 = skip)")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--pack-seeds", type=int, default=12, help="seeds of the 5-block packing leg (0 = skip)")
    ap.add_argument("--pack8-seeds", type=int, default=10, help="seeds of the 8-block packing leg (with --pack-seeds > 0)")
    ap.add_argument("--p2p-seeds", type=int, default=10, help="seeds of the point-to-point leg (0 = skip)")
    ap.add_argument("--ik-seeds", type=int, default=6,
                    help="10-block solves with the analytic lift IK, after timing both lift forms (0 = skip)")
    ap.add_argument("--sweep", action="store_true", help="run the N x M stage-1 sweep instead of the benchmark")
    ap.add_argument("--sweep-workloads", nargs="*", default=["tetris5", "tetris8", "tower10"])
    ap.add_argument("--sweep-trials", type=int, default=5)
    ap.add_argument("--sweep-seconds", type=float, default=90.0,
                    help="time budget of the reduced N x M sweep leg inside the benchmark line (0 = skip)")
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0])
    ap.add_argument("--override", action="append", default=[], metavar="PARAM=VALUE",
                    help="change a solver parameter (profiling of a reduced case only; recorded in config)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.sweep:
        if rank == 0:
            run_sweep(args)
        return
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, ws, rank, local)), flush=True)
        return
    if ws > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_native(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
