#!/usr/bin/env python
"""MB4 benchmark: site-steps/s of the MB4 step on one GB300 (per rank).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (N=1): the 512x512 single-instance FP64 run -- hopping t=1, disorder
uniform in [-0.5, 0.5], 1% of sites defects at V=20, chi=1, Gaussian
wavepacket sigma=8, k=(pi/4, 0), h=0.005, energy and norm logged every 10
steps.  One benchmark step is one MB4 time step (setup, the simplified-Newton
loop with its three shifted Krylov solves, accept).  ``value`` is the FP64
path; the mixed path (FP32 inner solves) runs the same workload and is
reported beside it.  The 512x512 working set fits in L2, so L2 is flushed
(a 256 MiB write) between timed steps, outside the timed intervals.

Under torchrun (N>1) every rank runs its own replica of the workload (the
path has no exchange step); rank 0 prints the line with the max over ranks.
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MB4 site-steps/s at |ΔH/H|≤1e-13, mixed vs FP64 path; served p50/p99 latency"
UNIT = "site-steps/s"
FP64_PEAK_DERIVED = 152 * 2070e6 * 2 * 2   # SMs x max SM clock x 2 DFMA/clk/SM x 2 flop (GB300, FP64)
FP64_ISSUE_PEAK = 152 * 2070e6 * 2         # FP64 instructions (per thread) per second
LOG_EVERY = 10
HBM_GBS = 6792.4                   # replaced by MEASURED_PEAKS.json's figure in run_ours
FP64_RATE = FP64_PEAK_DERIVED      # replaced by the FP64 rate measured in run_ours


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# Algorithmic work per kernel launch, per site (flops: FMA = 2), and bytes per site.
def kernel_model(kclass, precision, s, powers=True, pred_order=2):
    """Algorithmic work of one launch per site: flops (FMA = 2), FP64 instructions
    (DFMA, DADD and DMUL one each: what occupies the FP64 pipe) and bytes (each array
    read or written once; neighbours counted once).  ``powers``: the FP32 basis is the
    one-launch matrix-powers kernel (grid problems without preconditioning)."""
    tk = 8 if precision == "fp64" else 4
    ne = (s + 1) * (s + 2) // 2
    f64 = precision == "fp64"
    # FP64 instruction counts of the grid-stencil kernels with the x hopping factored
    # out (ncu counts 102 DFMA + 12 DADD + 18 DMUL and 18 + 12 + 0)
    if kclass == "residual":   # u0, (K+V)u0, D/tx, dU in; b = -Phibar (level 0) out
        return {"flops": 240, "fp64_ops": 132, "bytes": 16 + 16 + 8 + 48 + 6 * tk, "fp64": True}
    if kclass == "matvec":
        if not f64 and powers:  # J coefficients and level 0 in, levels 1..s out
            return {"flops": 54 * s, "fp64_ops": 0, "bytes": 4 * tk + 6 * tk + s * 6 * tk, "fp64": False}
        return {"flops": 54, "fp64_ops": 30 if f64 else 0, "bytes": 6 * tk + 4 * tk + 6 * tk, "fp64": f64}
    if kclass == "gram":       # all s+1 levels of the three systems in
        return {"flops": 3 * ne * 4, "fp64_ops": 3 * ne * 2 if f64 else 0, "bytes": (s + 1) * 6 * tk, "fp64": f64}
    if kclass == "update":     # s levels and dU in, dU out
        return {"flops": 3 * s * 4 + 6, "fp64_ops": 6 * (s + 1) if f64 else 6,
                "bytes": s * 6 * tk + 48 + 48, "fp64": f64}
    if kclass == "setup":      # u, D in; (K+V)u0, J coefficients, level 0 out
        return {"flops": 40, "fp64_ops": 0, "bytes": 16 + 8 + 16 + 4 * tk + 6 * tk, "fp64": True}
    if kclass == "accept":     # u, dU in; u out; the Newton-start history shifted by one step
        hist = 48 + (pred_order - 1) * 96 if pred_order > 0 else 0
        return {"flops": 12, "fp64_ops": 0, "bytes": 48 + 16 + 16 + hist, "fp64": True}
    return {"flops": 0, "fp64_ops": 0, "bytes": 0, "fp64": False}


def kernel_rooflines(prof, precision, s, hbm_gbs, fp64_flops, powers=True, pred_order=2):
    """Per kernel class, from (total ms, launches, sites computed): microseconds per
    launch, algorithmic GB/s (bytes per site x sites computed / time) and its fraction of
    the measured HBM copy bandwidth, and for FP64 kernels the FP64 flop rate and its
    fraction of the measured FP64 FMA rate.  Launches that skip their instance (the
    first residual of a step from U^0 = e3 (x) u0) add time but no sites."""
    out = {}
    for k, (ms, n, sites) in prof.items():
        if not n or not sites:
            continue
        m = kernel_model(k, precision, s, powers, pred_order)
        gbs = m["bytes"] * sites / (ms * 1e-3) / 1e9
        e = {"us_per_launch": 1e3 * ms / n, "launches": n, "ms_total": ms, "sites": sites,
             "bytes_per_site": m["bytes"], "gb_s": gbs, "hbm_frac": gbs / hbm_gbs}
        if m["fp64"] and m["fp64_ops"]:
            tf = m["flops"] * sites / (ms * 1e-3)
            e["fp64_tflops"] = tf / 1e12
            e["fp64_frac"] = tf / fp64_flops
            e["fp64_issue_frac"] = m["fp64_ops"] * sites / (ms * 1e-3) / (fp64_flops / 2.0)
        out[k] = e
    return out


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_grid512.txt")
KERNEL_SOURCES = ("paper_2003_04345_gb300/csrc/mb4_kernels.cu", "paper_2003_04345_gb300/csrc/mb4_device.cuh",
                  "paper_2003_04345_gb300/csrc/mb4_phases.cuh", "paper_2003_04345_gb300/csrc/mb4_persist.cu",
                  "paper_2003_04345_gb300/csrc/mb4_precond.cu", "paper_2003_04345_gb300/csrc/mb4_internal.h")


def kernel_source_hash():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kclass, precision):
    """DRAM bytes (read + write) per launch of a kernel class on the 512x512
    workload, from the committed ncu summary; None when the summary has no such
    line or was taken from other kernel sources than the ones built here."""
    try:
        digest = kernel_source_hash()
        with open(TRAFFIC_FILE) as fh:
            for line in fh:
                f = line.split()
                if len(f) >= 5 and f[0] == "traffic" and f[1] == kclass and f[2] == precision:
                    return float(f[3]) if f[4] == digest else None
    except OSError:
        pass
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_steps(it, K, flush, log_every=LOG_EVERY):
    """K MB4 steps queued with mb4_step_async, each bracketed by CUDA events on
    the library's stream (the current torch stream); L2 flushed between steps
    outside the brackets; energy and norm read back every log_every steps (inside
    the bracket of that step).  Returns (ms, Newton iterations, observable calls, H)."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    obs_calls = 0
    H = []
    for k in range(K):
        a, b = evs[k]
        a.record()
        it.step_async(1)
        if log_every and (k + 1) % log_every == 0:
            o = it.observables()
            H.append(o["H"])
            obs_calls += 1
        b.record()
        flush()
    st = it.wait()
    torch.cuda.synchronize()
    if st["steps_done"] != K:
        raise RuntimeError(f"{st['steps_done']} of {K} steps done")
    ms = sum(a.elapsed_time(b) for a, b in evs)
    return ms, st["newton_iters_total"], obs_calls, H


def run_ours(args):
    import numpy as np
    import torch

    from paper_2003_04345_gb300 import inputs, mb4

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = inputs.grid512_fp64()
    S = w.S
    K, W = args.steps, args.warmup
    peaks, peak_src = _peaks()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    flush = lambda: flush_buf.zero_()

    results = {}
    for precision in ("fp64", "mixed", "fp64_alg1", "fp64_persistent", "mixed_persistent"):
        # fp64_alg1: the FP64 path with Algorithm 1's Newton start U^0 = e3 (x) u0 instead
        # of the default extrapolated start (same equations, same tolerance);
        # *_persistent: each step one persistent cooperative kernel (same results bit for bit)
        start = 0 if precision == "fp64_alg1" else None
        pers = 1 if precision.endswith("_persistent") else 0
        it = mb4.from_workload(w, precision=precision.split("_")[0], stream=stream, newton_start=start,
                               persistent=pers)
        o0 = it.observables()
        it.step(W)
        torch.cuda.synchronize()
        if precision == "fp64":
            sampler = ClockSampler(local)
            time.sleep(0.25)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ms, newton, obs_calls, Hs = timed_steps(it, K, flush)
        torch.cuda.synchronize()
        barrier(world)
        wall = time.perf_counter() - t0
        if precision == "fp64_alg1":
            # the FP64 ceiling of the FP64-bound kernels, measured at the clocks of this run
            fp64_rate, fp64_probe_s = mb4.fp64_fma_rate(0.3)
            clocks = sampler.stop()
        o1 = it.observables()
        drift = max([abs(h - o0["H"]) / abs(o0["H"]) for h in Hs + [o1["H"]]])
        ms_max = max_over_ranks(ms, world, dev)
        s_dim = 4
        results[precision] = {
            "launch_shape": list(it.launch_shape()),
            "value": world * S * K / (ms_max / 1e3), "ms_per_step": ms_max / K, "wall_s": wall,
            "newton_per_step": newton / K, "energy_drift": drift,
            "norm_drift": abs(o1["norm2"] - o0["norm2"]), "krylov_s": s_dim,
            # per step: arm, setup, accept; per Newton iteration: residual, s basis
            # launches (one matrix-powers launch in mixed mode), Gram, update, loop test
            # (a step graph always runs its first two iterations, and every step here
            # takes at least two); 2 per log
            "launches": K * 3 + newton * ((s_dim if precision.startswith("fp64") else 1) + 4) + 2 * obs_calls,
            "obs_calls": obs_calls,
        }
        if precision == "fp64_alg1" or pers:
            it.close()
            continue
        # per-kernel device times from the event-instrumented run of the same steps;
        # the only region a profiler started with --profile-from-start off records
        kp = min(K, 100)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        _, prof = it.step_profiled(kp)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        results[precision]["kernels"] = {
            k: {"ms_total": v[0], "launches": v[1], "sites": v[2],
                "us_per_launch": (1e3 * v[0] / v[1]) if v[1] else 0.0}
            for k, v in prof.items() if v[1]}
        results[precision]["profiled_steps"] = kp
        if precision == "fp64":
            e2e_it = it
        else:
            it.close()

    # End to end through the C ABI with pinned host buffers: H2D of the state, one step,
    # D2H of the new state, every step.
    it = e2e_it
    hre = torch.empty(S, dtype=torch.float64).pin_memory()
    him = torch.empty(S, dtype=torch.float64).pin_memory()
    it.get_state_ptr(hre.data_ptr(), him.data_ptr(), 0)
    ke = min(K, 200)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for k in range(ke):
        a.record()
        it.set_state_ptr(hre.data_ptr(), him.data_ptr(), 0)
        it.step(1)
        it.get_state_ptr(hre.data_ptr(), him.data_ptr(), 0)
        b.record()
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
        flush()
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    it.close()

    fp = results["fp64"]
    # Roofline of the dominant kernel of the FP64 path: by the bench's own event times
    # (the host-driven copy of the timed steps), against the FP64 rate measured above.
    dom = max(fp["kernels"].items(), key=lambda kv: kv[1]["ms_total"])[0]
    model = kernel_model(dom, "fp64", fp["krylov_s"])
    kd = fp["kernels"][dom]
    # one launch's work is S sites; its duration is the time per site computed x S (a
    # launch that skips its instance adds time but no work, and is not counted)
    us = 1e3 * kd["ms_total"] / (kd["sites"] / S)
    flops_per_launch = model["flops"] * S
    bytes_per_launch = model["bytes"] * S
    t_alu = flops_per_launch / fp64_rate
    t_hbm = bytes_per_launch / (peaks["hbm_gbs"] * 1e9)
    probe_src = (f"measured in this run: mb4_fp64_fma_rate (DFMA chains over the whole device, "
                 f"{fp64_probe_s:.2f} s launch); nominal {FP64_PEAK_DERIVED / 1e12:.4f} TFLOP/s = "
                 f"152 SMs x 2070 MHz x 2 DFMA/clk/SM")
    if model["fp64"] and t_alu >= t_hbm:
        roof = {"bound": "alu", "kernel": dom, "achieved": flops_per_launch / (us * 1e-6) / 1e12,
                "peak": fp64_rate / 1e12, "unit": "TFLOP/s", "peak_source": probe_src,
                "frac_of_nominal": flops_per_launch / (us * 1e-6) / FP64_PEAK_DERIVED}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": bytes_per_launch / (us * 1e-6) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "peak_source": f"{peak_src} hbm_gbs"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if model["fp64_ops"]:
        # the same launch against the FP64 pipe's instruction rate (an add or a
        # multiply takes a DFMA's slot, so the flop fraction understates pipe use)
        ops = model["fp64_ops"] * S / (us * 1e-6)
        issue_peak = fp64_rate / 2.0
        roof["fp64_issue"] = {"ops_per_site": model["fp64_ops"], "achieved_gops": ops / 1e9,
                              "peak_gops": issue_peak / 1e9, "frac": ops / issue_peak}
    roof["traffic"] = measured_traffic(dom, "fp64")
    roof["algorithmic_per_site"] = {"flops": model["flops"], "bytes": model["bytes"]}
    roof["all_kernels"] = kernel_rooflines({k: (v["ms_total"], v["launches"], v["sites"])
                                            for k, v in fp["kernels"].items()},
                                           "fp64", fp["krylov_s"], peaks["hbm_gbs"], fp64_rate)
    global HBM_GBS, FP64_RATE
    HBM_GBS, FP64_RATE = peaks["hbm_gbs"], fp64_rate

    line = {
        "metric": METRIC, "value": fp["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": fp["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "grid512_fp64", "nx": w.nx, "ny": w.ny, "h": w.h, "chi": w.chi, "W": w.W,
                   "defect_fraction": w.defect_fraction, "V_defect": w.V_defect, "sigma": w.sigma,
                   "precision": "fp64", "krylov_s": fp["krylov_s"], "newton_start": 2, "log_every": LOG_EVERY,
                   "launch_shape": {"fp64": fp["launch_shape"], "mixed": results["mixed"]["launch_shape"],
                                    "order": "threads per block, then blocks per instance, of setup/accept, "
                                             "residual, basis, update (autotuned)"},
                   "l2": "flushed between timed steps (256 MiB write, outside the timed intervals)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "energy_drift": fp["energy_drift"], "newton_per_step": fp["newton_per_step"],
        "algorithm1_start": {"value": results["fp64_alg1"]["value"],
                             "ms_per_step": results["fp64_alg1"]["ms_per_step"],
                             "newton_per_step": results["fp64_alg1"]["newton_per_step"],
                             "energy_drift": results["fp64_alg1"]["energy_drift"],
                             "note": "FP64 path with U^0 = e3 (x) u0 (newton_start = 0)"},
        "persistent": {pr: {"value": results[pr + "_persistent"]["value"],
                            "ms_per_step": results[pr + "_persistent"]["ms_per_step"],
                            "newton_per_step": results[pr + "_persistent"]["newton_per_step"],
                            "energy_drift": results[pr + "_persistent"]["energy_drift"],
                            "launches_per_step": 2}
                       for pr in ("fp64", "mixed")},
        "mixed": {"value": results["mixed"]["value"], "ms_per_step": results["mixed"]["ms_per_step"],
                  "energy_drift": results["mixed"]["energy_drift"],
                  "newton_per_step": results["mixed"]["newton_per_step"],
                  "krylov_s": results["mixed"]["krylov_s"], "dtype": "f64 state/residual, f32 Krylov",
                  "speedup_vs_fp64": results["mixed"]["value"] / fp["value"],
                  "kernels": results["mixed"]["kernels"]},
        "kernels": fp["kernels"],
        "roofline": roof,
        "e2e": {"value": world * S * ke / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": 16 * S,
                "d2h_bytes_per_step": 16 * S, "steps": ke},
        "gpu_launches": fp["launches"],
        "clocks": clocks,
    }
    if not args.no_extra and world == 1:        # single-GPU lines: one process owns the device
        line["ensemble"] = bench_ensemble(args, flush)
        line["grid2048"] = bench_grid2048(args, flush)
        line["served"] = bench_served(args)
        line["served"]["rate_sweep"] = [bench_served(args, n_requests=8, rate=r) for r in (1.0, 4.0)]
        line["paper_setups"] = bench_paper_setups(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _timed_batch_steps(bt, K, flush):
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        evs[k][0].record()
        bt.step_async(1)
        evs[k][1].record()
        flush()
    stats, codes = bt.wait()
    torch.cuda.synchronize()
    if any(codes):
        raise RuntimeError(f"batch step failed: {sorted(set(codes))}")
    return sum(a.elapsed_time(b) for a, b in evs), sum(st["newton_iters_total"] for st in stats)


def bench_ensemble(args, flush, K=20):
    """The 1024-member 128x128 ensemble (chi ~ U[0, 2] per seed, 1% defects,
    sigma = 8, h = 0.01) as one batch, mixed precision: every launch covers all
    members (16.8M sites per step)."""
    import numpy as np
    import torch
    from paper_2003_04345_gb300 import inputs, mb4
    B, n = 1024, 128
    ws = [inputs.ensemble128(seed) for seed in range(B)]
    V = np.stack([w.potential() for w in ws])
    chi = np.array([w.chi for w in ws])
    psi = np.stack([w.psi0() for w in ws])
    out = {"workload": "ensemble1024_grid128", "members": B, "nx": n, "ny": n, "h": ws[0].h}
    for precision in ("mixed", "fp64"):
        with mb4.Batch(n, n, V, chi, ws[0].h, precision=precision,
                       stream=torch.cuda.current_stream()) as bt:
            bt.set_state(psi)
            H0 = bt.observables()[:, 0]
            bt.step(3)
            ms, newton = _timed_batch_steps(bt, K, flush)
            H1 = bt.observables()[:, 0]
            shape = list(bt.launch_shape())
            # per-kernel device times: the host-driven copy of 5 more steps, events around launches
            flush()
            _, codes, prof = bt.step_profiled(5)
            if any(codes):
                raise RuntimeError(f"profiled ensemble step failed: {sorted(set(codes))}")
        out[precision] = {"value": B * n * n * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K, "steps": K,
                          "launch_shape": shape,
                          "kernels": kernel_rooflines(prof, precision, 4, HBM_GBS, FP64_RATE),
                          "newton_per_member_step": newton / (B * K),
                          "energy_drift_max": float(np.max(np.abs(H1 - H0) / np.abs(H0)))}
    return out


def bench_grid2048(args, flush, K=20):
    """2048x2048, disorder in [-1, 1], 1% defects, chi = 2, h = 0.002: mixed and
    FP64 on the same inputs, and their difference after K steps."""
    import numpy as np
    import torch
    from paper_2003_04345_gb300 import inputs, mb4
    w = inputs.grid2048_mixed()
    out = {"workload": "grid2048_mixed", "nx": w.nx, "ny": w.ny, "h": w.h}
    finals = {}
    for precision in ("mixed", "fp64"):
        with mb4.from_workload(w, precision=precision, stream=torch.cuda.current_stream()) as it:
            H0 = it.energy()[0]
            it.step(3)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            newton = 0
            for k in range(K):
                evs[k][0].record()
                st = it.step(1)
                evs[k][1].record()
                newton += st["newton_iters_total"]
                flush()
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs)
            finals[precision] = it.get_state()
            H1 = it.energy()[0]
            # per-kernel device times: the host-driven copy of 5 more steps (the states above
            # are taken first, so the comparison covers the timed steps only)
            flush()
            _, prof = it.step_profiled(5)
        out[precision] = {"value": w.S * K / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / K,
                          "kernels": kernel_rooflines(prof, precision, 4, HBM_GBS, FP64_RATE),
                          "newton_per_step": newton / K, "energy_drift": abs(H1 - H0) / abs(H0)}
    a, b = finals["mixed"], finals["fp64"]
    out["mixed_vs_fp64_rel_linf"] = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    out["steps_compared"] = K + 3
    return out


def bench_served(args, n_requests=24, rate=200.0):
    """The served stream: Poisson arrivals at 200 req/s of simulations with grid
    sizes in {64^2 .. 1024^2}, step counts in [100, 5000], h in {0.002, 0.005,
    0.01}, per-request seed and defect density 0-2%, replayed for the first
    n_requests arrivals through the continuous-batching server (mixed precision,
    64 GiB HBM budget).  Latency = completion - arrival.  200 req/s offers ~100x
    what one GPU can serve, so this measures a saturated queue; the rate sweep
    replays the first requests of the same trace at lower rates (the arrival gaps
    scale with 1/rate) to show the unsaturated latency.  Every request's inputs are
    made before the server starts, and the trace starts after an offset long enough
    for all of them to be submitted, so that no request is submitted after its arrival."""
    import numpy as np
    from paper_2003_04345_gb300 import inputs, mb4
    trace = inputs.served_trace(n_requests, rate, seed=0)
    reqs = [(t, w, w.potential(), w.psi0()) for t, w in trace]
    site_steps = sum(w.S * w.steps for _, w, _, _ in reqs)
    offset = 1.0 + 0.004 * n_requests
    with mb4.Server(64 << 30, max_slots=64, keep_states=False, precision="mixed") as srv:
        ids = []
        for t, w, V, psi in reqs:
            ids.append(srv.submit(w.nx, w.ny, V, w.chi, psi, w.h, w.steps, arrival=offset + t))
        submitted = srv.clock()
        del reqs
        done = srv.run()
        makespan = srv.clock() - (offset + trace[0][0])
        res = [srv.result(i) for i in ids]
    lat = np.array([r["completed"] - r["arrival"] for r in res])
    drift = max(abs(r["energy_end"] - r["energy_start"]) / abs(r["energy_start"]) for r in res)
    return {"workload": "served_poisson200", "requests": n_requests, "completed": int(done),
            "rate_req_per_s": rate, "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)), "latency_max_s": float(lat.max()),
            "value": site_steps / makespan, "unit": UNIT, "makespan_s": makespan,
            "site_steps": site_steps, "energy_drift_max": drift,
            "errors": int(sum(1 for r in res if r["status"] != 0)),
            "submitted_before_first_arrival": bool(submitted <= offset + trace[0][0]),
            "trace_offset_s": offset}


def bench_paper_setups(args, K=60):
    """The paper's own setups (Sec. 3), spectrally preconditioned: the 70x70
    Laplacian run (u0 = 1 + 2 cos x + 2 cos y, gamma = 0.1, h = 0.01; K steps from
    t = 0, inside the collapse-free part of the run) and the 100x100 delta-potential
    run (gamma = 0.05, V0 = -50 at the origin).  Time per step, Newton iterations,
    energy drift."""
    import numpy as np
    import torch
    from paper_2003_04345_gb300 import inputs, mb4
    out = {}
    for name, n, gamma, V in (("paper70", 70, 0.1, None), ("paper_delta100", 100, 0.05, -50.0)):
        tx, ty, e0 = inputs.paper_laplacian_hopping(n, n)
        pot = np.zeros(n * n) if V is None else inputs.delta_potential(n, n, V)
        line = {"nx": n, "ny": n, "gamma": gamma, "h": 0.01, "steps": K}
        for precision in ("fp64", "mixed"):
            with mb4.Integrator(n, n, pot, -gamma, 0.01, tx=tx, ty=ty, onsite=e0, precision=precision,
                                precondition=1, newton_rtol=2e-14, stream=torch.cuda.current_stream()) as it:
                it.set_state(inputs.paper_initial_state(n, n))
                H0 = it.energy()[0]
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                it.step_async(K)
                b.record()
                st = it.wait()
                torch.cuda.synchronize()
                H1 = it.energy()[0]
            line[precision] = {"ms_per_step": a.elapsed_time(b) / K, "newton_per_step": st["newton_iters_total"] / K,
                               "energy_drift": abs(H1 - H0) / abs(H0)}
        out[name] = line
    return out


def _oracle_sample(n=64):
    from oracle import mb4_oracle as orc
    from paper_2003_04345_gb300 import inputs
    w = inputs.grid512_fp64()
    w.nx = w.ny = n
    prob = orc.Problem(n, n, w.potential(), w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    return orc, prob, w.psi0(), w.h, n * n


ONE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1",
                  "BLIS_NUM_THREADS": "1", "VECLIB_MAXIMUM_THREADS": "1", "NUMEXPR_NUM_THREADS": "1"}


def cpu_baseline(seconds=15.0, n=64):
    """The oracle, as it stands, on one host thread (its BLAS pinned to one thread in a
    fresh interpreter, so that ``cores`` is the number of threads actually used).  Its
    sparse LU and GMRES barely use more than one core anyway."""
    env = dict(os.environ, **ONE_THREAD_ENV)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-only",
                        "--cpu-seconds", str(seconds)], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(f"cpu baseline failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_baseline_here(seconds=15.0, n=64):
    """The oracle, as it stands, on a bounded sample of the workload: an n x n
    instance with the 512x512 physics, stepped for about ``seconds`` (run by
    cpu_baseline in a one-thread interpreter)."""
    orc, prob, u, h, S = _oracle_sample(n)
    u = orc.step(prob, u, h)   # warm-up (imports, caches)
    t0 = time.perf_counter()
    c0 = time.process_time()
    steps = 0
    while time.perf_counter() - t0 < seconds:
        u = orc.step(prob, u, h)
        steps += 1
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    return {"value": S * steps / wall, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n}x{n} instance with the 512x512 workload's physics, {steps} MB4 steps, "
                      f"{wall:.1f} s wall", "threads": "1 (BLAS and OpenMP pinned to one thread)",
            "cpu_busy_over_wall": cpu / wall, "host_threads_available": os.cpu_count()}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.update(ONE_THREAD_ENV)      # before numpy loads: the oracle runs on one thread
    n = 64
    orc, prob, u, h, S = _oracle_sample(n)
    for _ in range(args.warmup):
        u = orc.step(prob, u, h)
    t0 = time.perf_counter()
    c0 = time.process_time()
    for _ in range(args.steps):
        u = orc.step(prob, u, h)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    value = S * args.steps / wall
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "grid512_fp64", "sample": f"{n}x{n} instance with the same physics"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "cpu_busy_over_wall": cpu / wall,
                             "sample": f"{n}x{n} instance with the 512x512 workload's physics, "
                                       f"{args.steps} MB4 steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_case(case):
    """A few steps of the 512x512 workload (``fp64``, ``mixed``) or of the 2048x2048
    one (``fp64_2048``, ``mixed_2048``) with the host-driven Newton loop, so that every
    kernel is its own launch (the form ncu captures kernel by kernel); one step and
    one observables call sit in a profiler start/stop range, the range ncu
    --profile-from-start off records."""
    import torch
    from paper_2003_04345_gb300 import inputs, mb4
    precision, _, size = case.partition("_")
    w = inputs.grid2048_mixed() if size == "2048" else inputs.grid512_fp64()
    with mb4.from_workload(w, precision=precision, use_graph=False) as it:
        it.step(5)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()        # after the launch-shape tuning and the warm-up
        st = it.step(1)
        it.observables()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    print(json.dumps({"profile_case": case, "newton_iters_last": st["newton_iters_last"]}))


def full_runs():
    """The 2048x2048 configuration (500 steps) and the 1024-member 128x128 ensemble (2000
    steps) over their whole stated step counts, in both precisions: the largest relative
    energy drift over each run (H read every 10 and every 100 steps), Newton iterations per
    step and wall time; for 2048x2048 also mixed against FP64 at the end.  Prints one JSON
    line; a validation run, not a bench line."""
    import numpy as np
    import torch
    from paper_2003_04345_gb300 import inputs, mb4
    out = {}
    w = inputs.grid2048_mixed()
    res, finals = {}, {}
    for precision in ("mixed", "fp64"):
        with mb4.from_workload(w, precision=precision, stream=torch.cuda.current_stream()) as it:
            H0 = it.energy()[0]
            drift, newton = 0.0, 0
            t0 = time.perf_counter()
            for _ in range(w.steps // 10):
                newton += it.step(10)["newton_iters_total"]
                drift = max(drift, abs(it.energy()[0] - H0) / abs(H0))
            wall = time.perf_counter() - t0
            finals[precision] = it.get_state()
        res[precision] = {"steps": w.steps, "energy_drift_max": drift, "newton_per_step": newton / w.steps,
                          "wall_s": wall}
    a, b = finals["mixed"], finals["fp64"]
    res["mixed_vs_fp64_rel_linf"] = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    out["grid2048_mixed"] = res
    B, n = 1024, 128
    ws = [inputs.ensemble128(seed) for seed in range(B)]
    V = np.stack([x.potential() for x in ws])
    chi = np.array([x.chi for x in ws])
    psi = np.stack([x.psi0() for x in ws])
    steps = ws[0].steps
    res = {}
    for precision in ("mixed", "fp64"):
        with mb4.Batch(n, n, V, chi, ws[0].h, precision=precision, stream=torch.cuda.current_stream()) as bt:
            bt.set_state(psi)
            H0 = bt.observables()[:, 0]
            drift, newton = 0.0, 0
            t0 = time.perf_counter()
            for _ in range(steps // 100):
                stats, codes = bt.step(100)
                if any(codes):
                    raise RuntimeError(f"ensemble step failed: {sorted(set(codes))}")
                newton += sum(st["newton_iters_total"] for st in stats)
                H = bt.observables()[:, 0]
                drift = max(drift, float(np.max(np.abs(H - H0) / np.abs(H0))))
            wall = time.perf_counter() - t0
        res[precision] = {"members": B, "steps": steps, "energy_drift_max": drift,
                          "newton_per_member_step": newton / (B * steps), "wall_s": wall}
    out["ensemble1024_grid128"] = res
    print(json.dumps({"full_runs": out}))


def served_full():
    """The served stream at the size its p50/p99 need: the first 2000 arrivals of the
    200 req/s trace, and a rate sweep of 100 requests per rate at 0.5, 1 and 2 req/s (the
    first 100 requests of the same trace, arrival gaps scaled by 200/rate).  A validation
    run of tens of minutes: prints one JSON line, not a bench line."""
    out = {"served_poisson200_first2000": bench_served(None, n_requests=2000, rate=200.0),
           "rate_sweep_100": [bench_served(None, n_requests=100, rate=r) for r in (0.5, 1.0, 2.0)]}
    print(json.dumps({"served_full": out}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--profile-case", choices=["fp64", "mixed", "fp64_2048", "mixed_2048"],
                    help="run 6 host-driven steps of the 512x512 (or 2048x2048) workload for ncu and exit")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the ensemble, 2048^2 and served-stream lines")
    ap.add_argument("--served-full", action="store_true",
                    help="replay the first 2000 arrivals of the 200 req/s trace and a 100-request rate "
                         "sweep through the server, and exit")
    ap.add_argument("--full-runs", action="store_true",
                    help="run the 2048^2 and ensemble configurations over their whole step counts "
                         "(energy drift, Newton counts) and exit")
    args = ap.parse_args()
    if args.cpu_baseline_only:
        print(json.dumps(_cpu_baseline_here(seconds=args.cpu_seconds)))
        return
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.full_runs:
        full_runs()
        return
    if args.served_full:
        served_full()
        return
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
