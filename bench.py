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
LOG_EVERY = 10


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# Algorithmic work per kernel launch, per site (flops: FMA = 2), and bytes per site.
def kernel_model(kclass, precision, s):
    tk = 8 if precision == "fp64" else 4
    ne = (s + 1) * (s + 2) // 2
    if kclass == "residual":
        return {"flops": 264, "bytes": 16 + 16 + 8 + 48 + 6 * tk, "fp64": True}
    if kclass == "matvec":
        return {"flops": 54, "bytes": 6 * tk + 4 * tk + 6 * tk, "fp64": precision == "fp64"}
    if kclass == "gram":   # Gram partial sums (+ the last block's reduction and least squares)
        return {"flops": 3 * ne * 4, "bytes": (s + 1) * 6 * tk, "fp64": precision == "fp64"}
    if kclass == "update":
        return {"flops": 3 * s * 4 + 6 + 36, "bytes": s * 6 * tk + 48 + 48, "fp64": precision == "fp64"}
    if kclass == "setup":
        return {"flops": 40, "bytes": 16 + 8 + 16 + 48 + 4 * tk + 6 * tk, "fp64": True}
    if kclass == "accept":
        return {"flops": 12, "bytes": 48 + 16, "fp64": True}
    return {"flops": 0, "bytes": 0, "fp64": False}


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
    """K MB4 steps; each bracketed by CUDA events on the library's stream (the
    current torch stream); L2 flushed between steps outside the brackets."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    newton = 0
    obs_calls = 0
    H = []
    for k in range(K):
        a, b = evs[k]
        a.record()
        st = it.step(1)
        if log_every and (k + 1) % log_every == 0:
            o = it.observables()
            H.append(o["H"])
            obs_calls += 1
        b.record()
        newton += st["newton_iters_total"]
        flush()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    return ms, newton, obs_calls, H


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
    for precision in ("fp64", "mixed"):
        it = mb4.from_workload(w, precision=precision, stream=stream)
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
        if precision == "mixed":
            clocks = sampler.stop()
        o1 = it.observables()
        drift = max([abs(h - o0["H"]) / abs(o0["H"]) for h in Hs + [o1["H"]]])
        ms_max = max_over_ranks(ms, world, dev)
        s_dim = 4
        results[precision] = {
            "value": world * S * K / (ms_max / 1e3), "ms_per_step": ms_max / K, "wall_s": wall,
            "newton_per_step": newton / K, "energy_drift": drift,
            "norm_drift": abs(o1["norm2"] - o0["norm2"]), "krylov_s": s_dim,
            "launches": K * 2 + newton * (s_dim + 3) + 2 * obs_calls, "obs_calls": obs_calls,
        }
        # per-kernel device times from the event-instrumented run of the same steps
        kp = min(K, 100)
        _, prof = it.step_profiled(kp)
        results[precision]["kernels"] = {
            k: {"ms_total": v[0], "launches": v[1], "us_per_launch": (1e3 * v[0] / v[1]) if v[1] else 0.0}
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
    # Roofline of the dominant kernel of the FP64 path.
    dom = max(fp["kernels"].items(), key=lambda kv: kv[1]["ms_total"])[0]
    model = kernel_model(dom, "fp64", fp["krylov_s"])
    us = fp["kernels"][dom]["us_per_launch"]
    flops_per_launch = model["flops"] * S
    bytes_per_launch = model["bytes"] * S
    t_alu = flops_per_launch / FP64_PEAK_DERIVED
    t_hbm = bytes_per_launch / (peaks["hbm_gbs"] * 1e9)
    if model["fp64"] and t_alu >= t_hbm:
        roof = {"bound": "alu", "kernel": dom, "achieved": flops_per_launch / (us * 1e-6) / 1e12,
                "peak": FP64_PEAK_DERIVED / 1e12, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SMs x 2070 MHz x 2 DFMA/clk/SM (FP64)"}
    else:
        roof = {"bound": "hbm", "kernel": dom, "achieved": bytes_per_launch / (us * 1e-6) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "peak_source": f"{peak_src} hbm_gbs"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    roof["algorithmic_per_site"] = {"flops": model["flops"], "bytes": model["bytes"]}

    line = {
        "metric": METRIC, "value": fp["value"], "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": fp["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "grid512_fp64", "nx": w.nx, "ny": w.ny, "h": w.h, "chi": w.chi, "W": w.W,
                   "defect_fraction": w.defect_fraction, "V_defect": w.V_defect, "sigma": w.sigma,
                   "precision": "fp64", "krylov_s": fp["krylov_s"], "log_every": LOG_EVERY,
                   "l2": "flushed between timed steps (256 MiB write, outside the timed intervals)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "energy_drift": fp["energy_drift"], "newton_per_step": fp["newton_per_step"],
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
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _oracle_sample(n=64):
    from oracle import mb4_oracle as orc
    from paper_2003_04345_gb300 import inputs
    w = inputs.grid512_fp64()
    w.nx = w.ny = n
    prob = orc.Problem(n, n, w.potential(), w.chi, tx=w.tx, ty=w.ty, eps0=w.eps0)
    return orc, prob, w.psi0(), w.h, n * n


def cpu_baseline(seconds=15.0, n=64):
    """The oracle, as it stands, on a bounded sample of the workload: an n x n
    instance with the 512x512 physics, stepped for about ``seconds``."""
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
    return {"value": S * steps / wall, "unit": UNIT, "cores": max(1, round(cpu / wall)), "kind": "oracle",
            "sample": f"{n}x{n} instance with the 512x512 workload's physics, {steps} MB4 steps, "
                      f"{wall:.1f} s wall", "host_threads_available": os.cpu_count()}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
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
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": max(1, round(cpu / wall)), "kind": "oracle",
                             "sample": f"{n}x{n} instance with the 512x512 workload's physics, "
                                       f"{args.steps} MB4 steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
