#!/usr/bin/env python3
"""Benchmark of the immersed-boundary forcing step (one step = the n_F = 3
outer forcing iterations of Sec. 2.2.2 plus particle loads and the
Newton-Euler update) on the synthetic bidisperse bed: periodic 512x512x1024
grid, 1500 spheres D = 24h and 12000 spheres D = 12h (8,139,000 markers).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (a bounded sample of the same workload).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torchrun; every rank runs its own replica (no collective
on the data path), so scaling is weak.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IBM marker-iterations/s and HBM GB/s, FP32 vs plain FP64 form at stated slip"
UNIT = "marker-iterations/s"
WORKLOAD_DESC = {
    "bidisperse": "bidisperse bed: periodic 512x512x1024, 12000 spheres D=12h + 1500 D=24h, n_F=3, FP32",
    "mono": "monodisperse bed: periodic 256x256x512, 2000 spheres D=16h, n_F=3, FP32",
    "single64": "single sphere D=16h in a periodic 64^3 grid, n_F=3, FP32",
    "diff128": "differentiation workload: periodic 128^3, 150 spheres D=16h, n_F=3, FP32",
    "batched": "batched scenes: 512 periodic boxes, edge in {32,48,64,96,128}, 1-40 spheres each, "
               "D ~ U[8,20]h, n_F=3, FP32, all scenes in one persistent launch per step",
}
KERNEL_SOURCES = ["paper_2109_03972_gb300/csrc/ibm_cluster.cu", "paper_2109_03972_gb300/csrc/ibm_device.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bidisperse", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--mode", default="deterministic", choices=["cluster", "deterministic", "plain"])
    ap.add_argument("--threads", type=int, default=0, help="threads per block (0 = default, -1 = autotune)")
    ap.add_argument("--graph", dest="graph", action="store_true", default=True,
                    help="replay the step from a CUDA graph (default)")
    ap.add_argument("--no-graph", dest="graph", action="store_false", help="launch the step eagerly")
    ap.add_argument("--backward", action="store_true",
                    help="also time forward + adjoint (ibm_backward) steps, FP32 and FP64")
    ap.add_argument("--quick", action="store_true", help="skip the FP64, e2e and CPU legs")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--fluid", action="store_true",
                    help="run the fluid-solver leg also with --quick")
    ap.add_argument("--mean-force", action="store_true",
                    help="time the grid-pass mean force even with --quick")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_reduce(v, world, op, device):
    """A per-rank scalar reduced over the ranks (MAX for times, SUM for counts)."""
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, mode):
    """DRAM bytes per launch of the cluster kernel from the committed ncu summary,
    or None if the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", f"ibm_cluster_forcing_{workload}.md")
    try:
        with open(path) as fh:
            for line in fh:
                if line.startswith("traffic_per_launch:"):
                    parts = dict(kv.split("=") for kv in line.split(":", 1)[1].split())
                    if parts.get("source_hash") == kernel_source_hash() and parts.get("mode") == mode:
                        return float(parts["bytes"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def scene_arrays(W):
    sc = W.scenes
    x = np.concatenate([s.x_p for s in sc])
    up = np.concatenate([s.u_p for s in sc])
    om = np.concatenate([s.omega_p for s in sc])
    d = np.concatenate([s.d_p for s in sc])
    rho = np.concatenate([s.rho_p for s in sc])
    so = np.concatenate([np.full(s.n_p, i, dtype=np.int32) for i, s in enumerate(sc)])
    return x, up, om, d, rho, so


def cpu_sample(W, target_s, rng_seed=7):
    """Bounded sample of the workload for the oracle: the particles whose centres
    lie in a cubic sub-box of edge S (a periodic S^3 grid of its own), S chosen so
    one oracle step takes about target_s seconds on the oracle's threads (all host
    cores unless OMP_NUM_THREADS says otherwise)."""
    from oracle import oracle as O
    from paper_2109_03972_gb300 import synth
    sc = W.scenes[0]
    nx, ny, nz = sc.dims
    dmax = float(sc.d_p.max())

    def sub(S):
        keep = np.all(sc.x_p < S, axis=1) & np.all(sc.x_p >= 0, axis=1)
        return synth.Scene((S, S, S), sc.x_p[keep], sc.d_p[keep], sc.u_p[keep], sc.omega_p[keep],
                           sc.rho_p[keep], field_seed=rng_seed)

    S = int(min(nx, ny, nz, max(2 * dmax + 8, 64)))
    probe = sub(S)
    u = probe.field()
    t0 = time.perf_counter()
    O.forcing_step(u, probe.x_p, probe.u_p, probe.omega_p, probe.d_p, n_forcing=W.n_forcing, tau=W.tau,
                   want_slip=False)
    t1 = time.perf_counter() - t0
    grow = (target_s / max(t1, 1e-3)) ** (1.0 / 3.0)
    S2 = int(min(min(nx, ny, nz), max(S, int(S * grow) // 16 * 16)))
    return sub(S2), S2


def host_desc():
    """Host CPU of the oracle timing: architecture, logical cores, model name."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return f"{platform.machine()}, {os.cpu_count()} logical cores" + (f", {model}" if model else "")


def time_oracle(scene, W, steps):
    from oracle import oracle as O
    u = scene.field()
    n_mark = O.total_markers(scene.d_p)
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        O.forcing_step(u, scene.x_p, scene.u_p, scene.omega_p, scene.d_p, n_forcing=W.n_forcing, tau=W.tau,
                       want_slip=False)
        t.append(time.perf_counter() - t0)
    return n_mark, t


def reference_arm(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2109_03972_gb300 import synth
    O.build()
    W = synth.workload(args.workload)
    per_step = max(0.05, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    scene, S = cpu_sample(W, per_step)
    _, _ = time_oracle(scene, W, max(0, min(args.warmup, 1)))
    n_mark, t = time_oracle(scene, W, args.steps)
    ms = 1e3 * float(np.mean(t))
    value = n_mark * W.n_forcing / (ms / 1e3)
    sample = (f"particles with centres in a {S}^3 sub-box of the {args.workload} bed "
              f"({scene.n_p} spheres, {n_mark} markers), periodic {S}^3 grid, one step per timed step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_DESC[args.workload], "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                             "sample": sample, "host": host_desc()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def our_arm(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2109_03972_gb300 import build, synth
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2109_03972_gb300 import ibm

    def barrier():
        if world > 1:
            dist.barrier()

    W = synth.workload(args.workload, seed=2109 + rank)
    dims = [s.dims for s in W.scenes]
    x, up, om, d, rho, so = scene_arrays(W)
    n_p = len(d)
    fields64 = [s.field() for s in W.scenes]
    u_host = [torch.from_numpy(f.astype(np.float32)) for f in fields64]
    mode = {"cluster": ibm.IBM_SPREAD_CLUSTER, "deterministic": ibm.IBM_SPREAD_DETERMINISTIC,
            "plain": ibm.IBM_SPREAD_PLAIN}[args.mode]
    cfg = ibm.Config(dims=dims, n_forcing=W.n_forcing, precision=ibm.IBM_FP32, spread_mode=mode,
                     max_particles=n_p, newton_euler=True, rho_f=W.rho_f, g=W.g, profile=True,
                     threads_per_block=args.threads, use_graph=args.graph)
    stream = torch.cuda.current_stream()
    ctx = ibm.Context(cfg, stream)
    ctx.set_particles(x, up, om, d, rho, so if len(dims) > 1 else None)

    us = [t.cuda() for t in u_host]
    for _ in range(args.warmup):
        ctx.forcing_step(us, W.tau)
    torch.cuda.synchronize()
    stats = ctx.stats()
    n_mark = stats["markers"]
    ctx.kernel_timing(reset=True)
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.forcing_step(us, W.tau)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    ms = rank_reduce(ms, world, dist.ReduceOp.MAX if world > 1 else None, "cuda")
    # markers of all ranks' beds (each rank runs its own seeded bed)
    n_all = rank_reduce(n_mark, world, dist.ReduceOp.SUM if world > 1 else None, "cuda")
    stats = ctx.stats()
    kctx = ctx
    if args.graph:
        # graph replays record no kernel events: time the kernel on an eager twin
        # context running the same variant
        kcfg = ibm.Config(**{**cfg.__dict__, "use_graph": False,
                             "threads_per_block": stats["threads_per_block"]})
        kctx = ibm.Context(kcfg, stream)
        kctx.set_particles(x, up, om, d, rho, so if len(dims) > 1 else None)
        kctx.forcing_step(us, W.tau)
        kctx.kernel_timing(reset=True)
        for _ in range(min(args.steps, 20)):
            kctx.forcing_step(us, W.tau)
        torch.cuda.synchronize()
    k_ms, k_n = kctx.kernel_timing(reset=True)
    k_avg = k_ms / max(1, k_n)
    value = n_all * W.n_forcing / (ms / 1e3)

    peaks, peak_kind = measured_peaks()
    touched = stats["touched_cells"]
    n_p_smem = n_p   # particle records read/written by the kernel (upper bound: all particles)
    alg_bytes = touched * 3 * 4 * 2 * W.n_forcing + n_p_smem * (104 + 48)
    achieved = alg_bytes / (k_avg / 1e3) / 1e9 if k_avg > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
                "traffic": profiled_traffic(args.workload, args.mode),
                "kernel": "k_cluster_forcing" if mode != ibm.IBM_SPREAD_PLAIN else "k_plain_interp+k_plain_spread",
                "kernel_ms": k_avg, "algorithmic_bytes_per_launch": alg_bytes,
                "peak_kind": f"{peak_kind} hbm_gbs (STREAM-style copy)"}
    # slip after one step from the initial field (the same start as the FP64 leg)
    for dst, src in zip(us, u_host):
        dst.copy_(src)
    slip = ctx.forcing_step(us, W.tau, want_slip=True)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC[args.workload], "markers": n_mark, "particles": n_p,
                       "spread_mode": args.mode, "n_forcing": W.n_forcing,
                       "l2": "inputs larger than L2 (u field %.1f GB, touched cells %.0f MB)" % (
                           sum(t.numel() for t in us) * 4 / 1e9, touched * 12 / 1e6),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "cuda_graph": bool(args.graph), "threads_per_block": stats["threads_per_block"],
                       "scenes": len(dims)},
            "roofline": roofline,
            "hbm_gbs_algorithmic_step": alg_bytes / (ms / 1e3) / 1e9,
            "slip": {"rms": slip[0], "max": slip[1], "after": "one step from the initial field"},
            "stats": stats,
            "gpu_launches": int(stats["launches"]) * args.steps,
            "clocks": clocks}

    if not args.quick or args.mean_force:
        line["mean_force"] = mean_force_leg(ctx, us, W, dims, stream, peaks)
    if not args.quick or args.mean_force:
        line["particle_inertia"] = inertia_leg(ctx, us, u_host, peaks, stream)
    if not args.quick:
        line["contact_exclusion"] = exclusion_leg(cfg, us, u_host, W, (x, up, om, d, rho, so), dims, stream)
    if not args.quick:
        line["particle_substeps"] = collision_leg(W, (x, up, om, d, rho, so), dims, stream, ctx, peaks)
    if (not args.quick or args.fluid) and len(dims) == 1:
        line["fluid_stage"] = fluid_leg(W, (x, up, om, d, rho, so), dims[0], fields64[0], stream, peaks)
    if not args.quick:
        # end to end through the C ABI with host buffers: H2D of u and the particle
        # state, the step, D2H of u and the loads, every step
        pinned = [t.pin_memory() for t in u_host]
        back = [torch.empty_like(t).pin_memory() for t in u_host]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for dst, src in zip(us, pinned):
                dst.copy_(src, non_blocking=True)
            ctx.set_particles(x, up, om, d, rho, so if len(dims) > 1 else None)
            ctx.forcing_step(us, W.tau)
            loads = ctx.particle_loads()
            for dst, src in zip(back, us):
                dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = rank_reduce((time.perf_counter() - t0) / args.e2e_steps, world,
                            dist.ReduceOp.MAX if world > 1 else None, "cuda")
        ubytes = sum(t.numel() * 4 for t in u_host)
        pbytes = n_p * 8 * (3 * 3 + 2) + (n_p * 4 if len(dims) > 1 else 0)
        line["e2e"] = {"value": n_all * W.n_forcing / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": ubytes + pbytes, "d2h_bytes_per_step": ubytes + n_p * 8 * 15,
                       "ms_per_step": e2e_s * 1e3}
        # plain FP64 form (the denominator of the speed-up), same workload
        cfg64 = ibm.Config(dims=dims, n_forcing=W.n_forcing, precision=ibm.IBM_FP64,
                           spread_mode=ibm.IBM_SPREAD_PLAIN, max_particles=n_p, newton_euler=True,
                           rho_f=W.rho_f, g=W.g)
        c64 = ibm.Context(cfg64, stream)
        c64.set_particles(x, up, om, d, rho, so if len(dims) > 1 else None)
        u64 = [torch.from_numpy(f).cuda() for f in fields64]
        c64.forcing_step(u64, W.tau)
        torch.cuda.synchronize()
        n64 = 3
        e0.record(stream)
        for _ in range(n64):
            c64.forcing_step(u64, W.tau)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = rank_reduce(e0.elapsed_time(e1) / n64, world, dist.ReduceOp.MAX if world > 1 else None, "cuda")
        for dst, f in zip(u64, fields64):
            dst.copy_(torch.from_numpy(f))
        slip64 = c64.forcing_step(u64, W.tau, want_slip=True)
        line["fp64_plain"] = {"value": n_all * W.n_forcing / (ms64 / 1e3), "unit": UNIT,
                              "ms_per_step": ms64, "slip": {"rms": slip64[0], "max": slip64[1]}}
        line["speedup_vs_fp64_plain"] = ms64 / ms
        del u64, c64
        if rank == 0:
            from oracle import oracle as O
            O.build()
            scene, S = cpu_sample(W, 4.0)
            nm_cpu, t = time_oracle(scene, W, 3)
            cms = float(np.mean(t)) * 1e3
            line["cpu_baseline"] = {
                "value": nm_cpu * W.n_forcing / (cms / 1e3), "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                "host": host_desc(),
                "sample": f"particles with centres in a {S}^3 sub-box of the bed ({scene.n_p} spheres, "
                          f"{nm_cpu} markers) on a periodic {S}^3 grid; 3 steps, {cms:.0f} ms/step"}
    if args.backward:
        line["backward"] = backward_leg(args, W, dims, (x, up, om, d, rho, so), fields64, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def mean_force_leg(ctx, us, W, dims, stream, peaks):
    """Grid-pass mean IBM force (Eq. fe_IBM) over the f_out of one step: one
    read of every cell of the force field (12 B per cell, FP32), timed with
    CUDA events on the library's stream over back-to-back calls."""
    import torch
    fs = [torch.zeros_like(u) for u in us]
    ctx.forcing_step(us, W.tau, f_out=fs)
    F = ctx.particle_loads()["F"]
    out = torch.empty((len(dims), 3), dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.mean_force(fs, device=True)
    torch.cuda.synchronize()
    n = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        out = ctx.mean_force(fs, device=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    fbar = out.cpu().numpy()
    cells = sum(int(u[0].numel()) for u in us)
    nbytes = 3 * cells * 4
    gbs = nbytes / (ms / 1e3) / 1e9
    # one scene: the grid pass and the summed loads are the same sum (cells vs markers)
    resid = None
    if len(dims) == 1:
        resid = float(np.abs(fbar[0] * cells + F.sum(0)).max() / np.abs(F).sum())
    del fs
    return {"kernel": "k_mf_partial + k_mf_final", "ms": ms, "bytes_per_call": nbytes, "bound": "hbm",
            "achieved_gbs": gbs, "peak": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
            "fbar_scene0": [float(v) for v in fbar[0]], "loads_identity_residual": resid,
            "l2": "field %.1f GB, larger than L2" % (nbytes / 1e9)}


def inertia_leg(ctx, us, u_host, peaks, stream):
    """Fluid inertia inside every particle (Sec. 2.2.9): one block per particle
    over its box, timed with CUDA events over back-to-back calls.  Algorithmic
    bytes: the particles' cell-volume equivalent (sum V_p / h^3 cells) x 12 B of
    FP32 velocity, plus 152 B of particle record and 56 B of sums each."""
    import torch
    for dst, src in zip(us, u_host):
        dst.copy_(src)
    for _ in range(3):
        r = ctx.particle_inertia(us, device=True)
    torch.cuda.synchronize()
    n = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        r = ctx.particle_inertia(us, device=True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    V = r["V"].cpu().numpy()
    n_p = V.size
    nbytes = float(V.sum()) * 12 + n_p * (152 + 56)
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"kernel": "k_inertia", "ms": ms, "algorithmic_bytes": nbytes, "bound": "hbm", "achieved_gbs": gbs,
            "peak": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"], "particles": n_p,
            "solid_cells": float(V.sum())}


def collision_leg(W, parts, dims, stream, fctx, peaks):
    """Collision models and RK3 particle sub-steps (Sec. 2.2.6-2.2.10) on the
    workload's particles: one call advances them by one time step tau in 15
    sub-steps of three Runge-Kutta stages, with the hydrodynamic loads of the
    last forcing step (-rho_f times the fluid-side loads) held constant;
    T_c = 10 tau as in the paper, nu_f = 0.01 (grid units).  FP64, CUDA events
    over back-to-back calls (each call re-reads its neighbour-list and contact
    counts on the host)."""
    import torch
    from paper_2109_03972_gb300 import ibm
    x, up, om, d, rho, so = parts
    loads = fctx.particle_loads(device=True)
    Fh = (-W.rho_f * loads["F"]).contiguous()
    Th = (-W.rho_f * loads["T"]).contiguous()
    c = ibm.Context(ibm.Config(dims=dims, precision=ibm.IBM_FP64, spread_mode=ibm.IBM_SPREAD_PLAIN,
                               max_particles=len(d)), stream)
    c.set_particles(x, up, om, d, rho, so if len(dims) > 1 else None)
    prm = ibm.CollisionParams(rho_f=W.rho_f, nu_f=0.01, e_dry=0.97, t_c=10 * W.tau, g=W.g)
    for _ in range(2):
        c.particle_substeps(prm, W.tau, 15, F_h=Fh, T_h=Th)
    torch.cuda.synchronize()
    n = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    for _ in range(n):
        c.particle_substeps(prm, W.tau, 15, F_h=Fh, T_h=Th)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) / n * 1e3
    ms = e0.elapsed_time(e1) / n
    contacts = len(c.contact_history()[0])
    launches = c.stats()["launches"]
    del c
    return {"what": "one particle time step tau: 15 sub-steps x 3 RK stages, collision loads at the stage start "
                    "and the predicted state, FP64", "ms_per_call": ms, "wall_ms_per_call": wall,
            "particles": len(d), "pairs_in_contact": contacts, "kernel_launches_per_call": launches}


def fluid_leg(W, parts, dims, u0, stream, peaks):
    """One time step (three RK3 stages) of the collocated fractional-step solver
    of Sec. 2.2.1 and 2.2.4 on the workload's grid, FP64, with the IBM forcing loop
    of the workload's particles (plain FP64 path) inside every stage: step (a),
    n_F forcing iterations, the grid-pass mean force, the Crank-Nicolson
    Helmholtz solves and the Poisson solve (FP64 residuals around FP32 multigrid
    V-cycles, to 1e-12), the corrector.
    nu = 0.01, dt = tau, starting from the workload's velocity field.  CUDA
    events over one warm and one timed step; the finest-level smoothing launches
    (the dominant kernel) are timed one by one."""
    import torch
    from paper_2109_03972_gb300 import ibm
    x, up, om, d, rho, so = parts
    c = ibm.Context(ibm.Config(dims=[dims], n_forcing=W.n_forcing, precision=ibm.IBM_FP64,
                               spread_mode=ibm.IBM_SPREAD_PLAIN, max_particles=len(d)), stream)
    c.set_particles(x, up, om, d)
    fl = ibm.Fluid(dims, h=1.0, nu=0.01, theta=1.0, profile=True, stream=stream)
    F = ibm.FluidFields(dims)
    F.u.copy_(torch.from_numpy(u0))
    dt = W.tau
    fl.step(dt, F, ctx=c)                      # warm-up step (also first-call allocations)
    torch.cuda.synchronize()
    fl.kernel_timing(reset=True)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    cyc, res = [], []
    e[0].record(stream)
    for k in range(3):
        fl.stage(k, dt, F, ctx=c)
        e[k + 1].record(stream)
        s = fl.stats()
        cyc.append(s["cycles"])
        res.append(max(s["resid"]))
    torch.cuda.synchronize()
    stage_ms = [e[k].elapsed_time(e[k + 1]) for k in range(3)]
    k_ms, k_n = fl.kernel_timing(reset=True)
    nx, ny, nz = dims
    cells = nx * ny * nz
    k_avg = k_ms / max(1, k_n)
    alg = 12 * cells                            # one FP32 sweep: x and b read, x written (4 B each per cell)
    achieved = alg / (k_avg / 1e3) / 1e9 if k_avg > 0 else None
    uf = F.uf
    div = ((uf[0] - torch.roll(uf[0], 1, 2)) + (uf[1] - torch.roll(uf[1], 1, 1)) +
           (uf[2] - torch.roll(uf[2], 1, 0))).abs().max().item()
    levels = fl.stats()["levels"]
    del F, fl, c
    torch.cuda.empty_cache()
    return {"what": "one RK3 time step of the collocated fractional-step solver with the IBM loop in each stage, "
                    "FP64 state, solves by FP64 refinement around FP32 multigrid V-cycles to relative residual 1e-12",
            "grid": list(dims), "cells": cells, "particles": len(d), "ms_per_step": sum(stage_ms),
            "ms_per_stage": stage_ms, "cells_per_s": cells / (sum(stage_ms) / 1e3),
            "v_cycles_per_stage": cyc, "max_rel_residual": max(res), "multigrid_levels": levels,
            "max_abs_div_uf": div,
            "roofline": {"bound": "hbm", "kernel": "k_mg_rbgs<float> (finest-level red-black sweep)",
                         "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"] if achieved else None, "kernel_ms": k_avg,
                         "launches_timed": k_n, "share_of_step": k_ms / sum(stage_ms),
                         "algorithmic_bytes_per_launch": alg}}


def exclusion_leg(cfg, us, u_host, W, parts, dims, stream):
    """Marker exclusion near contact (Sec. 2.2.5) costs: the benchmark's step (same
    spread mode, the cluster kernel for the shared-memory modes) with and without
    it (eager, CUDA events, 10 steps each)."""
    import torch
    from paper_2109_03972_gb300 import ibm
    x, up, om, d, rho, so = parts
    res = {}
    for on in (False, True):
        c = ibm.Context(ibm.Config(**{**cfg.__dict__, "use_graph": False, "threads_per_block": 0,
                                      "profile": False}), stream)
        if on:
            c.set_contact_exclusion(True, 0.0, 2109)
        c.set_particles(x, up, om, d, rho, so if len(dims) > 1 else None)
        for dst, src in zip(us, u_host):
            dst.copy_(src)
        c.forcing_step(us, W.tau)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            c.forcing_step(us, W.tau)
        e1.record(stream)
        torch.cuda.synchronize()
        res["with" if on else "without"] = e0.elapsed_time(e1) / 10
        if on:
            res["markers_disabled"] = c.disabled_markers()[1]
        del c
    mode = {ibm.IBM_SPREAD_CLUSTER: "cluster", ibm.IBM_SPREAD_DETERMINISTIC: "deterministic",
            ibm.IBM_SPREAD_PLAIN: "plain"}[cfg.spread_mode]
    return {"path": f"FP32 {mode}", "ms_per_step_without": res["without"], "ms_per_step_with": res["with"],
            "overhead_ms": res["with"] - res["without"], "markers_disabled": res["markers_disabled"],
            "eps_sep_h": 1.5}


def backward_leg(args, W, dims, parts, fields64, stream):
    """Forward step with requires_grad plus ibm_backward, timed per step with CUDA
    events (loss L = 1/2 sum w |u|^2, so dL/du^{n_F} = w u), FP32 (plain spreading,
    as the adjoint kernels) and the FP64 plain form."""
    import torch
    from paper_2109_03972_gb300 import ibm, synth
    x, up, om, d, rho, so = parts
    out = {"what": "one forcing step (requires_grad) + ibm_backward to du0, dU_p, dw_p, dx_p"}
    for name, prec, dt in (("fp32", ibm.IBM_FP32, torch.float32), ("fp64", ibm.IBM_FP64, torch.float64)):
        cfg = ibm.Config(dims=dims, n_forcing=W.n_forcing, precision=prec, spread_mode=ibm.IBM_SPREAD_PLAIN,
                         max_particles=len(d), requires_grad=True)
        ctx = ibm.Context(cfg, stream)
        ctx.set_particles(x, up, om, d, rho, so if len(dims) > 1 else None)
        u0 = [torch.from_numpy(f).to(device="cuda", dtype=dt) for f in fields64]
        w = [torch.from_numpy(synth.loss_weights(dd, 7 + i)).to(device="cuda", dtype=dt)[None]
             for i, dd in enumerate(dims)]
        us = [t.clone() for t in u0]

        def one():
            for dst, src in zip(us, u0):
                dst.copy_(src)
            ctx.forcing_step(us, W.tau)
            ctx.backward([wi * ui for wi, ui in zip(w, us)])

        for _ in range(3):
            one()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = max(3, min(args.steps, 50))
        e0.record(stream)
        for _ in range(n):
            one()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_ms_per_step"] = e0.elapsed_time(e1) / n
        del ctx, us, u0
    out["speedup_fp32_vs_fp64"] = out["fp64_ms_per_step"] / out["fp32_ms_per_step"]
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    return our_arm(args)


if __name__ == "__main__":
    sys.exit(main())
