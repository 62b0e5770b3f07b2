#!/usr/bin/env python
"""Throughput of the time-reversible FDTD hot path on B300 (one JSON line on stdout).

A bench step is one whole forward + time-reversal gradient solve of the workload (every row of the
hot path: H and E updates with CPML, sources, detectors, face record, inverse step, adjoint sweep
and dL/deps). The default workload is the large single solve: a 600^3 grid (216 M cells) with a
12-cell CPML, a Si waveguide (eps 12.25) along x in SiO2 (eps 2.085), an Ey Gaussian sheet over the
core, a 200^3 random-density design box (seed 600) and a Poynting-flux objective, 4000 time steps
forward and 4000 reversed (about 72 GB on the device, of which 64 GB face history).

Metric: Gcell-steps/s = cells x time steps / device time of the fwd+grad solve (the forward-only
rate is reported beside it). Under torchrun each rank solves its own replica (weak scaling, no
collective on the data path); the value is the sum over ranks divided by the slowest rank's time.

`--impl reference` times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload (its full x-y cross-section in a z-slab, a few time steps per bench step).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2412_12360_b300 import scenes  # noqa: E402

METRIC = "Gcell-steps/s fwd+grad (time-reversal gradient)"
UNIT = "Gcell-steps/s"


def workload(name):
    if name == "design_96":
        sc = scenes.design_96()
        desc = ("design_96: 96^3 Yee grid, 10-cell CPML, Gaussian-beam Ex sheet, 40^3 design box "
                "eps=1+11.1*rho (rho~U[0,1), seed 1234), |E|^2 plane objective, 2000 steps fwd + 2000 reversed")
    elif name == "cavity_32":
        sc = scenes.cavity_32(500)
        desc = "cavity_32: 32^3 PEC box, 8^3 eps=2.25 cube, Ez dipole, 500 steps fwd + 500 reversed"
    elif name == "design_96_tfsf":
        sc = scenes.design_box_scene((96, 96, 96), 10, 40, 2000, 1234, 1.0, 12.1, 20.0, "design_96_tfsf", tfsf=True)
        desc = ("design_96_tfsf: design_96 with the Gaussian beam injected by a one-sided TFSF plane (+z) "
                "instead of a soft sheet, 2000 steps fwd + 2000 reversed")
    elif name == "design_96_interp":
        sc = scenes.design_box_scene((96, 96, 96), 10, 40, 2000, 1234, 1.0, 12.1, 20.0, "design_96_interp", interp=True)
        desc = ("design_96_interp: design_96 with the |E|^2 plane taken from E interpolated to the cell centres, "
                "2000 steps fwd + 2000 reversed")
    elif name == "waveguide_600":
        sc = scenes.waveguide_600()
        desc = ("waveguide_600: 600^3 grid, 12-cell CPML, Si core eps=12.25 in SiO2 eps=2.085, 200^3 design "
                "box, Poynting-flux objective, 4000 steps fwd + 4000 reversed")
    elif name.startswith("waveguide_600_slab") and name[18:].isdigit():
        nz = int(name[18:])
        sc = scenes.waveguide_600_slab(nz)
        desc = ("%s: the 600x600 cross-section of waveguide_600 over %d z-planes (12-cell CPML on every face), "
                "200x200x%d design box, Poynting-flux objective" % (name, nz, nz - 24))
    elif name.startswith("design_") and name[7:].isdigit():
        n = int(name[7:])
        sc = scenes.design_box_scene((n, n, n), 10, max(8, (2 * n) // 5), 2000, 1234, name=name)
        desc = ("%s: %d^3 Yee grid, 10-cell CPML, Gaussian-beam Ex sheet, centred design box, |E|^2 plane "
                "objective, 2000 steps fwd + 2000 reversed" % (name, n))
    else:
        raise SystemExit("unknown workload " + name)
    return sc, desc


def bench_config(sc, desc, world):
    """The `config` object of the bench line (the same in both arms)."""
    return {"workload": desc, "grid": list(sc.n), "cells": sc.ncells, "time_steps": sc.nsteps,
            "pml": list(sc.pml), "design": list(sc.design_shape()),
            "l2": ("flushed between steps (256 MB write outside the timed events); the solve's working set "
                   "(%.1f GB) is also larger than the 126 MB L2" % (state_bytes(sc) / 1e9)),
            "parallelism": "replicas" if world > 1 else "single"}


def state_bytes(sc):
    """Approximate device bytes of one fwd+grad solve: both field buffers, a, both adjoint buffers
    (fp32) and the face history (2 tangential H components on six planes, every time step)."""
    nx, ny, nz = sc.n
    nxp = (nx + 31) // 32 * 32
    r = [sc.n[d] - sc.pml[2 * d] - sc.pml[2 * d + 1] + 1 for d in range(3)]
    face = 2 * 2 * (r[1] * r[2] + r[0] * r[2] + r[0] * r[1]) * 4 * sc.nsteps
    return (12 + 1 + 12) * nxp * ny * nz * 4 + face


def objective_grad(sc, nsteps):
    """dL/d(detector) for L = sum of every detector output (the |E|^2 plane sum or the flux sum)."""
    n = 0
    for d in sc.detectors:
        per_cell = d.kind in (scenes.DET_PLANE_E2_SUM, scenes.DET_PLANE_E2_SUM_INTERP)
        n += int(np.prod([d.hi[k] - d.lo[k] for k in range(3)])) if per_cell else nsteps
    return np.ones(n, dtype=np.float64)


# ---- algorithmic bytes per launch (the roofline numerator) ------------------------------------------
def slab_cells(sc):
    """Cells inside the layer of each axis, summed over axes (a cell in two layers counts twice)."""
    nx, ny, nz = sc.n
    tot = 0
    for d in range(3):
        w = sc.pml[2 * d] + sc.pml[2 * d + 1]
        tot += w * (nx * ny * nz // sc.n[d])
    return tot


def algorithmic_bytes(kind, sc):
    """Bytes one launch of kernel `kind` must move at minimum (fp32 fields, fp64 dL/da)."""
    N = sc.ncells
    slab = slab_cells(sc)
    design = int(np.prod(sc.design_shape()))
    if kind == "rev_E":         # H r, E r/w, a r, E-bar r, H-bar r/w; psi-bar_E r + w; dL/da r/w
        return 76 * N + 16 * slab + 16 * design
    if kind == "rev_H":         # E r, H r/w, H-bar r, E-bar r/w; psi-bar_H r + w
        return 72 * N + 16 * slab
    if kind == "fused_fwd":     # E, H r/w, a r; psi_E and psi_H of 4 components per layer axis
        return 52 * N + 32 * slab
    if kind == "inv_fused":     # E, H r/w, a r; on design cells E-bar r and dL/da r/w
        return 52 * N + 28 * design
    if kind == "adj_fused":     # E-bar, H-bar r/w, a r; psi-bar_E and psi-bar_H of 4 components per layer axis
        return 52 * N + 32 * slab
    return None


KERNEL_SOURCE = {"fused_fwd": "fdtd_fused.cu", "rev_E": "fdtd_reverse.cu", "rev_H": "fdtd_reverse.cu",
                 "inv_fused": "fdtd_inverse.cu", "adj_fused": "fdtd_adjoint.cu"}


def kernel_source_hash(kind):
    import hashlib
    path = os.path.join(ROOT, "paper_2412_12360_b300", "csrc", KERNEL_SOURCE.get(kind, ""))
    if not os.path.isfile(path):
        return None
    return hashlib.sha256(open(path, "rb").read()).hexdigest()


def recorded_traffic(kind, workload_name):
    """DRAM bytes per launch of `kind` on this workload from a recorded ncu capture
    (profiles/traffic.json), or None if there is none or the kernel source changed since."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    e = rec.get(workload_name, {}).get(kind)
    if not e or e.get("source_sha256") != kernel_source_hash(kind):
        return None
    return e.get("dram_bytes_per_launch")


FWD_KERNELS = ("fused_fwd",)
REV_KERNELS = ("rev_E", "rev_H", "inv_fused", "adj_fused", "det_adj")


def roofline(prof, sc, args, fwd_step_ms, rev_step_ms):
    """Roofline of the dominant stencil kernel from the sampled CUDA events of the timed region.

    prof: {kernel: (total ms, launches timed)}. Every stencil kernel launches once per time step, so
    the largest mean launch time is the largest share. The event brackets around a sampled launch
    add a few microseconds to it; so that a kernel's time never exceeds the time of the step it is
    part of, the means of each phase (forward kernels; reverse kernels and detector adjoints) are
    scaled by min(1, measured unbracketed time per time step of that phase / their summed means)."""
    if not prof:
        return None
    mean = {k: v[0] / max(v[1], 1) for k, v in prof.items()}
    fwd_sum = sum(mean.get(k, 0.0) for k in FWD_KERNELS)
    rev_sum = sum(mean.get(k, 0.0) for k in REV_KERNELS)
    scale_f = min(1.0, fwd_step_ms / fwd_sum) if fwd_sum > 0 else 1.0
    scale_r = min(1.0, rev_step_ms / rev_sum) if rev_sum > 0 else 1.0
    ms = {k: v * (scale_f if k in FWD_KERNELS else (scale_r if k in REV_KERNELS else 1.0)) for k, v in mean.items()}
    kname = max((k for k in ms if algorithmic_bytes(k, sc)), key=ms.get)
    avg_ms = ms[kname]
    nbytes = algorithmic_bytes(kname, sc)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    src = "measured (copy bandwidth, MEASURED_PEAKS.json hbm_gbs)"
    if not peak:
        peak, src = 6400.0, "fallback"
    achieved = nbytes / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": src,
            "traffic": args.traffic if args.traffic is not None else recorded_traffic(kname, args.workload),
            "bytes_per_launch": nbytes, "avg_launch_ms": round(avg_ms, 5),
            "kernel_ms_per_launch": {k: round(v, 5) for k, v in ms.items() if k in FWD_KERNELS or k in REV_KERNELS},
            # the face copies run on a second stream beside the stencil kernels: their brackets measure the
            # time from their start until they finish, waiting for SM slots included
            "side_stream_ms_per_launch": {k: round(v, 5) for k, v in ms.items()
                                          if k not in FWD_KERNELS and k not in REV_KERNELS},
            "kernel_frac": {k: round(algorithmic_bytes(k, sc) / (v * 1e-3) / 1e9 / peak, 4)
                            for k, v in ms.items() if algorithmic_bytes(k, sc)},
            "timing": {"method": "CUDA events around every %d-th launch of each kernel on its own stream inside "
                                 "the timed solves; per-phase means scaled by min(1, unbracketed time per step / "
                                 "summed means)" % args.profile_every,
                       "fwd_step_ms": round(fwd_step_ms, 5), "fwd_kernels_ms": round(fwd_sum, 5),
                       "rev_step_ms": round(rev_step_ms, 5), "rev_kernels_ms": round(rev_sum, 5),
                       "scale_fwd": round(scale_f, 4), "scale_rev": round(scale_r, 4)}}


# ---- clocks during the timed region ------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu_id)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, power, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        loaded = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ---- distributed helpers ------------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours") else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    from paper_2412_12360_b300 import ranks
    return ranks.reduce_time_and_work(x, 0.0, device)[0] if world > 1 else x


# ---- CPU baseline (the oracle as it stands) ------------------------------------------------------------
# The oracle keeps FP64 fields, CPML memories (over the whole grid) and adjoints: about 70 GB for the
# 600^3 grid, allocated and zeroed on every call. It is timed on a z-slab of that grid (the full x-y
# cross-section with its CPML, core, source and flux planes), with the set-up of each call measured
# by a zero-step call and taken out, so the rate is the oracle's per-cell-step rate.
SAMPLE_OF = {"waveguide_600": "waveguide_600_slab64"}


def oracle_sample(sc, nsteps):
    """Seconds of the oracle's forward + time-reversal gradient of nsteps steps on the scene's grid."""
    from oracle import oracle as O
    g = np.ones(O.detector_total(sc, nsteps))
    t0 = time.perf_counter()
    O.gradient(sc, nsteps, g, O.METHOD_TIME_REVERSAL)
    return time.perf_counter() - t0


def oracle_setup_s(sc):
    """Seconds of one oracle call that runs no time step (allocation and set-up), median of 2."""
    return statistics.median([oracle_sample(sc, 0) for _ in range(2)])


def sample_scene(workload_name):
    name = SAMPLE_OF.get(workload_name, workload_name)
    sc, _ = workload(name)
    return sc, name


def cpu_baseline(workload_name, target_s=15.0, one_core=True):
    sc, sname = sample_scene(workload_name)
    setup = oracle_setup_s(sc)
    probe = 2
    t = oracle_sample(sc, probe) - setup
    steps = max(probe, min(400, int(probe * target_s / max(t, 1e-3))))
    t = oracle_sample(sc, steps) - setup
    cores = os.cpu_count()
    out = {"value": sc.ncells * steps / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%s: %dx%dx%d grid, %d time steps fwd + %d reversed (FP64 C++ oracle, OpenMP over "
                     "z-planes in the forward and inverse loops, serial adjoint loops), %.1f s after %.1f s of "
                     "per-call set-up (measured by a zero-step call, not counted)"
                     % (sname, sc.n[0], sc.n[1], sc.n[2], steps, steps, t, setup)}
    if one_core:  # the same oracle on one core (a child process with OMP_NUM_THREADS=1)
        code = ("import sys; sys.path.insert(0, %r); import bench; sc, _ = bench.workload(%r); "
                "print(bench.oracle_sample(sc, %d))")
        env = dict(os.environ, OMP_NUM_THREADS="1")
        try:
            run = lambda k, to: float(subprocess.run([sys.executable, "-c", code % (ROOT, sname, k)], env=env,
                                                     capture_output=True, text=True, timeout=to).stdout.split()[-1])
            s0 = run(0, 300)
            t1 = run(1, 600) - s0
            s1 = max(1, min(steps, int(target_s / 2 / max(t1, 1e-3))))
            t1 = run(s1, 900) - s0
            out["value_1core"] = sc.ncells * s1 / t1 / 1e9
            out["sample_1core"] = "%d time steps fwd + %d reversed on 1 core, %.1f s (set-up %.1f s not counted)" % (
                s1, s1, t1, s0)
        except (subprocess.SubprocessError, ValueError, IndexError) as e:
            out["value_1core"] = None
            out["sample_1core"] = "not measured: %s" % type(e).__name__
    return out


# ---- our arm ----------------------------------------------------------------------------------------------
def run_ours(args, world, rank, local):
    import torch
    from paper_2412_12360_b300 import fdtd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc, desc = workload(args.workload)
    if args.time_steps:
        sc.nsteps = args.time_steps
        desc += " [time steps overridden: %d]" % args.time_steps
    T = sc.nsteps
    stream = torch.cuda.Stream(device=dev)
    solver = fdtd.Solver(sc, stream=stream)
    gvec = objective_grad(sc, T)
    g_dev = torch.from_numpy(gvec).to(dev)
    grad_dev = torch.zeros(sc.design_shape(), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2

    def solve():
        solver.fdtd_forward(T, record_faces=True)
        solver.fdtd_backward(g_dev, grad_dev)

    def timed(fn, k):
        times = []
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            times.append((a, b))
        stream.synchronize()
        return [a.elapsed_time(b) for a, b in times]

    # forward-only rate (reported beside the headline): median of 3 after one untimed call that
    # captures its graph
    solver.fdtd_forward(T, record_faces=False)
    stream.synchronize()
    fwd_ms = statistics.median(timed(lambda: solver.fdtd_forward(T, record_faces=False), 3))

    # warm-up with the stencil-kernel sampling already on, so that the graphs the timed region
    # replays (captured per sampling setting) are built before it; then clear the warm-up samples
    solver.fdtd_profile(True, args.profile_every)
    for _ in range(args.warmup):
        solve()
    stream.synchronize()
    solver.fdtd_profile(True, args.profile_every)

    # timed region: K fwd+grad solves, stencil kernels sampled with CUDA events
    l0 = solver.fdtd_launch_count()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = ClockSampler(gpu_id)
    if rank == 0:
        clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    step_ms = timed(solve, args.steps)
    torch.cuda.synchronize(dev)
    barrier(world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop() if rank == 0 else None
    launches = solver.fdtd_launch_count() - l0
    prof = solver.fdtd_profile_read()
    solver.fdtd_profile(False)
    total_ms = sum(step_ms)
    total_ms_max = max_over_ranks(total_ms, world, dev)
    ms_per_step = total_ms_max / args.steps
    value = world * sc.ncells * T * args.steps / (total_ms_max * 1e-3) / 1e9
    fwd_value = sc.ncells * T / (fwd_ms * 1e-3) / 1e9 * world

    roof = roofline(prof, sc, args, fwd_ms / T, (statistics.median(step_ms) - fwd_ms) / T)

    # end to end through the C ABI with host buffers (copies inside the timed region), over a few
    # solves after one untimed one
    e2e = None
    if not args.no_e2e:
        dlo, dhi = sc.design_lo, sc.design_hi
        box = np.ascontiguousarray(sc.eps_inv[dlo[2]:dhi[2], dlo[1]:dhi[1], dlo[0]:dhi[0]])
        box_h = torch.from_numpy(box).pin_memory()
        g_h = torch.from_numpy(gvec).pin_memory()
        det_h = torch.zeros(solver.fdtd_detector_total(), dtype=torch.float64).pin_memory()
        grad_h = torch.zeros(sc.design_shape(), dtype=torch.float32).pin_memory()
        h2d = box_h.numel() * 4 + g_h.numel() * 8
        d2h = det_h.numel() * 8 + grad_h.numel() * 4

        def e2e_step():
            solver.fdtd_set_design_eps_inv(box_h)
            solver.fdtd_forward(T, record_faces=True)
            solver.fdtd_read_detectors(det_h)
            solver.fdtd_backward(g_h, grad_h)
            solver.fdtd_synchronize()

        e2e_step()
        barrier(world)
        tt = []
        for _ in range(args.e2e_steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            stream.synchronize()
            t1 = time.perf_counter()
            e2e_step()
            tt.append(time.perf_counter() - t1)
        tmax = max_over_ranks(sum(tt), world, dev)
        e2e = {"value": world * sc.ncells * T * args.e2e_steps / tmax / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps,
               "timing": "host wall clock around each call sequence (upload design eps, forward, read "
                         "detectors, upload dL/d(det), backward, read dL/deps, synchronise)"}
    solver.close()

    if rank != 0:
        return
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": bench_config(sc, desc, world),
            "fwd_value": round(fwd_value, 4), "fwd_ms": round(fwd_ms, 3),
            "roofline": roof, "e2e": e2e, "gpu_launches": int(launches * world),
            "wall_s": round(wall, 3), "clocks": clk}
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds, not args.time_steps)
    print(json.dumps(line), flush=True)


# ---- served stream (continuous batching) -----------------------------------------------------------------
def run_serve(args, world, rank, local):
    """Poisson arrivals of fwd+grad requests (grids from {64^3, 96^3, 128x128x256, 200^3}, 1000-3000
    steps, random densities), served with continuous batching (grouped launches), at several offered
    loads, against the same requests solved one after another."""
    import torch
    from paper_2412_12360_b300 import ranks, serve

    torch.cuda.set_device(local)
    rng = np.random.default_rng(7)
    ids = ranks.shard(args.serve_requests, world, rank)
    grids = scenes.SERVED_GRIDS if args.serve_grids == "mix" else scenes.SERVED_GRIDS[:2]
    all_scenes = [scenes.served_request(r, rng, grids) for r in range(args.serve_requests)]
    mine = [all_scenes[r] for r in ids]
    cells = sum(sc.ncells * sc.nsteps for sc in mine)
    serve.run_sequential(mine[:1])                     # warm-up: library load, first set-ups
    t0 = time.perf_counter()
    seq = serve.run_sequential(mine)
    t_seq = time.perf_counter() - t0
    mean_service = t_seq / max(1, len(mine))
    t_seq_max, cells_all = ranks.reduce_time_and_work(t_seq, cells)
    per_load = []
    for load in args.serve_loads:
        arng = np.random.default_rng(8 + rank)
        gaps = arng.exponential(mean_service / load, size=len(mine))
        with serve.Server(max_inflight=args.serve_slots, chunk_steps=args.serve_chunk,
                          group_bytes=args.serve_group_mb << 20) as srv:
            t0 = time.perf_counter()
            futs = []
            for sc, gap in zip(mine, gaps):
                time.sleep(float(gap))
                futs.append(srv.submit(sc))
            res = [f.result() for f in futs]
            t_srv = time.perf_counter() - t0
            peak, calls = srv.peak_inflight, srv.group_calls
        same = all(np.array_equal(a[0], r.detectors) and np.array_equal(a[1], r.dL_deps) for a, r in zip(seq, res))
        lat = serve.latency_stats(res)
        t_srv_max, _ = ranks.reduce_time_and_work(t_srv, cells)
        per_load.append({"offered_load": load, "value": round(cells_all / t_srv_max / 1e9, 4),
                         "p50_s": round(lat["p50_s"], 4), "p99_s": round(lat["p99_s"], 4),
                         "mean_latency_s": round(lat["mean_s"], 4), "peak_inflight": peak,
                         "grouped_calls": calls, "wall_s": round(t_srv_max, 3),
                         "results_equal_alone_and_in_mix": bool(same)})
    if rank != 0:
        return
    top = per_load[-1]
    line = {"metric": "served fwd+grad solves: p50/p99 latency and Gcell-steps/s", "unit": "Gcell-steps/s",
            "value": top["value"], "n_gpus": world, "higher_is_better": True,
            "sequential_value": round(cells_all / t_seq_max / 1e9, 4),
            "served_over_sequential": round(top["value"] / (cells_all / t_seq_max / 1e9), 4),
            "p50_s": top["p50_s"], "p99_s": top["p99_s"], "offered_load": top["offered_load"],
            "loads": per_load, "requests": args.serve_requests, "slots": args.serve_slots,
            "chunk_steps": args.serve_chunk, "group_mib": args.serve_group_mb,
            "results_equal_alone_and_in_mix": all(p["results_equal_alone_and_in_mix"] for p in per_load),
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "served stream: Poisson arrivals (seed 8) at offered loads %s of the sequential "
                                   "capacity, grids {%s} (seed 7), 1000-3000 steps, 10-cell CPML, random rho per "
                                   "request (seed 10000+id), %d requests; sequential: the same requests solved one "
                                   "after another with the same one-shot handles"
                                   % (args.serve_loads, ", ".join("x".join(map(str, g)) for g in grids),
                                      args.serve_requests)}}
    print(json.dumps(line), flush=True)


def run_batched(args, world, rank, local):
    """A batch of designs of one scene (default: 16 designs of a 240x240x960 waveguide, 12-cell CPML,
    120^3 design box each, rho seeds 500..515, flux objective, 3000 steps) through the
    torch.autograd.Function: forward of every design, then the backward. Each design's face history is
    kept whole while it fits in device memory beside the states and the histories planned before it,
    else kept as segments (the faces of the last segment and the segment start states; the reverse
    sweep regenerates the earlier segments), else recomputed (autograd.history_plan). Beside the
    throughput: the directional derivative of design 0 along a uniform density shift against central
    differences, and central differences on 4 voxels (indices from seed 99)."""
    import torch
    from paper_2412_12360_b300 import autograd, fdtd, ranks

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    T = args.time_steps or 3000
    ids = ranks.shard(args.batch, world, rank)
    scs = [scenes.waveguide_batch_member(b, T) for b in ids]
    free, _ = torch.cuda.mem_get_info(dev)
    plan, extra = autograd.history_plan(scs, T, int(0.85 * free))
    eps_lo, eps_hi = scs[0].extra["eps_lo"], scs[0].extra["eps_hi"]
    solvers = [fdtd.Solver(sc) for sc in scs]
    for s in solvers:  # each design solves once: direct launches rather than captured graphs
        s.fdtd_set_graphs(False)
    rho = torch.stack([torch.from_numpy(sc.extra["rho"]) for sc in scs]).to(dev).requires_grad_(True)

    def batch_step():
        rho.grad = None
        det = autograd.solve(rho, solvers, eps_lo, eps_hi, T, plan)
        loss = det.sum()          # L = sum over steps of the flux through the detector plane, per design
        loss.backward()
        return det

    torch.cuda.synchronize(dev)
    barrier(world)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    det = batch_step()
    b.record()
    torch.cuda.synchronize(dev)
    barrier(world)
    t = a.elapsed_time(b) * 1e-3
    cells = sum(sc.ncells * T for sc in scs)
    t_max, cells_all = ranks.reduce_time_and_work(t, cells)
    grad0 = rho.grad[0].detach().clone() if rank == 0 else None

    checks = None
    if rank == 0 and not args.no_fd:
        s0 = solvers[0]
        s0.fdtd_set_segment_steps(0)
        rho0 = rho[0].detach().clone()

        def loss_at(r):
            s0.fdtd_set_design_density(r, eps_lo, eps_hi)
            s0.fdtd_forward(T)
            return float(np.sum(s0.detectors()))

        checks = {"directional": [], "voxels": []}
        g0 = grad0.double()
        for h in (1e-3, 1e-2):   # every design voxel shifted by h: dL/dh = sum of dL/drho
            fd = (loss_at(rho0 + h) - loss_at(rho0 - h)) / (2 * h)
            ad = float(g0.sum())
            checks["directional"].append({"delta_rho": h, "fd": fd, "autograd": ad, "rel_err": abs(fd - ad) / abs(fd)})
        rng = np.random.default_rng(99)
        shape = scs[0].design_shape()
        vox = [tuple(int(rng.integers(d)) for d in shape) for _ in range(4)]
        for v in vox:
            row = {"voxel": list(v), "autograd": float(grad0[v])}
            for h in (2e-2, 5e-2):
                rp, rm = rho0.clone(), rho0.clone()
                rp[v] += h
                rm[v] -= h
                row["fd_%g" % h] = (loss_at(rp) - loss_at(rm)) / (2 * h)
            checks["voxels"].append(row)
        s0.fdtd_set_design_density(rho0, eps_lo, eps_hi)
    for s in solvers:
        s.close()
    if rank != 0:
        return
    counts = {"whole": sum(1 for p in plan if p == 0), "segmented": sum(1 for p in plan if p > 0),
              "recomputed": sum(1 for p in plan if p < 0)}
    line = {"metric": "Gcell-steps/s fwd+grad (batched autograd)", "unit": "Gcell-steps/s",
            "value": round(cells_all / t_max / 1e9, 4), "n_gpus": world, "higher_is_better": True,
            "seconds": round(t_max, 3), "designs": args.batch, "plan": plan, "histories": counts,
            "extra_forward_fraction": round(extra / (len(scs) * T), 4), "dtype": "f32", "data": "synthetic",
            "scaling": "weak", "gradient_checks": checks,
            "config": {"workload": "%d designs of a 240x240x960 waveguide (along z), 12-cell CPML, 120^3 design box "
                                   "each, rho~U[0,1) seeds 500.., flux objective, %d steps; per design the face "
                                   "history is kept whole (plan 0), as segments of L steps (plan L) or recomputed "
                                   "(plan -1), whichever fits first in device memory" % (args.batch, T)}}
    print(json.dumps(line), flush=True)


# ---- reference arm: the FP64 oracle on host cores -------------------------------------------------------
def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle as it stands on the host cores, each bench step a bounded
    sample of the workload (the slab sample for the 600^3 solve), the per-call set-up taken out."""
    if rank != 0:
        return
    sc_full, desc = workload(args.workload)
    sc, sname = sample_scene(args.workload)
    setup = oracle_setup_s(sc)
    probe = max(oracle_sample(sc, 2) - setup, 1e-3) / 2
    # time steps per bench step: the whole run (warm-up included) within about two minutes of compute
    per_step_budget = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    steps = max(1, min(200, int(per_step_budget / probe)))
    for _ in range(args.warmup):
        oracle_sample(sc, steps)
    ts = [oracle_sample(sc, steps) - setup for _ in range(args.steps)]
    total = sum(ts)
    value = sc.ncells * steps * args.steps / total / 1e9
    cores = os.cpu_count()
    sample = ("%s: %dx%dx%d grid, %d time steps fwd + %d reversed per bench step (FP64 C++ oracle); the "
              "per-call set-up (%.1f s, measured by a zero-step call) is not counted"
              % (sname, sc.n[0], sc.n[1], sc.n[2], steps, steps, setup))
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(sc_full, desc, world),
            "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_design(args, world, rank, local):
    """The inverse-design loop (design.DesignLoop) on the workload's design box: per iteration the
    projection, the density map, the recorded forward, the objective (the negated sum of the
    workload's detector outputs: maximise the |E|^2 plane or the flux), the reverse sweep for dL/drho
    and the Adam step. beta = 0 for the first half of the iterations, then 8 (binarisation)."""
    import torch
    from paper_2412_12360_b300 import design, fdtd

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sc, desc = workload(args.workload)
    if args.time_steps:
        sc.nsteps = args.time_steps
        desc += " [time steps overridden: %d]" % args.time_steps
    T = sc.nsteps
    eps_lo, eps_hi = sc.extra.get("eps_lo", 1.0), sc.extra.get("eps_hi", 12.1)
    stream = torch.cuda.Stream(device=dev)
    iters = args.design_iters
    theta0 = torch.full(sc.design_shape(), 0.5, dtype=torch.float32, device=dev)
    beta_of = lambda it: 0.0 if it < iters // 2 else 8.0
    with torch.cuda.stream(stream):
        solver = fdtd.Solver(sc, stream=stream)
        loop = design.DesignLoop(solver, theta0, eps_lo, eps_hi, T, lambda det: (-det.sum(), -torch.ones_like(det)),
                                 lr=0.02, beta_of=beta_of)
        for _ in range(args.warmup):       # warm-up iterations (graph captures), then a fresh loop
            loop.step()
        stream.synchronize()
        loop = design.DesignLoop(solver, theta0, eps_lo, eps_hi, T, lambda det: (-det.sum(), -torch.ones_like(det)),
                                 lr=0.02, beta_of=beta_of)
        barrier(world)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        losses = [loop.step() for _ in range(iters)]
        b.record(stream)
        stream.synchronize()
        ms = a.elapsed_time(b)
        losses = [float(x) for x in losses]
        rho = loop.rho.float()
        binary = float(((rho < 0.05) | (rho > 0.95)).float().mean())
        solver.close()
    ms_max = max_over_ranks(ms, world, dev)
    if rank != 0:
        return
    line = {"metric": "inverse-design iterations (fwd+grad+Adam) in Gcell-steps/s", "unit": UNIT,
            "value": round(world * sc.ncells * T * iters / (ms_max * 1e-3) / 1e9, 4), "n_gpus": world,
            "iterations": iters, "ms_per_iteration": round(ms_max / iters, 3), "higher_is_better": True,
            "loss_first": losses[0], "loss_last": losses[-1], "binary_fraction_last": round(binary, 4),
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc + "; design loop: theta0 = 0.5, Adam lr 0.02, projection beta 0 then 8",
                       "grid": list(sc.n), "time_steps": T, "design": list(sc.design_shape())}}
    print(json.dumps(line), flush=True)


def run_checkpoint(args, world, rank, local):
    """Time reversal against the checkpointing gradients of Sec. 2.2 on the same workload and device:
    per gradient method the device time of the forward + gradient, the forward steps evaluated and the
    device memory the method holds beyond the solver (face history, or stored full states)."""
    import torch
    from paper_2412_12360_b300 import fdtd

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sc, desc = workload(args.workload)
    if args.time_steps:
        sc.nsteps = args.time_steps
        desc += " [time steps overridden: %d]" % args.time_steps
    T = sc.nsteps
    stream = torch.cuda.Stream(device=dev)
    g_dev = torch.from_numpy(objective_grad(sc, T)).to(dev)
    grad = torch.zeros(sc.design_shape(), dtype=torch.float32, device=dev)
    nx, ny, nz = sc.n
    nxp = (nx + 31) // 32 * 32
    L = [sc.pml[0] + sc.pml[1], sc.pml[2] + sc.pml[3], sc.pml[4] + sc.pml[5]]
    pf = 2 * (nz * ny * L[0] + nz * L[1] * nxp + L[2] * ny * nxp)
    state_bytes = (6 * nxp * ny * nz + 2 * pf) * 4
    face_bytes = fdtd.footprint_bytes(sc, T, True) - fdtd.footprint_bytes(sc, T, False)
    runs = [("time_reversal", None, None), ("halving", 0, 0)] + [("treeverse", 1, k) for k in args.ckpt_slots]
    out = []
    with torch.cuda.stream(stream):
        solver = fdtd.Solver(sc, stream=stream)
        for name, method, slots in runs:
            def once():
                if method is None:
                    solver.fdtd_forward(T, record_faces=True)
                    solver.fdtd_backward(g_dev, grad)
                    return T
                solver.fdtd_forward(T)
                return solver.fdtd_backward_checkpointed(g_dev, grad, method, slots)
            once()  # warm-up (graph capture, tables)
            stream.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            steps = once()
            b.record(stream)
            stream.synchronize()
            ms = a.elapsed_time(b)
            nstates = None if method is None else (math.ceil(math.log2(T)) + 1 if method == 0 else slots)
            held = face_bytes if method is None else nstates * state_bytes
            out.append({"method": name, "slots": nstates, "ms": round(ms, 2),
                        "gcell_steps_per_s": round(sc.ncells * T / (ms * 1e-3) / 1e9, 4),
                        "forward_steps_in_gradient": steps, "held_bytes": int(held)})
        solver.close()
    if rank != 0:
        return
    line = {"metric": "fwd+grad time and memory: time reversal vs checkpointing (Sec. 2.2)", "unit": "ms",
            "value": out[0]["ms"], "higher_is_better": False, "n_gpus": world, "methods": out,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "grid": list(sc.n), "time_steps": T,
                       "state_bytes": state_bytes, "face_history_bytes": int(face_bytes)}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="waveguide_600")
    ap.add_argument("--time-steps", type=int, default=None,
                    help="override the workload's time steps (profiling runs only; not a bench line)")
    ap.add_argument("--profile-every", type=int, default=64,
                    help="time every Nth step's kernels with CUDA events (each bracket costs a few us)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture (null if stale)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2, help="solves timed end to end through host buffers")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve", action="store_true", help="measure the continuous-batching server instead")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-loads", type=float, nargs="+", default=[0.5, 0.9, 1.5],
                    help="offered loads (arrival rate / sequential capacity), one served run each")
    ap.add_argument("--serve-chunk", type=int, default=32, help="time steps per grouped call")
    ap.add_argument("--serve-grids", choices=["mix", "small"], default="mix",
                    help="served grids: the four-size mix, or only the 64^3 and 96^3 requests")
    ap.add_argument("--serve-slots", type=int, default=4, help="requests in flight at once (at most 8)")
    ap.add_argument("--serve-group-mb", type=int, default=64,
                    help="running requests stepped in groups of at most this many MiB of step bytes (0: one group)")
    ap.add_argument("--batched", action="store_true", help="measure the batched autograd workload instead")
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--no-fd", action="store_true", help="skip the finite-difference check of --batched")
    ap.add_argument("--checkpoint", action="store_true",
                    help="compare time reversal with the checkpointing gradients instead")
    ap.add_argument("--ckpt-slots", type=int, nargs="+", default=[4, 12])
    ap.add_argument("--design-loop", action="store_true", help="measure the inverse-design loop instead")
    ap.add_argument("--design-iters", type=int, default=10)
    args = ap.parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.serve:
        run_serve(args, world, rank, local)
    elif args.batched:
        run_batched(args, world, rank, local)
    elif args.design_loop:
        run_design(args, world, rank, local)
    elif args.checkpoint:
        run_checkpoint(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
