#!/usr/bin/env python
"""Benchmark of the HWENO-I hot path on GB300: FP64 2D Euler, 4096 x 4096 cells, periodic
[0, 2]^2, smooth wave rho = 1 + 0.2 sin(pi (x + y)), velocity (0.7, 0.3), P = 1, SSP-RK3 at CFL 0.6
with the step size computed on the device every step.

One benchmark step = one full SSP-RK3 step (three stages: cell, face and update kernels each) over
the whole grid.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 4096]

--impl reference times the CPU oracle (plain C++ FP64 on all host cores, lines of each sweep split
over threads) on the same workload: one oracle SSP-RK3 step of the full grid per benchmark step.
Multi-GPU (torchrun): every rank advances its own 4096^2 grid (independent replicas, weak
scaling); the time is the maximum over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D Euler HWENO-I Mcell-updates/s & HBM roofline %; batched/adjoint vs plain"
UNIT = "Mcell-updates/s"
# FP64 peak derived from the SM count (152), the maximum SM clock (2070 MHz) and the FP64 rate of
# GB300 (2 DFMA per SM per clock = 4 flop/clk/SM): 152 * 2.07e9 * 4, reported beside the peak the
# benchmark measures on its own GPU (hweno_selftest_fp64_peak).
FP64_PEAK_FLOPS_DERIVED = 152 * 2.07e9 * 4
# algorithmic HBM bytes of one SSP-RK3 step per 2D Euler cell: the state planes each stage must
# touch once (stage 1: read 12, write 12, write the 8-plane base; stages 2, 3: read 12, read the
# base 12, write 12) = 104 planes of 8 bytes
STEP_BYTES_PER_CELL = 104 * 8
HBM_PEAK_GBS_FALLBACK = 6800.0
# DRAM bytes per face of the 2D Euler face kernel from an ncu capture at 2048^2 (profiles/); the
# traffic grows in proportion to the faces, so a 4096^2 launch moves this times its faces.
FACE_TRAFFIC_BYTES_PER_FACE = 285.2  # ncu dram bytes per face, 2048^2 capture of the current face kernel
# device slots (each with its state, workspace and stream) of the end-to-end pipeline
E2E_DEPTH = 3
# from the same capture: FP64 pipe activity and FP64 instructions per face (the hardware's side of
# the roofline fraction, which counts the scheme's operations as written)
FACE_FP64_PIPE_ACTIVE = 0.958
FACE_FP64_INSTR_PER_FACE = 666


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The largest x of all ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws: int, cells: int, steps: int, ms_max: float) -> float:
    """Whole-job Mcell-updates/s: every rank advances its own grid (weak scaling)."""
    return ws * cells * steps / (ms_max * 1e-3) / 1e6


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def cpu_baseline(steps: int = 2, n: int = 4096):
    """The oracle on all host cores: `steps` SSP-RK3 steps of the benchmark's own workload (the
    4096^2 smooth wave), outside any GPU timing."""
    import oracle as O
    import workloads as W

    cores = O.set_threads(0)
    S, dx, dy = W.euler2d_smooth(n)
    cfg = O.make_cfg(2, O.EULER, n, n, dx=dx, dy=dy)
    dt = O.cfl_dt(cfg, S, 0.6)
    t0 = time.perf_counter()
    O.steps(cfg, S, dt, steps)
    sec = time.perf_counter() - t0
    return {"value": n * n * steps / sec / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} oracle SSP-RK3 steps of the same {n}x{n} smooth-wave grid, lines of each sweep "
                      f"split over {cores} host threads, {sec:.1f} s"}


def run_parity(dev, n: int, nsteps: int, envelope: bool = False):
    """The benchmark's workload advanced nsteps CFL steps on the GPU and by the oracle (all host
    cores), compared element by element: the relative max-norm of every (field, component) plane
    and the end times (dt of every step from each side's own state).  envelope: also the same
    distance between the oracle's run and its run from the input moved by one ulp (random signs),
    the rounding noise of the scheme on this workload.  Outside the timed region."""
    import numpy as np

    import oracle as O
    import workloads as W
    from paper_2411_11229_gb300 import Solver

    S, dx, dy = W.euler2d_smooth(n)
    s = Solver(2, "euler", n, n, dx=dx, dy=dy, device=dev)
    s.set_state(S)
    s.set_time(0.0, 0.0)
    s.step(0.0, nsteps)
    _, tg = s.last_dt()
    gpu = s.state.cpu().numpy()
    del s
    cores = O.set_threads(0)
    cfg = O.make_cfg(2, O.EULER, n, n, dx=dx, dy=dy)
    t0 = time.perf_counter()
    ref, k, t = O.run(cfg, S, 0.0, 0.6, 1.0, max_steps=nsteps)
    sec = time.perf_counter() - t0
    def rel_max(x):
        a, b = x.reshape(12, -1), ref.reshape(12, -1)
        return np.abs(a - b).max(axis=1) / np.maximum(np.abs(b).max(axis=1), 1e-300)

    rel = rel_max(gpu)
    out = {"workload": f"2D Euler {n}x{n} smooth wave, {nsteps} CFL steps", "steps": k,
           "rel_max_per_plane": [float(x) for x in rel], "rel_max": float(rel.max()), "t_gpu": tg, "t_oracle": t,
           "oracle_seconds": sec, "oracle_threads": cores}
    if envelope:
        del gpu
        sign = np.random.default_rng(11).choice([-1.0, 1.0], S.shape)
        pert, _, tp = O.run(cfg, S * (1.0 + sign * 2.0 ** -52), 0.0, 0.6, 1.0, max_steps=nsteps)
        env = rel_max(pert)
        out.update({"oracle_one_ulp_rel_max_per_plane": [float(x) for x in env],
                    "oracle_one_ulp_rel_max": float(env.max()), "t_oracle_one_ulp": tp})
    return out


def fp64_probe(dev) -> dict:
    """The library's FP64 issue probe on this GPU (independent register-operand DFMA chains on
    every SM, best of 5 launches): DFMA per second and flops per second (2 per DFMA)."""
    import ctypes

    import torch

    from paper_2411_11229_gb300 import _capi as C

    scratch = torch.zeros(4, dtype=torch.float64, device=dev)
    rate, per = ctypes.c_double(), ctypes.c_double()
    C.check(C.load().hweno_selftest_fp64_peak(ctypes.c_void_p(scratch.data_ptr()), 5,
                                              ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream),
                                              ctypes.byref(rate), ctypes.byref(per)), "hweno_selftest_fp64_peak")
    return {"dfma_per_s": rate.value, "flops": 2.0 * rate.value, "dfma_per_launch": per.value}


def run_batched(dev, steps: int = 3, only_1d: bool = False):
    """The uneven batched sweep: 256 1D Euler lines (N log-uniform in [128, 16384], seeded Riemann
    data) and 32 2D Euler grids (sides in {128, 256, 512, 1024}), every instance with its own CFL
    step.  Batched path (one persistent launch per stage, CUDA graph, autotuned launch shape)
    against one launch per instance and kernel.  only_1d: the 256 lines alone.  The timed batched
    steps of the full sweep run between cudaProfilerStart and cudaProfilerStop (no effect without a
    profiler; `ncu --profile-from-start off` records just those launches)."""
    import numpy as np
    import torch

    import workloads as W
    from paper_2411_11229_gb300 import Batch

    pairs = W.batched_states(W.batched_instances())
    if only_1d:
        pairs = [(d, S) for d, S in pairs if int(d["dim"]) == 1]
    cells = sum(int(np.prod(S.shape[2:])) for _, S in pairs)
    res = {"instances": len(pairs), "cells": cells}
    times = {}
    for mode in ("plain", "batched"):
        b = Batch([d for d, _ in pairs], device=dev)
        for i, (_, S) in enumerate(pairs):
            b.set_state(i, S)
        if mode == "batched":
            res["tuned_tiles_per_item"], res["tuned_blocks_per_sm"] = b.tune()
        b.set_time(0.0)
        run = b.step if mode == "batched" else b.step_plain
        run(1)
        b.sync()
        l0 = b.launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        window = mode == "batched" and not only_1d
        if window:
            torch.cuda.profiler.start()
        e0.record(b.stream)
        run(steps)
        e1.record(b.stream)
        b.sync()
        if window:
            torch.cuda.profiler.stop()
        times[mode] = e0.elapsed_time(e1) / steps
        res[f"launches_per_step_{mode}"] = (b.launch_count() - l0) // steps
        b.dts()
        del b
        torch.cuda.empty_cache()
    res["ms_per_step_plain"] = times["plain"]
    res["ms_per_step_batched"] = times["batched"]
    res["speedup_vs_plain"] = times["plain"] / times["batched"]
    res["mcell_updates_per_s_batched"] = cells / (times["batched"] * 1e-3) / 1e6
    return res


def run_adjoint(dev, n: int = 1024, nsteps: int = 200, every: int = 20):
    """The adjoint workload: 2D Euler 1024^2, smooth wave plus 8 seeded Fourier modes, J = 1/2 sum
    rho(T)^2 dx dy after 200 SSP-RK3 steps, gradient through the checkpointed rollout (checkpoints
    every 20 steps) and through the rollout that keeps every step's stage inputs.  Reports the cost
    of one adjoint step relative to one forward step.  n and nsteps only shrink it for a profiler
    capture."""
    import torch

    import workloads as W
    from paper_2411_11229_gb300 import Solver
    from paper_2411_11229_gb300.adjoint import Rollout

    S0n, dx, dy = W.euler2d_adjoint_init(n, seed=4000)
    s = Solver(2, "euler", n, n, dx=dx, dy=dy, device=dev)
    s.set_state(S0n)
    s.set_time(0.0, 0.0)
    rec = torch.empty(7, dtype=torch.float64, device=dev)
    s.step(0.0, 3)
    s.record(rec)
    s.sync()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    e0, e1 = ev(), ev()
    e0.record(s.stream)
    s.step(0.0, 10)
    e1.record(s.stream)
    torch.cuda.synchronize()
    fwd = e0.elapsed_time(e1) / 10
    Sn = s.state.clone()
    S1, S2 = torch.empty_like(Sn), torch.empty_like(Sn)
    lam = torch.randn_like(Sn)
    dt, al = float(rec[0].item()), rec[1:].contiguous()
    s.step_replay_stages(dt, al, S1, S2)
    lam = s.adjoint_step_stages(Sn, S1, S2, dt, al, lam)
    lam = s.adjoint_step(Sn, dt, al, lam)
    torch.cuda.synchronize()
    res = {"workload": f"2D Euler {n}^2 periodic, smooth wave + 8 seeded modes, J = 1/2 sum rho^2 dx dy",
           "ms_forward_step": fwd}
    for name, fn in (("from_stages", lambda l: s.adjoint_step_stages(Sn, S1, S2, dt, al, l)),
                     ("self_contained", lambda l: s.adjoint_step(Sn, dt, al, l))):
        e0.record(s.stream)
        for _ in range(5):
            lam = fn(lam)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        res[f"ms_adjoint_step_{name}"] = ms
        res[f"cost_ratio_{name}"] = ms / fwd
    S0 = torch.as_tensor(S0n, device=dev).requires_grad_(True)
    (0.5 * (S0.detach()[0, 0] ** 2).sum()).item()  # first use of these torch kernels loads them
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ST = Rollout.apply(S0, s, nsteps, every)
    J = 0.5 * (ST[0, 0] ** 2).sum() * dx * dy
    J.item()
    t1 = time.perf_counter()
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    res.update({"rollout_steps": nsteps, "checkpoint_every": every, "rollout_forward_s": t1 - t0,
                "rollout_backward_s": t2 - t1, "backward_over_forward": (t2 - t1) / (t1 - t0), "J": J.item(),
                "convention": "fixed recorded dt and per-stage alpha"})
    g_ckpt = S0.grad.detach().clone()
    del ST, J
    # the same rollout keeping every step's input and stage inputs (three states per step) instead of
    # checkpoints: no replay in the backward pass; run once first so that the timed run reuses the
    # allocator's block for the kept states
    kept = {}
    for rep in range(2):
        S0.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ST = Rollout.apply(S0, s, nsteps, every, True)
        J = 0.5 * (ST[0, 0] ** 2).sum() * dx * dy
        J.item()
        t1 = time.perf_counter()
        J.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        kept = {"forward_s": t1 - t0, "backward_s": t2 - t1, "backward_over_forward": (t2 - t1) / (t1 - t0),
                "kept_bytes": nsteps * 3 * s.state.numel() * 8,
                "gradient_equals_checkpointed": bool(torch.equal(S0.grad, g_ckpt))}
        del ST, J
    res["rollout_kept_stages"] = kept
    return res


def run_variants(dev, n: int, plain_ms: float, steps: int = 5):
    """The same workload with the per-cell characteristic decomposition (R2, one interpolation per
    cell and direction) and with the other two variants on the extended kernels (v^+/- with the
    nonlinear weights, Eq. Cd-2 D-terms): ms per step against the scheme of the paper."""
    import torch

    import workloads as W
    from paper_2411_11229_gb300 import Solver
    from paper_2411_11229_gb300 import _capi as C

    S, dx, dy = W.euler2d_smooth(n)
    out = {"workload": f"2D Euler {n}x{n}, the benchmark's state", "plain_ms_per_step": plain_ms}
    for name, flags in (("r2", C.HWENO_FLAG_R2), ("vw_cd2", C.HWENO_FLAG_V_WEIGHTED | C.HWENO_FLAG_CD2)):
        s = Solver(2, "euler", n, n, dx=dx, dy=dy, device=dev, flags=flags)
        s.set_state(S)
        s.set_time(0.0, 0.0)
        s.step(0.0, 3)
        s.sync()
        s.set_profiling(True)
        s.kernel_times()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s.stream)
        s.step(0.0, steps)
        e1.record(s.stream)
        torch.cuda.synchronize()
        kt = s.kernel_times()
        s.set_profiling(False)
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "speedup_vs_plain": plain_ms / ms,
                     "mcell_updates_per_s": n * n / (ms * 1e-3) / 1e6,
                     "kernel_avg_ms": {k: v[0] / max(v[1], 1) for k, v in kt.items()}}
        del s
        torch.cuda.empty_cache()
    return out


# CPU seconds of the HWENO-I scheme for Example 4.11 to t = 1.95 printed in the paper (its CPU-time
# table; serial MATLAB on one Apple M1 core): context for the wall time of the same runs here.
RT_PAPER_SECONDS = {(60, 240): 229.58, (120, 480): 1843.07, (240, 960): 17574.21}


def run_rayleigh_taylor(dev, meshes=((60, 240), (120, 480), (240, 960)), t_end: float = 1.95):
    """Example 4.11 (Rayleigh-Taylor, gravity, reflective sides, fixed top and bottom, gamma 5/3)
    to t = 1.95 on the paper's three meshes, through hweno_run: host wall time of the whole run."""
    import torch

    import workloads as W
    from paper_2411_11229_gb300 import Solver

    res = {"workload": "Example 4.11, Rayleigh-Taylor to t = 1.95, CFL 0.6", "runs": []}
    for nx, ny in meshes:
        S, dx, dy, fixed = W.rayleigh_taylor(nx, ny)
        kw = dict(gamma=5.0 / 3.0, grav=1.0, sides=("reflective", "reflective", "fixed", "fixed"), fixed=fixed)
        s = Solver(2, "euler", nx, ny, dx=dx, dy=dy, device=dev, **kw)
        s.set_state(S)
        s.run(0.01)  # first use: loads the kernels
        s.set_state(S)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nsteps = s.run(t_end)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        rho = s.state[0, 0]
        res["runs"].append({"mesh": f"{nx}x{ny}", "steps": nsteps, "seconds": sec,
                            "mcell_updates_per_s": nx * ny * nsteps / sec / 1e6,
                            "rho_min": float(rho.min()), "rho_max": float(rho.max()),
                            "paper_hweno_i_seconds": RT_PAPER_SECONDS.get((nx, ny))})
        del s
    return res


def run_reference(args, ws, rank):
    """The oracle on all host cores, one SSP-RK3 step of the full benchmark grid (4096^2 smooth
    wave) per benchmark step."""
    if rank != 0:
        return 0
    import oracle as O
    import workloads as W

    n = args.n
    cores = O.set_threads(0)
    S, dx, dy = W.euler2d_smooth(n)
    cfg = O.make_cfg(2, O.EULER, n, n, dx=dx, dy=dy)
    dt = O.cfl_dt(cfg, S, 0.6)
    for _ in range(args.warmup):
        S = O.steps(cfg, S, dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S = O.steps(cfg, S, dt, 1)
    sec = time.perf_counter() - t0
    value = n * n * args.steps / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"2D Euler HWENO-I {n}x{n} periodic [0,2]^2, smooth wave (0.7, 0.3), "
                               "SSP-RK3 CFL 0.6", "n": n, "cells": n * n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one oracle SSP-RK3 step of the full {n}x{n} grid per benchmark step, "
                                   f"{cores} host threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle as O
    import workloads as W
    from paper_2411_11229_gb300 import Solver

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    probe = fp64_probe(dev)  # the ALU roofline's peak, measured on this GPU before the workload
    S, dx, dy = W.euler2d_smooth(n)
    cells = n * n
    solver = Solver(2, "euler", n, n, dx=dx, dy=dy, device=dev)
    solver.set_state(S)
    stream = solver.stream
    solver.set_time(0.0, 0.0)
    for _ in range(args.warmup):
        solver.step(0.0)
    solver.sync()

    def barrier():
        if ws > 1:
            dist.barrier()

    gpu_idx = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and vis.split(",")[local].strip().isdigit():
        gpu_idx = int(vis.split(",")[local])
    sampler = ClockSampler(gpu_idx)

    # device-resident timed region
    solver.set_profiling(True)
    solver.kernel_times()
    launches0 = solver.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0.record(stream)
    for _ in range(args.steps):
        solver.step(0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    ms = e0.elapsed_time(e1)
    launches = solver.launch_count() - launches0
    ktimes = solver.kernel_times()
    solver.set_profiling(False)
    ms_max = max_over_ranks(ms, ws, dev)
    value = job_throughput(ws, cells, args.steps, ms_max)

    # end to end through the C ABI with host buffers: upload, step, download every step.  Each step
    # takes its input from pinned host memory and returns its result there, so consecutive steps are
    # independent problems: one hweno_pipeline call takes them, on three device slots in turn, so that
    # the copies of two run on the copy engines while the third steps (with two, a slot's next upload
    # waits for its own download, which the other slot's step does not cover when the host link is
    # slow).  The serial form (upload, step, download on one handle and one stream) is reported
    # beside it.
    host_in = torch.from_numpy(np.ascontiguousarray(solver.state.cpu().numpy())).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    nbytes = host_in.numel() * 8
    ke2e = max(2, args.steps)
    solver.upload(host_in)
    solver.step(0.0)
    solver.download(host_out)
    solver.sync()
    barrier()
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(ke2e):
        solver.upload(host_in)
        solver.step(0.0)
        solver.download(host_out)
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_serial = max_over_ranks(f0.elapsed_time(f1), ws, dev)
    serial_value = job_throughput(ws, cells, ke2e, ms_serial)
    depth = E2E_DEPTH
    ins = [host_in] + [torch.empty_like(host_in).pin_memory() for _ in range(depth - 1)]
    for h in ins[1:]:
        h.copy_(host_in)
    outs = [host_out] + [torch.empty_like(host_in).pin_memory() for _ in range(depth - 1)]
    seq_in = [ins[k % depth] for k in range(ke2e)]
    seq_out = [outs[k % depth] for k in range(ke2e)]
    solver.pipeline(ins, outs, 1, depth)  # allocates the slots' device memory outside the timed region
    barrier()
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    w0 = time.perf_counter()
    solver.pipeline(seq_in, seq_out, 1, depth)
    wall_ms = (time.perf_counter() - w0) * 1e3
    p1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = max_over_ranks(p0.elapsed_time(p1), ws, dev)
    e2e_value = job_throughput(ws, cells, ke2e, ms_e2e)
    e2e_wall_value = job_throughput(ws, cells, ke2e, max_over_ranks(wall_ms, ws, dev))
    # one more end-to-end step outside the timed region, with an event between its phases: where
    # the end-to-end time goes (the copies run at the host link's rate, which varies between boxes)
    g = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    g[0].record(stream)
    solver.upload(host_in)
    g[1].record(stream)
    solver.step(0.0)
    g[2].record(stream)
    solver.download(host_out)
    g[3].record(stream)
    torch.cuda.synchronize()
    phases = {"upload_ms": g[0].elapsed_time(g[1]), "step_ms": g[1].elapsed_time(g[2]),
              "download_ms": g[2].elapsed_time(g[3])}
    phases["copy_gbs"] = 2 * nbytes / ((phases["upload_ms"] + phases["download_ms"]) * 1e-3) / 1e9
    phases["h2d_gbs"] = nbytes / (phases["upload_ms"] * 1e-3) / 1e9
    phases["d2h_gbs"] = nbytes / (phases["download_ms"] * 1e-3) / 1e9

    if rank != 0:
        return 0
    # roofline of the dominant kernel (face kernel: FP64 ALU bound)
    cfg = O.make_cfg(2, O.EULER, n, n, dx=dx, dy=dy)
    counts = O.count_flops(cfg)
    faces = 2 * (n + 1) * n
    face_ms, face_n = ktimes["face"]
    face_avg_ms = face_ms / max(face_n, 1)
    flops_face_launch = counts["face"] * faces
    achieved = flops_face_launch / (face_avg_ms * 1e-3)
    total_ms = sum(v[0] for v in ktimes.values())
    traffic = None if FACE_TRAFFIC_BYTES_PER_FACE is None else FACE_TRAFFIC_BYTES_PER_FACE * faces
    peaks = _measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", HBM_PEAK_GBS_FALLBACK)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"2D Euler HWENO-I {n}x{n} periodic [0,2]^2, smooth wave (0.7, 0.3), "
                               "SSP-RK3 CFL 0.6, dt on device", "n": n, "cells": cells,
                   "parallelism": f"replicas x{ws}", "l2": "inputs larger than L2 (state 1.6 GB + workspace)"},
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "steps": ke2e,
                "path": f"one hweno_pipeline call: upload, one SSP-RK3 step and download per problem, pinned "
                        f"host buffers, {depth} device slots on their own streams in turn, so the copies of the "
                        "others overlap each slot's step (CUDA events on the handle's stream around the call)",
                "wall_value": e2e_wall_value,
                "serial": {"value": serial_value,
                           "path": "hweno_upload + hweno_step + hweno_download per step on one handle and one "
                                   "stream"},
                "phases_one_step": phases},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": probe["flops"] / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / probe["flops"], "traffic": traffic,
                     "kernel": "k_face<2,EULER>", "flops_per_face": counts["face"],
                     "faces_per_launch": faces, "avg_launch_ms": face_avg_ms,
                     "frac_note": "the scheme's operations per face as the oracle writes them (+, -, *, /, sqrt "
                                  "with nontrivial operands, counted on the oracle's own code) per second, over "
                                  "the FP64 peak measured on this GPU",
                     "peak_note": "measured on this GPU before the workload: register-operand DFMA issue rate "
                                  "(hweno_selftest_fp64_peak) x 2 flops",
                     "peak_derived": FP64_PEAK_FLOPS_DERIVED / 1e12,
                     "peak_derived_note": "152 SMs x 2070 MHz x 2 DFMA/clk x 2 flops",
                     "frac_of_derived": achieved / FP64_PEAK_FLOPS_DERIVED,
                     "fp64_pipe_active_ncu": None if traffic is None else FACE_FP64_PIPE_ACTIVE,
                     "fp64_instructions_per_face_ncu": None if traffic is None else FACE_FP64_INSTR_PER_FACE,
                     "frac_executed": None if traffic is None else
                     FACE_FP64_INSTR_PER_FACE * faces / (face_avg_ms * 1e-3) / probe["dfma_per_s"],
                     "frac_executed_note": "FP64 instructions the kernel executes per face (ncu) x faces per second, "
                                           "over the probe's DFMA issue rate",
                     "hbm_peak_gbs": hbm_peak},
        "hbm": {"bytes_per_cell_step_algorithmic": STEP_BYTES_PER_CELL,
                "achieved_gbs": value * 1e6 * STEP_BYTES_PER_CELL / 1e9,
                "frac": value * 1e6 * STEP_BYTES_PER_CELL / 1e9 / hbm_peak,
                "face_kernel_dram_gbs": None if traffic is None else traffic / (face_avg_ms * 1e-3) / 1e9,
                "face_kernel_frac": None if traffic is None else traffic / (face_avg_ms * 1e-3) / 1e9 / hbm_peak,
                "peak_gbs": hbm_peak, "peak_note": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback",
                "note": "the step is bound by the FP64 pipe; HBM is reported beside it"},
        "fp64_probe": probe,
        "kernel_share": {k: v[0] / total_ms for k, v in ktimes.items()} if total_ms > 0 else None,
        "kernel_avg_ms": {k: v[0] / max(v[1], 1) for k, v in ktimes.items()},
        "flops_per_cell_step": counts["per_cell_step"],
    }
    if ws == 1 and not args.no_variants:
        torch.cuda.empty_cache()
        line["variants"] = run_variants(dev, n, ms_max / args.steps)
    if ws == 1 and args.rt:
        line["rayleigh_taylor"] = run_rayleigh_taylor(dev)
    if ws == 1 and not args.no_batched:
        del solver
        torch.cuda.empty_cache()
        line["batched"] = run_batched(dev)
        torch.cuda.empty_cache()
        line["batched"]["lines_1d_only"] = run_batched(dev, only_1d=True)
    if ws == 1 and not args.no_adjoint:
        torch.cuda.empty_cache()
        line["adjoint"] = run_adjoint(dev, args.adjoint_n, args.adjoint_steps, min(20, args.adjoint_steps))
    if ws == 1 and args.parity_steps > 0:
        torch.cuda.empty_cache()
        line["parity"] = run_parity(dev, n, args.parity_steps, args.parity_envelope)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n=n)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--rt", action="store_true", help="also run Example 4.11 (Rayleigh-Taylor) on its three meshes")
    ap.add_argument("--no-rt", action="store_true", help=argparse.SUPPRESS)  # the default; kept for old commands
    ap.add_argument("--parity-steps", type=int, default=0,
                    help="also compare this many GPU steps of the workload with the oracle (all host cores)")
    ap.add_argument("--parity-envelope", action="store_true",
                    help="with --parity-steps: also the oracle's own drift from a one-ulp perturbed input")
    ap.add_argument("--adjoint-n", type=int, default=1024)
    ap.add_argument("--adjoint-steps", type=int, default=200)
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        return run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
