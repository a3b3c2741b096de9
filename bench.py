#!/usr/bin/env python
"""Benchmark of the STORM control step on B300.

Workload: the paper-scale control step -- 7-DOF seeded modified-DH chain, 500
particles x horizon 30, 6-knot cubic B-spline noise, 3 MPPI iterations with
mean + diagonal covariance update and shift, every cost term including 49 link
spheres against 20 boxes + 10 spheres.  Synthetic, seeded inputs (no dataset).

One JSON line on rank 0:
  value  rollout-steps/s (N * H * K per control step / device time per step),
         inputs resident in HBM, each step timed with CUDA events on the
         controller's stream, L2 flushed (256 MB write) before every step;
         the inputs are the closed-loop sequence of the e2e run (the step's
         work grows as the arm's links come close to each other)
  e2e    the same metric through the host API storm_step in a closed loop
         (pinned H2D of state + goal, D2H of the command, host wall clock):
         the arm driving to five goals on an ideal double-integrator plant
  latency_ms  p50 / p99 of the device-timed step
  latency_rest_ms  the same with the arm at rest at its start configuration
  roofline    the rollout kernel (ALU bound) against the FP32 FMA peak
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample

--impl reference times the FP64 oracle (the reference arm of this project) on
the same workload, each step a bounded particle sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2104_13542_b300 import workloads as W  # noqa: E402

METRIC = "MPC step latency p50/p99 (ms) and rollout-steps/s, 500x30 7-DOF, vs oracle"
LOOP_WARMUP, LOOP_STEPS = 50, 1000  # the closed loop every run records (five goals)
UNIT = "rollout-steps/s"
SM_COUNT = 148
FP32_LANES_PER_SM = 128


def algorithmic_flops_per_item(p: W.Params, robot: W.Robot, world: W.World) -> float:
    """FP32 flops of one (particle, step) item of the rollout kernel, counted
    from the method (FMA = 2 flops), not from the instruction stream.

    FK 48/joint, sphere centres 18/sphere, Jacobian 12/joint, manipulability
    by Gram-Schmidt 28 k + 22 per row k, pose + rotation + stop + joint +
    smoothness 100, world collision 14 per sphere-box and 8 per
    sphere-sphere check, self collision 8 per pair, plus the per-particle
    noise smoothing (2 S d H / H) and integration (4 d).
    """
    d, M, P = robot.dof, robot.spheres.shape[0], robot.pairs.shape[0]
    B, O = world.boxes.shape[0], world.spheres.shape[0]
    S = p.n_knots if p.n_knots > 0 else 1
    manip = sum(28 * k + 22 for k in range(6)) if p.w_manip else 0
    return (48 * d + 18 * M + 12 * d + manip + 100 + M * (14 * B + 8 * O) + 8 * P +
            2 * S * d + 4 * d)


def adjoint_flops_per_item(p: W.Params, robot: W.Robot, world: W.World) -> float:
    """FP32 flops of one (particle, step) item of the adjoint kernel, counted from
    the method: the forward pass it recomputes (algorithmic_flops_per_item), then
    the reverse pass -- twice the forward work of FK, the Jacobian,
    manipulability and the non-collision costs (reverse mode of each), the
    collision gradient at the minimising pair or sphere-obstacle (centres and
    distance, 2 x 30), and the integration adjoint (4 d)."""
    d = robot.dof
    manip = sum(28 * k + 22 for k in range(6)) if p.w_manip else 0
    return algorithmic_flops_per_item(p, robot, world) + 2 * (48 * d + 12 * d + manip + 100) + 2 * 60 + 4 * d


def fp32_peak_tflops(sm_mhz: float) -> float:
    return SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def kernel_source_hash() -> str:
    """Hash of what the warp rollout kernels are compiled from: the two headers
    that define them (and everything they call) and the compiler flags."""
    import hashlib
    from paper_2104_13542_b300.binding import NVCC_FLAGS
    h = hashlib.sha256()
    for f in ("storm_device.cuh", "storm_rollout_warp.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2104_13542_b300", "csrc", f), "rb").read())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


# the instantiations the paper-scale workload runs (the lean ones), as ncu names them
ROLLOUT_KERNELS = {"cta": "k_rollout", "warp": "k_rollout_warp<1, 0>", "pair": "k_rollout_warp<2, 0>",
                   "quad": "k_rollout_warp<4, 0>"}


def rollout_traffic(kernel: str):
    """DRAM bytes per launch of this rollout kernel from the committed ncu summary,
    or None when there is none for it or the kernels changed since the capture."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
    except Exception:
        return None
    return rec["dram_bytes_per_launch"] if rec.get("src_sha256_16") == kernel_source_hash() else None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks + throttle reasons, sampled every 100 ms from before the
    measured part until after it.  mark() records the edges of a window (the
    device-timed steps); summary() reports the samples inside it, or, when the
    window is shorter than the sampling period, those of the whole measured
    part (saying so).  The GPU is named by its UUID, so the sample is this
    process's GPU whatever CUDA_VISIBLE_DEVICES maps."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        import tempfile
        self.dev = device_index
        self.proc = None
        self.error = None
        self.marks = {}
        self.path = os.path.join(tempfile.gettempdir(), f"storm_bench_clocks_{os.getpid()}.csv")

    def _gpu_id(self):
        try:
            import torch
            u = getattr(torch.cuda.get_device_properties(self.dev), "uuid", None)
            if u:
                u = str(u)
                return u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [x.strip() for x in cvd.split(",") if x.strip()]
        return ids[self.dev] if self.dev < len(ids) else str(self.dev)

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self._gpu_id()}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.PIPE)
            t0 = time.time()
            while time.time() - t0 < 5.0:  # until the first sample is in
                if self.proc.poll() is not None:
                    self.error = "nvidia-smi exited: " + self.proc.stderr.read().decode(errors="replace")[:200]
                    self.proc = None
                    break
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.05)
        except Exception as e:  # no nvidia-smi: the record says why
            self.error = f"{type(e).__name__}: {e}"
            self.proc = None
        return self

    def mark(self, name):
        import datetime
        self.marks[name] = datetime.datetime.now()

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)  # one more sample after the last timed step
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if getattr(self, "fh", None):
            self.fh.close()

    def summary(self, window=("start", "end")):
        import datetime
        if not os.path.exists(self.path) or os.path.getsize(self.path) == 0:
            return {"unavailable": self.error or "no nvidia-smi samples"}
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            r = [x.strip() for x in line.strip().split(",")]
            try:
                ts = datetime.datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f")
                rows.append((ts, float(r[1]), float(r[2]),
                             {nm for k, nm in enumerate(names) if r[5 + k].lower() == "active"}))
            except (ValueError, IndexError):
                continue
        if not rows:
            return {"unavailable": "unparsable nvidia-smi samples"}
        a, b = self.marks.get(window[0]), self.marks.get(window[1])
        inside = [x for x in rows if a and b and a <= x[0] <= b]
        use, scope = (inside, "device-timed steps") if inside else (rows, "whole measured part")
        return {"sm_mhz": float(np.median([x[1] for x in use])), "sm_max_mhz": float(max(x[2] for x in use)),
                "reasons": sorted(set().union(*[x[3] for x in use])), "samples": len(use),
                "samples_total": len(rows), "scope": scope}


def goals_for(ctl, robot, seed: int, count: int, with_theta: bool = False):
    """Reachable goal poses X_g = FK(theta_g), theta_g ~ U[-2.24, 2.24] drawn until the
    configuration is at least 3 cm clear of self-collision (exact check of the library)."""
    import torch
    rng = np.random.default_rng([seed, 99])
    cand = rng.uniform(-2.24, 2.24, (64 * count, robot.dof)).astype(np.float32)
    sd = ctl.self_distance(torch.as_tensor(cand, device="cuda")).cpu().numpy()
    th = cand[sd > 0.03][:count]
    ee = ctl.forward_kinematics(torch.as_tensor(th, device="cuda")).cpu().numpy()
    goals = []
    for T in ee:
        Rm, p = T[:, :3].astype(np.float64), T[:, 3]
        # rotation -> quaternion (w, x, y, z) for the goal input format
        w = math.sqrt(max(0.0, 1 + Rm[0, 0] + Rm[1, 1] + Rm[2, 2])) / 2
        x = math.copysign(math.sqrt(max(0.0, 1 + Rm[0, 0] - Rm[1, 1] - Rm[2, 2])) / 2, Rm[2, 1] - Rm[1, 2])
        y = math.copysign(math.sqrt(max(0.0, 1 - Rm[0, 0] + Rm[1, 1] - Rm[2, 2])) / 2, Rm[0, 2] - Rm[2, 0])
        z = math.copysign(math.sqrt(max(0.0, 1 - Rm[0, 0] - Rm[1, 1] + Rm[2, 2])) / 2, Rm[1, 0] - Rm[0, 1])
        goals.append(np.array([p[0], p[1], p[2], w, x, y, z], dtype=np.float32))
    return (goals, th) if with_theta else goals


def max_over_ranks(value: float, world_size: int, device: str = "cuda") -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    if world_size <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step: int, steps: int, world_size: int, max_time_s: float) -> float:
    """Whole-job rollout-steps/s: every rank runs its own replica (weak scaling)."""
    return units_per_step * steps * world_size / max_time_s


def run_gpu(args, rank, world_size):
    import torch
    from paper_2104_13542_b300 import Controller

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    wl = W.config_paper(seed=args.seed + rank)
    p = wl.params
    units_per_step = p.N * p.H * p.K
    ctl = Controller(wl.robot, wl.world, p)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    state0 = wl.state.copy()
    state0[1:] = 0.0
    goals = goals_for(ctl, wl.robot, args.seed + rank, 5)
    # the library's autotuner picks the rollout launch shape for this workload
    ctl.step(state0.astype(np.float32), goals[0])
    if args.launch == "auto":
        tuned_us = ctl.autotune()
    else:  # a fixed rollout shape (profiling runs: the tuner's timings are not meaningful under a profiler)
        kind, _, shape = args.launch.partition(":")
        if kind == "warp":
            ctl.set_launch_warp(int(shape))
        elif kind == "pair":
            ctl.set_launch_warp_pair(int(shape))
        elif kind == "quad":
            ctl.set_launch_warp_quad(int(shape))
        else:
            ppc, threads = (int(x) for x in shape.split(","))
            ctl.set_launch(ppc, threads)
        tuned_us = None
    if args.dep_launch:
        ctl.set_dependent_launch(True)
    ctl.reset()

    clk = ClockSampler(torch.cuda.current_device())
    clk.__enter__()
    # ---------------- the closed loop through the host API (e2e): a fixed
    # LOOP_WARMUP + LOOP_STEPS steps whatever --steps is, the arm driving to five
    # goals in turn (LOOP_STEPS / 5 steps each) on an ideal double-integrator
    # plant stepped outside the timed call.  Every step's state and goal and the
    # controller's state before it (storm_get_state: mu, sigma, step counter) are
    # recorded, so the device-timed steps below replay exact steps of this loop.
    import ctypes
    dof = wl.robot.dof
    state = state0.astype(np.float32).copy()
    dt = float(p.dt[0])
    n_all = LOOP_WARMUP + LOOP_STEPS
    seg = LOOP_STEPS // len(goals)
    picks = np.linspace(LOOP_WARMUP, n_all - 1, args.steps).round().astype(int)
    want_blob = set(picks.tolist())
    e2e_ms, seq_state, seq_goal, blobs, final_err = [], [], [], {}, []
    for i in range(n_all):
        goal = goals[0] if i < LOOP_WARMUP else goals[min((i - LOOP_WARMUP) // seg, len(goals) - 1)]
        seq_state.append(state.reshape(-1).copy())
        seq_goal.append(np.asarray(goal, dtype=np.float32))
        if i in want_blob:
            blobs[i] = ctl.get_state()
        with torch.cuda.stream(ctl.stream):
            flush.fill_(float(i))
        ctl.stream.synchronize()
        t0 = time.perf_counter()
        cmd, info, rc = ctl.step(state, goal)
        t1 = time.perf_counter()
        if i >= LOOP_WARMUP:
            e2e_ms.append((t1 - t0) * 1e3)
        # ideal double-integrator plant
        state[2] = cmd
        state[1] = state[1] + dt * cmd
        state[0] = state[0] + dt * state[1]
        if i >= LOOP_WARMUP and (i - LOOP_WARMUP + 1) % seg == 0:
            T = ctl.forward_kinematics(torch.as_tensor(state[0:1], device="cuda")).cpu().numpy()[0]
            q = _quat_from_rot(T[:, :3].astype(np.float64))
            final_err.append({"pos_m": float(np.linalg.norm(T[:, 3] - goal[:3])),
                              "quat": float(1.0 - abs(np.dot(q, np.asarray(goal[3:], np.float64))))})
    e2e_ms = np.array(e2e_ms)
    e2e_time_s = max_over_ranks(float(e2e_ms.sum() / 1e3), world_size)

    # ---------------- device-resident timing (value): --steps steps of the loop,
    # evenly spaced over its LOOP_STEPS (after its warm-up), each replayed
    # exactly: before its events the controller's recorded state is restored
    # and the step's state and goal are copied into the handle's input buffers
    # (from HBM), and L2 is flushed
    s_ptr, g_ptr, _ = ctl.device_io_ptrs()
    io_state = torch.as_tensor(_DeviceFloats(s_ptr, 3 * dof), device="cuda")
    io_goal = torch.as_tensor(_DeviceFloats(g_ptr, 7), device="cuda")
    seq_state_d = torch.as_tensor(np.stack(seq_state), device="cuda")
    seq_goal_d = torch.as_tensor(np.stack(seq_goal), device="cuda")

    def place(i):
        ctl.set_state(blobs[i])
        with torch.cuda.stream(ctl.stream):
            io_state.copy_(seq_state_d[i], non_blocking=True)
            io_goal.copy_(seq_goal_d[i], non_blocking=True)

    for w in range(args.warmup):
        place(int(picks[w % len(picks)]))
        ctl.step_resident()
    ctl.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clk.mark("start")
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_steps")  # (profilers select the timed launches by this range)
    for k, i in enumerate(picks):
        with torch.cuda.stream(ctl.stream):
            flush.fill_(float(k))
        place(int(i))
        ev[k][0].record(ctl.stream)
        ctl.step_resident()
        ev[k][1].record(ctl.stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk.mark("end")
    ms = np.array([a.elapsed_time(b) for a, b in ev])
    dev_time_s = max_over_ranks(float(ms.sum() / 1e3), world_size)

    # the arm at rest at its start configuration, the first goal, every step
    # (the lightest collision load: for reference next to the trajectory)
    st_dev = torch.as_tensor(np.ascontiguousarray(state0, dtype=np.float32), device="cuda").reshape(-1)
    gl_dev = torch.as_tensor(goals[0], device="cuda")
    ctl.reset()
    with torch.cuda.stream(ctl.stream):
        io_state.copy_(st_dev)
        io_goal.copy_(gl_dev)
    for _ in range(args.warmup):
        ctl.step_resident()
    ms_rest = _time_steps(ctl.step_resident, ctl.stream, flush, min(max(args.steps, 20), 200))

    # ---------------- rollout-kernel roofline: the rollout kernel alone, timed
    # with events on the controller's stream, at states of the loop
    from paper_2104_13542_b300.binding import fp32_peak, lib
    n_rk = max(20, min(args.steps, 200))
    rk_picks = np.linspace(LOOP_WARMUP, n_all - 1, n_rk).round().astype(int)

    def rollout_ms():
        rk = []
        for j, i in enumerate(rk_picks):
            with torch.cuda.stream(ctl.stream):
                flush.fill_(float(j))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(ctl.stream)
            lib().storm_generate_rollouts(ctl.h, ctypes.c_void_p(seq_state_d[i].data_ptr()),
                                          ctypes.c_void_p(seq_goal_d[i].data_ptr()), 0, 0, None, None, None,
                                          None, None, None, None)
            b.record(ctl.stream)
            rk.append((a, b))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in rk]))

    rk_ms = rollout_ms()
    ctl.set_broadphase(False)  # the same kernel doing every exact collision test
    rk_bf_ms = rollout_ms()
    ctl.set_broadphase(True)
    clk.mark("fma_start")
    fma = fp32_peak(8192)  # this GPU's FP32 FMA rate, measured now
    clk.mark("fma_end")
    clk.__exit__(None, None, None)
    clocks = clk.summary(("start", "end"))
    fma_clocks = clk.summary(("fma_start", "fma_end"))
    flops_launch = algorithmic_flops_per_item(p, wl.robot, wl.world) * p.N * p.H
    peak = max(fma["scalar_tflops"], fma["paired_tflops"])
    achieved = flops_launch / (rk_ms * 1e-3) / 1e12
    achieved_bf = flops_launch / (rk_bf_ms * 1e-3) / 1e12

    res = dict(
        value=job_throughput(units_per_step, args.steps, world_size, dev_time_s),
        ms_per_step=float(ms.mean()),
        latency_ms={"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99)),
                    "max": float(ms.max())},
        latency_rest_ms={"p50": float(np.percentile(ms_rest, 50)), "p99": float(np.percentile(ms_rest, 99))},
        e2e={"value": job_throughput(units_per_step, len(e2e_ms), world_size, e2e_time_s), "unit": UNIT,
             "h2d_bytes_per_step": 4 * (3 * wl.robot.dof + 7),
             "d2h_bytes_per_step": 4 * wl.robot.dof + 16,
             "latency_ms": {"p50": float(np.percentile(e2e_ms, 50)),
                            "p99": float(np.percentile(e2e_ms, 99))},
             "closed_loop": {"warmup_steps": LOOP_WARMUP, "steps": LOOP_STEPS, "goals": len(goals),
                             "steps_per_goal": seg,
                             "final_error_per_goal": final_err}},
        roofline={"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                  "frac": achieved / peak, "traffic": rollout_traffic(ROLLOUT_KERNELS[ctl.launch_mapping()]),
                  "kernel": ROLLOUT_KERNELS[ctl.launch_mapping()], "kernel_ms": rk_ms,
                  "flops_per_launch": flops_launch,
                  "flops_basis": "brute-force count of the method's work per (particle, step); "
                                 "with the collision broad phase the kernel executes fewer",
                  "brute_force_kernel_ms": rk_bf_ms, "brute_force_frac": achieved_bf / peak,
                  "launch_shape": list(ctl.get_launch()), "autotune_us": tuned_us,
                  "dependent_launch": ctl.dependent_launch(),
                  "peak_basis": "measured: storm_fp32_peak (independent FMA chains on every SM), "
                                "the better of one and two FMAs per instruction, this run",
                  "fp32_peak_measured": fma, "fp32_peak_clocks": fma_clocks,
                  "fp32_peak_unit_count_tflops": fp32_peak_tflops(
                      (fma_clocks or {}).get("sm_mhz") or measured_peaks().get("sm_max_mhz", 2032.0))},
        clocks=clocks,
        gpu_launches=2 * p.K * args.steps,
        wall_s=wall,
    )
    ctl.close()
    return res, wl


class _DeviceFloats:
    """A float32 device buffer of the library (raw pointer), seen by torch
    without a copy."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4", "data": (ptr, False),
                                         "version": 3, "strides": None}


def _time_steps(step_fn, stream, flush, n):
    import torch
    ev = []
    for i in range(n):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step_fn()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in ev])


def run_variants(args, seed: int, fp32_peak: float | None = None):
    """The gradient-refined, batched and surrogate forms next to the plain step,
    same GPU, same timing rules (device time per step, L2 flushed before each)."""
    import torch
    from paper_2104_13542_b300 import BatchController, Controller, SurrogateMLP
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    n = max(20, min(args.steps, 200))
    out = {}
    # plain and gradient-refined paper-scale steps
    for name, wl in (("plain", W.config_paper(seed)), ("refined_grad5", W.config_differentiable(seed))):
        p = wl.params
        with Controller(wl.robot, wl.world, p) as c:
            st, gl = wl.state.astype(np.float32), wl.goal.astype(np.float32)
            c.step(st, gl)
            for _ in range(3):
                c.step_resident()
            ms = _time_steps(c.step_resident, c.stream, flush, n)
            entry = {"ms_p50": float(np.percentile(ms, 50)), "ms_p99": float(np.percentile(ms, 99)),
                     "rollout_steps_per_s": p.N * p.H * p.K * len(ms) / float(ms.sum() / 1e3)}
            if p.grad_steps:
                mu, _ = c.get_distribution()
                m = torch.as_tensor(mu, device="cuda")
                s_d, g_d = torch.as_tensor(st.reshape(-1), device="cuda"), torch.as_tensor(gl, device="cuda")
                # the adjoint alone (one k_adjoint launch: the sums are folded into it),
                # against the FP32 peak; called through the C ABI on preallocated outputs,
                # so that no host-side allocation or stream join sits between the events
                import ctypes
                from paper_2104_13542_b300.binding import lib
                g_out = torch.empty((p.H, wl.robot.dof), dtype=torch.float32, device="cuda")
                j_out = torch.empty(1, dtype=torch.float32, device="cuda")
                adj_args = (c.h, ctypes.c_void_p(s_d.data_ptr()), ctypes.c_void_p(g_d.data_ptr()),
                            ctypes.c_void_p(m.data_ptr()), 7, 0, ctypes.c_void_p(g_out.data_ptr()),
                            ctypes.c_void_p(j_out.data_ptr()), None)
                torch.cuda.synchronize()

                def adjoint_call():
                    if lib().storm_cost_grad(*adj_args) != 0:
                        raise RuntimeError("storm_cost_grad failed")

                adj_ms = _time_steps(adjoint_call, c.stream, flush, n)
                fl = adjoint_flops_per_item(p, wl.robot, wl.world) * p.N * p.H
                entry["adjoint"] = {"ms_p50": float(np.percentile(adj_ms, 50)),
                                    "flops_per_launch": fl,
                                    "tflops": fl / (float(np.percentile(adj_ms, 50)) * 1e-3) / 1e12}
                if fp32_peak:
                    entry["adjoint"]["frac_fp32_peak"] = entry["adjoint"]["tflops"] / fp32_peak
                J0, g = c.cost_grad(m, s_d, g_d, 7, 0)
                Js = [float(J0[0])]
                for _ in range(p.grad_steps):
                    m = m - p.grad_eta * g
                    J, g = c.cost_grad(m, s_d, g_d, 7, 0)
                    Js.append(float(J[0]))
                entry["grad_steps"] = p.grad_steps
                entry["J_along_refinement"] = Js
            out[name] = entry
    # the widened rows: variable-dt schedule with end-effector limits, mixed sampler, ball on a tray
    for name, wl in (("vardt_ee_limits", W.config_variable_dt(seed)), ("mixed_sampler", W.config_mixed(seed)),
                     ("ball_on_tray", W.config_ball(seed))):
        p = wl.params
        with Controller(wl.robot, wl.world, p) as c:
            if wl.ball is not None:
                c.set_ball(wl.ball[:3], wl.ball[3:])
            c.step(wl.state.astype(np.float32), wl.goal.astype(np.float32))
            for _ in range(3):
                c.step_resident()
            ms = _time_steps(c.step_resident, c.stream, flush, n)
            out[name] = {"ms_p50": float(np.percentile(ms, 50)), "ms_p99": float(np.percentile(ms, 99)),
                         "rollout_steps_per_s": p.N * p.H * p.K * len(ms) / float(ms.sum() / 1e3)}
    # batched uneven instances
    wls = W.config_batch(seed, 256)
    with BatchController([w.robot for w in wls], [w.world for w in wls], [w.params for w in wls]) as b:
        b.step([w.state.astype(np.float32) for w in wls], np.stack([w.goal for w in wls]).astype(np.float32))
        t_tune = b.autotune()
        for _ in range(3):
            b.step_resident()
        ms = _time_steps(b.step_resident, b.stream, flush, n)
        units = sum(w.params.N * w.params.H * w.params.K for w in wls)
        out["batched_256"] = {"ms_p50": float(np.percentile(ms, 50)), "ms_p99": float(np.percentile(ms, 99)),
                              "rollout_steps_per_s": units * len(ms) / float(ms.sum() / 1e3),
                              "instances": len(wls), "rollout_steps_per_step": units,
                              "mapping": b.launch_mapping(), "tile": b.get_launch(),
                              "autotune_rollout_us": t_tune}
    # learned self-collision surrogate at 1000 x 30, inside the rollout kernel,
    # next to the exact check; then the crossover: denser link spheres (more
    # self pairs) and the exact check without its broad phase
    wl = W.config_paper(seed, N=1000, H=30)
    margin = 0.05
    cross = {}
    for spl in (7, 9):
        robot = wl.robot if spl == 7 else W.make_robot(seed, 7, spheres_per_link=spl)
        with Controller(robot, wl.world, wl.params.replace(N=8)) as lab:
            rng = np.random.default_rng([seed, 77])
            th = torch.as_tensor(rng.uniform(-2.8, 2.8, (1 << 20, 7)).astype(np.float32), device="cuda")
            th_te = torch.as_tensor(rng.uniform(-2.8, 2.8, (65_536, 7)).astype(np.float32), device="cuda")
            sd, sd_te = lab.self_distance(th), lab.self_distance(th_te)
        if spl == 7:  # the first training call of the process also loads its kernels: untimed
            warm = SurrogateMLP(seed=seed + 1)
            warm.train(th[:8192], torch.clamp(sd[:8192], max=0.5), batch=4096, epochs=1, lr=2e-3, seed=seed)
            warm.close()
        net = SurrogateMLP(seed=seed)
        t0 = time.perf_counter()
        losses = net.train(th, torch.clamp(sd, max=0.5), batch=4096, epochs=8, lr=2e-3, seed=seed)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        y, ref = net.predict(th_te).cpu().numpy(), sd_te.cpu().numpy()
        near, coll = ref < 0.5, ref < 0.0
        acc = {"mae_m": float(np.abs(y[near] - ref[near]).mean()),
               "false_negative_rate": float(np.mean(y[coll] >= margin)) if coll.any() else 0.0,
               "skip_fraction": float(np.mean(y >= margin)), "margin_m": margin,
               "train_s": train_s, "train_samples": int(th.shape[0]), "epochs": len(losses),
               "final_loss": float(losses[-1])}
        row = {"spheres": int(robot.spheres.shape[0]), "self_pairs": int(robot.pairs.shape[0])}
        for mode in ("exact", "surrogate"):
            for bp in (True, False):
                with Controller(robot, wl.world, wl.params) as c:
                    if mode == "surrogate":
                        c.set_surrogate(net, margin)
                    c.set_broadphase(bp)
                    c.step(wl.state.astype(np.float32), wl.goal.astype(np.float32))
                    ms = _time_steps(c.step_resident, c.stream, flush, n)
                key = f"{mode}_{'broadphase' if bp else 'bruteforce'}_ms_p50"
                row[key] = float(np.percentile(ms, 50))
                if spl == 7 and bp:
                    out[f"{mode}_1000x30"] = {"ms_p50": float(np.percentile(ms, 50)),
                                              "ms_p99": float(np.percentile(ms, 99))}
        if spl == 7:
            out["surrogate_1000x30"].update(acc)
        else:
            row.update(acc)
        net.close()
        # the paper's own use (Eq. 13): jointNERF's depth as the self-collision
        # cost, no exact check at all
        nerf = SurrogateMLP(seed=seed, arch="jointnerf")
        nerf.train(th, torch.clamp(-sd, min=-0.5), batch=4096, epochs=8, lr=2e-3, seed=seed)
        d_te = -nerf.predict(th_te).cpu().numpy()
        row["learned_cost_jointnerf_mae_m"] = float(np.abs(d_te[near] - ref[near]).mean())
        for bp in (True, False):
            with Controller(robot, wl.world, wl.params) as c:
                c.set_surrogate_cost(nerf)
                c.set_broadphase(bp)
                c.step(wl.state.astype(np.float32), wl.goal.astype(np.float32))
                ms = _time_steps(c.step_resident, c.stream, flush, n)
            row[f"learned_cost_jointnerf_{'broadphase' if bp else 'bruteforce'}_ms_p50"] = float(np.percentile(ms, 50))
        nerf.close()
        cross[f"{spl}_spheres_per_link"] = row
    out["surrogate_crossover_1000x30"] = cross
    return out


def run_ablation(args):
    """Closed-loop sampling ablation (the paper's pseudo-random vs Halton and comb
    vs B-spline vs mixed studies, on the synthetic paper-scale workload): every
    sampler x filter x particle count reaches the same goals from the same start
    through the ideal double-integrator plant; reported per variant: position
    and quaternion error (1 - |q . q_g|) averaged over the last 50 steps of each
    goal, and the mean absolute joint jerk (smoothness)."""
    import torch
    from paper_2104_13542_b300 import Controller
    base = W.config_paper(args.seed)
    # pose reaching in free space with the paper's orientation-constrained weights
    base.world = W.World(np.zeros((0, 6)), np.zeros((0, 4)))
    base.params = base.params.replace(w_pos=100.0, w_rot=100.0)
    goals = None
    steps_per_goal = 400
    out = {}
    for N in (100, 500):
        for sampler, scr, sname in ((W.SAMPLER_PHILOX, 0, "pseudo_random"), (W.SAMPLER_HALTON, 0, "halton"),
                                    (W.SAMPLER_HALTON, 1, "halton_scrambled")):
            for filt, fname in ((W.FILTER_COMB, "comb"), (W.FILTER_DEFAULT, "bspline"),
                                (W.FILTER_MIXED, "mixed")):
                p = base.params.replace(N=N, sampler=sampler, halton_scramble=scr, filter=filt, n_null=2)
                with Controller(base.robot, base.world, p) as ctl:
                    if goals is None:
                        _, th = goals_for(ctl, base.robot, args.seed, 1, with_theta=True)
                        start = th[0]  # a configuration clear of self-collision, at rest
                        goals = _local_goals(ctl, start, args.seed, 3)
                    state = np.zeros((3, base.robot.dof), np.float32)
                    state[0] = start
                    dt = float(p.dt[0])
                    pos_e, rot_e, jerk, prev = [], [], [], None
                    for goal in goals:
                        for i in range(steps_per_goal):
                            cmd, info, rc = ctl.step(state, goal)
                            if prev is not None:
                                jerk.append(float(np.abs(cmd - prev).mean() / dt))
                            prev = cmd.copy()
                            state[2] = cmd
                            state[1] = state[1] + dt * cmd
                            state[0] = state[0] + dt * state[1]
                            if i >= steps_per_goal - 50:
                                T = ctl.forward_kinematics(torch.as_tensor(state[0:1], device="cuda")).cpu().numpy()[0]
                                pos_e.append(float(np.linalg.norm(T[:, 3] - goal[:3])))
                                R = T[:, :3].astype(np.float64)
                                tr = float(np.trace(_rot_from_quat(goal[3:]).T @ R))
                                rot_e.append(1.0 - 0.5 * np.sqrt(max(0.0, 1.0 + tr)))
                out[f"N{N}_{sname}_{fname}"] = {"pos_err_m": float(np.mean(pos_e)),
                                                "quat_err": float(np.mean(rot_e)),
                                                "mean_abs_jerk": float(np.mean(jerk))}
    return {"ablation": out, "workload": base.name, "goals": len(goals), "steps_per_goal": steps_per_goal,
            "data": "synthetic"}


def run_mlp_forward(args):
    """Forward passes of both surrogate networks on `--mlp-forward` random
    configurations (device time per pass, CUDA events, 3 warm-up passes): the
    fused whole-network kernel and the layer-by-layer kernels, with the
    tensor-core throughput of the three layers for each."""
    import torch
    from paper_2104_13542_b300 import SurrogateMLP
    rows = args.mlp_forward
    th = torch.as_tensor(np.random.default_rng(args.seed).uniform(-2.8, 2.8, (rows, 7)).astype(np.float32),
                         device="cuda")
    R = (rows + 127) // 128 * 128
    out = {}
    for arch, widths in (("distance", (256, 256, 256)), ("jointnerf", (256, 128, 64))):
        net = SurrogateMLP(seed=args.seed, arch=arch)
        flops = 2.0 * R * (16 * widths[0] + widths[0] * widths[1] + widths[1] * widths[2])
        y = torch.empty(rows, dtype=torch.float32, device="cuda")
        for mode in ("fused", "layers"):
            layers = mode == "layers"
            for _ in range(3):
                net.predict(th, layers=layers, out=y)
            if layers:  # each call waits on the host: per call, host round trip included
                ev = []
                for _ in range(10):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(net.stream)
                    net.predict(th, layers=True, out=y)
                    b.record(net.stream)
                    ev.append((a, b))
                torch.cuda.synchronize()
                ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
            else:  # 20 back-to-back kernels between two events on the network's stream
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(net.stream)
                for _ in range(20):
                    net.predict(th, out=y, wait=False)
                b.record(net.stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / 20
            out[f"{arch}_{mode}"] = {"ms": ms, "gemm_tflops": flops / (ms * 1e-3) / 1e12, "rows": rows}
        net.close()
    peak = measured_peaks().get("bf16_tflops")
    if peak:
        for k in out:
            out[k]["frac_bf16_peak"] = out[k]["gemm_tflops"] / peak
    return {"mlp_forward": out, "bf16_peak_tflops": peak,
            "note": "fused: device time per kernel, 20 back to back (inputs 1.8 MB, L2-resident); layers: "
                    "per predict call, encode + 3 layer kernels + output copy + the host wait"}


def _local_goals(ctl, theta0, seed: int, count: int):
    """Goal poses FK(theta_g) with theta_g = theta0 + U[-0.6, 0.6] rad per joint, within
    [-2.2, 2.2] and 3 cm clear of self-collision: reaching moves that a local
    optimiser can complete, so the samplers are compared on accuracy and smoothness."""
    import torch
    rng = np.random.default_rng([seed, 123])
    cand = np.clip(theta0 + rng.uniform(-0.6, 0.6, (64 * count, theta0.shape[0])), -2.2, 2.2).astype(np.float32)
    sd = ctl.self_distance(torch.as_tensor(cand, device="cuda")).cpu().numpy()
    th = cand[sd > 0.03][:count]
    ee = ctl.forward_kinematics(torch.as_tensor(th, device="cuda")).cpu().numpy()
    goals = []
    for T in ee:
        q = _quat_from_rot(T[:, :3].astype(np.float64))
        goals.append(np.concatenate([T[:, 3], q]).astype(np.float32))
    return goals


def _quat_from_rot(Rm):
    w = math.sqrt(max(0.0, 1 + Rm[0, 0] + Rm[1, 1] + Rm[2, 2])) / 2
    x = math.copysign(math.sqrt(max(0.0, 1 + Rm[0, 0] - Rm[1, 1] - Rm[2, 2])) / 2, Rm[2, 1] - Rm[1, 2])
    y = math.copysign(math.sqrt(max(0.0, 1 - Rm[0, 0] + Rm[1, 1] - Rm[2, 2])) / 2, Rm[0, 2] - Rm[2, 0])
    z = math.copysign(math.sqrt(max(0.0, 1 - Rm[0, 0] - Rm[1, 1] + Rm[2, 2])) / 2, Rm[1, 0] - Rm[0, 1])
    return np.array([w, x, y, z])


def _rot_from_quat(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_steps(wl, n, budget_s, threads):
    """Control steps of the FP64 oracle on n particles with `threads` host threads
    in its rollout loop, until budget_s seconds or 50 steps."""
    import oracle
    p = wl.params
    orc = oracle.Oracle(wl.robot, wl.world, p.replace(N=n))
    mu, sig = np.zeros((p.H, wl.robot.dof)), np.full(wl.robot.dof, p.sigma_init)
    prev = oracle.get_threads()
    oracle.set_threads(threads)
    times = []
    try:
        t_start = time.perf_counter()
        step = 0
        while True:
            t0 = time.perf_counter()
            _, mu, sig, _, _ = orc.step(wl.state, wl.goal, step, mu, sig)
            times.append(time.perf_counter() - t0)
            step += 1
            if time.perf_counter() - t_start > budget_s or step >= 50:
                break
    finally:
        oracle.set_threads(prev)
    return np.array(times)


def cpu_baseline(wl, budget_s: float = 12.0, n_sample: int | None = None):
    """Time the FP64 oracle's control step on the host cores: all cores (OpenMP
    over particles; the same bits as one thread) and a single thread, each for
    about budget_s / 2 seconds."""
    p = wl.params
    n = n_sample or p.N
    cores = os.cpu_count() or 1
    legs = {}
    for name, threads in (("all_cores", cores), ("single_thread", 1)):
        t = _oracle_steps(wl, n, budget_s / 2, threads)
        legs[name] = {"value": n * p.H * p.K / float(t.mean()), "unit": UNIT, "cores": threads,
                      "steps": len(t),
                      "latency_ms": {"p50": float(np.percentile(t, 50) * 1e3),
                                     "p99": float(np.percentile(t, 99) * 1e3)}}
    out = dict(legs["all_cores"])
    out.update({"kind": "oracle", "cpu_model": cpu_model(),
                "sample": f"{legs['all_cores']['steps']} control steps of the FP64 oracle with {n} of {p.N} "
                          f"particles (H={p.H}, K={p.K}) on {cores} threads (rollout loop over particles, "
                          f"OpenMP); single-thread leg: {legs['single_thread']['steps']} steps",
                "single_thread": legs["single_thread"]})
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle on all the host cores (OpenMP over
    particles), each step one oracle control step -- on all the workload's
    particles when (warm-up + steps) of them fit in about 150 s, else on the
    largest particle sample that does (--ref-particles N fixes the sample)."""
    import oracle
    wl = W.config_paper(seed=args.seed)
    p = wl.params
    cores = os.cpu_count() or 1
    prev = oracle.get_threads()
    oracle.set_threads(cores)
    try:
        n = args.ref_particles
        if n <= 0:  # size the sample from one full step
            t1 = _oracle_steps(wl, p.N, 0.0, cores)[0]
            total = (args.warmup + args.steps) * t1
            n = p.N if total <= 150.0 else max(8, int(p.N * 150.0 / total))
        ps = p.replace(N=n)
        orc = oracle.Oracle(wl.robot, wl.world, ps)
        mu, sig = np.zeros((p.H, wl.robot.dof)), np.full(wl.robot.dof, p.sigma_init)
        for w in range(args.warmup):
            _, mu, sig, _, _ = orc.step(wl.state, wl.goal, w, mu, sig)
        times = []
        for i in range(args.steps):
            t0 = time.perf_counter()
            _, mu, sig, _, _ = orc.step(wl.state, wl.goal, args.warmup + i, mu, sig)
            times.append(time.perf_counter() - t0)
    finally:
        oracle.set_threads(prev)
    t = np.array(times)
    value = n * p.H * p.K * len(t) / float(t.sum())
    sample = (f"each step: one FP64 oracle control step on {n} of the {p.N} particles "
              f"(H={p.H}, K={p.K}), {cores} threads (OpenMP over particles)")
    return {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(t.mean() * 1e3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "N": p.N, "H": p.H, "K": p.K, "dof": wl.robot.dof,
                       "sample_particles": n},
            "latency_ms": {"p50": float(np.percentile(t, 50) * 1e3),
                           "p99": float(np.percentile(t, 99) * 1e3)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["b300", "reference"], default="b300")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ref-particles", type=int, default=0,
                    help="reference arm: particles per oracle step (0: all of them when the run fits "
                         "in about 150 s, else the largest sample that does)")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--launch", default="auto",
                    help="rollout launch shape: auto (autotuned), warp:W (W warps per CTA), pair:W (W warp "
                         "pairs per CTA), quad:W (W four-warp groups per CTA) or cta:P,T")
    ap.add_argument("--dep-launch", action="store_true",
                    help="launch the step graph's rollouts and updates as programmatic dependents")
    ap.add_argument("--mlp-forward", type=int, default=0, metavar="ROWS",
                    help="time the surrogate networks' forward pass on ROWS configurations instead")
    ap.add_argument("--ablation", action="store_true",
                    help="run the closed-loop sampling ablation instead of the benchmark")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", 0))
    world_size = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)))
        return
    if args.ablation:
        if rank == 0:
            print(json.dumps(run_ablation(args)))
        return
    if args.mlp_forward:
        if rank == 0:
            print(json.dumps(run_mlp_forward(args)))
        return

    if world_size > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    res, wl = run_gpu(args, rank, world_size)
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    p = wl.params
    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world_size,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl.name, "N": p.N, "H": p.H, "K": p.K, "dof": wl.robot.dof,
                   "knots": p.n_knots, "spheres": int(wl.robot.spheres.shape[0]),
                   "self_pairs": int(wl.robot.pairs.shape[0]),
                   "boxes": int(wl.world.boxes.shape[0]),
                   "obstacle_spheres": int(wl.world.spheres.shape[0]),
                   "l2": "flushed (256 MB write) before every timed step",
                   "inputs": "the closed-loop sequence of the e2e run (the arm driving to 5 goals), "
                             "replayed from HBM",
                   "parallelism": f"replicas x{world_size}"},
        "latency_ms": res["latency_ms"], "latency_rest_ms": res["latency_rest_ms"],
        "e2e": res["e2e"], "roofline": res["roofline"],
        "clocks": res["clocks"], "gpu_launches": res["gpu_launches"],
    }
    if world_size == 1 and not args.no_variants:
        line["variants"] = run_variants(args, args.seed, res["roofline"]["peak"])
    if world_size == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_budget_s)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
