"""The rollout entry point that allocates no device memory.

Some callers cannot call cudaMalloc: code embedded in a host (a robot runtime,
a simulator) that owns the whole GPU memory budget and forbids allocation after
start-up, because an allocation can stall a real-time control loop or fail
under a fixed memory cap.  storm_rollout_costs_noalloc serves them with a
static device scratch array.  This file checks, through the C ABI, that it
returns the same rollout totals as the handle-based storm_generate_rollouts,
on two calls in a row (the second with another problem size, so the shared
scratch is rewritten), and that it rejects a problem larger than its scratch.
It is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2104_13542_b300 import Controller, binding
from paper_2104_13542_b300 import workloads as W

from gpu_helpers import TOL_COST, cuda, f32, host, max_rel

pytestmark = pytest.mark.gpu


def _reference_and_noalloc(wl, p, step, it, seed):
    mu = f32(W.make_mean(seed, p.H, wl.robot.dof, 0.5))
    sig = f32(W.make_sigma(seed, wl.robot.dof))
    state, goal = cuda(f32(W.make_state(seed, wl.robot.dof))), cuda(f32(wl.goal))
    with Controller(wl.robot, wl.world, p) as ctl:
        ctl.set_distribution(mu, sig)
        ref = host(ctl.generate_rollouts(state, goal, step, it, debug=False)["C"])
    stream = torch.cuda.current_stream()
    out = torch.full((p.N,), float("nan"), device="cuda")
    rc = binding.rollout_costs_noalloc(wl.robot, wl.world, p, state, goal, cuda(mu), cuda(sig),
                                       step, it, out, stream)
    stream.synchronize()
    return rc, ref, host(out)


def test_noalloc_matches_generate_rollouts_twice():
    paper = W.config_paper(0)
    small = W.config_small(1)
    cases = [(paper, paper.params, 4, 2, 0),
             (small, small.params.replace(N=200, H=25), 9, 0, 1)]
    for wl, p, step, it, seed in cases:
        rc, ref, got = _reference_and_noalloc(wl, p, step, it, seed)
        assert rc == 0
        assert np.all(np.isfinite(got))
        assert max_rel(got, ref, max(1.0, np.abs(ref).max())) < TOL_COST


def test_noalloc_rejects_problem_beyond_scratch():
    wl = W.config_small(0)
    p = wl.params.replace(N=16384, H=64)  # 29 MB of controls > 8 MiB scratch
    z = torch.zeros(64 * 7, device="cuda")
    out = torch.zeros(p.N, device="cuda")
    rc = binding.rollout_costs_noalloc(wl.robot, wl.world, p, z[:21], z[:7], z, z[:7], 0, 0, out)
    assert rc == binding.STORM_ERR_INVALID_ARG
