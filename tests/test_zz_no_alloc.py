"""The rollout entry point that allocates no device memory.

Some callers cannot call cudaMalloc: code embedded in a host (a robot runtime,
a simulator) that owns the whole GPU memory budget and forbids allocation after
start-up, because an allocation can stall a real-time control loop or fail
under a fixed memory cap.  storm_rollout_costs_noalloc serves them with a
static device scratch array.  This file checks, through the C ABI, that it
returns bitwise the same rollout totals as the handle-based
storm_generate_rollouts, on two calls in a row (the second with another problem
size, so the shared scratch is rewritten) with the collision terms active, that
those totals match the FP64 oracle, and that it rejects a problem larger than
its scratch and a stream under capture.
It is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2104_13542_b300 import Controller, binding
from paper_2104_13542_b300 import workloads as W

import oracle
from gpu_helpers import TOL_COST, cuda, f32, host, manip_flips, max_rel

pytestmark = pytest.mark.gpu


def _reference_and_noalloc(wl, p, step, it, seed, state=None):
    mu = f32(W.make_mean(seed, p.H, wl.robot.dof, 0.5))
    sig = f32(W.make_sigma(seed, wl.robot.dof))
    state = f32(W.make_state(seed, wl.robot.dof) if state is None else state)
    state_dev, goal = cuda(state), cuda(f32(wl.goal))
    with Controller(wl.robot, wl.world, p) as ctl:
        ctl.set_distribution(mu, sig)
        ref = host(ctl.generate_rollouts(state_dev, goal, step, it, debug=False)["C"])
    stream = torch.cuda.current_stream()
    out = torch.full((p.N,), float("nan"), device="cuda")
    rc = binding.rollout_costs_noalloc(wl.robot, wl.world, p, state_dev, goal, cuda(mu), cuda(sig),
                                       step, it, out, stream)
    stream.synchronize()
    return rc, ref, host(out), (mu, sig, state)


def _collision_state():
    """A start state whose rollouts hit both self and world collision (chosen on
    the oracle, which the test re-checks)."""
    state = W.make_state(21, 7)
    state[0, 3], state[1, 3] = 2.2, 0.8
    return state


def test_noalloc_matches_generate_rollouts_twice():
    """Two calls in a row, of different sizes, each bitwise equal to the handle's
    rollout totals (every rollout mapping computes the same bits).  The first
    case has active self and world collision terms, so the scratch path's pair
    blocks, link bounds and broad phase are all exercised."""
    paper = W.config_paper(0)
    small = W.config_small(1)
    cases = [(paper, paper.params, 2, 1, 3, _collision_state()),
             (small, small.params.replace(N=200, H=25), 9, 0, 1, None)]
    for wl, p, step, it, seed, state in cases:
        rc, ref, got, _ = _reference_and_noalloc(wl, p, step, it, seed, state)
        assert rc == 0
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, ref), max_rel(got, ref, max(1.0, np.abs(ref).max()))


def test_noalloc_collision_case_is_active_and_matches_the_oracle():
    """The collision case of the test above, against the FP64 oracle: some items
    have non-zero self and world collision terms, and the totals agree within the
    cost tolerance (particles with an item on the manipulability jump, where FP32
    and FP64 may take different branches, left out and counted)."""
    wl = W.config_paper(0)
    p = wl.params
    step, it, seed = 2, 1, 3
    rc, ref, got, (mu, sig, state) = _reference_and_noalloc(wl, p, step, it, seed, _collision_state())
    assert rc == 0 and np.array_equal(got, ref)
    with Controller(wl.robot, wl.world, p) as ctl:
        ctl.set_distribution(mu, sig)
        g_terms = host(ctl.generate_rollouts(cuda(state), cuda(f32(wl.goal)), step, it)["terms"])
    orc = oracle.Oracle(wl.robot, wl.world, p)
    o = orc.rollout(state, f32(wl.goal), mu, sig, orc.noise(step, it))
    assert (o["terms"][..., 5] > 0).any(), "self collision inactive"
    assert (o["terms"][..., 6] > 0).any(), "world collision inactive"
    flip, ok = manip_flips(orc, o["theta"], p.k_m, g_terms, o["terms"])
    assert ok and flip.mean() <= 1e-3
    rows = ~flip.any(axis=1)
    assert max_rel(got[rows], o["C"][rows], max(1.0, np.abs(o["C"]).max())) < TOL_COST


def test_noalloc_rejects_a_capturing_stream():
    """Its table copies come from host memory that the call frees on return, so a
    graph captured from it would replay copies from freed memory: it refuses a
    stream that is being captured, before enqueueing anything."""
    wl = W.config_small(0)
    p = wl.params
    z = torch.zeros(p.H * 7, device="cuda")
    out = torch.zeros(p.N, device="cuda")
    graph, s = torch.cuda.CUDAGraph(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        graph.capture_begin()
        rc = binding.rollout_costs_noalloc(wl.robot, wl.world, p, z[:21], z[:7], z, z[:7], 0, 0, out, s)
        out.add_(1.0)  # something to capture
        graph.capture_end()
    assert rc == binding.STORM_ERR_INVALID_ARG
    graph.replay()
    torch.cuda.synchronize()
    assert float(out.max()) == 1.0


def test_noalloc_rejects_problem_beyond_scratch():
    wl = W.config_small(0)
    p = wl.params.replace(N=16384, H=64)  # 29 MB of controls > 8 MiB scratch
    z = torch.zeros(64 * 7, device="cuda")
    out = torch.zeros(p.N, device="cuda")
    rc = binding.rollout_costs_noalloc(wl.robot, wl.world, p, z[:21], z[:7], z, z[:7], 0, 0, out)
    assert rc == binding.STORM_ERR_INVALID_ARG
