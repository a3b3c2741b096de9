"""GPU adjoint (dJ/dmu of the rollout cost) against the FP64 oracle's adjoint,
which is itself pinned by finite differences (tests/test_oracle_adjoint.py);
the autograd wrapper; and gradient refinement inside the control step."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13542_b300 import Controller, storm_cost
from paper_2104_13542_b300 import workloads as W

from gpu_helpers import TOL_COST, cuda, f32, host, max_rel, mu_tolerance

pytestmark = pytest.mark.gpu


def _pair(wl, p, seed=0, step=3, it=1):
    mu = f32(W.make_mean(seed, p.H, 7, 0.5))
    sig = f32(W.make_sigma(seed, 7))
    state, goal = f32(W.make_state(seed + 30, 7)), f32(wl.goal)
    with Controller(wl.robot, wl.world, p) as ctl:
        ctl.set_distribution(mu, sig)
        J, g, Cn = ctl.cost_grad(cuda(mu), cuda(state), cuda(goal), step, it, want_C=True)
        torch.cuda.synchronize()
        J, g, Cn = float(host(J)[0]), host(g), host(Cn)
    o = oracle.Oracle(wl.robot, wl.world, p)
    oJ, og = o.cost_grad(state, goal, mu, sig, o.noise(step, it))
    return (J, g, Cn), (oJ, og), o, (state, goal, mu, sig)


@pytest.mark.parametrize("name,N,kw", [
    ("paper", 64, {}),
    ("paper", 500, {}),
    ("paper_frob_null", 48, dict(rot_mode=W.ROT_FROBENIUS, rot_axis_w=(0.5, 1.0, 2.0), n_null=4)),
    ("paper_halton_smooth", 40, dict(sampler=W.SAMPLER_HALTON, w_smooth=2.0, k_m=0.3)),
    ("small", 64, {}),
])
def test_cost_grad_matches_oracle(name, N, kw):
    wl = W.config_small(0) if name == "small" else W.config_paper(2)
    p = wl.params.replace(N=N, **kw)
    (J, g, Cn), (oJ, og), o, _ = _pair(wl, p)
    assert abs(J - oJ) <= TOL_COST * max(1.0, abs(oJ))
    scale = max(1e-6, np.abs(og).max())
    assert max_rel(g, og, scale) < 1e-4, max_rel(g, og, scale)


@pytest.mark.parametrize("world", [(20, 10), (64, 64)])
def test_cost_grad_broadphase_is_exact(world):
    """The adjoint's collision broad phase (link bounds against obstacles and
    against each other) skips only tests that cannot penetrate: the gradient, J
    and every particle's total are bitwise those of the brute-force tests, on
    the paper world and on a dense one."""
    wl = W.config_paper(4)
    wl.world = W.make_world(4, *world)
    p = wl.params.replace(N=96)
    mu, sig = f32(W.make_mean(4, p.H, 7, 0.8)), f32(W.make_sigma(4, 7))
    state, goal = cuda(f32(W.make_state(34, 7))), cuda(f32(wl.goal))
    out = []
    for bp in (True, False):
        with Controller(wl.robot, wl.world, p) as ctl:
            ctl.set_broadphase(bp)
            ctl.set_distribution(mu, sig)
            J, g, Cn = ctl.cost_grad(cuda(mu), state, goal, 5, 2, want_C=True)
            torch.cuda.synchronize()
            out.append((host(J), host(g), host(Cn)))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    # the case has world and self contacts (some totals carry collision cost)
    assert (out[0][2] > 100.0).any()


def test_autograd_function_matches_adjoint():
    wl = W.config_paper(3)
    p = wl.params.replace(N=128)
    mu0 = f32(W.make_mean(3, p.H, 7, 0.5))
    state, goal = cuda(f32(wl.state)), cuda(f32(wl.goal))
    with Controller(wl.robot, wl.world, p) as ctl:
        ctl.set_distribution(mu0, f32(W.make_sigma(3, 7)))
        mu = cuda(mu0).requires_grad_(True)
        J = storm_cost(mu, ctl, state, goal, 2, 0)
        (gm,) = torch.autograd.grad(3.0 * J, mu)
        J2, g2 = ctl.cost_grad(cuda(mu0), state, goal, 2, 0)
        torch.cuda.synchronize()
    assert torch.allclose(gm, 3.0 * g2, rtol=0, atol=0)
    assert float(J) == float(J2[0])


def test_gradient_step_descends():
    wl = W.config_paper(0)
    p = wl.params.replace(N=500)
    mu = f32(W.make_mean(0, p.H, 7, 0.3))
    sig = f32(W.make_sigma(0, 7))
    state, goal = cuda(f32(wl.state)), cuda(f32(wl.goal))
    with Controller(wl.robot, wl.world, p) as ctl:
        ctl.set_distribution(mu, sig)
        m = cuda(mu)
        Js = []
        for _ in range(5):
            J, g = ctl.cost_grad(m, state, goal, 0, 3)
            Js.append(float(J[0]))
            m = m - 0.01 * g
        torch.cuda.synchronize()
    assert all(b < a for a, b in zip(Js, Js[1:])), Js


@pytest.mark.parametrize("N", [64, 500])
def test_refined_step_matches_oracle(N):
    wl = W.config_differentiable(1, N=N)
    p = wl.params
    state, goal = f32(W.make_state(41, 7)), f32(wl.goal)
    o = oracle.Oracle(wl.robot, wl.world, p)
    with Controller(wl.robot, wl.world, p) as ctl:
        cmd, info, rc = ctl.step(state, goal)
        mu, sig = ctl.get_distribution()
    ocmd, omu, osig, ost, obest = o.step(state, goal, 0, np.zeros((p.H, 7)),
                                         np.full(7, f32(p.sigma_init)))
    assert rc == 0 and info["step"] == 0
    tol = mu_tolerance([obest], p.beta)
    scale = max(1.0, np.abs(omu).max())
    assert max_rel(mu, omu, scale) < tol
    assert np.array_equal(cmd, mu[0])
    assert max_rel(sig, osig, max(1e-3, osig.max())) < tol
    # the refinement moved the mean: compare with the plain step
    with Controller(wl.robot, wl.world, p.replace(grad_steps=0)) as ctl0:
        ctl0.step(state, goal)
        mu0, _ = ctl0.get_distribution()
    assert np.abs(mu - mu0).max() > 1e-4


def _swap_spheres(robot, a, b):
    """The robot with spheres a and b (of one link) exchanged, pairs renumbered."""
    order = np.arange(len(robot.sphere_link))
    order[[a, b]] = order[[b, a]]
    pairs = np.sort(order[np.asarray(robot.pairs)], axis=1)
    return W.Robot(robot.dh, robot.q_min, robot.q_max, np.asarray(robot.sphere_link)[order],
                   np.asarray(robot.spheres)[order], pairs)


def test_cost_grad_more_than_eight_spheres_per_link():
    """Nine spheres per link, so that a pair block's first link has more rows
    than the eight slots of its second.  In this folded case every item
    self-collides, and with spheres 16 and 17 of link 2 exchanged the deepest
    pair of most items lies in that link's ninth row (checked on the oracle's
    FK).  The gradient and J match the oracle's adjoint, and the broad phase on
    and off give the same bits."""
    wl = W.config_paper(5)
    wl.robot = _swap_spheres(W.make_robot(5, 7, spheres_per_link=9), 16, 17)
    p = wl.params.replace(N=64)
    seed, step, it = 5, 3, 1
    mu, sig = f32(W.make_mean(seed, p.H, 7, 0.8)), f32(W.make_sigma(seed, 7))
    state, goal = f32(W.make_state(seed, 7)), f32(wl.goal)
    o = oracle.Oracle(wl.robot, wl.world, p)
    eps = o.noise(step, it)
    roll = o.rollout(state, goal, mu, sig, eps)
    active = roll["terms"][..., 5] > 0
    assert active.mean() > 0.5
    sl, sp, pairs = np.asarray(wl.robot.sphere_link), np.asarray(wl.robot.spheres), np.asarray(wl.robot.pairs)
    first = {int(l): int(np.argmax(sl == l)) for l in np.unique(sl)}
    late = 0
    for n, h in list(zip(*np.nonzero(active)))[::8]:
        fr = o.fk(roll["theta"][n, h])
        c = np.array([(fr[sl[s]] @ np.append(sp[s, :3], 1.0))[:3] for s in range(len(sl))])
        depth = sp[pairs[:, 0], 3] + sp[pairs[:, 1], 3] - np.linalg.norm(c[pairs[:, 0]] - c[pairs[:, 1]], axis=1)
        a = pairs[int(np.argmax(depth)), 0]
        late += a - first[int(sl[a])] >= 8
    assert late > 10
    oJ, og = o.cost_grad(state, goal, mu, sig, eps)
    out = []
    for bp in (True, False):
        with Controller(wl.robot, wl.world, p) as ctl:
            ctl.set_broadphase(bp)
            ctl.set_distribution(mu, sig)
            J, g = ctl.cost_grad(cuda(mu), cuda(state), cuda(goal), step, it)
            torch.cuda.synchronize()
            out.append((float(host(J)[0]), host(g)))
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])
    J, g = out[0]
    assert abs(J - oJ) <= TOL_COST * max(1.0, abs(oJ))
    scale = max(1e-6, np.abs(og).max())
    assert max_rel(g, og, scale) < 1e-4, max_rel(g, og, scale)
