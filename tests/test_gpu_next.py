"""GPU parity of the widened rows against the FP64 oracle: comb and mixed
samplers (Sec. 4.3), the variable time-step schedule with the end-effector
speed / acceleration limits built on Eq. 8's X_dot and X_ddot, and the
ball-on-tray cost (appendix); both work mappings stay bitwise identical on
them; and a closed-loop ball-balancing run on the GPU.  Tolerances are those of
tests/gpu_helpers.py."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13542_b300 import Controller, StormError
from paper_2104_13542_b300 import workloads as W

from gpu_helpers import TOL_COST, TOL_STATE, cuda, f32, host, manip_flips, max_rel, mu_tolerance

pytestmark = pytest.mark.gpu


def _cases():
    paper = W.config_paper(0)
    vardt = W.config_variable_dt(1)
    mixed = W.config_mixed(2)
    ball = W.config_ball(3)
    return {
        "vardt_ee": (vardt, vardt.params.replace(N=61)),
        "comb_philox": (paper, paper.params.replace(N=40, filter=W.FILTER_COMB, comb=(0.6, 0.25, 0.1))),
        "comb_halton_H50": (paper, paper.params.replace(N=23, H=50, filter=W.FILTER_COMB,
                                                        sampler=W.SAMPLER_HALTON)),
        "mixed": (mixed, mixed.params.replace(N=53)),
        "mixed_H12_null5": (mixed, mixed.params.replace(N=37, H=12, n_null=5, mix_bspline=0.3)),
        "ball": (ball, ball.params.replace(N=37)),
        "ball_H16_vardt": (ball, ball.params.replace(N=19, H=16, dt=0.015 * 1.1 ** np.arange(16),
                                                     w_ee_vel=10.0, ee_vel_max=0.2)),
    }


CASES = _cases()


def _inputs(wl, p, seed):
    mu = f32(W.make_mean(seed, p.H, 7, 0.5))
    sig = f32(W.make_sigma(seed, 7))
    state = f32(W.make_state(seed + 10, 7))
    return mu, sig, state, f32(wl.goal)


def _with_ball(wl, ctl=None, orc=None):
    if wl.ball is None:
        return
    if ctl is not None:
        ctl.set_ball(wl.ball[:3], wl.ball[3:])
    if orc is not None:
        orc.set_ball(f32(wl.ball[:3]), f32(wl.ball[3:]))


@pytest.mark.parametrize("name", list(CASES))
def test_rollout_parity(name):
    wl, p = CASES[name]
    mu, sig, state, goal = _inputs(wl, p, 4)
    orc = oracle.Oracle(wl.robot, wl.world, p)
    _with_ball(wl, orc=orc)
    with Controller(wl.robot, wl.world, p) as ctl:
        _with_ball(wl, ctl=ctl)
        ctl.set_distribution(mu, sig)
        g = {k: host(v) for k, v in ctl.generate_rollouts(cuda(state), cuda(goal), 2, 1).items()}
    o = orc.rollout(state, goal, mu, sig, orc.noise(2, 1))
    assert max_rel(g["u"], o["u"], max(1.0, np.abs(o["u"]).max())) < TOL_STATE
    assert max_rel(g["theta"], o["theta"], max(1.0, np.abs(o["theta"]).max())) < TOL_STATE
    assert max_rel(g["ee"], o["ee"], 1.0) < TOL_STATE
    flip, ok = manip_flips(orc, o["theta"], p.k_m, g["terms"], o["terms"])
    assert ok and flip.mean() <= 1e-3
    keep = ~flip
    for t in range(W.NTERMS):
        tscale = max(1.0, np.abs(o["terms"][..., t]).max())
        e = max_rel(g["terms"][..., t][keep], o["terms"][..., t][keep], tscale)
        assert e < TOL_COST, (W.TERM_NAMES[t], e)
    assert max_rel(g["cost"][keep], o["cost"][keep], max(1.0, np.abs(o["cost"]).max())) < TOL_COST
    rows = ~flip.any(axis=1)
    assert max_rel(g["C"][rows], o["C"][rows], max(1.0, np.abs(o["C"]).max())) < TOL_COST
    # the case exercises its row
    if p.w_ee_vel > 0:
        assert (o["terms"][..., 8] > 0).any()
    if p.w_ball > 0:
        assert (o["terms"][..., 10] > 0).all()


@pytest.mark.parametrize("name", list(CASES))
def test_mappings_bitwise_identical(name):
    wl, p = CASES[name]
    mu, sig, state, goal = _inputs(wl, p, 5)
    with Controller(wl.robot, wl.world, p) as ctl:
        _with_ball(wl, ctl=ctl)
        ctl.set_distribution(mu, sig)
        ctl.set_launch(2, 256)
        ref = {k: host(v) for k, v in ctl.generate_rollouts(cuda(state), cuda(goal), 3, 0).items()}
        for mapping, count in (("warp", 1), ("warp", 3), ("pair", 1), ("pair", 2), ("quad", 1), ("quad", 2)):
            {"warp": ctl.set_launch_warp, "pair": ctl.set_launch_warp_pair,
             "quad": ctl.set_launch_warp_quad}[mapping](count)
            g = {k: host(v) for k, v in ctl.generate_rollouts(cuda(state), cuda(goal), 3, 0).items()}
            for k in ref:
                assert np.array_equal(g[k], ref[k]), (mapping, count, k)


@pytest.mark.parametrize("name", ["vardt_ee", "mixed", "ball"])
def test_step_parity(name):
    wl, p = CASES[name]
    state, goal = f32(W.make_state(7, 7)), f32(wl.goal)
    orc = oracle.Oracle(wl.robot, wl.world, p)
    _with_ball(wl, orc=orc)
    with Controller(wl.robot, wl.world, p) as ctl:
        _with_ball(wl, ctl=ctl)
        mu0, sig0 = ctl.get_distribution()
        cmd, info, rc = ctl.step(state, goal)
        mu, sig = ctl.get_distribution()
    ocmd, omu, osig, ost, obest = orc.step(state, goal, 0, mu0, sig0)
    assert rc == ost == 0
    tol = mu_tolerance([obest, info["mean_weighted_cost"]], p.beta)
    scale = max(1.0, np.abs(omu).max())
    assert max_rel(mu, omu, scale) < tol
    assert max_rel(cmd, ocmd, scale) < tol
    assert max_rel(sig, osig, max(1e-3, osig.max())) < tol


def test_ee_twist_matches_oracle():
    wl = W.config_paper(6)
    o = oracle.Oracle(wl.robot, wl.world, wl.params)
    rng = np.random.default_rng(8)
    n = 300
    th = f32(rng.uniform(-2.8, 2.8, (n, 7)))
    thd = f32(rng.uniform(-2, 2, (n, 7)))
    thdd = f32(rng.uniform(-5, 5, (n, 7)))
    with Controller(wl.robot, wl.world, wl.params) as ctl:
        xd, xdd = ctl.ee_twist(cuda(th), cuda(thd), cuda(thdd))
        xd, xdd = host(xd), host(xdd)
    ref = [o.ee_twist(th[i], thd[i], thdd[i]) for i in range(n)]
    rxd = np.array([r[0] for r in ref])
    rxdd = np.array([r[1] for r in ref])
    assert max_rel(xd, rxd, max(1.0, np.abs(rxd).max())) < 2e-5
    assert max_rel(xdd, rxdd, max(1.0, np.abs(rxdd).max())) < 2e-5


def test_unsupported_combinations_are_rejected():
    wl = W.config_paper(0)
    with Controller(wl.robot, wl.world, wl.params.replace(N=16, H=10, w_ee_vel=1.0)) as ctl:
        s, g = cuda(f32(wl.state)), cuda(f32(wl.goal))
        with pytest.raises(StormError):
            ctl.cost_grad(cuda(np.zeros((10, 7), np.float32)), s, g, 0, 0)
        with pytest.raises(StormError):
            ctl.set_ball([0.0, np.nan, 0.0], [0.0, 0.0, 0.0])


def _tray_plant(ctl, theta, x, v, gravity, dt):
    """The ball on the tray one control period later (the controller's own model:
    in-plane gravity in the tray frame, semi-implicit step), and its world
    position / velocity for the next measurement."""
    T = host(ctl.forward_kinematics(cuda(f32(theta)[None])))[0]
    R, pe = T[:, :3].astype(np.float64), T[:, 3].astype(np.float64)
    a = R.T @ np.asarray(gravity)
    a[2] = 0.0
    v = v + dt * a
    x = x + dt * v
    return x, v, R @ x + pe, R @ v


def test_ball_balancing_closed_loop():
    """Ball on a level tray, 9.4 cm off centre: the controller tilts the tray and
    brings the ball back within 2 cm and holds it there (the plant is the same
    rolling model, stepped at the first time step of the schedule)."""
    wl = W.config_ball(0)
    p = wl.params.replace(N=500)
    state = f32(wl.state)
    state[1:] = 0.0
    dt = float(p.dt[0])
    with Controller(wl.robot, wl.world, p) as probe:
        T = host(probe.forward_kinematics(cuda(state[:1])))[0]
    R0, p0 = T[:, :3].astype(np.float64), T[:, 3].astype(np.float64)
    gravity = -9.81 * R0[:, 2]  # the tray starts level
    goal = np.concatenate([p0, [1.0, 0.0, 0.0, 0.0]]).astype(np.float32)  # hold position (w_rot = 0)
    p = p.replace(gravity=tuple(gravity))
    x, v = np.array([0.08, -0.05, 0.0]), np.zeros(3)
    dist = []
    with Controller(wl.robot, wl.world, p) as ctl:
        xw, vw = R0 @ x + p0, np.zeros(3)
        for t in range(400):
            ctl.set_ball(xw, vw)
            cmd, info, rc = ctl.step(state, goal)
            assert rc == 0
            state[2] = cmd
            state[1] += dt * cmd
            state[0] += dt * state[1]
            x, v, xw, vw = _tray_plant(ctl, state[0], x, v, gravity, dt)
            dist.append(np.hypot(x[0], x[1]))
    dist = np.array(dist)
    assert np.isfinite(dist).all()
    assert dist[-100:].max() < 0.02, dist[::40]
