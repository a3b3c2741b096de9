"""Pins of the oracle's samplers (comb and mixed filters, Sec. 4.3), end-effector
velocity / acceleration (Eq. 8) with the task-space limit terms, and the
ball-on-tray model (appendix, ball balancing).

Each is checked against something other than itself: the comb filter against
scipy's recursive-filter routine and its impulse response, the mixed sampler
against scipy's B-spline design matrix, X_dot / X_ddot against central finite
differences of the oracle's forward kinematics along theta(t) = theta +
t theta_dot + t^2/2 theta_ddot, and the ball against the constant-acceleration
closed form on a static tray.
"""
import numpy as np
import pytest
import scipy.interpolate
import scipy.signal

import oracle
from paper_2104_13542_b300 import workloads as W


# ----------------------------------------------------------------------------- comb filter

def test_comb_filter_is_the_second_order_recursive_filter():
    rng = np.random.default_rng(0)
    eps = rng.normal(size=(30, 7))
    c = (0.5, 0.3, 0.2)
    ref = scipy.signal.lfilter([c[0]], [1.0, -c[1], -c[2]], eps, axis=0)
    assert np.allclose(oracle.comb_filter(c, eps), ref, atol=1e-13)
    imp = np.zeros((6, 1))
    imp[0] = 1.0
    y = oracle.comb_filter(c, imp)[:, 0]
    assert np.allclose(y[:3], [c[0], c[0] * c[1], c[0] * (c[1] ** 2 + c[2])], atol=1e-15)
    # a pure gain passes the samples through scaled
    assert np.allclose(oracle.comb_filter((2.0, 0.0, 0.0), eps), 2.0 * eps)


def _clamped_basis(H, S):
    knots = np.concatenate([[0.0] * 4, np.arange(1, S - 3) / (S - 3), [1.0] * 4])
    return scipy.interpolate.BSpline.design_matrix(np.arange(H) / (H - 1), knots, 3).toarray()


@pytest.mark.parametrize("filt", [W.FILTER_COMB, W.FILTER_MIXED])
def test_filtered_controls(filt):
    wl = W.config_paper(0)
    c = (0.6, 0.25, 0.1)
    p = wl.params.replace(N=11, H=24, n_knots=6, n_null=2, filter=filt, comb=c, mix_bspline=0.6)
    o = oracle.Oracle(wl.robot, wl.world, p)
    assert o.n_noise == 24  # one sample per step for both filters
    rng = np.random.default_rng(1)
    mu, sig = rng.normal(size=(24, 7)), rng.uniform(0.1, 0.9, 7)
    eps = o.noise(3, 1)
    assert eps.shape == (11, 24, 7)
    u = o.controls(mu, sig, eps)
    n_bs = int(np.floor(0.6 * (11 - 2) + 0.5)) if filt == W.FILTER_MIXED else 0
    assert n_bs in (0, 5)
    B = _clamped_basis(24, 6)
    for n in range(11):
        if n < 2:
            assert np.all(u[n] == 0.0)
            continue
        if n < 2 + n_bs:
            e = B @ eps[n, :6]
        else:
            e = scipy.signal.lfilter([c[0]], [1.0, -c[1], -c[2]], eps[n], axis=0)
        assert np.allclose(u[n], mu + sig * e, atol=1e-12), n


# ----------------------------------------------------------------------------- Eq. 8 twist

def _pose(o, th, thd, thdd, t):
    F = o.fk(th + t * thd + 0.5 * t * t * thdd)[-1]
    return F[:3, :3], F[:3, 3]


def _omega(o, th, thd, thdd, t, h):
    Rp, _ = _pose(o, th, thd, thdd, t + h)
    Rm, _ = _pose(o, th, thd, thdd, t - h)
    R0, _ = _pose(o, th, thd, thdd, t)
    Wm = (Rp - Rm) / (2 * h) @ R0.T
    return np.array([Wm[2, 1], Wm[0, 2], Wm[1, 0]])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ee_twist_matches_finite_differences(seed):
    wl = W.config_paper(seed)
    o = oracle.Oracle(wl.robot, wl.world, wl.params)
    rng = np.random.default_rng(10 + seed)
    th, thd, thdd = rng.uniform(-2, 2, 7), rng.uniform(-1.5, 1.5, 7), rng.uniform(-3, 3, 7)
    xd, xdd = o.ee_twist(th, thd, thdd)
    h = 1e-4
    _, p0 = _pose(o, th, thd, thdd, 0.0)
    _, pp = _pose(o, th, thd, thdd, h)
    _, pm = _pose(o, th, thd, thdd, -h)
    v = (pp - pm) / (2 * h)
    a = (pp - 2 * p0 + pm) / (h * h)
    w = _omega(o, th, thd, thdd, 0.0, 1e-5)
    al = (_omega(o, th, thd, thdd, h, 1e-5) - _omega(o, th, thd, thdd, -h, 1e-5)) / (2 * h)
    assert np.allclose(xd[:3], v, atol=1e-7 * max(1, np.abs(v).max()))
    assert np.allclose(xd[3:], w, atol=1e-7 * max(1, np.abs(w).max()))
    assert np.allclose(xdd[:3], a, atol=2e-5 * max(1, np.abs(a).max()))
    assert np.allclose(xdd[3:], al, atol=2e-5 * max(1, np.abs(al).max()))
    # X_dot is the Jacobian times theta_dot, and linear in it; X_ddot at rest is J theta_ddot
    assert np.allclose(xd, o.jacobian(th) @ thd, atol=1e-12)
    xd0, xdd0 = o.ee_twist(th, np.zeros(7), thdd)
    assert np.allclose(xd0, 0.0) and np.allclose(xdd0, o.jacobian(th) @ thdd, atol=1e-12)


def test_ee_limit_terms_are_hinges():
    wl = W.config_paper(0)
    p = wl.params.replace(ee_vel_max=0.3, ee_acc_max=2.0)
    o = oracle.Oracle(wl.robot, wl.world, p)
    rng = np.random.default_rng(5)
    th, thd, u = rng.uniform(-2, 2, 7), rng.uniform(-1.5, 1.5, 7), rng.uniform(-3, 3, 7)
    terms, _ = o.running_cost(wl.goal, 3, th, thd, u, np.zeros(7))
    xd, xdd = o.ee_twist(th, thd, u)
    assert terms[8] == pytest.approx(max(0.0, np.linalg.norm(xd[:3]) - 0.3), abs=1e-12)
    assert terms[9] == pytest.approx(max(0.0, np.linalg.norm(xdd[:3]) - 2.0), abs=1e-12)
    terms0, _ = o.running_cost(wl.goal, 3, th, np.zeros(7), np.zeros(7), np.zeros(7))
    assert terms0[8] == 0.0 and terms0[9] == 0.0


# ----------------------------------------------------------------------------- ball on tray

def _ball_workload(seed=0, H=15):
    wl = W.config_ball(seed)
    return wl, wl.params.replace(N=3, H=H)


def test_ball_static_tray_closed_form():
    wl, p = _ball_workload()
    o = oracle.Oracle(wl.robot, wl.world, p)
    pos, vel = wl.ball[:3], wl.ball[3:]
    o.set_ball(pos, vel)
    state = wl.state.copy()
    state[1:] = 0.0
    theta = np.tile(state[0], (p.H, 1))
    xb, vb = o.ball_states(state, theta)
    F = o.fk(state[0])[-1]
    R0, p0 = F[:3, :3], F[:3, 3]
    x0, v0 = R0.T @ (pos - p0), R0.T @ vel
    v0[2] = 0.0
    g = R0.T @ np.array(p.gravity)
    a = np.array([g[0], g[1], 0.0])
    dt = p.dt[0]
    for h in range(p.H):
        k = h + 1
        assert np.allclose(vb[h], v0 + a * k * dt, atol=1e-13)
        assert np.allclose(xb[h], x0 + k * dt * v0 + a * dt * dt * k * (k + 1) / 2, atol=1e-13)


def test_ball_cost_in_rollout():
    """A static arm (every particle null, zero velocity): the running cost is
    the ball's in-plane distance from the tray centre, w_ball = 1."""
    wl, p = _ball_workload(1, H=12)
    zero = {k: 0.0 for k in ("w_pos", "w_rot", "w_stop", "w_joint", "w_manip", "w_coll", "w_smooth")}
    p = p.replace(n_null=p.N, w_ball=1.0, tray_center=(0.01, -0.02, 0.0), **zero)
    o = oracle.Oracle(wl.robot, wl.world, p)
    o.set_ball(wl.ball[:3], wl.ball[3:])
    state = wl.state.copy()
    state[1:] = 0.0
    out = o.rollout(state, wl.goal, np.zeros((p.H, 7)), np.full(7, 0.3), o.noise(0, 0))
    xb, _ = o.ball_states(state, np.tile(state[0], (p.H, 1)))
    ref = np.hypot(xb[:, 0] - 0.01, xb[:, 1] + 0.02)
    for n in range(p.N):
        assert np.allclose(out["terms"][n, :, 10], ref, atol=1e-13)
        assert np.allclose(out["cost"][n], ref, atol=1e-13)


def test_ball_level_tray_rolls_straight():
    """With gravity along the tray normal the ball keeps its in-plane velocity."""
    wl, p = _ball_workload(2)
    o = oracle.Oracle(wl.robot, wl.world, p)
    state = wl.state.copy()
    state[1:] = 0.0
    F = o.fk(state[0])[-1]
    n_w = F[:3, 2]  # tray normal (end-effector z) in the world
    o2 = oracle.Oracle(wl.robot, wl.world, p.replace(gravity=tuple(-9.81 * n_w)))
    o2.set_ball(F[:3, 3], np.array([0.1, -0.05, 0.02]))
    xb, vb = o2.ball_states(state, np.tile(state[0], (p.H, 1)))
    v0 = F[:3, :3].T @ np.array([0.1, -0.05, 0.02])
    v0[2] = 0.0
    assert np.allclose(vb, v0, atol=1e-12)
    assert np.allclose(xb[-1], v0 * p.dt[0] * p.H, atol=1e-12)
