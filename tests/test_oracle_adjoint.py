"""Pins of the oracle's hand-derived adjoint (dJ/dmu of the rollout cost).

The integration adjoint is checked against the explicit transposes of the
S_l(1) diag(dt) matrices of Eq. 7; every cost term's gradient and the full
dJ/dmu against FP64 central finite differences (h = 1e-6) of the oracle's own
forward cost at random points (away from kinks with probability ~1).
"""
import numpy as np
import pytest

import oracle
from paper_2104_13542_b300 import workloads as W

TERMS = ["w_pos", "w_rot", "w_stop", "w_joint", "w_manip", "w_coll", "w_smooth"]


def _only(p, name, **kw):
    z = {t: 0.0 for t in TERMS}
    z[name] = 1.0
    z.update(kw)
    return p.replace(**z)


def test_integration_adjoint_is_explicit_transpose():
    rng = np.random.default_rng(0)
    H, d = 9, 3
    dt = rng.uniform(0.01, 0.05, H)
    L = np.tril(np.ones((H, H))) @ np.diag(dt)  # S_l(1) diag(dt)
    gth, gthd, gu = rng.normal(size=(H, d)), rng.normal(size=(H, d)), rng.normal(size=(H, d))
    # theta_dot = L u + c, theta = L theta_dot + c' = L L u + c''
    ref = gu + L.T @ gthd + (L @ L).T @ gth
    assert np.allclose(oracle.integrate_adjoint(dt, gth, gthd, gu), ref, atol=1e-13)


def _fd_running(o, goal, h, th, thd, u, up, eps=1e-6):
    def f(a, b, c, e):
        return o.running_cost(goal, h, a, b, c, e)[1]
    out = []
    for which in range(4):
        args = [th, thd, u, up]
        g = np.zeros_like(args[which])
        for j in range(len(g)):
            ap = [a.copy() for a in args]
            am = [a.copy() for a in args]
            ap[which][j] += eps
            am[which][j] -= eps
            g[j] = (f(*ap) - f(*am)) / (2 * eps)
        out.append(g)
    return out


@pytest.mark.parametrize("term", TERMS)
@pytest.mark.parametrize("rot_mode", [W.ROT_QUAT, W.ROT_FROBENIUS])
def test_running_cost_gradient_per_term(term, rot_mode):
    if rot_mode == W.ROT_FROBENIUS and term != "w_rot":
        pytest.skip("rotation mode only changes the rotation term")
    wl = W.config_paper(5, N=1, H=12)
    extra = dict(k_m=10.0) if term == "w_manip" else {}
    p = _only(wl.params, term, rot_mode=rot_mode, rot_axis_w=(0.7, 1.3, 2.0),
              pos_axis_w=(1.0, 0.5, 2.0), **extra)
    o = oracle.Oracle(wl.robot, wl.world, p)
    rng = np.random.default_rng(1 + TERMS.index(term))
    hits = 0
    for trial in range(6):
        th = rng.uniform(-2.7, 2.7, 7)
        thd = rng.uniform(-1.5, 1.5, 7)
        u, up = rng.normal(size=7), rng.normal(size=7)
        h = int(rng.integers(0, p.H))
        terms, c = o.running_cost(wl.goal, h, th, thd, u, up)
        if c == 0.0:
            continue
        hits += 1
        g = o.running_cost_grad(wl.goal, h, th, thd, u, up)
        fd = _fd_running(o, wl.goal, h, th, thd, u, up)
        scale = max(1e-3, max(np.abs(x).max() for x in fd))
        for a, b in zip(g, fd):
            assert np.allclose(a, b, atol=2e-6 * scale + 1e-8), (term, trial, a, b)
    assert hits >= 2, f"term {term} never active"


def test_cost_gradient_matches_finite_differences():
    wl = W.config_paper(6, N=4, H=8)
    p = wl.params.replace(N=4, H=8, n_knots=0, n_null=1, w_smooth=0.5, k_m=0.3)
    o = oracle.Oracle(wl.robot, wl.world, p)
    state = W.make_state(6, 7)
    mu = W.make_mean(6, p.H, 7, 0.5)
    sig = W.make_sigma(6, 7)
    eps = o.noise(3, 0)
    J, grad = o.cost_grad(state, wl.goal, mu, sig, eps)
    # J is the mean total cost of the forward rollout
    out = o.rollout(state, wl.goal, mu, sig, eps)
    assert J == pytest.approx(out["C"].mean(), rel=1e-14)
    h = 1e-6
    fd = np.zeros_like(mu)
    for k in range(mu.size):
        mp, mm = mu.copy(), mu.copy()
        mp.flat[k] += h
        mm.flat[k] -= h
        fd.flat[k] = (o.cost_grad(state, wl.goal, mp, sig, eps)[0] -
                      o.cost_grad(state, wl.goal, mm, sig, eps)[0]) / (2 * h)
    scale = np.abs(fd).max()
    assert np.allclose(grad, fd, atol=1e-5 * scale), np.abs(grad - fd).max() / scale


def test_cost_gradient_null_particles_and_spline():
    wl = W.config_paper(7, N=3, H=10)
    p = wl.params.replace(N=3, H=10, n_knots=5, n_null=0)
    o = oracle.Oracle(wl.robot, wl.world, p)
    mu, sig = W.make_mean(7, 10, 7), W.make_sigma(7, 7)
    eps = o.noise(0, 1)
    J, grad, dcdu = o.cost_grad(wl.state, wl.goal, mu, sig, eps, per_particle=True)
    assert np.allclose(grad, dcdu.mean(0))
    p0 = p.replace(n_null=3)  # every particle null: u does not depend on mu
    o0 = oracle.Oracle(wl.robot, wl.world, p0)
    J0, g0 = o0.cost_grad(wl.state, wl.goal, mu, sig, eps)
    assert np.all(g0 == 0.0)
