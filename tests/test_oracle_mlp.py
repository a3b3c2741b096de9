"""Pins of the oracle's surrogate network: a hand-computed tiny case, the BF16
rounding rule, and finite differences of the FP64 loss gradient."""
import math

import numpy as np
import pytest

import oracle

H, I = 256, 16
P = H * I + 2 * (H * H + H) + H + 1


def _split(p):
    o = 0
    parts = {}
    for name, n in [("W1", H * I), ("W2", H * H), ("b2", H), ("W3", H * H), ("b3", H), ("w4", H),
                    ("b4", 1)]:
        parts[name] = p[o:o + n]
        o += n
    return parts


def test_param_count():
    assert oracle.mlp_param_count() == P


def test_bf16_rounding_rule():
    assert oracle.bf16_round(1.0) == 1.0
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert oracle.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert oracle.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert oracle.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert oracle.bf16_round(-3.0) == -3.0
    assert math.isinf(oracle.bf16_round(float("inf")))


def test_tiny_network_by_hand():
    p = np.zeros(P)
    d = _split(p)
    d["W1"][0 * I + 0] = 2.0          # unit 0: 2 x0
    d["W1"][1 * I + 7] = -1.0         # unit 1: -1 (bias input) -> relu 0
    d["W2"][0 * H + 0] = 3.0          # layer 2 unit 0: 3 a1_0 + b2_0
    d["b2"][0] = 0.5
    d["W3"][5 * H + 0] = 1.0          # layer 3 unit 5: a2_0 - 0.25
    d["b3"][5] = -0.25
    d["w4"][5] = 2.0
    d["b4"][0] = 0.1
    th = np.array([[0.9, 0, 0, 0, 0, 0, 0], [-0.9, 0, 0, 0, 0, 0, 0]])
    y = oracle.mlp_forward(p, th, bf16=False)
    x0 = 0.9 / 3.0
    assert y[0] == pytest.approx(2.0 * (3.0 * (2.0 * x0) + 0.5 - 0.25) + 0.1)
    assert y[1] == pytest.approx(2.0 * (0.5 - 0.25) + 0.1)  # relu cuts unit 0


def test_loss_gradient_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.2, P)
    th = rng.uniform(-2.8, 2.8, (5, 7))
    t = rng.uniform(-0.1, 0.4, 5)
    loss, g = oracle.mlp_loss_grad(p, th, t, bf16=False)
    assert loss == pytest.approx(np.mean((oracle.mlp_forward(p, th, bf16=False) - t) ** 2))
    idx = np.concatenate([rng.choice(P, 60, replace=False), [P - 1, P - 2, H * I + 3]])
    h = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (oracle.mlp_loss_grad(pp, th, t, bf16=False)[0] -
              oracle.mlp_loss_grad(pm, th, t, bf16=False)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, abs=1e-6 * max(1.0, abs(fd)))


def test_bf16_mode_close_to_fp64():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.1, P)
    th = rng.uniform(-2.8, 2.8, (20, 7))
    y64 = oracle.mlp_forward(p, th, bf16=False)
    y16 = oracle.mlp_forward(p, th, bf16=True)
    assert np.max(np.abs(y64 - y16)) < 0.05 * max(1.0, np.max(np.abs(y64)))
    assert not np.array_equal(y64, y16)


# ----------------------------------------------------------------------------- jointNERF (Sec. 4.2)

NERF = oracle.ARCH_JOINTNERF
PN = 256 * 16 + 128 * 256 + 128 + 64 * 128 + 64 + 64 + 1


def _split_nerf(p):
    o, parts = 0, {}
    for name, n in [("W1", 256 * 16), ("W2", 128 * 256), ("b2", 128), ("W3", 64 * 128), ("b3", 64),
                    ("w4", 64), ("b4", 1)]:
        parts[name] = p[o:o + n]
        o += n
    return parts


def test_jointnerf_shape_and_encoding():
    assert oracle.mlp_arch_param_count(NERF) == PN == 45313
    assert oracle.mlp_arch_param_count(oracle.ARCH_DISTANCE) == P
    th = np.array([0.3, -1.2, 2.0, 0.0, -2.7, 1.1, 0.5])
    x = oracle.mlp_arch_encode(NERF, th)
    assert np.allclose(x[:7], np.sin(th)) and np.allclose(x[7:14], np.cos(th))
    assert x[14] == 1.0 and x[15] == 0.0


def test_jointnerf_routes_by_hand():
    """Single paths through the three layers, at asymmetric indices: y = relu(sin th_0)
    through units (5, 3, 2), plus 0.5 relu(cos th_1 - 0.2) through (9, 100, 40)."""
    p = np.zeros(PN)
    d = _split_nerf(p)
    d["W1"][5 * 16 + 0] = 1.0        # a1_5 = relu(sin th0)
    d["W2"][3 * 256 + 5] = 1.0       # a2_3 = a1_5
    d["W3"][2 * 128 + 3] = 1.0       # a3_2 = a2_3
    d["w4"][2] = 1.0
    d["W1"][9 * 16 + 8] = 1.0        # a1_9 = relu(cos th1 - 0.2)  (x_8 = cos th1, x_14 = 1)
    d["W1"][9 * 16 + 14] = -0.2
    d["W2"][100 * 256 + 9] = 2.0     # a2_100 = 2 a1_9
    d["W3"][40 * 128 + 100] = 0.25   # a3_40 = 0.5 a1_9
    d["w4"][40] = 1.0
    d["b4"][0] = -0.05
    rng = np.random.default_rng(3)
    th = rng.uniform(-3, 3, (20, 7))
    y = oracle.mlp_arch_forward(NERF, p, th, bf16=False)
    ref = np.maximum(0, np.sin(th[:, 0])) + 0.5 * np.maximum(0, np.cos(th[:, 1]) - 0.2) - 0.05
    assert np.allclose(y, ref, atol=1e-14)


def test_jointnerf_loss_gradient_finite_differences():
    rng = np.random.default_rng(1)
    p = rng.normal(0, 0.15, PN)
    th = rng.uniform(-2.8, 2.8, (4, 7))
    t = rng.uniform(-0.1, 0.4, 4)
    loss, g = oracle.mlp_arch_loss_grad(NERF, p, th, t, bf16=False)
    y = oracle.mlp_arch_forward(NERF, p, th, bf16=False)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-12)
    idx = np.concatenate([rng.choice(PN, 60, replace=False), [PN - 1, PN - 2, 4096 + 32768 + 5]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_arch_loss_grad(NERF, pp, th, t, bf16=False)[0] -
              oracle.mlp_arch_loss_grad(NERF, pm, th, t, bf16=False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, abs=1e-7 + 1e-5 * abs(fd)), i


def test_jointnerf_bf16_mode_close_to_fp64():
    rng = np.random.default_rng(2)
    p = rng.normal(0, 0.1, PN)
    th = rng.uniform(-2.8, 2.8, (50, 7))
    y64 = oracle.mlp_arch_forward(NERF, p, th, bf16=False)
    y16 = oracle.mlp_arch_forward(NERF, p, th, bf16=True)
    assert np.abs(y16 - y64).max() < 0.03 * max(1.0, np.abs(y64).max())
    assert not np.array_equal(y16, y64)


# ----------------------------------------------------------------------------- network in the rollout

def _collision_rollout(mode=None, params=None, margin=None):
    """Paper workload, a start whose rollouts self-collide, a few particles."""
    from paper_2104_13542_b300 import workloads as W
    wl = W.config_paper(0)
    p = wl.params.replace(N=12)
    orc = oracle.Oracle(wl.robot, wl.world, p)
    if params is not None:
        orc.set_surrogate(oracle.ARCH_DISTANCE, params, margin)
    state = W.make_state(21, 7)
    state[0, 3], state[1, 3] = 2.2, 0.8
    mu, sig = W.make_mean(3, p.H, 7, 0.5), W.make_sigma(3, 7)
    return p, orc.rollout(state, wl.goal, mu, sig, orc.noise(2, 1))


def _constant_net(c):
    p = np.zeros(P)
    p[-1] = c  # b4: the output is c whatever the input
    return p


def test_learned_cost_mode_is_max_of_zero_and_the_network():
    """Eq. 13 mode: every self term is max(0, net); the other terms and the
    running cost otherwise are the exact rollout's."""
    p, ex = _collision_rollout()
    assert (ex["terms"][..., 5] > 0).any()  # the exact check finds contact here
    for c in (0.03, -0.2):
        _, got = _collision_rollout(params=_constant_net(c))
        assert np.all(got["terms"][..., 5] == max(0.0, c))
        for t in range(oracle.NTERMS):
            if t != 5:
                assert np.array_equal(got["terms"][..., t], ex["terms"][..., t])
        shift = p.w_coll * (max(0.0, c) - ex["terms"][..., 5])
        assert np.allclose(got["cost"], ex["cost"] + shift, rtol=1e-12, atol=1e-9)


def test_gate_mode_constant_networks():
    """Gate mode: a network predicting 'clear' (at or above the margin) drops every
    self term; one predicting 'near' keeps the exact check everywhere."""
    p, ex = _collision_rollout()
    _, far = _collision_rollout(params=_constant_net(0.05), margin=0.05)
    assert np.all(far["terms"][..., 5] == 0.0)
    assert np.allclose(far["cost"], ex["cost"] - p.w_coll * ex["terms"][..., 5], rtol=1e-12, atol=1e-9)
    _, near = _collision_rollout(params=_constant_net(0.049), margin=0.05)
    assert np.array_equal(near["terms"], ex["terms"]) and np.array_equal(near["C"], ex["C"])


def test_gate_mode_decides_per_item():
    """A hand-routed network y = 3 relu(theta_3 / 3 - 0.8) = max(0, theta_3 - 2.4)
    (BF16 rounds the bias weight -0.8 to -0.80078125 and theta_3 / 3 by up to
    2^-9 relative, so the switch sits at theta_3 = 2.4523 +- 0.006 for the 5 cm
    margin): items clearly above it lose their self term, the others keep the
    exact one."""
    net = np.zeros(P)
    d = _split(net)
    d["W1"][0 * I + 3] = 1.0   # unit 0: x3 = theta_3 / 3 ...
    d["W1"][0 * I + 7] = -0.8  # ... minus 0.8 (x7 = 1 carries the bias)
    d["W2"][0 * H + 0] = 1.0
    d["W3"][0 * H + 0] = 1.0
    d["w4"][0] = 3.0
    margin = 0.05
    p, ex = _collision_rollout()
    _, got = _collision_rollout(params=net, margin=margin)
    th3 = ex["theta"][..., 3]
    switch = 3 * 0.80078125 + margin
    above, below = th3 > switch + 0.02, th3 < switch - 0.02
    assert above.sum() > 20 and below.sum() > 20
    assert (ex["terms"][..., 5][above] > 0).any()  # the gate really drops contact there
    assert np.all(got["terms"][..., 5][above] == 0.0)
    assert np.array_equal(got["terms"][..., 5][below], ex["terms"][..., 5][below])
