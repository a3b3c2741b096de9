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
