"""Learned self-collision surrogate on tcgen05 tensor cores.

Forward and loss gradient of the BF16 network against the FP64 oracle with the
same BF16 rounding points (the oracle's FP64 gradient is pinned by finite
differences in tests/test_oracle_mlp.py); the exact labeller against the
oracle's pair distance; training on labels from the exact check; the rollout
with the surrogate against the exact rollout; accuracy (MAE, false-negative
rate) judged by the exact check."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13542_b300 import Controller, SurrogateMLP
from paper_2104_13542_b300 import workloads as W

from gpu_helpers import cuda, f32, host, max_rel

pytestmark = pytest.mark.gpu


def _random_params(seed, scale=0.08):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, oracle.mlp_param_count()).astype(np.float32)


@pytest.mark.parametrize("count", [128, 300, 1000])
def test_forward_matches_oracle(count):
    p = _random_params(1)
    th = f32(np.random.default_rng(count).uniform(-2.8, 2.8, (count, 7)))
    net = SurrogateMLP(seed=3)
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    y = host(net.predict(cuda(th)))
    torch.cuda.synchronize()
    o = oracle.mlp_forward(p.astype(np.float64), th, bf16=True)
    o64 = oracle.mlp_forward(p.astype(np.float64), th, bf16=False)
    scale = max(1e-3, np.abs(o).max())
    assert max_rel(y, o, scale) < 5e-3, max_rel(y, o, scale)
    # and far closer to the BF16-emulating oracle than BF16 is to FP64
    assert np.abs(y - o).mean() < np.abs(o64 - o).mean()
    net.close()


def test_loss_gradient_matches_oracle():
    p = _random_params(2)
    rng = np.random.default_rng(5)
    th = f32(rng.uniform(-2.8, 2.8, (256, 7)))
    t = f32(rng.uniform(-0.1, 0.3, 256))
    net = SurrogateMLP(seed=4)
    net.set_params(p)
    loss, g = net.loss_grad(cuda(th), cuda(t))
    oloss, og = oracle.mlp_loss_grad(p.astype(np.float64), th, t, bf16=True)
    assert loss == pytest.approx(oloss, rel=1e-2)
    H, I = 256, 16
    blocks = [("W1", 0, H * I), ("W2", H * I, H * H), ("b2", H * I + H * H, H),
              ("W3", H * I + H * H + H, H * H), ("b3", H * I + 2 * H * H + H, H),
              ("w4", H * I + 2 * H * H + 2 * H, H), ("b4", H * I + 2 * H * H + 3 * H, 1)]
    for name, o0, n in blocks:
        gs, os_ = g[o0:o0 + n], og[o0:o0 + n]
        scale = max(1e-8, np.abs(os_).max())
        assert max_rel(gs, os_, scale) < 3e-2, (name, max_rel(gs, os_, scale))
        # direction: cosine similarity
        assert gs @ os_ / (np.linalg.norm(gs) * np.linalg.norm(os_) + 1e-30) > 0.999, name
    net.close()


def test_exact_labeller_matches_oracle():
    wl = W.config_paper(0)
    o = oracle.from_workload(wl)
    th = f32(np.random.default_rng(7).uniform(-2.8, 2.8, (500, 7)))
    with Controller(wl.robot, wl.world, wl.params.replace(N=8)) as ctl:
        sd = host(ctl.self_distance(cuda(th)))
    ref = np.array([o.self_min_sd_theta(t) for t in th])
    assert max_rel(sd, ref, 1.0) < 1e-5


def _labelled(ctl, n, seed):
    th = cuda(np.random.default_rng(seed).uniform(-2.8, 2.8, (n, 7)))
    sd = ctl.self_distance(th)
    return th, sd


def test_training_learns_the_distance():
    wl = W.config_paper(0)
    with Controller(wl.robot, wl.world, wl.params.replace(N=8)) as ctl:
        th, sd = _labelled(ctl, 262_144, 11)
        th_te, sd_te = _labelled(ctl, 32_768, 12)
    target = torch.clamp(sd, max=0.5)
    net = SurrogateMLP(seed=5)
    y0 = host(net.predict(th_te))
    losses = net.train(th, target, batch=4096, epochs=6, lr=2e-3, seed=1)
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.5 * losses[0], losses
    y = host(net.predict(th_te))
    ref = np.minimum(host(sd_te), 0.5)
    mae0, mae = np.abs(y0 - ref).mean(), np.abs(y - ref).mean()
    assert mae < 0.5 * mae0, (mae0, mae)
    net.close()


def test_surrogate_rollout_fallback_is_exact():
    wl = W.config_paper(1)
    p = wl.params.replace(N=96)
    net = SurrogateMLP(seed=6)
    state, goal = cuda(f32(wl.state)), cuda(f32(wl.goal))
    mu, sig = f32(W.make_mean(1, p.H, 7, 0.3)), f32(W.make_sigma(1, 7))
    with Controller(wl.robot, wl.world, p) as a:
        a.set_distribution(mu, sig)
        ref = [a.step(f32(wl.state), f32(wl.goal)) for _ in range(2)]
        mu_a, _ = a.get_distribution()
    with Controller(wl.robot, wl.world, p) as b:
        b.set_surrogate(net, margin=float("inf"))  # always fall back: bitwise exact
        b.set_distribution(mu, sig)
        got = [b.step(f32(wl.state), f32(wl.goal)) for _ in range(2)]
        mu_b, _ = b.get_distribution()
    for (c1, i1, _), (c2, i2, _) in zip(ref, got):
        assert np.array_equal(c1, c2) and i1["best_cost"] == i2["best_cost"]
    assert np.array_equal(mu_a, mu_b)
    net.close()


def test_surrogate_accuracy_and_gain(record_property):
    """What the trained network gains: the share of (particle, step) items whose
    exact self check it skips, the rollout time with and without it, and its
    error judged by the exact check (MAE, false negatives = predicted clear by
    the margin but in collision).  Reported; the asserts are sanity bounds."""
    wl = W.config_paper(0)
    p = wl.params.replace(N=1000, H=30)
    margin = 0.05
    with Controller(wl.robot, wl.world, p.replace(N=8)) as lab:
        th, sd = _labelled(lab, 262_144, 21)
        th_te, sd_te = _labelled(lab, 65_536, 22)
    net = SurrogateMLP(seed=9)
    net.train(th, torch.clamp(sd, max=0.5), batch=4096, epochs=8, lr=2e-3, seed=2)
    y, ref = host(net.predict(th_te)), host(sd_te)
    near = ref < 0.5
    mae = float(np.abs(y[near] - ref[near]).mean())
    collide = ref < 0.0
    fn = float(np.mean(y[collide] >= margin)) if collide.any() else 0.0
    skip = float(np.mean(y >= margin))
    state, goal = cuda(f32(wl.state)), cuda(f32(wl.goal))
    times = {}
    for mode in ("exact", "surrogate"):
        with Controller(wl.robot, wl.world, p) as c:
            if mode == "surrogate":
                c.set_surrogate(net, margin)
            c.step(f32(wl.state), f32(wl.goal))
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(20)]
            for a, b in ev:
                a.record(c.stream)
                c.step_resident()
                b.record(c.stream)
            torch.cuda.synchronize()
            times[mode] = float(np.median([a.elapsed_time(b) for a, b in ev]))
    print(f"surrogate: MAE {mae:.4f} m (|sd| < 0.5), false negatives {fn:.4f}, "
          f"exact checks skipped {skip:.3f}, step {times['surrogate']:.3f} ms vs exact "
          f"{times['exact']:.3f} ms")
    record_property("surrogate_mae_m", mae)
    record_property("surrogate_false_negative_rate", fn)
    record_property("surrogate_skip_fraction", skip)
    record_property("step_ms_surrogate", times["surrogate"])
    record_property("step_ms_exact", times["exact"])
    assert mae < 0.05 and fn < 0.2
    net.close()
