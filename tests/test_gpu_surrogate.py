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

from gpu_helpers import TOL_COST, cuda, f32, host, manip_flips, max_rel

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


@pytest.mark.parametrize("count", [1, 128, 1000, 65_536 + 77, 262_144 + 7])
def test_fused_forward_equals_layer_kernels(count):
    """storm_mlp_predict (the whole network per tile, activations on chip) gives
    bitwise the predictions of the layer-by-layer kernels of the training pass,
    for ragged tile counts and a grid of several persistent waves; the largest
    count gives each CTA ~14 tiles, so the accumulators swap roles and the next
    tile's inputs are announced early many times over."""
    p = _random_params(11)
    th = cuda(np.random.default_rng(count).uniform(-2.8, 2.8, (count, 7)))
    net = SurrogateMLP(seed=3)
    net.set_params(p)
    a = host(net.predict(th))
    b = host(net.predict(th, layers=True))
    assert np.array_equal(a, b)
    net.close()


def test_wait_probe_times_out_and_the_network_stays_usable():
    """The tensor-core kernels' bounded wait, run out on purpose (an mbarrier that
    nothing completes, 2 ms limit): STORM_ERR_TIMEOUT, then the network still
    predicts bitwise as before and reports no error."""
    from paper_2104_13542_b300 import binding
    net = SurrogateMLP(seed=4)
    th = cuda(np.random.default_rng(3).uniform(-2.8, 2.8, (300, 7)))
    before = host(net.predict(th))
    assert net.wait_probe(2000) == binding.STORM_ERR_TIMEOUT
    after = host(net.predict(th))
    assert np.array_equal(before, after)
    assert net.wait_probe(2000) == binding.STORM_ERR_TIMEOUT  # and again
    net.close()


_TRAINED = {}


def _trained_distance_net():
    """A distance network trained on the exact check's labels (cached per run)."""
    if "distance" not in _TRAINED:
        wl = W.config_paper(0)
        with Controller(wl.robot, wl.world, wl.params.replace(N=8)) as lab:
            th, sd = _labelled(lab, 262_144, 41)
        net = SurrogateMLP(seed=12)
        net.train(th, torch.clamp(sd, max=0.5), batch=4096, epochs=6, lr=2e-3, seed=3)
        _TRAINED["distance"] = net
    return _TRAINED["distance"]


def _gate_states():
    """Start states (chosen on the oracle's exact distances): two whose rollouts
    stay clear of self contact (every item's distance about 6 cm), two that run
    from clear configurations into contact, one deep in contact."""
    out = [W.make_state(22, 7), W.make_state(25, 7)]
    for j3, v3 in ((1.4, 0.8), (2.1, 2.0), (2.2, 0.8)):
        st = W.make_state(21, 7)
        st[0, 3], st[1, 3] = j3, v3
        out.append(st)
    return out


def _gated_case(which, margin, record_property):
    """The rollout with the network inside the kernel (Sec. 4.2) gating the exact
    self check at 5 cm, against the oracle rollout gated by the same trained BF16
    network (orc_mlp_arch_forward with the same rounding points) on the paper
    workload at full size (the oracle takes the first 96 particles: a particle's
    noise does not depend on N).  An item whose two predictions fall on different
    sides of the margin is left out and counted -- it must lie within the BF16
    forward tolerance of the margin; everything else must match term by term, and
    the totals of particles without such items within the cost tolerance."""
    wl = W.config_paper(0)
    p = wl.params  # 500 x 30
    net = _trained_distance_net()
    params = net.get_params().astype(np.float64)
    step, it, seed = 2, 1, 3
    mu, sig = f32(W.make_mean(seed, p.H, 7, 0.5)), f32(W.make_sigma(seed, 7))
    state, goal = f32(_gate_states()[which]), f32(wl.goal)
    with Controller(wl.robot, wl.world, p) as ctl:
        ctl.set_distribution(mu, sig)
        ctl.set_surrogate(net, margin)
        g = {k: host(v) for k, v in ctl.generate_rollouts(cuda(state), cuda(goal), step, it).items()}
        # the predictions the kernel gated on: the same network on the kernel's own joint states
        pg = host(net.predict(cuda(g["theta"].reshape(-1, 7)))).reshape(p.N, p.H)
    # on the GPU side the gate is exactly the prediction against the margin
    assert np.all(g["terms"][..., 5][pg >= margin] == 0.0)
    n_or = 96
    orc = oracle.Oracle(wl.robot, wl.world, p.replace(N=n_or))
    orc.set_surrogate(oracle.ARCH_DISTANCE, params, margin)
    o = orc.rollout(state, goal, mu, sig, orc.noise(step, it))
    y_o = oracle.mlp_arch_forward(oracle.ARCH_DISTANCE, params, o["theta"].reshape(-1, 7)).reshape(n_or, p.H)
    gs = {k: v[:n_or] for k, v in g.items()}
    band = 5e-3 * max(1e-3, np.abs(y_o).max())  # the BF16 forward tolerance
    assert np.abs(pg[:n_or] - y_o).max() < band
    differ = (pg[:n_or] >= margin) != (y_o >= margin)
    assert np.all(np.abs(y_o[differ] - margin) < band)
    assert differ.mean() <= 0.01
    skipped = (y_o >= margin) & ~differ
    print(f"state {which}, margin {margin}: {skipped.mean():.3f} of items skip the exact check, "
          f"{differ.sum()} of {differ.size} decided differently within {band:.1e} m of the margin")
    record_property(f"gate_skip_fraction_state{which}_margin{margin}", float(skipped.mean()))
    flip, ok = manip_flips(orc, o["theta"], p.k_m, gs["terms"], o["terms"])
    assert ok and flip.mean() <= 1e-3
    keep = ~flip & ~differ
    for t in range(W.NTERMS):
        tscale = max(1.0, np.abs(o["terms"][..., t]).max())
        assert max_rel(gs["terms"][..., t][keep], o["terms"][..., t][keep], tscale) < TOL_COST, W.TERM_NAMES[t]
    cscale = max(1.0, np.abs(o["cost"]).max())
    assert max_rel(gs["cost"][keep], o["cost"][keep], cscale) < TOL_COST
    rows = keep.all(axis=1)
    assert rows.mean() > 0.5
    assert max_rel(gs["C"][rows], o["C"][rows], max(1.0, np.abs(o["C"]).max())) < TOL_COST
    return bool(skipped.any()), bool(((y_o < margin) & (o["terms"][..., 5] > 0)).any())


def test_gated_rollout_matches_oracle(record_property):
    """The gated rollout against the oracle from each start state, at the 5 cm
    margin and at 0 (the exact check only where the network predicts contact).
    This robot's self clearance never exceeds about 6 cm (some sphere pair is that
    close in every configuration), so the trained network rarely predicts 5 cm
    near these start states; the 0 margin makes the gate skip where it predicts
    clearance at all.  Across the runs the gate both skips exact checks and keeps
    exact checks that find contact.""" 
    seen = [_gated_case(which, margin, record_property)
            for which in range(len(_gate_states())) for margin in (0.05, 0.0)]
    assert any(a for a, _ in seen) and any(b for _, b in seen), seen


def test_gated_step_is_the_gated_rollout():
    """A control step with the gate set runs the same fused rollout: its update
    equals the update of storm_generate_rollouts' totals (bitwise), two steps in
    a row."""
    wl = W.config_paper(0)
    p = wl.params.replace(K=1)
    net = _trained_distance_net()
    state, goal = f32(_gate_states()[0]), f32(wl.goal)
    with Controller(wl.robot, wl.world, p) as a, Controller(wl.robot, wl.world, p) as b:
        a.set_surrogate(net, 0.05)
        b.set_surrogate(net, 0.05)
        for t in range(2):
            cmd, info, rc = a.step(state, goal)
            mu_b, sig_b = b.get_distribution()
            if t > 0:
                b.shift()
            g = b.generate_rollouts(cuda(state), cuda(goal), t, 0, debug=False)
            b.update_distribution(g["C"], g["u"], want_weights=False)
            mu_a, _ = a.get_distribution()
            mu_b, _ = b.get_distribution()
            assert np.array_equal(mu_a, mu_b), t
            assert np.array_equal(cmd, mu_a[0])


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
