"""jointNERF (Sec. 4.2: [sin theta, cos theta] encoding, layers [256, 128, 64],
ReLU) on the tcgen05 path: forward and loss gradient against the FP64 oracle
with the same BF16 rounding points, training on the paper's sign convention
(positive = penetration depth), and its use as the self-collision cost of
Eq. 13 (max(0, jointNERF(theta)), no exact check) in the control step."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13542_b300 import Controller, SurrogateMLP
from paper_2104_13542_b300 import workloads as W

from gpu_helpers import cuda, f32, host, max_rel

pytestmark = pytest.mark.gpu

NERF = oracle.ARCH_JOINTNERF
H1, H2, H3, I = 256, 128, 64, 16
BLOCKS = [("W1", 0, H1 * I), ("W2", H1 * I, H2 * H1), ("b2", H1 * I + H2 * H1, H2),
          ("W3", H1 * I + H2 * H1 + H2, H3 * H2), ("b3", H1 * I + H2 * H1 + H2 + H3 * H2, H3),
          ("w4", H1 * I + H2 * H1 + H2 + H3 * H2 + H3, H3), ("b4", H1 * I + H2 * H1 + H2 + H3 * H2 + 2 * H3, 1)]


def _random_params(seed, scale=0.1):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, oracle.mlp_arch_param_count(NERF)).astype(np.float32)


def test_shape():
    net = SurrogateMLP(seed=1, arch="jointnerf")
    assert net.n_params == oracle.mlp_arch_param_count(NERF) == 45313
    assert net.get_params().shape == (45313,)
    net.close()


@pytest.mark.parametrize("count", [128, 300, 1000])
def test_forward_matches_oracle(count):
    p = _random_params(1)
    th = f32(np.random.default_rng(count).uniform(-3.1, 3.1, (count, 7)))
    net = SurrogateMLP(seed=3, arch="jointnerf")
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    y = host(net.predict(cuda(th)))
    o = oracle.mlp_arch_forward(NERF, p.astype(np.float64), th, bf16=True)
    o64 = oracle.mlp_arch_forward(NERF, p.astype(np.float64), th, bf16=False)
    scale = max(1e-3, np.abs(o).max())
    assert max_rel(y, o, scale) < 5e-3, max_rel(y, o, scale)
    assert np.abs(y - o).mean() < np.abs(o64 - o).mean()
    net.close()


def test_loss_gradient_matches_oracle():
    p = _random_params(2)
    rng = np.random.default_rng(5)
    th = f32(rng.uniform(-3.1, 3.1, (384, 7)))
    t = f32(rng.uniform(-0.3, 0.1, 384))
    net = SurrogateMLP(seed=4, arch="jointnerf")
    net.set_params(p)
    loss, g = net.loss_grad(cuda(th), cuda(t))
    oloss, og = oracle.mlp_arch_loss_grad(NERF, p.astype(np.float64), th, t, bf16=True)
    assert loss == pytest.approx(oloss, rel=1e-2)
    for name, o0, n in BLOCKS:
        gs, os_ = g[o0:o0 + n], og[o0:o0 + n]
        scale = max(1e-8, np.abs(os_).max())
        assert max_rel(gs, os_, scale) < 3e-2, (name, max_rel(gs, os_, scale))
        assert gs @ os_ / (np.linalg.norm(gs) * np.linalg.norm(os_) + 1e-30) > 0.999, name
    net.close()


def _depth_labels(ctl, n, seed):
    th = cuda(np.random.default_rng(seed).uniform(-2.8, 2.8, (n, 7)))
    return th, torch.clamp(-ctl.self_distance(th), min=-0.5)  # paper's sign: positive = penetrating


def test_training_learns_the_depth():
    wl = W.config_paper(0)
    with Controller(wl.robot, wl.world, wl.params.replace(N=8)) as ctl:
        th, dep = _depth_labels(ctl, 262_144, 11)
        th_te, dep_te = _depth_labels(ctl, 32_768, 12)
    net = SurrogateMLP(seed=5, arch="jointnerf")
    y0 = host(net.predict(th_te))
    losses = net.train(th, dep, batch=4096, epochs=6, lr=2e-3, seed=1)
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.5 * losses[0], losses
    y, ref = host(net.predict(th_te)), host(dep_te)
    assert np.abs(y - ref).mean() < 0.5 * np.abs(y0 - ref).mean()
    net.close()


def _constant_net(c):
    net = SurrogateMLP(seed=7, arch="jointnerf")
    p = np.zeros(net.n_params, np.float32)
    p[-1] = c  # b4: the network outputs c everywhere
    net.set_params(p)
    return net


def test_learned_cost_replaces_the_exact_check():
    """Eq. 13 as the paper uses it.  A network that outputs a constant depth
    c > 0 adds w_coll c to every running cost (the MPPI weights, and so the
    update, are unchanged up to rounding); one that outputs c < 0 adds nothing;
    both skip the exact check, so on a robot without self contact the c < 0
    step is bitwise the exact step."""
    wl = W.config_paper(1)
    p = wl.params.replace(N=96)
    st, gl = f32(wl.state), f32(wl.goal)
    mu, sig = f32(W.make_mean(1, p.H, 7, 0.3)), f32(W.make_sigma(1, 7))

    def run(net):
        with Controller(wl.robot, wl.world, p) as c:
            if net is not None:
                c.set_surrogate_cost(net)
            c.set_distribution(mu, sig)
            cmd, info, rc = c.step(st, gl)
            m, _ = c.get_distribution()
            return cmd, info, m

    # the exact rollout of this state has no self contact (checked through the debug rollout)
    with Controller(wl.robot, wl.world, p) as c:
        c.set_distribution(mu, sig)
        g = c.generate_rollouts(cuda(st), cuda(gl), 0, 0)
        exact_self = host(g["terms"])[..., 5]
    ref_cmd, ref_info, ref_mu = run(None)
    neg = _constant_net(-0.2)
    cmd, info, m = run(neg)
    if not exact_self.any():
        assert np.array_equal(cmd, ref_cmd) and info["best_cost"] == ref_info["best_cost"]
    pos = _constant_net(0.01)
    cmd2, info2, m2 = run(pos)
    shift = p.w_coll * 0.01 * float(np.sum(p.gamma ** np.arange(p.H)))
    assert info2["best_cost"] - info["best_cost"] == pytest.approx(shift, rel=2e-3)
    assert max_rel(m2, m, max(1.0, np.abs(m).max())) < 1e-3
    neg.close()
    pos.close()


def test_learned_cost_rollout_matches_oracle():
    """Eq. 13 as the paper uses it, with a trained jointNERF inside the rollout
    kernel: every item's self term is max(0, jointNERF(theta)), against the
    oracle rollout whose self term is the same BF16 network
    (orc_mlp_arch_forward).  The self term may differ by the BF16 forward
    tolerance (5e-3 of the largest output), the running cost by w_coll times
    that; every other term within the cost tolerance.  On the GPU side the term
    is exactly max(0, prediction) of storm_mlp_predict on the kernel's own joint
    states."""
    wl = W.config_paper(0)
    p = wl.params
    with Controller(wl.robot, wl.world, p.replace(N=8)) as lab:
        th, dep = _depth_labels(lab, 262_144, 51)
    net = SurrogateMLP(seed=13, arch="jointnerf")
    net.train(th, dep, batch=4096, epochs=6, lr=2e-3, seed=4)
    params = net.get_params().astype(np.float64)
    step, it, seed = 2, 1, 3
    mu, sig = f32(W.make_mean(seed, p.H, 7, 0.5)), f32(W.make_sigma(seed, 7))
    state = W.make_state(21, 7)  # rollouts from here run from clear into self contact
    state[0, 3], state[1, 3] = 1.4, 0.8
    state, goal = f32(state), f32(wl.goal)
    with Controller(wl.robot, wl.world, p) as ctl:
        ctl.set_distribution(mu, sig)
        ctl.set_surrogate_cost(net)
        g = {k: host(v) for k, v in ctl.generate_rollouts(cuda(state), cuda(goal), step, it).items()}
        pg = host(net.predict(cuda(g["theta"].reshape(-1, 7)))).reshape(p.N, p.H)
    assert np.array_equal(g["terms"][..., 5], np.maximum(0.0, pg).astype(np.float32).astype(np.float64))
    n_or = 96
    orc = oracle.Oracle(wl.robot, wl.world, p.replace(N=n_or))
    orc.set_surrogate(NERF, params)
    o = orc.rollout(state, goal, mu, sig, orc.noise(step, it))
    y_o = oracle.mlp_arch_forward(NERF, params, o["theta"].reshape(-1, 7)).reshape(n_or, p.H)
    assert (y_o > 0).any() and (y_o <= 0).any()  # both sides of the hinge occur
    gs = {k: v[:n_or] for k, v in g.items()}
    band = 5e-3 * max(1e-3, np.abs(y_o).max())
    assert np.abs(gs["terms"][..., 5] - o["terms"][..., 5]).max() < band
    from gpu_helpers import TOL_COST, manip_flips
    flip, ok = manip_flips(orc, o["theta"], p.k_m, gs["terms"], o["terms"])
    assert ok and flip.mean() <= 1e-3
    keep = ~flip
    for t in range(W.NTERMS):
        if t == 5:
            continue
        tscale = max(1.0, np.abs(o["terms"][..., t]).max())
        assert max_rel(gs["terms"][..., t][keep], o["terms"][..., t][keep], tscale) < TOL_COST, W.TERM_NAMES[t]
    cscale = max(1.0, np.abs(o["cost"]).max())
    assert np.abs(gs["cost"][keep] - o["cost"][keep]).max() < TOL_COST * cscale + p.w_coll * band
    rows = ~flip.any(axis=1)
    disc = float(np.sum(p.gamma ** np.arange(p.H)))
    Cscale = max(1.0, np.abs(o["C"]).max())
    assert np.abs(gs["C"][rows] - o["C"][rows]).max() < TOL_COST * Cscale + p.w_coll * band * disc
    net.close()


def test_jointnerf_against_the_distance_network(record_property):
    """Same labels (sign flipped for jointNERF), same training budget: the
    accuracy of the paper's architecture next to the 256-256-256 network.
    Reported; the asserts are sanity bounds."""
    wl = W.config_paper(0)
    with Controller(wl.robot, wl.world, wl.params.replace(N=8)) as lab:
        th = cuda(np.random.default_rng(31).uniform(-2.8, 2.8, (262_144, 7)))
        th_te = cuda(np.random.default_rng(32).uniform(-2.8, 2.8, (65_536, 7)))
        sd, sd_te = lab.self_distance(th), lab.self_distance(th_te)
    ref = host(sd_te)
    near, coll = ref < 0.5, ref < 0.0
    out = {}
    for arch, target, sign in (("distance", torch.clamp(sd, max=0.5), 1.0),
                               ("jointnerf", torch.clamp(-sd, min=-0.5), -1.0)):
        net = SurrogateMLP(seed=9, arch=arch)
        net.train(th, target, batch=4096, epochs=8, lr=2e-3, seed=2)
        d = sign * host(net.predict(th_te))  # predicted distance
        out[arch] = (float(np.abs(d[near] - ref[near]).mean()),
                     float(np.mean(d[coll] >= 0.05)) if coll.any() else 0.0)
        net.close()
    print(f"MAE / false negatives at 5 cm: distance net {out['distance']}, jointNERF {out['jointnerf']}")
    record_property("distance_net_mae_m", out["distance"][0])
    record_property("jointnerf_mae_m", out["jointnerf"][0])
    assert out["jointnerf"][0] < 0.06 and out["distance"][0] < 0.06
