"""Parity of the CUDA control step with the FP64 oracle, through the C ABI.

Stage by stage (noise, rollouts, distribution update, shift, FK) and end to end
(one and several control steps), on the seeded workloads: the 64 x 20 plain
MPPI step and the 500 x 30 paper-scale step at full size, plus ragged and
degenerate variants.  Tolerances are stated in tests/gpu_helpers.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_13542_b300 import Controller, StormError
from paper_2104_13542_b300 import workloads as W

from gpu_helpers import (TOL_COST, TOL_STATE, TOL_UPDATE, cuda, f32, host, manip_flips,
                         max_rel, mu_tolerance)

pytestmark = pytest.mark.gpu


def _ctl(wl, p=None):
    return Controller(wl.robot, wl.world, p or wl.params)


def _variants():
    small, paper = W.config_small(0), W.config_paper(0)
    return {
        "small": (small, small.params),
        "paper": (paper, paper.params),
        "paper_ragged_N37": (paper, paper.params.replace(N=37)),
        "paper_halton": (paper, paper.params.replace(N=96, sampler=W.SAMPLER_HALTON)),
        "paper_halton_scrambled": (paper, paper.params.replace(N=96, sampler=W.SAMPLER_HALTON, halton_scramble=1)),
        "paper_null_frob": (paper, paper.params.replace(N=64, n_null=5,
                                                        rot_mode=W.ROT_FROBENIUS,
                                                        rot_axis_w=(0.5, 1.0, 2.0),
                                                        pos_axis_w=(1.0, 2.0, 0.5))),
        "small_H1": (small, small.params.replace(N=16, H=1)),
        "small_N1": (small, small.params.replace(N=1)),
        "paper_H50_knots10": (paper, paper.params.replace(N=40, H=50, n_knots=10)),
    }


VARIANTS = _variants()


# ----------------------------------------------------------------------------- noise

@pytest.mark.parametrize("name", ["small", "paper", "paper_ragged_N37", "paper_halton", "paper_halton_scrambled"])
def test_noise_matches_oracle(name):
    wl, p = VARIANTS[name]
    orc = oracle.Oracle(wl.robot, wl.world, p)
    with _ctl(wl, p) as ctl:
        for step, it in [(0, 0), (3, 2), (17, 1)]:
            g = host(ctl.sample_noise(step, it))
            o = orc.noise(step, it)
            assert g.shape == o.shape
            err = np.abs(g - o) / np.maximum(1.0, np.abs(o))
            assert err.max() < 2e-6, (step, it, err.max())


@pytest.mark.parametrize("name", ["small", "paper", "paper_ragged_N37"])
def test_philox_words_bit_exact(name):
    """The integer Philox4x32-10 stream behind the noise, GPU against the oracle's
    own implementation of the published generator (itself pinned by the Random123
    known-answer vectors), word for word, over every block of a step's noise and
    a far block range (counter words past 2^31)."""
    wl, p = VARIANTS[name]
    blocks = (p.N * (p.n_knots if p.n_knots > 0 else p.H) * 7 + 3) // 4
    key = [p.seed & 0xFFFFFFFF, p.seed >> 32]
    with _ctl(wl, p) as ctl:
        for step, it, first, count in [(0, 0, 0, blocks), (3, 2, 0, blocks), (17, 1, 0, blocks),
                                       (2**31 - 5, 255, 2**31 + 7, 1000)]:
            g = ctl.philox_words(step, it, first, count)
            o = np.array([oracle.philox([first + b, step, (p.instance << 8) | it, 0], key)
                          for b in range(count)], dtype=np.uint32)
            assert g.dtype == np.uint32 and g.shape == (count, 4)
            assert np.array_equal(g, o), (step, it, int(np.sum(g != o)))


# ----------------------------------------------------------------------------- rollouts

def _rollout_pair(wl, p, seed=0, step=2, it=1, state=None):
    orc = oracle.Oracle(wl.robot, wl.world, p)
    mu = f32(W.make_mean(seed, p.H, 7, 0.5))
    sig = f32(W.make_sigma(seed, 7))
    state = f32(W.make_state(seed + 10, 7) if state is None else state)
    goal = f32(wl.goal)
    with _ctl(wl, p) as ctl:
        ctl.set_distribution(mu, sig)
        g = ctl.generate_rollouts(cuda(state), cuda(goal), step, it)
        g = {k: host(v) for k, v in g.items()}
    o = orc.rollout(state, goal, mu, sig, orc.noise(step, it))
    return orc, g, o


@pytest.mark.parametrize("name", list(VARIANTS))
def test_rollout_stage_parity(name):
    wl, p = VARIANTS[name]
    orc, g, o = _rollout_pair(wl, p)
    assert max_rel(g["u"], o["u"], max(1.0, np.abs(o["u"]).max())) < TOL_STATE
    assert max_rel(g["theta"], o["theta"], max(1.0, np.abs(o["theta"]).max())) < TOL_STATE
    assert max_rel(g["theta_dot"], o["theta_dot"], max(1.0, np.abs(o["theta_dot"]).max())) < TOL_STATE
    assert max_rel(g["ee"], o["ee"], 1.0) < TOL_STATE
    flip, ok = manip_flips(orc, o["theta"], p.k_m, g["terms"], o["terms"])
    assert ok and flip.mean() <= 1e-3, f"manipulability branch flips: {flip.sum()}"
    keep = ~flip
    cscale = max(1.0, np.abs(o["cost"]).max())
    for t in range(W.NTERMS):
        tscale = max(1.0, np.abs(o["terms"][..., t]).max())
        e = max_rel(g["terms"][..., t][keep], o["terms"][..., t][keep], tscale)
        assert e < TOL_COST, (W.TERM_NAMES[t], e)
    assert max_rel(g["cost"][keep], o["cost"][keep], cscale) < TOL_COST
    rows = ~flip.any(axis=1)
    assert max_rel(g["C"][rows], o["C"][rows], max(1.0, np.abs(o["C"]).max())) < TOL_COST
    # discounted total is the gamma-weighted sum of the GPU's own running costs
    gam = p.gamma ** np.arange(p.H)
    assert max_rel(g["C"], g["cost"] @ gam, max(1.0, np.abs(g["C"]).max())) < 1e-5


def test_rollout_collision_terms_active():
    """The paper-scale workload exercises every cost term (none identically zero)."""
    wl, p = VARIANTS["paper"]
    state = W.make_state(21, 7)  # chosen on the oracle: every term active
    state[0, 3], state[1, 3] = 2.2, 0.8  # joint 4 heading through its soft limit (2.24)
    orc, g, o = _rollout_pair(wl, p, seed=3, state=state)
    for t, name in enumerate(W.TERM_NAMES[:8]):  # the paper's terms (the added ones: test_gpu_next)
        if name == "smooth":
            continue
        assert (o["terms"][..., t] > 0).any(), name
        assert (g["terms"][..., t] > 0).any(), name


# ----------------------------------------------------------------------------- update

def _update_pair(N, H, beta, C=None, seed=0, **kw):
    wl = W.config_small(0)
    p = wl.params.replace(N=N, H=H, beta=beta, **kw)
    orc = oracle.Oracle(wl.robot, wl.world, p)
    u = f32(W.make_controls(seed, N, H, 7, 0.7))
    Cv = f32(W.make_costs(seed, N, 0.0, 30.0) if C is None else C)
    mu0 = f32(W.make_mean(seed, H, 7))
    sig0 = f32(W.make_sigma(seed, 7))
    with _ctl(wl, p) as ctl:
        ctl.set_distribution(mu0, sig0)
        w = host(ctl.update_distribution(cuda(Cv), cuda(u)))
        mu, sig = ctl.get_distribution()
        info, st = ctl.sync()
    omu, osig, ost, ow = orc.update(Cv, u, mu0, sig0)
    return (mu, sig, w, st), (omu, osig, ow, ost), mu0, sig0, u


# (4096, 30): 512 particle rows per CTA of the update's cluster, more than one
# batch of loads in flight per thread; (37, 7): chunks of 5 rows of 49 floats
@pytest.mark.parametrize("N,H,beta,amu,asg", [(64, 20, 0.1, 1.0, 0.5), (500, 30, 10.0, 1.0, 0.5),
                                              (1000, 30, 1.0, 0.7, 0.3), (37, 7, 3.0, 0.5, 1.0),
                                              (1, 5, 1.0, 1.0, 0.5), (2048, 10, 2.0, 1.0, 0.5),
                                              (4096, 30, 1.0, 1.0, 0.5)])
def test_update_stage_parity(N, H, beta, amu, asg):
    (mu, sig, w, st), (omu, osig, ow, ost), *_ = _update_pair(N, H, beta, alpha_mu=amu,
                                                             alpha_sigma=asg)
    assert st == 0 and ost == 0
    assert max_rel(w, ow, 1.0) < TOL_UPDATE
    assert abs(w.sum() - 1.0) < 1e-5
    assert max_rel(mu, omu, max(1.0, np.abs(omu).max())) < TOL_UPDATE
    assert max_rel(sig, osig, max(osig.max(), 1e-3)) < TOL_UPDATE


def _update_explicit(C, u, mu0, sig0, beta, **kw):
    wl = W.config_small(0)
    N, H = u.shape[:2]
    p = wl.params.replace(N=N, H=H, beta=beta, **kw)
    orc = oracle.Oracle(wl.robot, wl.world, p)
    with _ctl(wl, p) as ctl:
        ctl.set_distribution(f32(mu0), f32(sig0))
        ctl.update_distribution(cuda(f32(C)), cuda(f32(u)))
        mu, sig = ctl.get_distribution()
    omu, osig, ost, ow = orc.update(f32(C), f32(u), f32(mu0), f32(sig0))
    return mu, sig, omu, osig


@pytest.mark.parametrize("case", ["zero_controls_win", "far_tight_cloud", "uniform_far"])
def test_update_far_from_old_mean(case):
    """Eq. 5 evaluated far from the mean the iteration started from: the weight on
    zero controls (null particles) while |mu_old| >> sigma, and tight clouds of
    samples several units from mu_old (sigma floor 0, so nothing masks an error
    in the deviation sum)."""
    rng = np.random.default_rng(7)
    N, H = 300, 12
    mu0 = np.full((H, 7), 3.0) + rng.normal(0, 0.1, (H, 7))
    sig0 = np.full(7, 0.05)
    if case == "zero_controls_win":
        u = mu0 + 0.05 * rng.normal(size=(N, H, 7))
        u[:10] = 0.0
        C = np.where(np.arange(N) < 10, 1.0, 40.0) + rng.uniform(0, 0.5, N)
        beta = 1.0
    elif case == "far_tight_cloud":
        u = mu0 + 5.0 + 1e-3 * rng.normal(size=(N, H, 7))
        C = rng.uniform(0, 5, N)
        beta = 2.0
    else:
        u = mu0 - 4.0 + 1e-2 * rng.normal(size=(N, H, 7))
        C = np.full(N, 3.0)
        beta = 10.0
    mu, sig, omu, osig = _update_explicit(C, u, mu0, sig0, beta, sigma_min=0.0, alpha_sigma=1.0)
    assert max_rel(mu, omu, max(1.0, np.abs(omu).max())) < TOL_UPDATE
    # sigma to the update tolerance, or to the FP32 resolution of the mean it is
    # measured about (a few ulps of max|mu|), whichever is larger; the deviation
    # sum formed in one pass about mu_old misses this by ~1e-3 in the first case
    bound = max(TOL_UPDATE * osig.max(), 4 * np.finfo(np.float32).eps * np.abs(mu0).max())
    assert np.abs(sig - osig).max() <= bound, (sig, osig, bound)


def test_degenerate_step_keeps_the_shifted_mean():
    """Alg. 1's shift is folded into the first iteration of a step; an iteration with
    no finite total (a NaN sigma, no null particles) still leaves the shifted mean
    (rows h + 1, the last row zero) and commands its first row."""
    wl = W.config_paper(0)
    p = wl.params.replace(N=64, n_null=0, K=1)
    st, gl = f32(wl.state), f32(wl.goal)
    with _ctl(wl, p) as ctl:
        ctl.step(st, gl)
        mu1, _ = ctl.get_distribution()
        ctl.set_distribution(mu1, np.full(7, np.nan, np.float32))
        cmd, info, rc = ctl.step(st, gl)
        mu2, _ = ctl.get_distribution()
    assert rc == 1 and info["status"] == 1
    shifted = np.vstack([mu1[1:], np.zeros((1, 7), np.float32)])
    assert np.array_equal(mu2, shifted)
    assert np.array_equal(cmd, shifted[0])


def test_update_zero_temperature_and_ties():
    C = np.full(50, 9.0)
    C[[7, 30]] = 2.0  # tie: lowest index wins
    (mu, sig, w, st), (omu, osig, ow, ost), mu0, sig0, u = _update_pair(50, 6, 0.0, C=C)
    assert np.array_equal(w, np.eye(50)[7])
    assert np.allclose(mu, u[7], atol=1e-7)
    assert max_rel(sig, osig, 1.0) < TOL_UPDATE


def test_update_nonfinite_costs():
    C = W.make_costs(1, 40, 0.0, 5.0)
    C[[3, 11]] = np.inf
    C[20] = np.nan
    (mu, sig, w, st), (omu, osig, ow, ost), *_ = _update_pair(40, 6, 1.0, C=C)
    assert w[3] == 0 and w[11] == 0 and w[20] == 0
    assert max_rel(mu, omu, max(1.0, np.abs(omu).max())) < TOL_UPDATE


def test_update_degenerate_keeps_distribution():
    C = np.full(16, np.inf)
    (mu, sig, w, st), (omu, osig, ow, ost), mu0, sig0, _ = _update_pair(16, 5, 1.0, C=C)
    assert st == 1 and ost == 1
    assert np.array_equal(mu, mu0.astype(np.float32)) and np.array_equal(sig, sig0.astype(np.float32))


# ----------------------------------------------------------------------------- control step

def _step_pair(wl, p, n_steps=1, state_seed=0):
    orc = oracle.Oracle(wl.robot, wl.world, p)
    state = f32(W.make_state(state_seed + 20, 7))
    goal = f32(wl.goal)
    omu, osig = np.zeros((p.H, 7)), np.full(7, f32(p.sigma_init))
    res = []
    with _ctl(wl, p) as ctl:
        for t in range(n_steps):
            cmd, info, rc = ctl.step(state, goal)
            mu, sig = ctl.get_distribution()
            ocmd, omu, osig, ost, obest = orc.step(state, goal, t, omu, osig)
            res.append((cmd, info, rc, mu, sig, ocmd, omu.copy(), osig.copy(), ost, obest))
    return res


@pytest.mark.parametrize("name", ["small", "paper", "paper_ragged_N37", "paper_halton", "paper_halton_scrambled",
                                  "paper_null_frob", "small_N1"])
def test_step_parity(name):
    wl, p = VARIANTS[name]
    (cmd, info, rc, mu, sig, ocmd, omu, osig, ost, obest), = _step_pair(wl, p)
    assert rc == ost == 0
    assert info["step"] == 0
    tol = mu_tolerance([obest, info["mean_weighted_cost"]], p.beta)
    scale = max(1.0, np.abs(omu).max())
    assert max_rel(mu, omu, scale) < tol
    assert max_rel(cmd, ocmd, scale) < tol
    assert np.array_equal(cmd, mu[0])
    assert max_rel(sig, osig, max(1e-3, osig.max())) < tol
    assert abs(info["best_cost"] - obest) <= TOL_COST * max(1.0, abs(obest))


def test_multi_step_parity_with_shift():
    """Four steps, the GPU and the oracle each carrying its own distribution
    forward (no oracle input comes from the GPU).  The bound after step t is
    (t + 1) times the one-step bound: a mean update with alpha_mu = 1 is
    mu_t = sum_n w_n (shift(mu_{t-1}) + sigma eps_n) with sum_n w_n = 1, so a
    difference in mu_{t-1} reappears in mu_t with gain one, plus the step's own
    error; the weights' response to that difference is of the same size as the
    FP32 cost error the one-step bound already covers."""
    wl, p = VARIANTS["small"]
    res = _step_pair(wl, p, n_steps=4)
    for t, (cmd, info, rc, mu, sig, ocmd, omu, osig, ost, obest) in enumerate(res):
        assert info["step"] == t
        tol = mu_tolerance([obest], p.beta) * (t + 1)
        scale = max(1.0, np.abs(omu).max())
        assert max_rel(mu, omu, scale) < tol, t
        assert max_rel(sig, osig, max(1e-3, osig.max())) < tol, t


def test_shift_stage():
    wl, p = VARIANTS["small"]
    mu0 = W.make_mean(4, p.H, 7).astype(np.float32)
    with _ctl(wl, p) as ctl:
        ctl.set_distribution(mu0, np.full(7, 0.2))
        ctl.shift()
        mu, sig = ctl.get_distribution()
    assert np.array_equal(mu[:-1], mu0[1:]) and np.all(mu[-1] == 0)
    assert np.allclose(sig, 0.2)


# ----------------------------------------------------------------------------- other entry points

def test_forward_kinematics_matches_oracle():
    wl = W.config_paper(2)
    orc = oracle.from_workload(wl)
    th = f32(np.random.default_rng(0).uniform(-2.8, 2.8, (1000, 7)))
    with _ctl(wl) as ctl:
        ee = host(ctl.forward_kinematics(cuda(th)))
    o = np.stack([orc.fk(t)[-1][:3] for t in th])
    assert max_rel(ee, o, 1.0) < TOL_STATE


def test_joint_sin_cos_accuracy():
    """The chain's sin / cos of a joint angle, read out through a one-joint
    chain with a = alpha = d = 0 (its frame is Rz(theta): R[0,0] = cos theta,
    R[1,0] = sin theta), against the FP64 values of the same float32 angles:
    within 1.5e-7 absolute over |theta| <= 40 (multiples of pi/2 and their
    neighbours included) and up to 1e4, odd symmetry exact, NaN for NaN / inf."""
    robot = W.Robot(dh=np.zeros((1, 4)), q_min=np.array([-3.0]), q_max=np.array([3.0]),
                    sphere_link=np.array([1], np.int32), spheres=np.array([[0.0, 0.0, 0.0, 0.05]]),
                    pairs=np.zeros((0, 2), np.int32))
    world = W.World(boxes=np.zeros((0, 6)), spheres=np.zeros((0, 4)))
    quarter = np.arange(-25, 26) * (np.pi / 2)
    th = np.concatenate([np.linspace(-40.0, 40.0, 400_001), quarter, np.nextafter(quarter, 0),
                         np.nextafter(quarter, 100), np.linspace(-1e4, 1e4, 20_001),
                         [0.0, 1e-30, -1e-30, 1e-8, np.pi / 4, -np.pi / 4]]).astype(np.float32)
    with Controller(robot, world, W.Params(N=4, H=4, n_knots=0, dt=np.full(4, 0.02))) as ctl:
        R = host(ctl.forward_kinematics(cuda(th[:, None])))
        c, s = R[:, 0, 0].astype(np.float64), R[:, 1, 0].astype(np.float64)
        x = th.astype(np.float64)
        assert np.abs(s - np.sin(x)).max() < 1.5e-7
        assert np.abs(c - np.cos(x)).max() < 1.5e-7
        Rm = host(ctl.forward_kinematics(cuda(-th[:, None])))
        assert np.array_equal(Rm[:, 1, 0], -R[:, 1, 0]) and np.array_equal(Rm[:, 0, 0], R[:, 0, 0])
        small = np.abs(x) < 1e-4  # sin x = x to within an ulp near zero
        assert np.all(np.abs(s[small] - x[small]) <= np.spacing(np.abs(th[small])).astype(np.float64))
        bad = host(ctl.forward_kinematics(cuda(np.array([[np.nan], [np.inf], [-np.inf]], np.float32))))
        assert np.isnan(bad[:, 0, 0]).all() and np.isnan(bad[:, 1, 0]).all()


def test_checkpoint_resume_is_bitwise():
    wl, p = VARIANTS["small"]
    state, goal = f32(wl.state), f32(wl.goal)
    with _ctl(wl, p) as a:
        a.step(state, goal)
        blob = a.get_state()
        ref = [a.step(state, goal)[0] for _ in range(3)]
        mu_a, sig_a = a.get_distribution()
    with _ctl(wl, p) as b:
        b.set_state(blob)
        got = [b.step(state, goal)[0] for _ in range(3)]
        mu_b, sig_b = b.get_distribution()
        with pytest.raises(StormError):
            b.set_state(blob[:-4])
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    assert np.array_equal(mu_a, mu_b) and np.array_equal(sig_a, sig_b)


def test_rewound_handle_reruns_bitwise():
    """A handle rewound to a checkpoint of its own (set_state after further
    steps) reruns those steps bit for bit: nothing of the later steps (the
    step counter, the mean, sigma) leaks into the rerun."""
    wl, p = VARIANTS["paper"]
    state, goal = f32(wl.state), f32(wl.goal)
    with _ctl(wl, p) as a:
        a.step(state, goal)
        blob = a.get_state()
        ref = [a.step(state, goal)[0] for _ in range(3)]
        mu_a, sig_a = a.get_distribution()
        a.set_state(blob)
        got = [a.step(state, goal)[0] for _ in range(3)]
        mu_b, sig_b = a.get_distribution()
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)
    assert np.array_equal(mu_a, mu_b) and np.array_equal(sig_a, sig_b)


def test_determinism_across_handles():
    wl, p = VARIANTS["paper"]
    state, goal = f32(wl.state), f32(wl.goal)
    outs = []
    for _ in range(2):
        with _ctl(wl, p) as c:
            cmds = [c.step(state, goal)[0] for _ in range(2)]
            outs.append((cmds, c.get_distribution()))
    assert all(np.array_equal(x, y) for x, y in zip(outs[0][0], outs[1][0]))
    assert np.array_equal(outs[0][1][0], outs[1][1][0])


def test_set_world_then_rollout_parity():
    wl = W.config_paper(1)
    p = wl.params.replace(N=48)
    new_world = W.make_world(7, n_boxes=5, n_spheres=3)
    orc = oracle.Oracle(wl.robot, new_world, p)
    mu, sig = f32(W.make_mean(1, p.H, 7)), f32(W.make_sigma(1, 7))
    state, goal = f32(wl.state), f32(wl.goal)
    with _ctl(wl, p) as ctl:
        ctl.set_world(new_world)
        ctl.set_distribution(mu, sig)
        g = {k: host(v) for k, v in ctl.generate_rollouts(cuda(state), cuda(goal), 0, 0).items()}
    o = orc.rollout(state, goal, mu, sig, orc.noise(0, 0))
    for t in (5, 6):
        assert max_rel(g["terms"][..., t], o["terms"][..., t], 1.0) < TOL_COST


def test_nonfinite_inputs_rejected():
    wl, p = VARIANTS["small"]
    with _ctl(wl, p) as ctl:
        bad = f32(wl.state).copy()
        bad[1, 2] = np.nan
        with pytest.raises(StormError) as e:
            ctl.step(bad, wl.goal)
        assert e.value.code == -4
        g = f32(wl.goal).copy()
        g[5] = np.inf
        with pytest.raises(StormError):
            ctl.step(wl.state, g)
        cmd, info, rc = ctl.step(wl.state, wl.goal)  # handle still usable
        assert rc == 0 and info["step"] == 0


def test_step_async_device_buffers_match_host_step():
    wl, p = VARIANTS["paper"]
    state, goal = f32(wl.state), f32(wl.goal)
    with _ctl(wl, p) as a:
        ref = [a.step(state, goal)[0] for _ in range(2)]
    with _ctl(wl, p) as b:
        s, g, c = cuda(state), cuda(goal), torch.zeros(7, device="cuda")
        got = []
        for _ in range(2):
            b.step_async(s, g, c)
            b.sync()
            got.append(c.cpu().numpy().copy())
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("grad_steps", [0, 2])
def test_host_step_outputs_match_the_device_step(grad_steps):
    """storm_step's outputs (the command and the step record, written into pinned
    memory by the step's last update and awaited there; with gradient refinement,
    copied out after the stream) equal the device-resident step's, bit for bit,
    over a closed loop that includes a degenerate step (NaN sigma, no null
    particles: every total non-finite)."""
    wl = W.config_paper(1)
    p = wl.params.replace(N=96, n_null=0, grad_steps=grad_steps, grad_eta=0.01)
    goal = f32(wl.goal)
    runs = []
    for host in (True, False):
        with _ctl(wl, p) as ctl:
            state = f32(wl.state)
            s, g, c = cuda(state.reshape(-1)), cuda(goal), torch.zeros(7, device="cuda")
            out = []
            for k in range(5):
                if k == 3:  # a degenerate step; the next one starts from a sane sigma again
                    mu, sig = ctl.get_distribution()
                    ctl.set_distribution(mu, np.full(7, np.nan, np.float32))
                if k == 4:
                    mu, sig = ctl.get_distribution()
                    ctl.set_distribution(mu, np.full(7, 0.3, np.float32))
                if host:
                    cmd, info, rc = ctl.step(state, goal)
                else:
                    s.copy_(torch.as_tensor(state.reshape(-1)))
                    ctl.step_async(s, g, c)
                    info, rc = ctl.sync()
                    cmd = c.cpu().numpy().copy()
                out.append((cmd, info["best_cost"], info["mean_weighted_cost"], info["status"], info["step"], rc))
                state = state.copy()
                state[2] = np.nan_to_num(cmd)
                state[1] += 0.02 * state[2]
                state[0] += 0.02 * state[1]
            runs.append(out)
    for k, (a, b) in enumerate(zip(*runs)):
        assert np.array_equal(a[0], b[0], equal_nan=True), k
        assert np.array_equal(np.asarray(a[1:3]), np.asarray(b[1:3]), equal_nan=True), (k, a[1:3], b[1:3])
        assert a[3:] == b[3:], (k, a[3:], b[3:])
    assert [r[4] for r in runs[0]] == [0, 1, 2, 3, 4]
    assert runs[0][3][3] == 1 and runs[0][3][5] == 1  # STORM_WARN_DEGENERATE
    if grad_steps == 0:  # the distribution was kept: the next step is sane again
        assert all(r[3] == 0 for k, r in enumerate(runs[0]) if k != 3)
    # (with refinement the gradient of the sample-average cost, J(mu) over
    # mu + sigma o eps, carries the NaN sigma into the mean: garbage in, and
    # both paths report it the same way)


# ----------------------------------------------------------------------------- launch shapes

def test_launch_shapes_are_bitwise_identical_and_autotune():
    wl = W.config_paper(4)
    p = wl.params.replace(N=130)
    state, goal = cuda(f32(wl.state)), cuda(f32(wl.goal))
    mu, sig = f32(W.make_mean(4, p.H, 7, 0.5)), f32(W.make_sigma(4, 7))
    ref = None
    with _ctl(wl, p) as ctl:
        ctl.set_distribution(mu, sig)
        for ppc, threads in [(2, 256), (1, 64), (5, 512), (3, 128), (4, 256)]:
            ctl.set_launch(ppc, threads)
            assert ctl.get_launch() == (ppc, threads)
            g = {k: host(v) for k, v in ctl.generate_rollouts(state, goal, 1, 0).items()}
            if ref is None:
                ref = g
            for k in ref:
                assert np.array_equal(g[k], ref[k]), (ppc, threads, k)
        with pytest.raises(StormError):
            ctl.set_launch(0, 256)
        with pytest.raises(StormError):
            ctl.set_launch(2, 100)
        ctl.step(f32(wl.state), f32(wl.goal))
        t = ctl.autotune()
        assert 0 < t < 1e4
        ctl.set_distribution(mu, sig)  # the step above moved the distribution
        g = {k: host(v) for k, v in ctl.generate_rollouts(state, goal, 1, 0).items()}
        for k in ref:
            assert np.array_equal(g[k], ref[k]), k


def _mapping_cases():
    paper = W.config_paper(0)
    dense = W.config_paper(3)
    dense.world = W.make_world(43, n_boxes=64, n_spheres=64)
    return {
        # every cost term active (state chosen on the oracle, see the collision test)
        "paper_terms": (paper, paper.params.replace(N=61), 21),
        "dense_world": (dense, dense.params.replace(N=40, w_smooth=0.3), 63),
        "H5_N37_white": (paper, paper.params.replace(N=37, H=5, n_knots=0, n_null=3), 1),
        "H12_N37_halton": (paper, paper.params.replace(N=37, H=12, sampler=W.SAMPLER_HALTON), 2),
        "H16_N9_frob": (paper, paper.params.replace(N=9, H=16, rot_mode=W.ROT_FROBENIUS,
                                                    rot_axis_w=(0.5, 1.0, 2.0)), 4),
        "H50_N23": (paper, paper.params.replace(N=23, H=50, n_knots=10), 5),
        "H64_N3": (paper, paper.params.replace(N=3, H=64, n_knots=0), 6),
        # the arm folded onto itself: many overlapping frame pairs per item, so
        # the pair mapping's two warps share the self-collision tests
        "folded_arm": (paper, paper.params.replace(N=48), 77),
    }


def _folded_state(wl, seed=77, draws=200):
    """The configuration, of `draws` uniform ones, closest to (or deepest in)
    self-collision (chosen on the oracle), at rest."""
    orc = oracle.Oracle(wl.robot, wl.world, wl.params)
    rng = np.random.default_rng([seed, 5])
    th = rng.uniform(-2.6, 2.6, (draws, 7))
    sd = np.array([orc.self_min_sd_theta(t) for t in th])
    state = np.zeros((3, 7))
    state[0] = th[int(np.argmin(sd))]
    return state


@pytest.mark.parametrize("name", list(_mapping_cases()))
def test_warp_mapping_is_bitwise_identical_to_cta_mapping(name):
    """Both work mappings, every warp count and both collision modes give the
    same bits in every output (controls, joint states, EE poses, cost terms,
    running and total costs)."""
    wl, p, sseed = _mapping_cases()[name]
    state = W.make_state(sseed, 7) if sseed != 77 else _folded_state(wl)
    if sseed == 21:
        state[0, 3], state[1, 3] = 2.2, 0.8
    state, goal = cuda(f32(state)), cuda(f32(wl.goal))
    mu, sig = f32(W.make_mean(sseed, p.H, 7, 0.8)), f32(W.make_sigma(sseed, 7, 0.2, 0.6))
    with _ctl(wl, p) as ctl:
        assert ctl.launch_mapping() == "pair" and ctl.get_launch()[1] == 64
        ctl.set_distribution(mu, sig)
        ctl.set_launch(2, 256)
        assert ctl.launch_mapping() == "cta"
        ref = {k: host(v) for k, v in ctl.generate_rollouts(state, goal, 3, 1).items()}
        for bp in (True, False):
            ctl.set_broadphase(bp)
            for mapping, count in (("warp", 1), ("warp", 3), ("warp", 8), ("pair", 1), ("pair", 3),
                                   ("quad", 1), ("quad", 2)):
                {"warp": ctl.set_launch_warp, "pair": ctl.set_launch_warp_pair,
                 "quad": ctl.set_launch_warp_quad}[mapping](count)
                assert ctl.launch_mapping() == mapping
                ppc, threads = ctl.get_launch()
                assert threads == {"warp": 32, "pair": 64, "quad": 128}[mapping] * count
                g = {k: host(v) for k, v in ctl.generate_rollouts(state, goal, 3, 1).items()}
                for k in ref:
                    assert np.array_equal(g[k], ref[k]), (bp, mapping, count, k)
        with pytest.raises(StormError):
            ctl.set_launch_warp(0)
        with pytest.raises(StormError):
            ctl.set_launch_warp(9)
        with pytest.raises(StormError):
            ctl.set_launch_warp_pair(5)
        with pytest.raises(StormError):
            ctl.set_launch_warp_quad(3)
    active = {nm for t, nm in enumerate(W.TERM_NAMES) if (ref["terms"][..., t] > 0).any()}
    assert {"pos", "rot", "manip"} <= active
    if name == "paper_terms":  # both collision phases exercised (checked on the oracle)
        assert {"self", "world"} <= active, active
    if name == "dense_world":
        assert "world" in active, active
    if name == "folded_arm":
        assert "self" in active, active


@pytest.mark.parametrize("mapping", ["cta", "warp", "pair"])
def test_dependent_launch_is_bitwise_identical(mapping):
    """The step graph with its rollouts and updates launched as programmatic
    dependents and launched ordinarily (the default): the same commands, means,
    sigmas and step records, bit for bit, over several closed-loop steps of
    K = 3 iterations."""
    wl = W.config_paper(2)
    p = wl.params.replace(N=300)
    goal = f32(wl.goal)
    runs = []
    for dep in (True, False):
        with _ctl(wl, p) as ctl:
            assert not ctl.dependent_launch()
            {"cta": lambda: ctl.set_launch(4, 256), "warp": lambda: ctl.set_launch_warp(4),
             "pair": lambda: ctl.set_launch_warp_pair(2)}[mapping]()
            ctl.set_dependent_launch(dep)
            assert ctl.dependent_launch() == dep
            state = f32(wl.state)
            out = []
            for _ in range(6):
                cmd, info, rc = ctl.step(state, goal)
                mu, sig = ctl.get_distribution()
                out.append((cmd, mu, sig, info["best_cost"], info["mean_weighted_cost"], rc))
                state[2] = cmd
                state[1] += 0.02 * cmd
                state[0] += 0.02 * state[1]
            runs.append(out)
    for a, b in zip(*runs):
        for x, y in zip(a, b):
            assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("seed,world", [(0, None), (3, (64, 64)), (5, (8, 0))])
def test_broadphase_is_bitwise_identical(seed, world):
    wl = W.config_paper(seed)
    if world is not None:
        wl.world = W.make_world(seed + 40, n_boxes=world[0], n_spheres=world[1])
    p = wl.params.replace(N=200)
    state, goal = cuda(f32(W.make_state(seed + 60, 7))), cuda(f32(wl.goal))
    mu, sig = f32(W.make_mean(seed, p.H, 7, 0.8)), f32(W.make_sigma(seed, 7, 0.2, 0.6))
    outs = []
    with _ctl(wl, p) as ctl:
        ctl.set_distribution(mu, sig)
        for on in (True, False):
            ctl.set_broadphase(on)
            outs.append({k: host(v) for k, v in ctl.generate_rollouts(state, goal, 4, 1).items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    assert (outs[0]["terms"][..., 5] > 0).any() or (outs[0]["terms"][..., 6] > 0).any()


@pytest.mark.parametrize("per_link", [1, 2])
def test_broadphase_with_point_and_short_capsules_is_bitwise_identical(per_link):
    """Links with one sphere (the capsule's segment a point) and two spheres:
    the capsule cull passes every pair that touches, so every output equals the
    brute-force tests bit for bit, at a folded configuration (self collision)
    among a dense world; the self and world terms are non-zero somewhere."""
    wl = W.config_paper(6)
    wl.robot = W.make_robot(6, 7, spheres_per_link=per_link)
    wl.world = W.make_world(46, n_boxes=64, n_spheres=64)
    p = wl.params.replace(N=200)
    state, goal = cuda(f32(_folded_state(wl))), cuda(f32(wl.goal))
    mu, sig = f32(W.make_mean(6, p.H, 7, 0.8)), f32(W.make_sigma(6, 7, 0.2, 0.6))
    outs = []
    with _ctl(wl, p) as ctl:
        ctl.set_distribution(mu, sig)
        for on in (True, False):
            ctl.set_broadphase(on)
            outs.append({k: host(v) for k, v in ctl.generate_rollouts(state, goal, 2, 1).items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    assert (outs[0]["terms"][..., 5] > 0).any() and (outs[0]["terms"][..., 6] > 0).any()


@pytest.mark.parametrize("dof", [1, 2, 3, 4])
def test_short_chains(dof):
    """Chains of one to four joints (one to five frames; self-collision pairs
    only from three joints on), in a world of boxes and spheres: every rollout
    mapping gives the same bits, with the broad phase on and off, and the
    control step matches the oracle.  The manipulability weight is 0: with
    fewer than six joints J J^T is singular and m is 0 up to rounding."""
    s = 30 + dof
    robot = W.make_robot(s, dof)
    world = W.make_world(s, n_boxes=12, n_spheres=6)
    p = W.config_paper(0).params.replace(N=48, H=12, n_knots=4, dt=np.full(12, 0.02), w_manip=0.0)
    wl = W.Workload(f"chain{dof}", robot, world, p, W.make_state(s, dof), W.make_goal(s))
    state, goal = f32(wl.state), f32(wl.goal)
    mu0, sig0 = f32(W.make_mean(s, p.H, dof, 0.8)), f32(W.make_sigma(s, dof, 0.2, 0.6))
    with _ctl(wl, p) as ctl:
        ctl.set_distribution(mu0, sig0)
        ref = None
        for bp in (True, False):
            ctl.set_broadphase(bp)
            for mapping, count in (("cta", 0), ("warp", 1), ("pair", 1), ("quad", 1)):
                if mapping == "cta":
                    ctl.set_launch(2, 128)
                else:
                    {"warp": ctl.set_launch_warp, "pair": ctl.set_launch_warp_pair,
                     "quad": ctl.set_launch_warp_quad}[mapping](count)
                g = {k: host(v) for k, v in ctl.generate_rollouts(cuda(state), cuda(goal), 1, 0).items()}
                if ref is None:
                    ref = g
                for k in ref:
                    assert np.array_equal(g[k], ref[k]), (bp, mapping, k)
        ctl.set_broadphase(True)
        ctl.set_launch_warp_pair(1)
        ctl.reset()
        cmd, info, rc = ctl.step(state, goal)
        mu, sig = ctl.get_distribution()
    orc = oracle.Oracle(robot, world, p)
    ocmd, omu, osig, ost, obest = orc.step(state, goal, 0, np.zeros((p.H, dof)), np.full(dof, f32(p.sigma_init)))
    assert rc == ost == 0
    tol = mu_tolerance([obest, info["mean_weighted_cost"]], p.beta)
    scale = max(1.0, np.abs(omu).max())
    assert max_rel(mu, omu, scale) < tol
    assert max_rel(cmd, ocmd, scale) < tol
    assert max_rel(sig, osig, max(1e-3, osig.max())) < tol
    assert abs(info["best_cost"] - obest) <= TOL_COST * max(1.0, abs(obest))
