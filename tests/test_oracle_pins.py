"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks one oracle routine against something other than itself: a
published known-answer vector, a closed form, an invariant, a special case
that reduces to a library routine, or brute force on a tiny input.  The aim is
that a dropped term, a wrong sign or index, or a transposed operand anywhere in
the oracle fails at least one of these.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2104_13542_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- noise

def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_from_bits_open_interval():
    assert oracle.uniform_from_bits(0) == 2.0 ** -24
    assert oracle.uniform_from_bits(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # 23 high bits only: the low 9 bits do not matter
    assert oracle.uniform_from_bits(0x12345600) == oracle.uniform_from_bits(0x123457FF)
    assert oracle.uniform_from_bits(1 << 31) == 0.5 + 2.0 ** -24


def test_box_muller_special_values():
    u1 = math.exp(-0.5)  # radius sqrt(-2 ln u1) = 1
    for u2, expect in [(0.0, (1.0, 0.0)), (0.25, (0.0, 1.0)), (0.5, (-1.0, 0.0)),
                       (0.75, (0.0, -1.0))]:
        z0, z1 = oracle.box_muller(u1, u2)
        assert z0 == pytest.approx(expect[0], abs=1e-15)
        assert z1 == pytest.approx(expect[1], abs=1e-15)
    z0, z1 = oracle.box_muller(math.exp(-2.0), 0.125)  # radius 2 at 45 degrees
    assert z0 == pytest.approx(math.sqrt(2.0), abs=1e-14)
    assert z1 == pytest.approx(math.sqrt(2.0), abs=1e-14)


def test_noise_counter_layout():
    seed, step, inst, it, tag = 0x1234_5678_9ABC_DEF0, 7, 3, 2, 0
    eps = oracle.noise_philox(seed, step, inst, it, tag, 10)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for e in range(10):
        x = oracle.philox([e // 4, step, (inst << 8) | it, tag], key)
        pair = (e % 4) // 2
        z = oracle.box_muller(oracle.uniform_from_bits(x[2 * pair]),
                              oracle.uniform_from_bits(x[2 * pair + 1]))
        assert eps[e] == z[e % 2]
    # distinct iterations, steps and instances give distinct streams
    a = oracle.noise_philox(seed, step, inst, it + 1, tag, 8)
    b = oracle.noise_philox(seed, step + 1, inst, it, tag, 8)
    c = oracle.noise_philox(seed, step, inst + 1, it, tag, 8)
    for other in (a, b, c):
        assert not np.allclose(eps[:8], other)


def test_noise_is_standard_normal():
    eps = oracle.noise_philox(42, 0, 0, 0, 0, 200_000)
    n = eps.size
    assert abs(eps.mean()) < 5 / math.sqrt(n)
    assert abs(eps.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert stats.kstest(eps, "norm").pvalue > 1e-4
    # lanes 0/1 of one block are independent (correlation ~ 0)
    x = eps[: n - n % 4].reshape(-1, 4)
    assert abs(np.corrcoef(x[:, 0], x[:, 1])[0, 1]) < 0.02


def test_halton_radical_inverse_exact():
    for i, v in zip(range(1, 5), [1 / 2, 1 / 4, 3 / 4, 1 / 8]):
        assert oracle.radical_inverse(i, 2) == v
    for i, v in zip(range(1, 4), [1 / 3, 2 / 3, 1 / 9]):
        assert oracle.radical_inverse(i, 3) == pytest.approx(v, rel=1e-15)
    assert oracle.radical_inverse(7, 5) == pytest.approx(11 / 25, rel=1e-15)  # 7 = (12)_5
    assert [oracle.nth_prime(n) for n in range(10)] == [2, 3, 5, 7, 11, 13, 17, 19, 23, 29]
    assert oracle.nth_prime(41) == 181


def test_norm_ppf_matches_library():
    ps = np.concatenate([[1e-10, 1e-4, 0.025, 0.3, 0.5, 0.7, 0.975, 1 - 1e-6],
                         np.random.default_rng(0).uniform(0, 1, 50)])
    for p in ps:
        assert oracle.norm_ppf(p) == pytest.approx(stats.norm.ppf(p), abs=1e-11, rel=1e-11)
    assert oracle.norm_ppf(0.5) == pytest.approx(0.0, abs=1e-15)


def test_halton_noise_dimension_layout():
    N, S, d = 5, 3, 4
    eps = oracle.noise_halton(N, S, d)
    primes = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37]
    for n in range(N):
        for s in range(S):
            for j in range(d):
                i = n + 1
                b = primes[s * d + j]
                # radical inverse written out digit by digit
                r, f = 0.0, 1.0 / b
                while i:
                    r += (i % b) * f
                    i //= b
                    f /= b
                assert eps[n, s, j] == pytest.approx(stats.norm.ppf(r), abs=1e-10)


# ----------------------------------------------------------------------------- B-spline

@pytest.mark.parametrize("H,S", [(30, 6), (20, 4), (50, 10), (7, 5)])
def test_bspline_partition_of_unity_and_ends(H, S):
    B = oracle.bspline_basis(H, S)
    assert np.allclose(B.sum(1), 1.0, atol=1e-14)
    assert np.all(B >= -1e-15)
    assert np.allclose(B[0], np.eye(S)[0])
    assert np.allclose(B[-1], np.eye(S)[-1])
    # linear precision: Greville abscissae reproduce x_h exactly
    knots = np.concatenate([[0, 0, 0, 0], np.arange(1, S - 3) / (S - 3), [1, 1, 1, 1]])
    grev = np.array([(knots[s + 1] + knots[s + 2] + knots[s + 3]) / 3 for s in range(S)])
    x = np.arange(H) / (H - 1)
    assert np.allclose(B @ grev, x, atol=1e-13)


def test_bspline_single_span_is_bernstein():
    H = 11
    B = oracle.bspline_basis(H, 4)
    x = np.arange(H) / (H - 1)
    bern = np.stack([(1 - x) ** 3, 3 * x * (1 - x) ** 2, 3 * x ** 2 * (1 - x), x ** 3], 1)
    assert np.allclose(B, bern, atol=1e-14)


def test_bspline_interior_span_uniform_blending():
    # S = 10 control points -> knots 0,0,0,0,1/7,..,6/7,1,1,1,1.  Basis functions
    # 3..6 have five equally spaced knots, so on the span [3/7, 4/7) they are the
    # uniform cubic blending polynomials.
    H, S = 50, 10
    B = oracle.bspline_basis(H, S)
    hits = 0
    for h in range(H):
        x = h / (H - 1)
        if not (3 / 7 <= x < 4 / 7):
            continue
        hits += 1
        t = (x - 3 / 7) * 7
        blend = np.array([(1 - t) ** 3, 3 * t ** 3 - 6 * t ** 2 + 4,
                          -3 * t ** 3 + 3 * t ** 2 + 3 * t + 1, t ** 3]) / 6
        assert np.allclose(B[h, 3:7], blend, atol=1e-13)
        assert np.all(np.abs(np.delete(B[h], [3, 4, 5, 6])) < 1e-15)
    assert hits >= 6


def test_controls_null_particles_and_no_spline():
    wl = W.config_small(0)
    p = wl.params.replace(N=6, n_null=2)
    o = oracle.Oracle(wl.robot, wl.world, p)
    mu = W.make_mean(1, p.H, 7)
    sig = W.make_sigma(1, 7)
    eps = np.random.default_rng(3).normal(size=(p.N, p.H, 7))
    u = o.controls(mu, sig, eps)
    assert np.all(u[:2] == 0.0)
    assert np.allclose(u[2:], mu[None] + sig[None, None] * eps[2:], atol=1e-15)


def test_controls_with_spline_constant_knots():
    wl = W.config_paper(0, N=4, H=30)
    o = oracle.Oracle(wl.robot, wl.world, wl.params.replace(n_null=0))
    mu = W.make_mean(2, 30, 7)
    sig = W.make_sigma(2, 7)
    eps = np.broadcast_to(np.arange(7.0)[None, None, :], (4, 6, 7)).copy()
    u = o.controls(mu, sig, eps)  # constant control points -> constant curve
    assert np.allclose(u, mu[None] + sig * np.arange(7.0), atol=1e-13)


# ----------------------------------------------------------------------------- integration

def test_integration_constant_acceleration_closed_form():
    H, d, dt = 25, 3, 0.02
    a = np.array([0.7, -1.3, 0.2])
    th0, thd0 = np.array([0.1, -0.4, 1.0]), np.array([0.3, 0.0, -0.2])
    state = np.stack([th0, thd0, np.zeros(d)])
    th, thd = oracle.integrate(np.full(H, dt), state, np.tile(a, (H, 1)))
    k = np.arange(1, H + 1)[:, None]
    assert np.allclose(thd, thd0 + k * a * dt, atol=1e-13)
    assert np.allclose(th, th0 + k * thd0 * dt + a * dt ** 2 * k * (k + 1) / 2, atol=1e-13)


def test_integration_variable_dt_matches_cumsum():
    rng = np.random.default_rng(1)
    H, d = 17, 4
    dt = rng.uniform(0.005, 0.05, H)
    state = rng.normal(size=(3, d))
    u = rng.normal(size=(H, d))
    th, thd = oracle.integrate(dt, state, u)
    thd_ref = state[1] + np.cumsum(dt[:, None] * u, axis=0)
    th_ref = state[0] + np.cumsum(dt[:, None] * thd_ref, axis=0)
    assert np.allclose(thd, thd_ref, atol=1e-13)
    assert np.allclose(th, th_ref, atol=1e-13)


# ----------------------------------------------------------------------------- FK / Jacobian

def _robot_from_dh(dh):
    d = len(dh)
    return W.Robot(np.asarray(dh, float), np.full(d, -2.8), np.full(d, 2.8),
                   np.zeros(0, np.int32), np.zeros((0, 4)), np.zeros((0, 2), np.int32))


def _empty_world():
    return W.World(np.zeros((0, 6)), np.zeros((0, 4)))


def _oracle_for(robot, **kw):
    d = robot.dof
    p = W.Params(N=1, H=1, dt=np.array([0.02]), **kw)
    return oracle.Oracle(robot, _empty_world(), p)


def test_fk_planar_arm_closed_form():
    L1, L2 = 0.35, 0.25
    o = _oracle_for(_robot_from_dh([[0, 0, 0, 0], [L1, 0, 0, 0], [L2, 0, 0, 0]]))
    for t1, t2 in [(0.0, 0.0), (0.3, -1.1), (2.0, 0.7)]:
        Te = o.fk([t1, t2, 0.0])[-1]
        assert Te[0, 3] == pytest.approx(L1 * math.cos(t1) + L2 * math.cos(t1 + t2), abs=1e-14)
        assert Te[1, 3] == pytest.approx(L1 * math.sin(t1) + L2 * math.sin(t1 + t2), abs=1e-14)
        assert Te[2, 3] == pytest.approx(0.0, abs=1e-14)
        assert np.arctan2(Te[1, 0], Te[0, 0]) == pytest.approx(
            math.atan2(math.sin(t1 + t2), math.cos(t1 + t2)), abs=1e-14)


def test_fk_zero_configuration_alpha_zero():
    rng = np.random.default_rng(5)
    a, dd = rng.uniform(0, 0.4, 7), rng.uniform(0, 0.4, 7)
    o = _oracle_for(_robot_from_dh(np.stack([a, np.zeros(7), dd, np.zeros(7)], 1)))
    Te = o.fk(np.zeros(7))[-1]
    assert np.allclose(Te[:3, :3], np.eye(3), atol=1e-15)
    assert np.allclose(Te[:3, 3], [a.sum(), 0.0, dd.sum()], atol=1e-14)


def test_fk_zero_configuration_twisted_chain():
    # alpha = +pi/2 then -pi/2: frame 2 maps z -> -y, so d_2 moves along -y
    o = _oracle_for(_robot_from_dh([[0.1, 0, 0.2, 0], [0.3, math.pi / 2, 0.4, 0],
                                    [0.0, -math.pi / 2, 0.0, 0]]))
    Te = o.fk(np.zeros(3))[-1]
    assert np.allclose(Te[:3, 3], [0.1 + 0.3, -0.4, 0.2], atol=1e-14)
    assert np.allclose(Te[:3, :3], np.eye(3), atol=1e-14)


def _rodrigues(axis, ang):
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_fk_single_joint_is_rodrigues_rotation():
    robot = W.make_robot(3, 7)
    o = _oracle_for(robot)
    base = np.random.default_rng(2).uniform(-1, 1, 7)
    F0 = o.fk(base)
    for k in range(7):
        ang = 0.9 - 0.3 * k
        th = base.copy()
        th[k] += ang
        F = o.fk(th)
        z, org = F0[k + 1][:3, 2], F0[k + 1][:3, 3]
        Rk = _rodrigues(z, ang)
        assert np.allclose(F[-1][:3, 3], Rk @ (F0[-1][:3, 3] - org) + org, atol=1e-13)
        assert np.allclose(F[-1][:3, :3], Rk @ F0[-1][:3, :3], atol=1e-13)
        # frames before joint k are untouched
        assert np.allclose(F[: k + 1], F0[: k + 1], atol=1e-15)


def test_fk_rotations_orthonormal():
    robot = W.make_robot(4, 7)
    o = _oracle_for(robot)
    for th in np.random.default_rng(4).uniform(-2.8, 2.8, (20, 7)):
        for T in o.fk(th):
            R = T[:3, :3]
            assert np.allclose(R.T @ R, np.eye(3), atol=1e-12)
            assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
            assert np.allclose(T[3], [0, 0, 0, 1])


def _vee(S):
    return np.array([S[2, 1], S[0, 2], S[1, 0]])


def test_jacobian_matches_central_differences():
    robot = W.make_robot(6, 7)
    o = _oracle_for(robot)
    h = 1e-6
    for th in np.random.default_rng(6).uniform(-2.5, 2.5, (5, 7)):
        J = o.jacobian(th)
        for k in range(7):
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            Fp, Fm = o.fk(tp)[-1], o.fk(tm)[-1]
            lin = (Fp[:3, 3] - Fm[:3, 3]) / (2 * h)
            Rp, Rm = Fp[:3, :3], Fm[:3, :3]
            ang = _vee((Rp @ Rm.T - Rm @ Rp.T) / 2) / (2 * h)
            assert np.allclose(J[:3, k], lin, atol=1e-8)
            assert np.allclose(J[3:, k], ang, atol=1e-8)


def test_det_matches_library():
    rng = np.random.default_rng(7)
    for n in (1, 2, 3, 6):
        A = rng.normal(size=(n, n))
        assert oracle.det(A) == pytest.approx(np.linalg.det(A), rel=1e-12)
    P = np.eye(6)[[1, 0, 2, 3, 5, 4]]  # two transpositions -> +1
    assert oracle.det(P) == pytest.approx(1.0)
    assert oracle.det(np.eye(6)[[1, 0, 2, 3, 4, 5]]) == pytest.approx(-1.0)


def test_manipulability_singular_values():
    rng = np.random.default_rng(8)
    J6 = rng.normal(size=(6, 6))
    assert oracle.manipulability(J6) == pytest.approx(abs(np.linalg.det(J6)), rel=1e-11)
    J7 = rng.normal(size=(6, 7))
    assert oracle.manipulability(J7) == pytest.approx(np.prod(np.linalg.svd(J7)[1]), rel=1e-11)
    J7[5] = J7[4]  # rank deficient
    assert oracle.manipulability(J7) < 1e-6


# ----------------------------------------------------------------------------- rotations

def test_quaternion_round_trip_and_trace_identity():
    rng = np.random.default_rng(9)
    for _ in range(50):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        Rm = oracle.rot_from_quat(q)
        assert np.allclose(Rm.T @ Rm, np.eye(3), atol=1e-14)
        q2 = oracle.quat_from_rot(Rm)
        assert abs(abs(q @ q2) - 1.0) < 1e-13
        # rotation about z by angle a: quaternion (cos a/2, 0, 0, sin a/2)
    a = 0.8
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    assert np.allclose(oracle.quat_from_rot(Rz), [math.cos(a / 2), 0, 0, math.sin(a / 2)])
    assert np.allclose(oracle.rot_from_quat([math.cos(a / 2), 0, 0, math.sin(a / 2)]), Rz)
    # |q1 . q2| = cos(phi/2) = sqrt(1 + tr(R1^T R2)) / 2
    for _ in range(20):
        q1, q2 = rng.normal(size=4), rng.normal(size=4)
        q1 /= np.linalg.norm(q1)
        q2 /= np.linalg.norm(q2)
        tr = np.trace(oracle.rot_from_quat(q1).T @ oracle.rot_from_quat(q2))
        assert abs(q1 @ q2) == pytest.approx(math.sqrt(max(0.0, 1 + tr)) / 2, abs=1e-12)


# ----------------------------------------------------------------------------- collision

def test_box_sdf_on_axis_and_inside():
    box = np.array([0.1, -0.2, 0.5, 0.2, 0.1, 0.3])
    assert oracle.box_sdf([0.1 + 0.2 + 0.3, -0.2, 0.5], box) == pytest.approx(0.3)
    assert oracle.box_sdf([0.1, -0.2 - 0.1 - 0.05, 0.5], box) == pytest.approx(0.05)
    assert oracle.box_sdf([0.1, -0.2, 0.5], box) == pytest.approx(-0.1)  # centre: nearest face y
    assert oracle.box_sdf([0.1 + 0.2 + 0.3, -0.2 + 0.1 + 0.4, 0.5], box) == pytest.approx(0.5)


def test_box_sdf_brute_force():
    rng = np.random.default_rng(10)
    box = np.array([0.0, 0.0, 0.0, 0.3, 0.2, 0.1])
    g = np.linspace(-1, 1, 81)
    # dense sample of the surface: each face as a grid
    faces = []
    for ax in range(3):
        o1, o2 = [a for a in range(3) if a != ax]
        for s in (-1, 1):
            U, V = np.meshgrid(g * box[3 + o1], g * box[3 + o2])
            P = np.zeros(U.shape + (3,))
            P[..., ax] = s * box[3 + ax]
            P[..., o1] = U
            P[..., o2] = V
            faces.append(P.reshape(-1, 3))
    surf = np.concatenate(faces)
    for _ in range(30):
        p = rng.uniform(-0.6, 0.6, 3)
        dmin = np.min(np.linalg.norm(surf - p, axis=1))
        inside = np.all(np.abs(p) <= box[3:])
        sd = oracle.box_sdf(p, box)
        assert sd == pytest.approx(-dmin if inside else dmin, abs=2e-3)


def test_sphere_collisions_constructed():
    # planar two-link arm along x; one sphere on each link frame
    dh = [[0, 0, 0, 0], [0.5, 0, 0, 0], [0.5, 0, 0, 0]]
    robot = _robot_from_dh(dh)
    robot.sphere_link = np.array([1, 3], np.int32)
    robot.spheres = np.array([[0.0, 0.0, 0.0, 0.1], [0.0, 0.0, 0.0, 0.2]])
    robot.pairs = np.array([[0, 1]], np.int32)
    world = W.World(np.array([[1.0, 0.0, 0.0, 0.05, 0.05, 0.05]]),
                    np.array([[0.0, 0.0, 0.25, 0.1]]))
    o = oracle.Oracle(robot, world, W.Params(N=1, H=1, dt=np.array([0.02])))
    th = np.zeros(3)  # sphere 0 at origin, sphere 1 at x = 1.0
    assert o.self_min_sd(th) == pytest.approx(1.0 - 0.3)
    # sphere 1 (r 0.2) at box centre: box sdf -0.05 -> -0.25; sphere 0 to obstacle
    # sphere: 0.25 - 0.1 - 0.1 = 0.05
    assert o.world_min_sd(th) == pytest.approx(-0.25)
    th = np.array([0.0, math.pi, 0.0])  # fold back: sphere 1 returns to the origin
    assert o.self_min_sd(th) == pytest.approx(-0.3, abs=1e-12)
    assert o.world_min_sd(th) == pytest.approx(0.25 - 0.2 - 0.1, abs=1e-12)


# ----------------------------------------------------------------------------- costs

def _goal_from_frame(T):
    q = oracle.quat_from_rot(T[:3, :3])
    return np.concatenate([T[:3, 3], q])


def test_costs_vanish_at_goal_at_rest():
    wl = W.config_paper(1, N=1, H=30)
    p = wl.params.replace(N=1, k_m=0.0)
    world = W.World(np.zeros((0, 6)), np.zeros((0, 4)))
    robot = wl.robot
    robot_nc = W.Robot(robot.dh, robot.q_min, robot.q_max, robot.sphere_link, robot.spheres,
                       np.zeros((0, 2), np.int32))
    o = oracle.Oracle(robot_nc, world, p)
    th = np.array([0.3, -0.2, 0.1, 0.5, -0.4, 0.2, 0.0])
    goal = _goal_from_frame(o.fk(th)[-1])
    terms, tot = o.running_cost(goal, 0, th, np.zeros(7), np.zeros(7), np.zeros(7))
    assert np.allclose(terms, 0.0, atol=1e-12)
    assert tot == pytest.approx(0.0, abs=1e-9)


def test_cost_terms_closed_forms():
    wl = W.config_paper(1, N=1, H=10)
    p = wl.params.replace(N=1, H=10, k_m=0.0)
    robot = W.Robot(wl.robot.dh, wl.robot.q_min, wl.robot.q_max, wl.robot.sphere_link,
                    wl.robot.spheres, np.zeros((0, 2), np.int32))
    o = oracle.Oracle(robot, W.World(np.zeros((0, 6)), np.zeros((0, 4))), p)
    th = np.zeros(7)
    T = o.fk(th)[-1]
    goal = _goal_from_frame(T)
    goal[:3] += [0.03, -0.04, 0.0]  # 5 cm away
    terms, _ = o.running_cost(goal, 0, th, np.zeros(7), np.zeros(7), np.zeros(7))
    assert terms[0] == pytest.approx(0.05, abs=1e-12)
    assert terms[1] == pytest.approx(0.0, abs=1e-12)
    # rotation about the goal z axis by a: 1 - cos(a/2)
    a = 0.6
    g2 = goal.copy()
    Rg = T[:3, :3] @ _rodrigues(np.array([0, 0, 1.0]), a)
    g2[3:] = oracle.quat_from_rot(Rg)
    terms, _ = o.running_cost(g2, 0, th, np.zeros(7), np.zeros(7), np.zeros(7))
    assert terms[1] == pytest.approx(1 - math.cos(a / 2), abs=1e-12)
    # joint limit: soft limits at +-(2.8 - 0.1 * 5.6) = +-2.24
    th2 = th.copy()
    th2[2] = 2.24 + 0.1
    th2[4] = -2.24 - 0.2
    terms, _ = o.running_cost(goal, 0, th2, np.zeros(7), np.zeros(7), np.zeros(7))
    assert terms[3] == pytest.approx(math.hypot(0.1, 0.2), abs=1e-12)
    # stop: limit at h is qdd_max * sum_{k>=h} dt_k = 2 * 0.02 * (10 - h)
    h = 6
    vlim = 2.0 * 0.02 * (10 - h)
    thd = np.zeros(7)
    thd[1] = -(vlim + 0.3)
    thd[5] = vlim - 0.01  # below the limit: no cost
    terms, _ = o.running_cost(goal, h, th, thd, np.zeros(7), np.zeros(7))
    assert terms[2] == pytest.approx(0.3, abs=1e-12)
    # smoothness
    du = np.arange(7.0) * 0.1
    terms, _ = o.running_cost(goal, 0, th, np.zeros(7), du, np.zeros(7))
    assert terms[7] == pytest.approx(float(du @ du), abs=1e-12)


def test_manip_cost_threshold():
    wl = W.config_paper(2, N=1, H=5)
    robot = W.Robot(wl.robot.dh, wl.robot.q_min, wl.robot.q_max, wl.robot.sphere_link,
                    wl.robot.spheres, np.zeros((0, 2), np.int32))
    empty = W.World(np.zeros((0, 6)), np.zeros((0, 4)))
    th = np.full(7, 0.4)
    o = oracle.Oracle(robot, empty, wl.params.replace(N=1, H=5))
    m = oracle.manipulability(o.jacobian(th))
    goal = W.make_goal(0)
    for k_m, expect in [(m * 1.01, 1 - m), (m * 0.99, 0.0)]:
        o = oracle.Oracle(robot, empty, wl.params.replace(N=1, H=5, k_m=k_m))
        terms, _ = o.running_cost(goal, 0, th, np.zeros(7), np.zeros(7), np.zeros(7))
        assert terms[4] == pytest.approx(expect, abs=1e-12)


def test_rotation_frobenius_mode():
    wl = W.config_small(0)
    p = wl.params.replace(N=1, rot_mode=W.ROT_FROBENIUS, rot_axis_w=(0.0, 0.0, 2.0))
    o = oracle.Oracle(wl.robot, wl.world, p)
    th = np.zeros(7)
    T = o.fk(th)[-1]
    a = 0.5  # rotate about goal x: ee z axis tilts by a; only the z column is weighted
    goal = _goal_from_frame(T)
    goal[3:] = oracle.quat_from_rot(T[:3, :3] @ _rodrigues(np.array([1.0, 0, 0]), a))
    terms, _ = o.running_cost(goal, 0, th, np.zeros(7), np.zeros(7), np.zeros(7))
    # column z of I - Rx(-a): (0, -sin a, 1 - cos a) -> norm 2 sin(a/2), times 2
    assert terms[1] == pytest.approx(2 * 2 * math.sin(a / 2), abs=1e-12)


# ----------------------------------------------------------------------------- discount / rollout

def test_discount_special_cases():
    wl = W.config_small(3)
    for gamma in (1.0, 0.0, 0.9):
        p = wl.params.replace(N=5, gamma=gamma)
        o = oracle.Oracle(wl.robot, wl.world, p)
        eps = o.noise(0, 0)
        out = o.rollout(wl.state, wl.goal, W.make_mean(0, p.H, 7), W.make_sigma(0, 7), eps)
        if gamma == 1.0:
            assert np.allclose(out["C"], out["cost"].sum(1), rtol=1e-14)
        elif gamma == 0.0:
            assert np.allclose(out["C"], out["cost"][:, 0], rtol=1e-14)
        else:
            assert np.allclose(out["C"], out["cost"] @ (gamma ** np.arange(p.H)), rtol=1e-13)


def test_rollout_stage_consistency():
    wl = W.config_paper(0, N=3, H=30)
    o = oracle.from_workload(wl)
    mu, sig = W.make_mean(0, 30, 7), W.make_sigma(0, 7)
    eps = o.noise(0, 0)
    out = o.rollout(wl.state, wl.goal, mu, sig, eps)
    assert np.allclose(out["u"], o.controls(mu, sig, eps))
    for n in range(3):
        th, thd = oracle.integrate(wl.params.dt, wl.state, out["u"][n])
        assert np.allclose(out["theta"][n], th) and np.allclose(out["theta_dot"][n], thd)
        for h in (0, 17, 29):
            assert np.allclose(out["ee"][n, h], o.fk(th[h])[-1][:3])
    w = np.array([wl.params.w_pos, wl.params.w_rot, wl.params.w_stop, wl.params.w_joint,
                  wl.params.w_manip, wl.params.w_coll, wl.params.w_coll, wl.params.w_smooth,
                  wl.params.w_ee_vel, wl.params.w_ee_acc, wl.params.w_ball])
    assert np.allclose(out["terms"] @ w, out["cost"], rtol=1e-13)


# ----------------------------------------------------------------------------- MPPI update

def _upd_oracle(N, H, d, **kw):
    wl = W.config_small(0)
    robot = _robot_from_dh(np.zeros((d, 4)))
    return oracle.Oracle(robot, _empty_world(), wl.params.replace(N=N, H=H, **kw))


def test_update_single_particle_returns_it():
    H, d = 5, 3
    o = _upd_oracle(1, H, d, alpha_mu=1.0, alpha_sigma=0.5)
    u = np.random.default_rng(0).normal(size=(1, H, d))
    mu, sig, st, w = o.update(np.array([3.0]), u, np.zeros((H, d)), np.full(d, 0.2))
    assert st == 0 and w[0] == 1.0
    assert np.allclose(mu, u[0])
    assert np.allclose(sig, math.sqrt(0.5) * 0.2)  # u - mu_new = 0


def test_update_zero_temperature_is_argmin_lowest_index():
    H, d, N = 4, 2, 6
    o = _upd_oracle(N, H, d, beta=0.0)
    u = np.random.default_rng(1).normal(size=(N, H, d))
    C = np.array([5.0, 2.0, 7.0, 2.0, np.nan, 3.0])
    mu, _, st, w = o.update(C, u, np.zeros((H, d)), np.ones(d))
    assert np.array_equal(w, np.eye(N)[1])
    assert np.allclose(mu, u[1])


def test_update_small_temperature_tends_to_argmin():
    H, d, N = 4, 2, 6
    o = _upd_oracle(N, H, d, beta=1e-3)
    u = np.random.default_rng(2).normal(size=(N, H, d))
    C = np.array([5.0, 2.5, 7.0, 2.0, 9.0, 3.0])
    mu, _, _, w = o.update(C, u, np.zeros((H, d)), np.ones(d))
    assert np.allclose(mu, u[3], atol=1e-12)


def test_update_weights_softmax_and_equal_costs():
    H, d, N = 6, 3, 40
    rng = np.random.default_rng(3)
    u = rng.normal(size=(N, H, d))
    o = _upd_oracle(N, H, d, beta=0.7, alpha_mu=1.0, alpha_sigma=1.0)
    C = rng.uniform(0, 4, N)
    mu, sig, _, w = o.update(C, u, np.zeros((H, d)), np.ones(d))
    assert w.sum() == pytest.approx(1.0, abs=1e-14)
    ref = np.exp(-C / 0.7)
    assert np.allclose(w, ref / ref.sum(), rtol=1e-12)
    # equal costs: plain sample mean and the population variance about it
    mu, sig, _, w = o.update(np.full(N, 1.5), u, np.zeros((H, d)), np.ones(d))
    assert np.allclose(mu, u.mean(0), atol=1e-14)
    assert np.allclose(sig ** 2, u.var(axis=0).mean(axis=0), rtol=1e-12)


def test_update_step_sizes():
    H, d, N = 3, 2, 10
    rng = np.random.default_rng(4)
    u = rng.normal(size=(N, H, d))
    mu0, sig0 = rng.normal(size=(H, d)), np.array([0.3, 0.4])
    o = _upd_oracle(N, H, d, alpha_mu=0.0, alpha_sigma=0.0)
    mu, sig, _, _ = o.update(rng.uniform(0, 1, N), u, mu0, sig0)
    assert np.array_equal(mu, mu0) and np.allclose(sig, sig0)
    o = _upd_oracle(N, H, d, alpha_mu=0.25, alpha_sigma=0.5, beta=0.0)
    C = np.arange(N, dtype=float)
    mu, sig, _, _ = o.update(C, u, mu0, sig0)
    assert np.allclose(mu, 0.75 * mu0 + 0.25 * u[0])
    e = u[0] - mu
    assert np.allclose(sig ** 2, 0.5 * sig0 ** 2 + 0.5 * (e ** 2).mean(0))
    o = _upd_oracle(N, H, d, alpha_mu=1.0, alpha_sigma=1.0, beta=0.0, sigma_min=0.7)
    _, sig, _, _ = o.update(C, u, mu0, sig0)  # one-hot: zero spread, floored
    assert np.allclose(sig, 0.7)


def test_update_all_nonfinite_is_degenerate():
    o = _upd_oracle(3, 2, 2)
    mu0 = np.ones((2, 2))
    mu, sig, st, _ = o.update(np.array([np.inf, np.nan, -np.inf]), np.zeros((3, 2, 2)), mu0,
                              np.ones(2))
    assert st == 1 and np.array_equal(mu, mu0)


def test_shift_and_step_semantics():
    wl = W.config_small(2)
    p = wl.params.replace(N=8, H=6, K=2)
    o = oracle.Oracle(wl.robot, wl.world, p)
    mu0 = W.make_mean(3, 6, 7)
    sig0 = np.full(7, 0.1)
    cmd, mu, sig, st, _ = o.step(wl.state, wl.goal, 0, mu0, sig0)
    assert np.allclose(cmd, mu[0])
    # the same step done by hand (no shift at step 0)
    m, s = mu0.copy(), sig0.copy()
    for k in range(2):
        out = o.rollout(wl.state, wl.goal, m, s, o.noise(0, k))
        m, s, _, _ = o.update(out["C"], out["u"], m, s)
    assert np.allclose(m, mu) and np.allclose(s, sig)
    # step 1 shifts first: mu_h <- mu_{h+1}, last row zero
    m1 = np.vstack([mu[1:], np.zeros((1, 7))])
    out = o.rollout(wl.state, wl.goal, m1, sig, o.noise(1, 0))
    m2, s2, _, _ = o.update(out["C"], out["u"], m1, sig)
    out = o.rollout(wl.state, wl.goal, m2, s2, o.noise(1, 1))
    m3, s3, _, _ = o.update(out["C"], out["u"], m2, s2)
    cmd1, mu1, sig1, _, _ = o.step(wl.state, wl.goal, 1, mu, sig)
    assert np.allclose(mu1, m3) and np.allclose(sig1, s3) and np.allclose(cmd1, m3[0])


# ----------------------------------------------------------------------------- scrambled Halton

def test_scrambled_radical_inverse_by_hand():
    # 5 = (12)_3 with digits 2, 1 (least significant first)
    assert oracle.radical_inverse_scrambled(5, 3, 1) == pytest.approx(2 / 3 + 1 / 9, abs=1e-15)
    assert oracle.radical_inverse_scrambled(5, 3, 2) == pytest.approx(1 / 3 + 2 / 9, abs=1e-15)
    # 10 = (1010)_2: multiplier 1 is the only one in base 2
    assert oracle.radical_inverse_scrambled(10, 2, 1) == pytest.approx(0.5 ** 2 + 0.5 ** 4, abs=1e-15)
    # 23 = (43)_5, mult 3: digits 3, 4 -> 9 mod 5 = 4, 12 mod 5 = 2
    assert oracle.radical_inverse_scrambled(23, 5, 3) == pytest.approx(4 / 5 + 2 / 25, abs=1e-15)


@pytest.mark.parametrize("base,mult", [(7, 3), (11, 5), (13, 12)])
def test_scrambled_sequence_keeps_the_stratification(base, mult):
    """b^k consecutive points (from 0) still hit every cell j / b^k once: the
    digit map is a permutation of each digit position."""
    k = 2
    pts = sorted(oracle.radical_inverse_scrambled(i, base, mult) for i in range(base ** k))
    assert np.allclose(pts, np.arange(base ** k) / base ** k, atol=1e-12)


def test_halton_multipliers_and_decorrelation():
    seed = 2000
    primes = [oracle.nth_prime(k) for k in range(42)]
    mults = [oracle.halton_multiplier(seed, k, b) for k, b in enumerate(primes)]
    assert mults[0] == 1 and all(1 <= m < b for m, b in zip(mults, primes))
    assert len(set(mults[10:])) > 20  # drawn, not constant
    # the unscrambled leading points of two large-prime dimensions are i / p: collinear
    plain = oracle.noise_halton(100, 6, 7)
    scr = oracle.noise_halton(100, 6, 7, scramble=True, seed=seed)
    a, b = 40, 41
    r_plain = np.corrcoef(plain[:, a // 7, a % 7], plain[:, b // 7, b % 7])[0, 1]
    r_scr = np.corrcoef(scr[:, a // 7, a % 7], scr[:, b // 7, b % 7])[0, 1]
    assert r_plain > 0.95 and abs(r_scr) < 0.5, (r_plain, r_scr)
    # marginals stay standard normal-like
    assert abs(scr.mean()) < 0.05 and abs(scr.std() - 1.0) < 0.1


def test_rollout_threads_give_the_same_bits():
    """The particle-parallel rollout loop (the all-cores CPU baseline) computes
    exactly what the sequential loop computes: particles are independent and no
    reduction crosses them."""
    from paper_2104_13542_b300 import workloads as W
    wl = W.config_paper(1)
    p = wl.params.replace(N=24)
    orc = oracle.Oracle(wl.robot, wl.world, p)
    mu, sig = W.make_mean(2, p.H, 7, 0.4), W.make_sigma(2, 7)
    eps = orc.noise(1, 0)
    prev = oracle.get_threads()
    try:
        oracle.set_threads(1)
        a = orc.rollout(wl.state, wl.goal, mu, sig, eps)
        oracle.set_threads(4)
        b = orc.rollout(wl.state, wl.goal, mu, sig, eps)
    finally:
        oracle.set_threads(prev)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
