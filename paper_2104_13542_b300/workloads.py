"""Seeded synthetic workloads shaped like the paper's (Sec. 5, App. D).

This module only draws inputs: robot chains, obstacle sets, start states, goal
poses and the parameter sets of the five workload configurations.  It holds no
arithmetic of the control method itself, so both the CUDA path and the FP64
oracle may consume its output.

Recipe (all draws from ``numpy.random.default_rng(seed)``):
  * robot: d revolute joints in modified DH form; a_{i-1}, d_i ~ U[0, 0.4] m,
    alpha_{i-1} ~ U{0, +pi/2, -pi/2}, offsets 0, redrawn while a moving link's
    segment to the next joint is shorter than 0.2 m; limits +-2.8 rad.  Seven
    collision spheres per moving link, evenly spaced on the segment from the
    link's frame origin to the next joint's origin (a fixed 0.1 m stub along z
    for the last link), radii ~ U[0.04, 0.10] m.  Self-collision pairs: every
    sphere pair whose links are at least two joints apart.
  * world: axis-aligned boxes with centres ~ U([-0.75, 0.75]^2 x [0, 1.5]) and
    half extents ~ U[0.03, 0.15] m, spheres with radii ~ U[0.03, 0.15] m; any
    obstacle reaching within 0.15 m of the base axis below 0.5 m is redrawn.
  * state: theta ~ U[-1, 1], theta_dot ~ U[-v, v] (v = 0.5 for parity cases,
    0 for closed loop), theta_ddot ~ U[-a, a].
  * goal: position ~ U([-0.6, 0.6]^2 x [0.1, 0.9]), orientation a uniformly
    random unit quaternion (normalised Gaussian 4-vector), as (x, y, z, w, x, y, z).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

SAMPLER_PHILOX = 0
SAMPLER_HALTON = 1
ROT_QUAT = 0
ROT_FROBENIUS = 1
N_TERMS = 8
TERM_NAMES = ("pos", "rot", "stop", "joint", "manip", "self", "world", "smooth", "ee_vel", "ee_acc",
              "ball")
NTERMS = len(TERM_NAMES)
FILTER_DEFAULT, FILTER_COMB, FILTER_MIXED = 0, 1, 2


@dataclass
class Robot:
    dh: np.ndarray           # (d, 4) a_{i-1}, alpha_{i-1}, d_i, theta_offset_i
    q_min: np.ndarray        # (d,)
    q_max: np.ndarray        # (d,)
    sphere_link: np.ndarray  # (M,) int32, frame index 0..d
    spheres: np.ndarray      # (M, 4) x, y, z in link frame, radius
    pairs: np.ndarray        # (P, 2) int32 sphere indices

    @property
    def dof(self) -> int:
        return int(self.dh.shape[0])


@dataclass
class World:
    boxes: np.ndarray    # (B, 6) cx, cy, cz, hx, hy, hz
    spheres: np.ndarray  # (S, 4) cx, cy, cz, r


@dataclass
class Params:
    N: int = 64
    H: int = 20
    K: int = 1
    n_knots: int = 0
    sampler: int = SAMPLER_PHILOX
    n_null: int = 0
    dt: np.ndarray = field(default_factory=lambda: np.full(20, 0.02))
    beta: float = 0.1
    gamma: float = 0.99
    alpha_mu: float = 1.0
    alpha_sigma: float = 0.5
    sigma_init: float = 0.1
    sigma_min: float = 0.0
    w_pos: float = 1.0
    w_rot: float = 1.0
    w_stop: float = 0.0
    w_joint: float = 1.0
    w_manip: float = 0.0
    w_coll: float = 0.0
    w_smooth: float = 1.0
    pos_axis_w: tuple = (1.0, 1.0, 1.0)
    rot_axis_w: tuple = (1.0, 1.0, 1.0)
    rot_mode: int = ROT_QUAT
    k_jl: float = 0.1
    k_m: float = 0.05
    qdd_max: float = 2.0
    seed: int = 0
    instance: int = 0
    grad_steps: int = 0
    grad_eta: float = 0.0
    # noise smoothing along the horizon: FILTER_DEFAULT (B-spline when n_knots > 0),
    # FILTER_COMB (comb coefficients), FILTER_MIXED (mix_bspline of the particles
    # B-spline, the rest comb)
    filter: int = 0
    comb: tuple = (0.5, 0.3, 0.2)
    mix_bspline: float = 0.6
    # task-space limits on the end-effector speed / acceleration (m/s, m/s^2)
    w_ee_vel: float = 0.0
    w_ee_acc: float = 0.0
    ee_vel_max: float = 1.0
    ee_acc_max: float = 10.0
    # ball on a tray held by the end effector
    w_ball: float = 0.0
    gravity: tuple = (0.0, 0.0, -9.81)
    tray_center: tuple = (0.0, 0.0, 0.0)
    # Halton sampler: linearly scrambled digits (per-dimension multipliers from the seed)
    halton_scramble: int = 0

    def replace(self, **kw) -> "Params":
        p = dataclasses.replace(self, **kw)
        if "H" in kw and "dt" not in kw:
            p.dt = np.full(p.H, float(self.dt[0]) if len(self.dt) else 0.02)
        return p


@dataclass
class Workload:
    name: str
    robot: Robot
    world: World
    params: Params
    state: np.ndarray  # (3, d) theta, theta_dot, theta_ddot
    goal: np.ndarray   # (7,) x, y, z, qw, qx, qy, qz
    ball: np.ndarray = None  # (6,) ball position and velocity, world frame (ball-on-tray only)


def _segment_end(dh: np.ndarray, i: int) -> np.ndarray:
    """Origin of joint i+1 in frame i (modified DH row i), or a 0.1 m stub along z
    after the last joint: where the spheres of link i are placed."""
    if i < dh.shape[0]:
        a_i, al_i, d_next = dh[i, 0], dh[i, 1], dh[i, 2]
        return np.array([a_i, -np.sin(al_i) * d_next, np.cos(al_i) * d_next])
    return np.array([0.0, 0.0, 0.1])


def make_robot(seed: int, dof: int = 7, spheres_per_link: int = 7,
               min_link: float = 0.2) -> Robot:
    """Chains are redrawn while any moving link is shorter than `min_link`
    (a link of near-zero length would put the spheres of its neighbours on top
    of each other, i.e. in self-collision in every configuration)."""
    rng = np.random.default_rng([seed, 1])
    while True:
        a = rng.uniform(0.0, 0.4, dof)
        d = rng.uniform(0.0, 0.4, dof)
        alpha = rng.choice(np.array([0.0, np.pi / 2, -np.pi / 2]), dof)
        dh = np.stack([a, alpha, d, np.zeros(dof)], axis=1)
        if all(np.linalg.norm(_segment_end(dh, i)) >= min_link for i in range(1, dof)):
            break
    q_min = np.full(dof, -2.8)
    q_max = np.full(dof, 2.8)
    links, centres = [], []
    for i in range(1, dof + 1):
        end = _segment_end(dh, i)  # segment from frame i's origin to frame i+1's origin
        for k in range(spheres_per_link):
            f = (k + 0.5) / spheres_per_link
            links.append(i)
            centres.append(f * end)
    M = len(links)
    radii = rng.uniform(0.04, 0.10, M)
    spheres = np.concatenate([np.array(centres).reshape(M, 3), radii[:, None]], axis=1)
    sphere_link = np.array(links, dtype=np.int32)
    pairs = [(p, q) for p in range(M) for q in range(p + 1, M)
             if abs(int(sphere_link[p]) - int(sphere_link[q])) >= 2]
    pairs = np.array(pairs, dtype=np.int32).reshape(-1, 2)
    return Robot(dh, q_min, q_max, sphere_link, spheres, pairs)


def make_world(seed: int, n_boxes: int = 20, n_spheres: int = 10) -> World:
    rng = np.random.default_rng([seed, 2])

    def centre():
        while True:
            c = np.array([rng.uniform(-0.75, 0.75), rng.uniform(-0.75, 0.75),
                          rng.uniform(0.0, 1.5)])
            if np.hypot(c[0], c[1]) > 0.35 or c[2] > 0.65:
                return c

    boxes = np.zeros((n_boxes, 6))
    for b in range(n_boxes):
        boxes[b, :3] = centre()
        boxes[b, 3:] = rng.uniform(0.03, 0.15, 3)
    spheres = np.zeros((n_spheres, 4))
    for s in range(n_spheres):
        spheres[s, :3] = centre()
        spheres[s, 3] = rng.uniform(0.03, 0.15)
    return World(boxes, spheres)


def make_state(seed: int, dof: int, vel: float = 0.5, acc: float = 0.5) -> np.ndarray:
    rng = np.random.default_rng([seed, 3])
    return np.stack([rng.uniform(-1.0, 1.0, dof), rng.uniform(-vel, vel, dof),
                     rng.uniform(-acc, acc, dof)])


def make_goal(seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 4])
    p = np.array([rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(0.1, 0.9)])
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    return np.concatenate([p, q])


def make_mean(seed: int, H: int, dof: int, scale: float = 0.3) -> np.ndarray:
    """A nonzero mean control sequence, for stage-wise checks."""
    rng = np.random.default_rng([seed, 5])
    return rng.uniform(-scale, scale, (H, dof))


def make_sigma(seed: int, dof: int, lo: float = 0.05, hi: float = 0.3) -> np.ndarray:
    rng = np.random.default_rng([seed, 6])
    return rng.uniform(lo, hi, dof)


def make_costs(seed: int, N: int, lo: float = 0.0, hi: float = 5.0) -> np.ndarray:
    """Synthetic total costs for checking the distribution update on its own."""
    rng = np.random.default_rng([seed, 7])
    return rng.uniform(lo, hi, N)


def make_controls(seed: int, N: int, H: int, dof: int, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng([seed, 8])
    return rng.normal(0.0, scale, (N, H, dof))


def config_small(seed: int = 0) -> Workload:
    """Plain MPPI step: 64 particles x horizon 20, 7 joints, Gaussian noise sigma 0.1,
    temperature 0.1, discount 0.99, goal position + orientation + joint limits +
    acceleration smoothness, one iteration."""
    robot = make_robot(seed, 7)
    world = World(np.zeros((0, 6)), np.zeros((0, 4)))
    p = Params(N=64, H=20, K=1, n_knots=0, dt=np.full(20, 0.02), beta=0.1, gamma=0.99,
               sigma_init=0.1, w_pos=1.0, w_rot=1.0, w_joint=1.0, w_smooth=1.0, w_stop=0.0,
               w_manip=0.0, w_coll=0.0, seed=1000 + seed)
    return Workload("mppi_64x20_7dof", robot, world, p, make_state(seed, 7), make_goal(seed))


def config_paper(seed: int = 0, N: int = 500, H: int = 30) -> Workload:
    """Paper-scale step: 500 particles x horizon 30, 7 joints, 6-knot cubic B-spline
    noise, 3 iterations with mean + diagonal covariance update (sigma floored at
    0.1: without a floor the near-argmin weights collapse sigma and the arm
    stalls), 2 null particles, all cost terms, 49 link spheres, 20 boxes + 10
    spheres."""
    robot = make_robot(seed, 7)
    world = make_world(seed, 20, 10)
    p = Params(N=N, H=H, K=3, n_knots=6, dt=np.full(H, 0.02), beta=10.0, gamma=0.99,
               alpha_mu=1.0, alpha_sigma=0.5, sigma_init=0.5, sigma_min=0.1, n_null=2,
               w_pos=150.0, w_rot=20.0, w_stop=10.0, w_joint=100.0, w_manip=30.0,
               w_coll=1000.0, w_smooth=0.0, seed=2000 + seed)
    return Workload(f"storm_{N}x{H}_7dof_k3_spline6", robot, world, p, make_state(seed, 7),
                    make_goal(seed))


def config_differentiable(seed: int = 0, N: int = 500, H: int = 30) -> Workload:
    """Differentiable rollout: the paper-scale step followed by 5 gradient steps on
    the mean, mu <- mu - 0.01 dJ/dmu, J the mean discounted rollout cost."""
    wl = config_paper(seed, N, H)
    wl.params = wl.params.replace(grad_steps=5, grad_eta=0.01)
    wl.name = f"storm_{N}x{H}_7dof_k3_spline6_grad5"
    return wl


def config_variable_dt(seed: int = 0, N: int = 500, H: int = 30) -> Workload:
    """Paper-scale step on a variable time-step schedule (Sec. 4.1: small steps near
    the current state, growing along the horizon): dt_h = 0.01 * 1.08^h (0.01 s to
    0.093 s, 1.13 s in all), with end-effector speed (0.5 m/s) and acceleration
    (4 m/s^2) limits weighted into the cost."""
    wl = config_paper(seed, N, H)
    wl.params = wl.params.replace(dt=0.01 * 1.08 ** np.arange(H), w_ee_vel=50.0, w_ee_acc=5.0,
                                  ee_vel_max=0.5, ee_acc_max=4.0)
    wl.name = f"storm_{N}x{H}_7dof_k3_spline6_vardt_eelimits"
    return wl


def config_mixed(seed: int = 0, N: int = 500, H: int = 30) -> Workload:
    """Paper-scale step with the mixed sampler: 0.6 of the particles B-spline
    smoothed (6 knots), 0.4 comb filtered (coefficients 0.5, 0.3, 0.2)."""
    wl = config_paper(seed, N, H)
    wl.params = wl.params.replace(filter=FILTER_MIXED, mix_bspline=0.6, comb=(0.5, 0.3, 0.2))
    wl.name = f"storm_{N}x{H}_7dof_k3_mixed"
    return wl


def config_ball(seed: int = 0, N: int = 500, H: int = 30) -> Workload:
    """Ball on a tray held by the end effector: the paper-scale sampler and
    update, no obstacles, the ball-centring cost with a weak position hold of
    the end effector and no orientation term (the tray must tilt).  Variable
    time steps dt_h = 0.02 * 1.05^h (Sec. 4.1; 1.33 s of horizon: with uniform
    0.02 s steps the 0.6 s horizon is too short to stop the rolling ball and the
    closed loop diverges).  The ball state (world frame) is a seeded point with
    a small velocity."""
    rng = np.random.default_rng([seed, 17])
    robot = make_robot(seed, 7)
    world = make_world(seed, 0, 0)
    p = Params(N=N, H=H, K=3, n_knots=6, dt=0.02 * 1.05 ** np.arange(H), beta=10.0, gamma=0.99,
               alpha_mu=1.0, alpha_sigma=0.5, sigma_init=0.5, sigma_min=0.1, n_null=2,
               w_pos=20.0, w_rot=0.0, w_stop=10.0, w_joint=100.0, w_manip=0.0,
               w_coll=1000.0, w_smooth=0.0, w_ball=200.0, gravity=(0.0, 0.0, -9.81),
               tray_center=(0.0, 0.0, 0.0), seed=4000 + seed)
    ball = np.concatenate([rng.uniform([-0.5, -0.5, 0.2], [0.5, 0.5, 0.8]), rng.uniform(-0.1, 0.1, 3)])
    return Workload(f"storm_ball_{N}x{H}_7dof", robot, world, p, make_state(seed, 7), make_goal(seed),
                    ball)


def config_batch(seed: int = 0, count: int = 256) -> list:
    """Batched uneven MPC: `count` independent instances, particles ~ U{64..1024},
    horizon ~ U{10..50}, 6 or 7 joints, 0..64 obstacles (boxes and spheres), each
    with its own robot, world, start, goal and Philox stream; one MPPI iteration."""
    rng = np.random.default_rng([seed, 10])
    out = []
    for i in range(count):
        N = int(rng.integers(64, 1025))
        H = int(rng.integers(10, 51))
        dof = int(rng.choice([6, 7]))
        n_obs = int(rng.integers(0, 65))
        s = 100_000 + 1000 * seed + i
        robot = make_robot(s, dof)
        world = make_world(s, n_boxes=(n_obs + 1) // 2, n_spheres=n_obs // 2)
        p = Params(N=N, H=H, K=1, n_knots=6, dt=np.full(H, 0.02), beta=10.0, gamma=0.99,
                   alpha_mu=1.0, alpha_sigma=0.5, sigma_init=0.5, sigma_min=0.1, n_null=2,
                   w_pos=150.0, w_rot=20.0,
                   w_stop=10.0, w_joint=100.0, w_manip=30.0, w_coll=1000.0, w_smooth=0.0,
                   seed=3000 + seed, instance=i)
        out.append(Workload(f"batch{i}_{N}x{H}_{dof}dof_{n_obs}obs", robot, world, p,
                            make_state(s, dof), make_goal(s)))
    return out
