"""Closed loop: the controller drives an ideal double-integrator arm to a goal.

Parity of a 300-step trajectory with the oracle is not meaningful (the loop is
chaotic under FP32 vs FP64 rounding), and the paper prints no trajectories, so
this checks task success only: from a collision-free start to a collision-free
goal pose X_g = FK(theta_g) (both chosen with the oracle), with the paper's
orientation-constrained weights (alpha_p = [100, 100], supplement), position
error under 5 mm and orientation error 1 - |q . q_g| under 0.01 after 600 steps,
with no joint-limit or collision violation along the way (checked with the
oracle)."""
import numpy as np
import pytest

import oracle
from paper_2104_13542_b300 import Controller
from paper_2104_13542_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _clear(o, rng):
    while True:
        th = rng.uniform(-2.0, 2.0, 7)
        if o.self_min_sd_theta(th) > 0.03 and o.world_min_sd(th) > 0.03:
            return th


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_reaches_goal_without_violations(seed):
    wl = W.config_paper(seed)
    wl.params = wl.params.replace(w_pos=100.0, w_rot=100.0)
    o = oracle.from_workload(wl)
    rng = np.random.default_rng(seed + 50)
    th0, thg = _clear(o, rng), _clear(o, rng)
    Tg = o.fk(thg)[-1]
    goal = np.concatenate([Tg[:3, 3], oracle.quat_from_rot(Tg[:3, :3])]).astype(np.float32)
    st = np.zeros((3, 7), np.float32)
    st[0] = th0
    worst_self, worst_world, over_limit = np.inf, np.inf, -np.inf
    with Controller(wl.robot, wl.world, wl.params) as c:
        for _ in range(600):
            cmd, info, rc = c.step(st, goal)
            assert rc == 0
            st[2] = cmd
            st[1] = st[1] + 0.02 * cmd
            st[0] = st[0] + 0.02 * st[1]
            th = st[0].astype(np.float64)
            worst_self = min(worst_self, o.self_min_sd_theta(th))
            worst_world = min(worst_world, o.world_min_sd(th))
            over_limit = max(over_limit, float(np.max(np.abs(th)) - 2.8))
    T = o.fk(st[0].astype(np.float64))[-1]
    pos_err = float(np.linalg.norm(T[:3, 3] - goal[:3]))
    q = oracle.quat_from_rot(T[:3, :3])
    rot_err = 1.0 - abs(float(q @ goal[3:].astype(np.float64)))
    assert pos_err < 0.005, pos_err
    assert rot_err < 0.01, rot_err
    assert worst_self > 0.0 and worst_world > 0.0 and over_limit < 0.0
