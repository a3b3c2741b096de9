"""Batched uneven instances: every instance of a batch step equals the same
instance stepped alone by its own handle (bitwise: the same kernels in another
launch order), and matches the FP64 oracle within the tolerance model."""
import numpy as np
import pytest

import oracle
from paper_2104_13542_b300 import BatchController, Controller, StormError
from paper_2104_13542_b300 import workloads as W

from gpu_helpers import f32, max_rel, mu_tolerance

pytestmark = pytest.mark.gpu


def _batch(count, seed=0):
    wls = W.config_batch(seed, count)
    # keep the oracle affordable: cap the particle count of the parity batch
    for wl in wls:
        wl.params = wl.params.replace(N=min(wl.params.N, 160))
    return wls


def test_batch_equals_individual_handles_bitwise():
    wls = _batch(10, seed=1)
    states = [f32(wl.state) for wl in wls]
    goals = np.stack([f32(wl.goal) for wl in wls])
    with BatchController([w.robot for w in wls], [w.world for w in wls],
                         [w.params for w in wls]) as b:
        steps = [b.step(states, goals) for _ in range(2)]
        dists = [b.get_distribution(i) for i in range(len(wls))]
    for i, wl in enumerate(wls):
        with Controller(wl.robot, wl.world, wl.params) as c:
            ref = [c.step(states[i], goals[i])[0] for _ in range(2)]
            mu, sg = c.get_distribution()
        for t in range(2):
            assert np.array_equal(steps[t][0][i], ref[t]), (i, t)
        assert np.array_equal(dists[i][0], mu) and np.array_equal(dists[i][1], sg)
    assert all(np.all(s[1] == 0) for s in steps)


def test_batch_matches_oracle_per_instance():
    wls = _batch(8, seed=2)
    states = [f32(wl.state) for wl in wls]
    goals = np.stack([f32(wl.goal) for wl in wls])
    with BatchController([w.robot for w in wls], [w.world for w in wls],
                         [w.params for w in wls]) as b:
        cmds, st = b.step(states, goals)
        dists = [b.get_distribution(i) for i in range(len(wls))]
    for i, wl in enumerate(wls):
        p = wl.params
        o = oracle.Oracle(wl.robot, wl.world, p)
        ocmd, omu, osig, ost, obest = o.step(states[i], goals[i], 0, np.zeros((p.H, wl.robot.dof)),
                                             np.full(wl.robot.dof, f32(p.sigma_init)))
        tol = mu_tolerance([obest], p.beta)
        scale = max(1.0, np.abs(omu).max())
        assert max_rel(dists[i][0], omu, scale) < tol, (i, wl.name)
        assert max_rel(cmds[i], ocmd, scale) < tol, (i, wl.name)
        assert max_rel(dists[i][1], osig, max(1e-3, osig.max())) < tol, (i, wl.name)


def test_batch_autotune_keeps_results():
    wls = _batch(6, seed=3)
    states = [f32(wl.state) for wl in wls]
    goals = np.stack([f32(wl.goal) for wl in wls])
    args = ([w.robot for w in wls], [w.world for w in wls], [w.params for w in wls])
    with BatchController(*args) as b:
        ref, _ = b.step(states, goals)
    with BatchController(*args) as b:
        t = b.autotune()
        assert 0 < t < 1e5
        items, threads = b.get_launch()
        if b.launch_mapping() == "cta":
            assert items in (32, 48, 64, 96, 128) and threads in (128, 256, 512)
        else:
            assert items == threads and threads in (32, 64, 128, 256)
        got, _ = b.step(states, goals)
    for x, y in zip(ref, got):
        assert np.array_equal(x, y)


def test_batch_mappings_bitwise_identical():
    """The CTA-tile and warp-task mappings of the batched rollout, at several
    shapes, give the same commands and distributions bit for bit."""
    wls = _batch(9, seed=4)
    # short horizons too, so that the warp mapping packs 2 and 4 particles per warp
    for i, h in ((0, 6), (1, 8), (2, 12)):
        p = wls[i].params
        wls[i].params = p.replace(H=h, dt=np.full(h, 0.02))
    states = [f32(wl.state) for wl in wls]
    goals = np.stack([f32(wl.goal) for wl in wls])
    args = ([w.robot for w in wls], [w.world for w in wls], [w.params for w in wls])
    runs = []
    for shape in (("warp", 4), ("cta", 64, 256), ("warp", 1), ("warp", 8), ("cta", 32, 128)):
        with BatchController(*args) as b:
            assert b.launch_mapping() == "warp"
            if shape[0] == "warp":
                b.set_launch_warp(shape[1])
            else:
                b.set_launch(shape[1], shape[2])
            assert b.launch_mapping() == shape[0]
            cmds = [b.step(states, goals)[0] for _ in range(2)]
            runs.append((cmds, [b.get_distribution(i) for i in range(len(wls))]))
    for cmds, dists in runs[1:]:
        for t in range(2):
            for x, y in zip(cmds[t], runs[0][0][t]):
                assert np.array_equal(x, y)
        for (m, s), (m0, s0) in zip(dists, runs[0][1]):
            assert np.array_equal(m, m0) and np.array_equal(s, s0)


def test_batch_launch_shapes_are_validated():
    wls = _batch(2, seed=5)
    with BatchController([w.robot for w in wls], [w.world for w in wls], [w.params for w in wls]) as b:
        for bad in (0, 9):
            with pytest.raises(StormError):
                b.set_launch_warp(bad)
        for items, threads in ((0, 128), (64, 48), (64, 1024)):
            with pytest.raises(StormError):
                b.set_launch(items, threads)
        assert b.launch_mapping() == "warp"


def test_full_size_batch_runs():
    wls = W.config_batch(0, 256)
    states = [f32(wl.state) for wl in wls]
    goals = np.stack([f32(wl.goal) for wl in wls])
    with BatchController([w.robot for w in wls], [w.world for w in wls],
                         [w.params for w in wls]) as b:
        cmds, st = b.step(states, goals)
        cmds2, st2 = b.step(states, goals)
        # spot-check three instances against their own handles
        for i in (0, 97, 255):
            wl = wls[i]
            with Controller(wl.robot, wl.world, wl.params) as c:
                r1 = c.step(states[i], goals[i])[0]
                r2 = c.step(states[i], goals[i])[0]
            assert np.array_equal(cmds[i], r1) and np.array_equal(cmds2[i], r2)
    assert len(cmds) == 256 and all(np.all(np.isfinite(c)) for c in cmds)


def test_full_size_batch_matches_oracle():
    """The 256-instance uneven batch at its drawn sizes (N up to 1024, H up to 50,
    6 and 7 joints, 0 to 64 obstacles), stepped once as one batch, against the
    oracle's control step of a spread of its instances: the largest N x H, the
    largest N and H, both joint counts, the most and the fewest obstacles, and
    the smallest N."""
    wls = W.config_batch(0, 256)
    states = [f32(wl.state) for wl in wls]
    goals = np.stack([f32(wl.goal) for wl in wls])
    with BatchController([w.robot for w in wls], [w.world for w in wls],
                         [w.params for w in wls]) as b:
        cmds, st = b.step(states, goals)
        dists = [b.get_distribution(i) for i in range(len(wls))]
    assert all(s == 0 for s in st)
    size = [wl.params.N * wl.params.H for wl in wls]
    n_obs = [len(wl.world.boxes) + len(wl.world.spheres) for wl in wls]
    dof = [wl.robot.dof for wl in wls]
    pick = {int(np.argmax(size)), int(np.argmax([wl.params.N for wl in wls])),
            int(np.argmax([wl.params.H for wl in wls])), int(np.argmax(n_obs)), int(np.argmin(n_obs)),
            int(np.argmin([wl.params.N for wl in wls])),
            next(i for i in range(len(wls)) if dof[i] == 6), next(i for i in range(len(wls)) if dof[i] == 7)}
    picked = [wls[i] for i in sorted(pick)]
    assert max(w.params.N for w in picked) >= 1000 and max(w.params.H for w in picked) >= 48
    assert {w.robot.dof for w in picked} == {6, 7} and max(n_obs[i] for i in pick) >= 60
    for i in sorted(pick):
        wl, p = wls[i], wls[i].params
        o = oracle.Oracle(wl.robot, wl.world, p)
        ocmd, omu, osig, ost, obest = o.step(states[i], goals[i], 0, np.zeros((p.H, wl.robot.dof)),
                                             np.full(wl.robot.dof, f32(p.sigma_init)))
        assert ost == 0
        tol = mu_tolerance([obest], p.beta)
        scale = max(1.0, np.abs(omu).max())
        assert max_rel(dists[i][0], omu, scale) < tol, (i, wl.name)
        assert max_rel(cmds[i], ocmd, scale) < tol, (i, wl.name)
        assert max_rel(dists[i][1], osig, max(1e-3, osig.max())) < tol, (i, wl.name)
