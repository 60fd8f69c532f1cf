"""The FP64 reference planner (oracle side, CPU): invariants of Alg. 1/2 that
hold for any correct run, determinism of its own random stream, and the
obstacle-free optimum of Thm. 1.  Its trajectories are not those of the GPU
planner (independent random streams); parity of the planner is unpinned and
rests on these invariants."""
import numpy as np
import pytest

from paper_2609_30644_gb300 import synth

RES = 0.02


def _start_goal(orc, scene, seed, margin=1e-4):
    o = orc.OracleScene(scene)
    stream = synth.config_stream(scene, seed)
    ok = lambda q: o.config_valid(q, margin + 2e-3)[0]
    return synth.first_accepted(stream, ok).astype(np.float64), \
        synth.first_accepted(stream, ok).astype(np.float64), o


def _plan(orc, scene, qs, qg, **kw):
    args = dict(resolution=RES, margin=1e-4, delta=0.8, n_per_round=64, max_iters=1000,
                round_budget=40, seed=1)
    args.update(kw)
    return orc.plan_reference(scene, qs, qg, **args)


@pytest.mark.parametrize("seed", [0, 3])   # seeds whose roadmaps connect (joint limits
def test_ref_planner_invariants(orc, seed):  # split the free space of some others)
    scene = synth.planar_pair_scene(seed)
    qs, qg, o = _start_goal(orc, scene, seed)
    r = _plan(orc, scene, qs, qg, iter_budget=2500, seed=seed)
    assert r["status"] == 0
    path, cost = r["path"], r["cost"]
    np.testing.assert_array_equal(path[0], qs)
    np.testing.assert_array_equal(path[-1], qg)
    # C(sigma): the summed segment lengths, in FP64
    segs = np.linalg.norm(np.diff(path, axis=0), axis=1)
    assert cost == pytest.approx(segs.sum(), rel=1e-12)
    assert cost >= np.linalg.norm(qg - qs) - 1e-12
    # the oracle re-validates the path at 4x finer resolution
    ok, bad = o.path_valid(path.astype(np.float32), RES / 4, 0.0)
    assert ok, bad
    # incumbents strictly decrease; times and iteration counts never go back
    c = r["costs"]
    assert len(c) >= 1 and c[-1] == cost
    assert (np.diff(c) < 0).all()
    assert (np.diff(r["times"]) >= 0).all() and (np.diff(r["trace_iters"]) >= 0).all()


def test_ref_planner_deterministic_and_prefix(orc):
    """Same seed, same iteration budget: identical runs; a shorter budget
    reproduces a prefix of the longer run's incumbents."""
    scene = synth.planar_pair_scene(2)
    qs, qg, _ = _start_goal(orc, scene, 2)
    a = _plan(orc, scene, qs, qg, iter_budget=2000)
    b = _plan(orc, scene, qs, qg, iter_budget=2000)
    assert a["status"] == 0
    np.testing.assert_array_equal(a["path"], b["path"])
    np.testing.assert_array_equal(a["costs"], b["costs"])
    np.testing.assert_array_equal(a["trace_iters"], b["trace_iters"])
    short = _plan(orc, scene, qs, qg, iter_budget=int(a["trace_iters"][0]))
    assert short["costs"][0] == a["costs"][0]


def test_ref_planner_obstacle_free_approaches_straight_line(orc):
    """Thm. 1 on far-apart planar arms without obstacles: C* = |q_goal -
    q_start|; the incumbent stays above it and comes within 20 %."""
    b1 = synth._yaw_base(-5.0, 0.0, 0.0, np.pi / 2)
    b2 = synth._yaw_base(5.0, 0.0, 0.0, np.pi / 2)
    scene = synth.Scene([synth.planar_arm(b1), synth.planar_arm(b2)],
                        np.zeros((0, 4), np.float32), np.zeros((0, 15), np.float32))
    rng = np.random.default_rng(3)
    qs, qg = rng.uniform(-2.0, 2.0, 6), rng.uniform(-2.0, 2.0, 6)
    cstar = np.linalg.norm(qg - qs)
    r = _plan(orc, scene, qs, qg, iter_budget=3000, seed=2)
    assert r["status"] == 0
    assert cstar - 1e-12 <= r["cost"] <= 1.2 * cstar


def test_ref_planner_single_robot_and_errors(orc):
    scene = synth.planar_pair_scene(0)
    one = synth.Scene([scene.robots[0]], scene.obs_spheres, scene.obs_cuboids)
    qs, qg, o = _start_goal(orc, one, 4)
    r = _plan(orc, one, qs, qg, iter_budget=2000)
    assert r["status"] == 0
    assert o.path_valid(r["path"].astype(np.float32), RES / 4, 0.0)[0]
    # a start in collision is an error; so is a call without any budget
    rng = np.random.default_rng(11)
    bad = qs.copy()
    while o.config_valid(bad, 1e-4)[0]:
        bad = rng.uniform(-np.pi, np.pi, 3)
    assert _plan(orc, one, bad, qg, iter_budget=10)["status"] == -1
    assert _plan(orc, one, qs, qg)["status"] == -1
