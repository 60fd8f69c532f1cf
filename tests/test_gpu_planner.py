"""GPU planner (mrpop_plan): every returned path is re-validated by the FP64
oracle at a quarter of the planning resolution, its reported cost equals the
summed segment lengths C(sigma) (Sec. III-A), it runs from q_start to q_goal,
and the incumbent costs decrease strictly over time (Alg. 1; Lem. C1: a
connection is accepted only below c_best).  Trajectories themselves are not
compared: the planner is randomised."""
import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree

from paper_2609_30644_gb300 import synth

pytestmark = pytest.mark.gpu
RES = 0.02


@pytest.fixture(scope="module")
def mp():
    import paper_2609_30644_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return m


def _robot_connected(orc, scene, k, qs, qg, n=1500, delta=0.8, self_collision=False):
    """Dense FP64 PRM of robot k alone (oracle checks): are its start and goal
    in one free-space component?  Joint limits without wrap-around can split
    free space, so a random start/goal pair may have no path at all."""
    sub = synth.Scene([scene.robots[k]], scene.obs_spheres, scene.obs_cuboids)
    o = orc.OracleScene(sub, self_collision=self_collision)
    r = scene.robots[k]
    off = sum(rr.dof for rr in scene.robots[:k])
    rng = np.random.default_rng(k)
    samp = rng.uniform(r.q_lo, r.q_hi, (n, r.dof)).astype(np.float32)
    keep = [q for q in samp if o.config_valid(q, 2e-4)[0]]
    V = np.array([qs[off:off + r.dof], qg[off:off + r.dof]] + keep, np.float32)
    pairs = np.array(sorted(cKDTree(V).query_pairs(delta)))
    res = o.validate_edges(np.ascontiguousarray(V[pairs[:, 0]].T),
                           np.ascontiguousarray(V[pairs[:, 1]].T), RES, 2e-4, early_exit=True)
    adj = [[] for _ in range(len(V))]
    for (a, b), v in zip(pairs, res["valid"]):
        if v:
            adj[a].append(b)
            adj[b].append(a)
    seen, st = {0}, [0]
    while st:
        for w in adj[st.pop()]:
            if w not in seen:
                seen.add(w)
                st.append(w)
    return 1 in seen


def _start_goal(orc, scene, seed, margin=1e-4, delta=0.8, check=True):
    """Collision-free start/goal (oracle, with clearance above the margin)
    whose robots each connect start and goal in a dense oracle PRM."""
    o = orc.OracleScene(scene)
    stream = synth.config_stream(scene, seed)
    ok = lambda q: o.config_valid(q, margin + 1e-3)[0]
    for _ in range(20):
        qs, qg = synth.first_accepted(stream, ok), synth.first_accepted(stream, ok)
        if not check or all(_robot_connected(orc, scene, k, qs, qg, delta=delta)
                            for k in range(scene.K)):
            return qs, qg, o
    raise AssertionError("no feasible start/goal pair found")


def _check_path(orc, o, path, cost, qs, qg):
    assert path is not None and path.shape[0] >= 2
    np.testing.assert_array_equal(path[0], qs)
    np.testing.assert_array_equal(path[-1], qg)
    ok, bad = o.path_valid(path, RES / 4, 0.0)
    assert ok, f"segment {bad} invalid at res/4"
    assert cost == pytest.approx(orc.path_cost(path), rel=1e-5)
    assert cost >= np.linalg.norm(qg.astype(float) - qs.astype(float)) - 1e-6


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plan_planar_pair(mp, orc, seed):
    scene = synth.planar_pair_scene(seed)
    qs, qg, o = _start_goal(orc, scene, seed)
    with mp.Problem(scene, resolution=RES, margin=1e-4, delta=0.8, n_per_round=64,
                    tree_cap=1 << 16, roadmap_cap=1 << 14, max_iters=4096, seed=seed,
                    start=qs, goal=qg) as p:
        path, cost = mp.plan(p, 2.0)
        t, c, iters = mp.plan_trace(p)
    _check_path(orc, o, path, cost, qs, qg)
    assert len(c) >= 1 and c[-1] == pytest.approx(cost)
    assert np.all(np.diff(c) < 0), "incumbents must decrease strictly"
    assert np.all(np.diff(t) >= 0) and iters > 0


def test_plan_reassigned_fine_stage(mp, orc):
    """The planner's batched validation launches with the reassigned fine
    stage: the returned path is oracle-valid at res/4."""
    scene = synth.planar_pair_scene(0)
    qs, qg, o = _start_goal(orc, scene, 0)
    with mp.Problem(scene, resolution=RES, margin=1e-4, delta=0.8, n_per_round=64,
                    tree_cap=1 << 16, roadmap_cap=1 << 14, max_iters=4096, seed=5,
                    start=qs, goal=qg) as p:
        mp.set_launch(p, 0, 0, 1)
        path, cost = mp.plan(p, 1.5)
    _check_path(orc, o, path, cost, qs, qg)


def test_plan_with_self_collision(mp, orc):
    """Planning with self-collision on (default adjacency mask): the returned
    path is valid for the self-colliding oracle at res/4."""
    scene = synth.planar_pair_scene(0)
    o = orc.OracleScene(scene, self_collision=True)
    stream = synth.config_stream(scene, 0)
    ok = lambda q: o.config_valid(q, 1e-4 + 1e-3)[0]
    for _ in range(20):
        qs, qg = synth.first_accepted(stream, ok), synth.first_accepted(stream, ok)
        if all(_robot_connected(orc, scene, k, qs, qg, delta=0.8, self_collision=True)
               for k in range(scene.K)):
            break
    with mp.Problem(scene, resolution=RES, margin=1e-4, delta=0.8, n_per_round=64,
                    tree_cap=1 << 16, roadmap_cap=1 << 14, max_iters=4096, seed=3,
                    start=qs, goal=qg, self_collision=True) as p:
        path, cost = mp.plan(p, 2.0)
    _check_path(orc, o, path, cost, qs, qg)


def test_plan_table_pair(mp, orc):
    scene = synth.table_pair_scene(0)
    qs, qg, o = _start_goal(orc, scene, 5, delta=2.5)
    with mp.Problem(scene, resolution=RES, margin=1e-4, delta=2.5, n_per_round=64,
                    tree_cap=1 << 16, roadmap_cap=1 << 14, max_iters=4096, seed=3,
                    start=qs, goal=qg) as p:
        path, cost = mp.plan(p, 4.0)
        t, c, _ = mp.plan_trace(p)
    _check_path(orc, o, path, cost, qs, qg)
    assert np.all(np.diff(c) < 0)


def test_plan_continues_and_improves(mp, orc):
    """A second call continues from the device-resident state: the incumbent
    never gets worse (Alg. 1 keeps c_best)."""
    scene = synth.planar_pair_scene(4)
    qs, qg, o = _start_goal(orc, scene, 4)
    with mp.Problem(scene, resolution=RES, margin=1e-4, delta=0.8, seed=9, start=qs, goal=qg) as p:
        _, c1 = mp.plan(p, 1.0)
        path, c2 = mp.plan(p, 1.0)
    assert c2 <= c1
    _check_path(orc, o, path, c2, qs, qg)


def test_plan_rejects_colliding_start(mp, orc):
    scene = synth.table_pair_scene(0)
    o = orc.OracleScene(scene)
    stream = synth.config_stream(scene, 77)
    bad = synth.first_accepted(stream, lambda q: not o.config_valid(q, 0.0)[0])
    good = synth.first_accepted(stream, lambda q: o.config_valid(q, 1e-3)[0])
    with mp.Problem(scene, start=bad, goal=good) as p:
        with pytest.raises(mp.MrpopError) as ei:
            mp.plan(p, 0.5)
    assert ei.value.status == 1


def test_plan_obstacle_free_converges_to_straight_line(mp):
    """Far-apart planar arms without obstacles: C* = |q_goal - q_start| (the
    straight line is free).  The incumbent must approach it (Thm. 1)."""
    scene = synth.planar_pair_scene(0)
    scene.robots[0].base[3] = -2.0
    scene.robots[1].base[3] = 2.0
    scene = synth.Scene(scene.robots, np.zeros((0, 4), np.float32), np.zeros((0, 15), np.float32))
    rng = np.random.default_rng(3)
    qs = rng.uniform(-2.5, 2.5, 6).astype(np.float32)
    qg = rng.uniform(-2.5, 2.5, 6).astype(np.float32)
    cstar = float(np.linalg.norm(qg.astype(float) - qs.astype(float)))
    with mp.Problem(scene, delta=0.8, seed=1, start=qs, goal=qg) as p:
        path, cost = mp.plan(p, 3.0)
    assert cost >= cstar - 1e-6
    assert cost <= 1.5 * cstar, (cost, cstar)


def _planar_problem(mp, orc, seed, **kw):
    scene = synth.planar_pair_scene(seed)
    qs, qg, o = _start_goal(orc, scene, seed)
    p = mp.Problem(scene, resolution=RES, margin=1e-4, delta=0.8, n_per_round=64,
                   tree_cap=1 << 15, roadmap_cap=1 << 13, max_iters=4096, seed=seed,
                   start=qs, goal=qg, **kw)
    return p, qs, qg, o


def test_plan_batch_paths_valid(mp, orc):
    """Four problems planned together: every result is oracle-valid."""
    probs = [_planar_problem(mp, orc, s) for s in (0, 2, 3, 6)]
    st = mp.plan_batch([p for p, *_ in probs], 3.0)
    assert (st == 0).all()
    for p, qs, qg, o in probs:
        path, cost = mp.plan_result(p)
        _check_path(orc, o, path, cost, qs, qg)
        _, c, _ = mp.plan_trace(p)
        assert np.all(np.diff(c) < 0)
        p.close()


def test_plan_batch_alone_equals_mix(mp, orc):
    """The same problem, same seed and same number of steps gives exactly the
    same path and cost alone and in a mix with other problems."""
    steps = 40
    a, *_ = _planar_problem(mp, orc, 2)
    mp.plan_batch([a], 60.0, max_steps=steps)
    alone = mp.plan_result(a)
    a.close()
    a2, *_ = _planar_problem(mp, orc, 2)
    # partners of another size (14-DOF, other tables) change the shared launch
    # configuration of the batch, not the result
    table = synth.table_pair_scene(0)
    tqs, tqg, _ = _start_goal(orc, table, 5, check=False)
    big = mp.Problem(table, resolution=RES, margin=1e-4, delta=2.5, seed=1, start=tqs, goal=tqg)
    others = [_planar_problem(mp, orc, 0)[0], big]
    mp.plan_batch([others[0], a2, others[1]], 60.0, max_steps=steps)
    mixed = mp.plan_result(a2)
    assert alone[0] is not None
    np.testing.assert_array_equal(alone[0], mixed[0])
    assert alone[1] == mixed[1]
    for p in [a2] + others:
        p.close()


def test_plan_batch_stepped_form(mp, orc):
    """The stepped batch form (a captured graph per step, host bookkeeping
    between steps) on the same kind of batch: every result is oracle-valid."""
    probs = [_planar_problem(mp, orc, s) for s in (0, 3)]
    st = mp.plan_batch([p for p, *_ in probs], 3.0, form=mp.BATCH_STEPPED)
    assert (st == 0).all()
    for p, qs, qg, o in probs:
        path, cost = mp.plan_result(p)
        _check_path(orc, o, path, cost, qs, qg)
        p.close()


def test_plan_batch_persistent_heterogeneous(mp, orc):
    """One persistent launch over problems of different robot counts and
    dimensions (planar 6-DOF, single-robot, two 7-DOF arms, four arms):
    whatever each found is oracle-valid at res/4, its incumbents decrease,
    and a second call continues from the device state."""
    probs = [_planar_problem(mp, orc, s) for s in (0, 6)]
    table = synth.table_pair_scene(0)
    tqs, tqg, to = _start_goal(orc, table, 5, check=False)
    probs.append((mp.Problem(table, resolution=RES, margin=1e-4, delta=2.5, seed=3,
                             start=tqs, goal=tqg), tqs, tqg, to))
    arm = synth.Scene([table.robots[0]], table.obs_spheres, table.obs_cuboids)
    aqs, aqg, ao = _start_goal(orc, arm, 3, check=False)
    probs.append((mp.Problem(arm, resolution=RES, margin=1e-4, delta=0.6, seed=4,
                             start=aqs, goal=aqg), aqs, aqg, ao))
    ps = [p for p, *_ in probs]
    st = mp.plan_batch(ps, 4.0)
    assert (st == 0).all()
    st = mp.plan_batch(ps, 2.0)
    assert (st == 0).all()
    solved = 0
    for p, qs, qg, o in probs:
        path, cost = mp.plan_result(p)
        t, c, _ = mp.plan_trace(p)
        if path is not None:
            solved += 1
            _check_path(orc, o, path, cost, qs, qg)
            assert c[-1] == pytest.approx(cost)
            # (times count from the start of the call that found each incumbent)
            assert np.all(np.diff(c) < 0) and np.all(t >= 0)
        p.close()
    assert solved >= 3


def test_plan_batch_bounded_wait_times_out(mp, orc):
    """The persistent launch's only wait is a CTA polling for work.  With
    more CTAs than the problem has chunks and a poll limit of four, idle CTAs
    give up: the call reports MRPOP_ETIMEOUT instead of waiting, whatever was
    found stays valid, and the context and the planner keep working."""
    p, qs, qg, o = _planar_problem(mp, orc, 0)
    mp.set_persistent_limits(ctas=16, idle_polls=4)
    try:
        with pytest.raises(mp.MrpopError) as ei:
            mp.plan_batch([p], 2.0, max_steps=60)
        assert ei.value.status == 5          # MRPOP_ETIMEOUT
    finally:
        mp.set_persistent_limits(0, 0)
    path, cost = mp.plan_result(p)
    if path is not None:
        _check_path(orc, o, path, cost, qs, qg)
    st = mp.plan_batch([p], 2.0)
    assert (st == 0).all()
    path, cost = mp.plan_result(p)
    _check_path(orc, o, path, cost, qs, qg)
    p.close()


def test_plan_batch_stops_at_target(mp, orc):
    p, qs, qg, o = _planar_problem(mp, orc, 3)
    st = mp.plan_batch([p], 5.0, targets=[1e9])   # any solution reaches the target
    path, cost = mp.plan_result(p)
    t, c, _ = mp.plan_trace(p)
    assert len(c) == 1 and t[0] < 1.0
    _check_path(orc, o, path, cost, qs, qg)
    p.close()


@pytest.mark.parametrize("kind", ["planar", "spatial"])
def test_plan_single_robot_direct(mp, orc, kind):
    """K = 1 skips the roadmap and plans directly in configuration space
    (Sec. V-C); the result obeys the same checks."""
    if kind == "planar":
        base = synth.planar_pair_scene(2)
        delta = 0.8
    else:
        base = synth.table_pair_scene(0)
        delta = 1.0
    scene = synth.Scene([base.robots[0]], base.obs_spheres, base.obs_cuboids)
    qs, qg, o = _start_goal(orc, scene, 3, delta=max(delta, 0.8 if kind == "planar" else 2.5))
    with mp.Problem(scene, resolution=RES, margin=1e-4, delta=delta, seed=2, start=qs, goal=qg) as p:
        path, cost = mp.plan(p, 2.0)
        t, c, it = mp.plan_trace(p)
        hist = [mp.plan_history(p, k) for k in range(len(c))]
    _check_path(orc, o, path, cost, qs, qg)
    assert np.all(np.diff(c) < 0)
    # every recorded incumbent is itself a valid path with its recorded cost
    for (hp, hc), ck in zip(hist, c):
        assert hc == ck
        _check_path(orc, o, hp, hc, qs, qg)
    np.testing.assert_array_equal(hist[-1][0], path)


def test_plan_planar_within_2000_iterations(mp, orc):
    """The planar pair's iteration budget: a solution within 2,000 search
    iterations (steps that only grow roadmaps do not count), oracle-valid at
    res/4.  Runs are deterministic for a seed."""
    scene = synth.planar_pair_scene(1)
    qs, qg, o = _start_goal(orc, scene, 1)
    with mp.Problem(scene, resolution=RES, margin=1e-4, delta=0.8, n_per_round=64,
                    tree_cap=1 << 16, roadmap_cap=1 << 14, max_iters=4096, seed=1,
                    start=qs, goal=qg) as p:
        for _ in range(200):
            mp.plan_batch([p], 60.0, max_steps=1)
            if mp.plan_trace(p)[2] >= 2000:
                break
        t, c, iters = mp.plan_trace(p)
        path, cost = mp.plan_result(p)
    assert iters <= 2048 and len(c) >= 1
    _check_path(orc, o, path, cost, qs, qg)


def test_plan_grid4(mp, orc):
    """Four 7-DOF arms over a shared cube (28-DOF) with 128 obstacles: a path
    within a 2 s budget (the workload allows 10 s), oracle-valid at res/4."""
    scene = synth.grid4_scene(0)
    o = orc.OracleScene(scene)
    stream = synth.config_stream(scene, 0)
    ok = lambda q: o.config_valid(q, 2e-3)[0]
    qs, qg = synth.first_accepted(stream, ok), synth.first_accepted(stream, ok)
    with mp.Problem(scene, resolution=RES, margin=1e-4, delta=2.5, n_per_round=64,
                    tree_cap=1 << 16, roadmap_cap=1 << 13, max_iters=4096, seed=1,
                    start=qs, goal=qg) as p:
        path, cost = mp.plan(p, 2.0)
        t, c, iters = mp.plan_trace(p)
    assert np.all(np.diff(c) < 0)
    _check_path(orc, o, path, cost, qs, qg)


# ----------------------------------------------------------------------------
# the planner's own NEAREST and NEIGHBORS kernels against the oracle
# ----------------------------------------------------------------------------

def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("pass_", [0, 1])
@pytest.mark.parametrize("D,N", [(14, 3000), (28, 1500), (7, 257), (21, 1)])
def test_planner_nearest_kernel_parity(mp, orc, D, N, pass_):
    """k_nearest (both passes of a search step) on a tree with duplicated
    vertices, queries placed exactly on vertices (exact ties: lowest g, then
    lowest index), unbounded, tight and empty budgets: indices equal the
    oracle's, with the primitives' allowance for genuine FP32/FP64 near-ties."""
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree(D, N, lo, hi, seed=60 + D, dup_frac=0.1)
    Q = 256
    qs, cs = synth.nn_queries(D, Q, lo, hi, seed=70 + D, budget_lo=0.0, budget_hi=25.0)
    k = min(N, 48)
    qs[:, :k] = tree[:D, :k]                       # on (duplicated) vertices
    cs[200:216] = np.inf                           # unbounded
    cs[216:232] = -1.0                             # nothing admissible
    got = mp.planner_nearest_pass(_dev(tree), _dev(qs), _dev(cs), pass_).cpu().numpy()
    assert (got[216:232] == -1).all()
    ties = 0
    for i in range(Q):
        ref, bd, sd, gap = orc.nearest(tree, qs[:, i], cs[i])
        if got[i] == ref:
            continue
        scale = max(1.0, abs(float(cs[i])) if np.isfinite(cs[i]) else 1.0)
        assert (np.isfinite(sd) and sd - bd <= 1e-5 * max(bd, 1e-30)) or gap <= 1e-5 * scale, \
            (i, got[i], ref, bd, sd, gap)
        ties += 1
    assert ties <= 3
    # fewer queries than a step holds: the rest of the step is padding
    part = mp.planner_nearest_pass(_dev(tree), _dev(qs[:, :37]), _dev(cs[:37]), pass_)
    np.testing.assert_array_equal(part.cpu().numpy(), got[:37])


@pytest.mark.parametrize("dof,N,Q,delta", [(7, 3000, 300, 2.5), (7, 500, 64, 1.2),
                                           (3, 40, 33, 10.0), (16, 2000, 100, 6.0)])
def test_planner_neighbors_kernel_parity(mp, orc, dof, N, Q, delta):
    """k_rmb_neighbors on a roadmap: ascending indices within delta, capped at
    64 per vertex (the roadmap degree cap; the rest of the row -1), and the
    full count, against the oracle's radius query.  Queries sitting on
    vertices and duplicated vertices are included."""
    rng = np.random.default_rng(dof + N)
    V = rng.uniform(-2.9, 2.9, (dof, N)).astype(np.float32)
    V[:, N // 2:N // 2 + 8] = V[:, :8]              # duplicated vertices
    qs = rng.uniform(-2.9, 2.9, (dof, Q)).astype(np.float32)
    qs[:, :8] = V[:, :8]
    idx, cnt = mp.planner_neighbors_pass(_dev(V), _dev(qs), delta)
    idx, cnt = idx.cpu().numpy(), cnt.cpu().numpy()
    tree = np.vstack([V, np.zeros((1, N), np.float32)])   # g row: ignored
    cap = mp.ROADMAP_DEGREE_CAP
    for i in range(Q):
        ref, rc, gap = orc.neighbors(tree, qs[:, i], np.float32(delta), cap, dims=dof)
        if gap > 1e-5 * delta:
            assert cnt[i] == rc, (i, cnt[i], rc)
            np.testing.assert_array_equal(idx[i, :len(ref)], ref)
        else:
            assert abs(int(cnt[i]) - rc) <= 2
        kept = min(int(cnt[i]), cap)
        assert (np.diff(idx[i, :kept]) > 0).all()
        assert (idx[i, kept:] == -1).all()
    if N > 2 * cap and delta >= 5:           # the cap is exercised on the wide radius
        assert cnt.max() > cap


def test_plan_batch_phase_stats(mp, orc):
    """The persistent launch accounts its CTA time by phase kind: ROADMAP and
    search phases both ran, chunk counts are positive where time is, and the
    busy time fits in the launch's CTA time."""
    probs = [_planar_problem(mp, orc, s)[0] for s in (0, 1)]
    mp.plan_batch(probs, 2.0, max_steps=40)
    st = mp.plan_batch_phase_stats()
    busy = sum(st[k][0] for k in mp.PLAN_PHASE_NAMES)
    assert st["ctas"] > 0 and st["wall_ns"] > 0
    assert 0 < busy <= st["ctas"] * st["wall_ns"]
    for k in mp.PLAN_PHASE_NAMES:
        ns, n = st[k]
        assert n >= 0 and not (ns > 0 and n == 0)   # time only where chunks ran
    assert st["roadmap_edge_check"][1] > 0 and st["search_sample"][1] > 0
    assert st["phase_transitions"][1] > 0
    for p in probs:
        p.close()
