"""GPU parity of forward kinematics and motion validation against the FP64
oracle, through the C ABI.

Tolerances (stated by the method's target, derived for FP32):
  * sphere centres and clearances: |gpu - oracle| <= 1e-5 * (1 + |oracle|)
    (FP32 distances within 1e-5 relative at the ~1 m workspace scale);
  * verdicts: bit-exact for every edge whose oracle minimum clearance lies
    outside [margin - 1e-4, margin + 1e-4] m (the contact band, where FP32
    and FP64 may legitimately disagree);
  * interval counts: bit-exact (an integer both sides decide in FP32).
"""
import numpy as np
import pytest
import torch

from paper_2609_30644_gb300 import synth

pytestmark = pytest.mark.gpu

BAND = 1e-4
REL = 1e-5


@pytest.fixture(scope="module")
def mp():
    import paper_2609_30644_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return m


SCENES = {
    "planar_pair": lambda: synth.planar_pair_scene(0),
    "table_pair": lambda: synth.table_pair_scene(0),
    "grid4": lambda: synth.grid4_scene(0),
}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_verdicts(valid_gpu, ref, margin, report=None, label=""):
    """Bit-exact verdicts outside the contact band; the band itself is a thin
    shell of the clearance range, so it may hold only a few edges of a batch
    (at most 3, or 2 % of a large batch).  Returns the in-band count; with a
    report list, also records how the GPU decided the in-band edges: 'toward
    collision' (GPU rejects an edge the oracle accepts) or 'toward free'."""
    valid_gpu = np.asarray(valid_gpu).astype(np.uint8)
    inband = np.abs(ref["min_clear"] - margin) <= BAND
    bad = (valid_gpu != ref["valid"]) & ~inband
    assert not bad.any(), f"{bad.sum()} verdict mismatches outside the contact band: {np.nonzero(bad)[0][:10]}"
    n_in = int(inband.sum())
    assert n_in <= max(3, 0.02 * valid_gpu.size), f"{n_in} of {valid_gpu.size} edges in the band"
    if report is not None:
        to_coll = int((inband & (valid_gpu == 0) & (ref["valid"] == 1)).sum())
        to_free = int((inband & (valid_gpu == 1) & (ref["valid"] == 0)).sum())
        report.append(f"{label}: margin {margin:g} m, {valid_gpu.size} edges, {n_in} in band, "
                      f"differing toward collision {to_coll}, toward free {to_free}")
    return n_in


@pytest.mark.parametrize("name", list(SCENES))
def test_fk_parity(mp, orc, name):
    scene = SCENES[name]()
    o = orc.OracleScene(scene)
    rng = np.random.default_rng(0)
    q = synth.uniform_configs(scene, 257, rng)
    with mp.Problem(scene) as p:
        out = mp.fk(p, _dev(q)).cpu().numpy()
    for i in range(0, 257, 16):
        ref = o.fk(q[:, i])
        got = out[:, :, i].T
        err = np.abs(got - ref[:, :3])
        assert (err <= REL * (1 + np.abs(ref[:, :3]))).all(), err.max()


@pytest.mark.parametrize("name,n_edges", [("planar_pair", 300), ("table_pair", 160), ("grid4", 40)])
def test_clearance_parity(mp, orc, name, n_edges):
    scene = SCENES[name]()
    o = orc.OracleScene(scene)
    qa, qb = synth.candidate_edges(scene, n_edges, seed=5, step_hi=1.5)
    ref = o.validate_edges(qa, qb, 0.02, 0.0, early_exit=False)
    with mp.Problem(scene, resolution=0.02) as p:
        got = mp.edge_clearance(p, _dev(qa), _dev(qb)).cpu().numpy().astype(np.float64)
    err = np.abs(got - ref["min_clear"])
    assert (err <= REL * (1 + np.abs(ref["min_clear"]))).all(), err.max()


@pytest.mark.parametrize("margin", [0.0, 1e-4, 0.02])
@pytest.mark.parametrize("name,n_edges", [("planar_pair", 600), ("table_pair", 300), ("grid4", 60)])
def test_verdict_parity(mp, orc, band_report, name, n_edges, margin):
    """Mixed candidate edges, long enough to span several 32-point tiles with
    ragged tails (step up to 3 rad)."""
    scene = SCENES[name]()
    o = orc.OracleScene(scene)
    qa, qb = synth.candidate_edges(scene, n_edges, seed=11, step_hi=3.0)
    ref = o.validate_edges(qa, qb, 0.02, margin, early_exit=False)
    assert ref["npoints"].max() >= 64            # several tiles
    assert 0 < ref["valid"].sum() < n_edges      # a real mix
    with mp.Problem(scene, resolution=0.02, margin=margin) as p:
        n = qa.shape[1]
        valid = torch.empty(n, dtype=torch.uint8, device="cuda")
        length = torch.empty(n, dtype=torch.float32, device="cuda")
        npts = torch.empty(n, dtype=torch.int32, device="cuda")
        mp.validate_edges(p, _dev(qa), _dev(qb), valid, length, npts)
        v = valid.cpu().numpy()
        np.testing.assert_array_equal(npts.cpu().numpy(), ref["npoints"])
        L = np.linalg.norm(qb.astype(np.float64) - qa.astype(np.float64), axis=0)
        np.testing.assert_allclose(length.cpu().numpy(), L, rtol=1e-6, atol=1e-7)
        # repeated launches reuse the self-resetting work counter
        v2 = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
        np.testing.assert_array_equal(v, v2)
        # the reassigned fine stage (load-proportional work items)
        mp.set_launch(p, 0, 0, 1)
        v3 = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
    _check_verdicts(v, ref, margin, band_report, f"{name} union")
    _check_verdicts(v3, ref, margin, band_report, f"{name} reassigned")


def test_verdict_matches_gpu_clearance(mp):
    """Culling never changes a verdict: the culled early-exit kernel agrees
    with the unculled full-clearance kernel wherever FP32 itself is decided."""
    scene = synth.table_pair_scene(1)
    qa, qb = synth.candidate_edges(scene, 8192, seed=13)
    with mp.Problem(scene, margin=1e-4) as p:
        v = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
        c = mp.edge_clearance(p, _dev(qa), _dev(qb)).cpu().numpy()
    decided = np.abs(c - 1e-4) > 1e-6
    np.testing.assert_array_equal(v[decided], (c[decided] >= 1e-4).astype(np.uint8))


def test_full_size_batch_sampled(mp, orc, band_report):
    """65,536-edge batch of the 2 x 7-DOF table scene in the benchmark's launch
    configuration; a seeded sample of edges is re-checked by the oracle, at the
    kernel's margin and (the planner's safety property) at margin 0."""
    scene = synth.table_pair_scene(0)
    qa, qb = synth.candidate_edges(scene, 65536, seed=0)
    with mp.Problem(scene, resolution=0.02, margin=1e-4) as p:
        v = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(65536, 256, replace=False))
    o = orc.OracleScene(scene)
    ref = o.validate_edges(qa[:, idx], qb[:, idx], 0.02, 1e-4, early_exit=False)
    _check_verdicts(v[idx], ref, 1e-4, band_report, "table_pair 65,536-edge batch, sample")
    assert 0.2 < v.mean() < 0.8
    ref0 = o.validate_edges(qa[:, idx], qb[:, idx], 0.02, 0.0, early_exit=False)
    unsafe = (v[idx] == 1) & (ref0["valid"] == 0)
    assert not unsafe.any(), f"GPU accepted at 1e-4 what the oracle rejects at 0: {idx[unsafe]}"


def _eight_arm_scene():
    for i in range(40):
        sc = synth.batched_scene(i)
        if sc.K >= 7:
            return sc
    raise AssertionError("no batched scene with 7 or more arms")


SAFETY_CASES = {
    "planar_pair": (lambda: synth.planar_pair_scene(0), 600, dict(step_hi=3.0)),
    "table_pair": (lambda: synth.table_pair_scene(0), 300, dict(step_hi=3.0)),
    "grid4": (lambda: synth.grid4_scene(0), 60, dict(step_hi=3.0)),
    "eight_arm_batched": (_eight_arm_scene, 24, dict(step_lo=0.02, step_hi=0.2)),
}


@pytest.mark.parametrize("name", list(SAFETY_CASES))
def test_planner_margin_never_admits_a_collision(mp, orc, band_report, name):
    """The planner's safety property on the primitive itself.  The planner
    validates with margin 1e-4 m and its paths must pass the FP64 oracle at
    margin 0, so on every edge -- in the contact band included -- a GPU
    verdict 'free' at 1e-4 implies an oracle verdict 'free' at 0: FP32
    rounding (micrometres here) never exceeds the 1e-4 m of inflation.  The
    same batch is also compared at equal margins, where verdicts must be
    bit-exact outside the band and the in-band edges are counted by the
    direction in which the GPU differs."""
    make, n_edges, kw = SAFETY_CASES[name]
    scene = make()
    o = orc.OracleScene(scene)
    qa, qb = synth.candidate_edges(scene, n_edges, seed=19, **kw)
    ref0 = o.validate_edges(qa, qb, 0.02, 0.0, early_exit=False)
    ref1 = o.validate_edges(qa, qb, 0.02, 1e-4, early_exit=False)
    assert 0 < ref0["valid"].sum() < n_edges
    with mp.Problem(scene, resolution=0.02, margin=1e-4) as p:
        v1 = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
    with mp.Problem(scene, resolution=0.02, margin=0.0) as p:
        v0 = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
    unsafe = (v1 == 1) & (ref0["valid"] == 0)
    assert not unsafe.any(), f"GPU accepted at 1e-4 what the oracle rejects at 0: {np.nonzero(unsafe)[0]}"
    _check_verdicts(v1, ref1, 1e-4, band_report, f"{name} (safety batch)")
    _check_verdicts(v0, ref0, 0.0, band_report, f"{name} (safety batch)")


def test_edge_cases(mp, orc):
    scene = synth.table_pair_scene(0)
    o = orc.OracleScene(scene)
    rng = np.random.default_rng(3)
    with mp.Problem(scene) as p:
        # empty batch: no launch, no error
        z = torch.empty((p.D, 0), dtype=torch.float32, device="cuda")
        assert mp.validate_edges(p, z, z).numel() == 0
        # zero-length edges (n = 1, both checkpoints equal) and single edge
        q = synth.uniform_configs(scene, 33, rng)
        v = mp.validate_edges(p, _dev(q), _dev(q)).cpu().numpy()
        for i in range(33):
            assert v[i] == o.config_valid(q[:, i], 0.0)[0] or abs(o.config_valid(q[:, i])[1]) <= BAND
        v1 = mp.validate_edges(p, _dev(q[:, :1]), _dev(q[:, 1:2])).cpu().numpy()
        ref = o.validate_edges(q[:, :1], q[:, 1:2], 0.02, 0.0)
        _check_verdicts(v1, ref, 0.0)


def test_single_robot_and_obstacle_variants(mp, orc):
    """K = 1 (no robot-robot tests), no obstacles, cuboids only, and a link
    with 16 spheres (the per-link maximum)."""
    base = synth.table_pair_scene(0)
    arm = base.robots[0]
    big = synth.planar_arm(np.array([0, -1, 0, 0.1, 1, 0, 0, -0.2, 0, 0, 1, 0], np.float32),
                           spheres_per_link=16, radius=0.02)
    empty4 = np.zeros((0, 4), np.float32)
    empty15 = np.zeros((0, 15), np.float32)
    variants = [
        synth.Scene([arm], base.obs_spheres, base.obs_cuboids),
        synth.Scene(base.robots, empty4, empty15),
        synth.Scene(base.robots, empty4, base.obs_cuboids),
        synth.Scene([big, arm], base.obs_spheres, empty15),
    ]
    for sc in variants:
        o = orc.OracleScene(sc)
        qa, qb = synth.candidate_edges(sc, 120, seed=21, step_hi=2.0)
        ref = o.validate_edges(qa, qb, 0.02, 0.0)
        with mp.Problem(sc) as p:
            v = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
            c = mp.edge_clearance(p, _dev(qa), _dev(qb)).cpu().numpy().astype(np.float64)
        _check_verdicts(v, ref, 0.0)
        fin = ref["min_clear"] < 1e300
        assert np.all(np.abs(c[fin] - ref["min_clear"][fin]) <= REL * (1 + np.abs(ref["min_clear"][fin])))


def test_batched_scene_eight_arms(mp, orc):
    """Largest composite problem of the batched workload (up to 8 arms,
    56-DOF, hundreds of obstacles): fewer warps per block, same verdicts."""
    sc = _eight_arm_scene()
    o = orc.OracleScene(sc)
    qa, qb = synth.candidate_edges(sc, 24, seed=2, step_lo=0.02, step_hi=0.2)
    ref = o.validate_edges(qa, qb, 0.02, 0.0)
    with mp.Problem(sc) as p:
        v = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
    _check_verdicts(v, ref, 0.0)


def test_work_counters_structure(mp, orc):
    """Counters on edges the oracle finds valid (no early exit): every
    checkpoint is evaluated once, every tile bounds every link once and tests
    it against every obstacle (a cuboid first through its bounding sphere)
    and every earlier robot's link, and checkpoint tests never exceed their
    tile candidates."""
    scene = synth.table_pair_scene(0)
    o = orc.OracleScene(scene)
    qa, qb = synth.candidate_edges(scene, 400, seed=17, step_hi=0.3)
    ref = o.validate_edges(qa, qb, 0.02, 0.0)
    keep = np.nonzero((ref["valid"] == 1) & (ref["min_clear"] > 1e-3))[0][:64]
    assert keep.size >= 8
    qa, qb = np.ascontiguousarray(qa[:, keep]), np.ascontiguousarray(qb[:, keep])
    with mp.Problem(scene) as p:
        cnt = mp.validate_work(p, _dev(qa), _dev(qb)).cpu().numpy()
    npts = ref["npoints"][keep]
    pts = int((npts + 1).sum())
    tiles = int(((npts >> 5) + 1).sum())
    L = scene.D
    n_obs = len(scene.obs_spheres) + len(scene.obs_cuboids)
    assert cnt[0] == pts
    assert cnt[1] == pts * L
    NS, NC = len(scene.obs_spheres), len(scene.obs_cuboids)
    assert cnt[9] == tiles * L
    # tile level: every obstacle sphere and every cuboid's bounding sphere,
    # robot 1's links vs robot 0's 7; exact box tests where the sphere is near
    assert cnt[8] == tiles * (L * NS + L * NC + 7 * 7)
    assert 0 < cnt[11] <= tiles * L * NC
    assert cnt[2] <= pts * L * NS and cnt[10] <= pts * L * NC and cnt[3] <= pts * 7 * 7
    assert cnt[7] >= pts * L


def test_robot_robot_contact_spatial(mp, orc):
    """Two 7-DOF arms with bases 0.5 m apart and no obstacles: every verdict
    is decided by robot-robot sphere pairs (tile, link and sphere levels)."""
    scene = synth.table_pair_scene(0)
    scene.robots[0].base[7] = -0.25
    scene.robots[1].base[7] = 0.25
    scene = synth.Scene(scene.robots, np.zeros((0, 4), np.float32), np.zeros((0, 15), np.float32))
    o = orc.OracleScene(scene)
    qa, qb = synth.candidate_edges(scene, 400, seed=31, step_hi=1.0)
    ref = o.validate_edges(qa, qb, 0.02, 1e-4)
    assert 0.1 < ref["valid"].mean() < 0.9
    with mp.Problem(scene, margin=1e-4) as p:
        v = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
        c = mp.edge_clearance(p, _dev(qa), _dev(qb)).cpu().numpy().astype(np.float64)
        cnt = mp.validate_work(p, _dev(qa), _dev(qb)).cpu().numpy()
    _check_verdicts(v, ref, 1e-4)
    assert np.all(np.abs(c - ref["min_clear"]) <= REL * (1 + np.abs(ref["min_clear"])))
    assert cnt[6] > 0        # sphere-level robot-robot tests did run


def test_launch_configs_and_autotune_same_verdicts(mp, orc):
    """Every launch the autotuner may pick (warps per block, checkpoint order,
    union or reassigned fine tests) gives the same verdicts, also on edges
    long enough for many tiles."""
    scene = synth.table_pair_scene(0)
    qa, qb = synth.candidate_edges(scene, 4096, seed=41, step_hi=2.5)
    with mp.Problem(scene, margin=1e-4) as p:
        ref = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
        for w in (1, 2, 4):
            for order in (0, 1):
                for fine in (0, 1):
                    for regs in (0, 1):
                        mp.set_launch(p, w, order, fine, regs)
                        got = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
                        np.testing.assert_array_equal(got, ref)
        with pytest.raises(mp.MrpopError):
            mp.set_launch(p, 4, 0, 2)
        with pytest.raises(mp.MrpopError):
            mp.set_launch(p, 4, 0, 0, 2)
        w, order, fine, ms = mp.autotune(p, _dev(qa), _dev(qb))
        assert w in (1, 2, 4) and order in (0, 1) and fine in (0, 1) and ms > 0
        tuned = mp.get_launch(p)
        assert tuned[:3] == (w, order, fine) and tuned[3] in (0, 1)
        np.testing.assert_array_equal(mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy(), ref)
    # a new problem of the same shape starts with the tuned launch (cache)
    with mp.Problem(synth.table_pair_scene(3), margin=1e-4) as p2:
        assert mp.get_launch(p2) == tuned
    # another shape does not
    with mp.Problem(synth.planar_pair_scene(0)) as p3:
        assert mp.get_launch(p3) == (0, 0, 0, 0)
    o = orc.OracleScene(scene)
    idx = np.arange(0, 4096, 97)
    _check_verdicts(ref[idx], o.validate_edges(qa[:, idx], qb[:, idx], 0.02, 1e-4), 1e-4)


# ----------------------------------------------------------------------------
# optional self-collision with an adjacency mask
# ----------------------------------------------------------------------------

def _zero_pose_mask_scene(orc, scene, slack=0.01):
    """Adjacency masks in the usual allowed-collision style: pair links i and
    j >= i + 2 of each arm unless their spheres come within ``slack`` of each
    other at the zero configuration (oracle FK)."""
    import dataclasses
    w = orc.OracleScene(scene).fk(np.zeros(scene.D))
    arms, s0 = [], 0
    for rb in scene.robots:
        ww = w[s0:s0 + rb.n_spheres]
        s0 += rb.n_spheres
        lk = rb.sphere_link
        m = np.zeros(rb.dof, np.uint16)
        for j in range(rb.dof):
            for i in range(j - 1):
                a, b = ww[lk == i], ww[lk == j]
                d = (np.linalg.norm(a[:, None, :3] - b[None, :, :3], axis=2)
                     - a[:, None, 3] - b[None, :, 3])
                if d.min() >= slack:
                    m[j] |= 1 << i
        arms.append(dataclasses.replace(rb, self_mask=m))
    return synth.Scene(arms, scene.obs_spheres, scene.obs_cuboids, scene.name)


@pytest.mark.parametrize("name,n_edges,masked", [("planar_pair", 600, False),
                                                  ("table_pair", 300, True),
                                                  ("grid4", 60, True)])
def test_self_collision_parity(mp, orc, name, n_edges, masked):
    """Verdicts, clearances and interval counts with self-collision on: the
    default mask (links two or more apart) on the planar arms and zero-pose
    adjacency masks on the 7-DOF arms.  Self-collision must change verdicts
    (the test is not vacuous) and the kernel must follow the oracle."""
    scene = SCENES[name]()
    if masked:
        scene = _zero_pose_mask_scene(orc, scene)
    qa, qb = synth.candidate_edges(scene, n_edges, seed=11, step_hi=3.0)
    ref0 = orc.OracleScene(scene).validate_edges(qa, qb, 0.02, 0.0, early_exit=False)
    ref = orc.OracleScene(scene, self_collision=True).validate_edges(qa, qb, 0.02, 0.0,
                                                                     early_exit=False)
    assert (ref["valid"] != ref0["valid"]).sum() > 0
    assert ref["valid"].sum() > 0
    with mp.Problem(scene, resolution=0.02, self_collision=True) as p:
        n = qa.shape[1]
        valid = torch.empty(n, dtype=torch.uint8, device="cuda")
        length = torch.empty(n, dtype=torch.float32, device="cuda")
        npts = torch.empty(n, dtype=torch.int32, device="cuda")
        mp.validate_edges(p, _dev(qa), _dev(qb), valid, length, npts)
        np.testing.assert_array_equal(npts.cpu().numpy(), ref["npoints"])
        c = mp.edge_clearance(p, _dev(qa), _dev(qb)).cpu().numpy().astype(np.float64)
        v = valid.cpu().numpy()
    err = np.abs(c - ref["min_clear"])
    assert (err <= REL * (1 + np.abs(ref["min_clear"]))).all(), err.max()
    _check_verdicts(v, ref, 0.0)
    # self-collision off ignores the masks: the plain verdicts come back
    with mp.Problem(scene, resolution=0.02) as p:
        v0 = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
    _check_verdicts(v0, ref0, 0.0)


def _max_size_scene():
    """At the ABI limits: 4 planar arms of 16 links (64 links, the maximum
    composite dimension) with 16 spheres on every link (1,024 robot spheres),
    and 512 sphere + 512 cuboid obstacles (the obstacle maximum)."""
    bases = [synth._yaw_base(x, y, 0.0, a) for x, y, a in   # arms point outward
             ((-0.45, -0.45, -2.3), (0.45, -0.45, -0.8), (-0.45, 0.45, 2.3), (0.45, 0.45, 0.8))]
    arms = [synth.planar_arm(b, n_links=16, link_len=0.05, spheres_per_link=16, radius=0.008)
            for b in bases]
    for a in arms:   # joint limits +-0.5 rad: a 16-link chain folds onto itself less often
        a.q_lo[:] = -0.5
        a.q_hi[:] = 0.5
    rng = np.random.default_rng(77)
    sph, cub = synth._clutter(rng, 512, 512, (-1.6, -1.6, -0.3), (1.6, 1.6, 0.3),
                              [a.base for a in arms], keep_out=0.1)
    sph[:, 3] *= 0.12
    cub[:, 3:6] *= 0.12
    return synth.Scene(arms, sph, cub, "max_size")


@pytest.mark.parametrize("self_collision", [False, True])
def test_max_size_scene(mp, orc, self_collision):
    """64 links, 16 spheres per link, 1,024 obstacles (one warp per block fits
    the tables and scratch): verdicts and clearances against the oracle."""
    scene = _max_size_scene()
    assert scene.D == 64 and sum(r.n_spheres for r in scene.robots) == 1024
    o = orc.OracleScene(scene, self_collision=self_collision)
    qa, qb = synth.candidate_edges(scene, 24, seed=3, step_lo=0.05, step_hi=0.4)
    ref = o.validate_edges(qa, qb, 0.02, 0.0)
    assert 0 < ref["valid"].sum() < 24
    with mp.Problem(scene, resolution=0.02, self_collision=self_collision) as p:
        v = mp.validate_edges(p, _dev(qa), _dev(qb)).cpu().numpy()
        c = mp.edge_clearance(p, _dev(qa[:, :6]), _dev(qb[:, :6])).cpu().numpy().astype(np.float64)
    _check_verdicts(v, ref, 0.0)
    err = np.abs(c - ref["min_clear"][:6])
    assert (err <= REL * (1 + np.abs(ref["min_clear"][:6]))).all(), err.max()
