"""Pins for the FP64 oracle: each check compares it with something other than
itself -- hand-derived closed forms (tests/golden), an independent
quaternion-based kinematics, brute-force surface sampling, brute-force dense
edge sampling, and library routines (scipy cKDTree) for special cases.

No GPU needed.  Chosen so that a dropped term, a wrong sign or index, or a
transposed operand anywhere in the oracle fails at least one of them.
"""
import dataclasses
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

from paper_2609_30644_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# independent kinematics used as pins
# ----------------------------------------------------------------------------

def planar_closed_form(robot, theta):
    """Textbook planar chain: phi_j = yaw + sum_{i<=j} theta_i; link j starts
    at base + sum_{i<j} L_i (cos phi_i, sin phi_i)."""
    yaw = math.atan2(robot.base[4], robot.base[0])
    bx, by = float(robot.base[3]), float(robot.base[7])
    L = robot.dh[:, 0].astype(float)
    out = []
    for s in range(robot.n_spheres):
        j = int(robot.sphere_link[s])
        f = float(robot.sphere_xyzr[s, 0]) / L[j]
        x, y, phi = bx, by, yaw
        for i in range(j):
            phi_i = yaw + sum(theta[: i + 1])
            x += L[i] * math.cos(phi_i)
            y += L[i] * math.sin(phi_i)
        phi = yaw + sum(theta[: j + 1])
        out.append((x + f * L[j] * math.cos(phi), y + f * L[j] * math.sin(phi), 0.0,
                    float(robot.sphere_xyzr[s, 3])))
    return np.array(out)


def quaternion_fk(robot, q):
    """DH chain composed with rotation objects and explicit translations in the
    base frame: F_j' = F_{j-1} Rz(theta_j + off_j); next origin = origin +
    R_j' (a_j, 0, d_j); next rotation = R_j' Rx(alpha_j); sphere = origin_{j-1}
    + R_j' p.  The (float32, not exactly orthonormal) base matrix is applied
    last, as given.  Returns world spheres and per-link (R, origin) in world."""
    B = robot.base.astype(float).reshape(3, 4)
    BR, Bt = B[:, :3], B[:, 3]
    rot = Rotation.identity()
    org = np.zeros(3)
    frames = []
    for j in range(robot.dof):
        a, al, d, off = robot.dh[j].astype(float)
        rj = rot * Rotation.from_euler("z", q[j] + off)
        frames.append((rj, org.copy()))
        org = org + rj.apply([a, 0.0, d])
        rot = rj * Rotation.from_euler("x", al)
    out = []
    for s in range(robot.n_spheres):
        rj, o = frames[int(robot.sphere_link[s])]
        p = BR @ (o + rj.apply(robot.sphere_xyzr[s, :3].astype(float))) + Bt
        out.append((*p, float(robot.sphere_xyzr[s, 3])))
    world = [(BR @ rj.as_matrix(), BR @ o + Bt) for rj, o in frames]
    return np.array(out), world


def box_clearance_bruteforce(c, r, cub, n=161):
    """Min distance from c to a dense sample of the box surface, or -r when
    c is inside (inside test in box coordinates)."""
    ctr = cub[:3].astype(float)
    h = cub[3:6].astype(float)
    R = cub[6:].astype(float).reshape(3, 3)
    p = R.T @ (np.asarray(c, float) - ctr)
    if np.all(np.abs(p) <= h):
        return -r
    u = np.linspace(-1, 1, n)
    U, V = np.meshgrid(u, u)
    pts = []
    for ax in range(3):
        o1, o2 = [a for a in range(3) if a != ax]
        for sgn in (-1, 1):
            P = np.zeros((U.size, 3))
            P[:, ax] = sgn * h[ax]
            P[:, o1] = U.ravel() * h[o1]
            P[:, o2] = V.ravel() * h[o2]
            pts.append(P)
    P = np.concatenate(pts)
    return float(np.min(np.linalg.norm(P - p[None], axis=1))) - r


# ----------------------------------------------------------------------------
# forward kinematics
# ----------------------------------------------------------------------------

def test_planar_fk_golden(orc):
    scene = synth.planar_pair_scene(0)
    o = orc.OracleScene(scene)
    rows = [l.split() for l in open(os.path.join(GOLDEN, "planar_fk.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 8
    for row in rows:
        th = [float(x) for x in row[:3]]
        link, k = int(row[3]), int(row[4])
        x, y = float(row[5]), float(row[6])
        w = o.fk_robot(0, th)
        s = link * 4 + k
        # scene parameters are float32 (|rounding| < 3e-8 per value)
        assert w[s, 0] == pytest.approx(x, abs=2e-7)
        assert w[s, 1] == pytest.approx(y, abs=2e-7)
        assert w[s, 2] == pytest.approx(0.0, abs=1e-12)


def test_planar_fk_closed_form(orc):
    """DH with alpha = d = 0 reduces to the textbook planar chain."""
    scene = synth.planar_pair_scene(3)
    o = orc.OracleScene(scene)
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.uniform(-math.pi, math.pi, 6)
        for k in range(2):
            ref = planar_closed_form(scene.robots[k], q[3 * k:3 * k + 3])
            got = o.fk_robot(k, q[3 * k:3 * k + 3])
            np.testing.assert_allclose(got, ref, atol=1e-12)


@pytest.mark.parametrize("make", [synth.table_pair_scene, synth.grid4_scene])
def test_spatial_fk_vs_quaternion_chain(orc, make):
    scene = make(1)
    o = orc.OracleScene(scene)
    rng = np.random.default_rng(2)
    for _ in range(20):
        for k, rb in enumerate(scene.robots):
            q = rng.uniform(rb.q_lo, rb.q_hi)
            ref, frames = quaternion_fk(rb, q)
            np.testing.assert_allclose(o.fk_robot(k, q), ref, atol=1e-12)
            F = o.link_frames(k, q)
            for j, (rj, org) in enumerate(frames):
                np.testing.assert_allclose(F[j, :3, :3], rj, atol=1e-12)
                np.testing.assert_allclose(F[j, :3, 3], org, atol=1e-12)
                # joint rotations are exact rotations: the frame is as
                # orthonormal as the float32 base rotation it starts from
                Rm = F[j, :3, :3]
                B = rb.base.astype(float).reshape(3, 4)[:, :3]
                base_err = np.abs(B.T @ B - np.eye(3)).max()
                assert np.abs(Rm.T @ Rm - np.eye(3)).max() <= base_err + 1e-12
                np.testing.assert_array_equal(F[j, 3], [0, 0, 0, 1])


def test_fk_theta_offset_is_added(orc):
    """theta_offset shifts the joint angle: q + off with off=0 equals q' = q + off."""
    scene = synth.table_pair_scene(0)
    rb = scene.robots[0]
    rng = np.random.default_rng(3)
    q = rng.uniform(-1, 1, rb.dof)
    off = rng.uniform(-1, 1, rb.dof).astype(np.float32)
    rb2 = synth.Robot(rb.dof, rb.dh.copy(), rb.q_lo, rb.q_hi, rb.sphere_link,
                      rb.sphere_xyzr, rb.base)
    rb2.dh[:, 3] = off
    s1 = synth.Scene([rb2], scene.obs_spheres, scene.obs_cuboids)
    s0 = synth.Scene([rb], scene.obs_spheres, scene.obs_cuboids)
    a = orc.OracleScene(s1).fk_robot(0, q)
    b = orc.OracleScene(s0).fk_robot(0, q + off.astype(float))
    np.testing.assert_allclose(a, b, atol=1e-12)


# ----------------------------------------------------------------------------
# distances
# ----------------------------------------------------------------------------

def test_clearance_golden(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "clearance_cases.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 8
    for row in rows:
        v = [float(x) for x in row[1:]]
        if row[0] == "ss":
            got = orc.sphere_sphere_clearance(v[0:3], v[3], v[4:7], v[7])
            assert got == pytest.approx(v[8], abs=1e-12)
        else:
            cub = np.array(v[4:19], dtype=np.float32)
            got = orc.sphere_cuboid_clearance(v[0:3], v[3], cub)
            assert got == pytest.approx(v[19], abs=1e-7)


def test_sphere_cuboid_vs_bruteforce(orc):
    rng = np.random.default_rng(4)
    scene = synth.table_pair_scene(0)
    for i in range(40):
        cub = scene.obs_cuboids[1 + i % 31]
        c = cub[:3].astype(float) + rng.uniform(-0.25, 0.25, 3)
        r = float(rng.uniform(0.0, 0.05))
        got = orc.sphere_cuboid_clearance(c, r, cub)
        ref = box_clearance_bruteforce(c, r, cub)
        # surface grid spacing 2h/160 <= 1.25e-3 m
        if ref > -r:
            assert got <= ref + 1e-9
            assert got == pytest.approx(ref, abs=1.5e-3)
        else:
            assert got == pytest.approx(-r, abs=1e-12)


def test_sphere_sphere_symmetric_and_scaled(orc):
    rng = np.random.default_rng(5)
    for _ in range(100):
        a, b = rng.normal(size=3), rng.normal(size=3)
        r1, r2 = rng.uniform(0, 1, 2)
        d = orc.sphere_sphere_clearance(a, r1, b, r2)
        assert d == pytest.approx(orc.sphere_sphere_clearance(b, r2, a, r1), abs=1e-15)
        assert d == pytest.approx(np.linalg.norm(a - b) - r1 - r2, abs=1e-12)


# ----------------------------------------------------------------------------
# configuration validity (composite free space)
# ----------------------------------------------------------------------------

def _planar_min_clearance(scene, q):
    """All-pairs clearance with closed-form planar FK and scipy-free numpy."""
    offs = np.cumsum([0] + [rb.dof for rb in scene.robots])
    w = [planar_closed_form(rb, q[offs[k]:offs[k + 1]]) for k, rb in enumerate(scene.robots)]
    mc = np.inf
    for k, wk in enumerate(w):
        oc = scene.obs_spheres.astype(float)
        d = np.linalg.norm(wk[:, None, :3] - oc[None, :, :3], axis=2) - wk[:, None, 3] - oc[None, :, 3]
        mc = min(mc, d.min())
        for j in range(k + 1, len(w)):
            d = (np.linalg.norm(wk[:, None, :3] - w[j][None, :, :3], axis=2)
                 - wk[:, None, 3] - w[j][None, :, 3])
            mc = min(mc, d.min())
    return mc


def test_config_valid_planar_allpairs(orc):
    scene = synth.planar_pair_scene(0)
    o = orc.OracleScene(scene)
    rng = np.random.default_rng(6)
    n_valid = 0
    for _ in range(200):
        q = rng.uniform(-math.pi, math.pi, 6)
        ok, mc = o.config_valid(q, 0.0)
        ref = _planar_min_clearance(scene, q)
        assert mc == pytest.approx(ref, abs=1e-12)
        assert ok == (ref >= 0.0)
        n_valid += ok
        # margin shifts the threshold
        ok2, _ = o.config_valid(q, 0.05)
        assert ok2 == (ref >= 0.05)
    assert 20 < n_valid < 180


def test_config_valid_spatial_composition(orc):
    """Spatial scene: quaternion FK spheres, numpy sphere-sphere and robot-robot
    pairs, oracle box clearance (pinned above) -> same minimum and verdict."""
    scene = synth.table_pair_scene(2)
    o = orc.OracleScene(scene)
    rng = np.random.default_rng(7)
    for _ in range(20):
        q = synth.uniform_configs(scene, 1, rng)[:, 0].astype(float)
        w = [quaternion_fk(rb, q[off:off + rb.dof])[0]
             for rb, off in zip(scene.robots, scene.dof_offsets)]
        mc = np.inf
        for k, wk in enumerate(w):
            oc = scene.obs_spheres.astype(float)
            d = np.linalg.norm(wk[:, None, :3] - oc[None, :, :3], axis=2) - wk[:, None, 3] - oc[None, :, 3]
            mc = min(mc, d.min())
            for s in range(wk.shape[0]):
                for cub in scene.obs_cuboids:
                    mc = min(mc, orc.sphere_cuboid_clearance(wk[s, :3], wk[s, 3], cub))
            for j in range(k + 1, len(w)):
                d = (np.linalg.norm(wk[:, None, :3] - w[j][None, :, :3], axis=2)
                     - wk[:, None, 3] - w[j][None, :, 3])
                mc = min(mc, d.min())
        ok, got = o.config_valid(q, 1e-4)
        assert got == pytest.approx(mc, abs=1e-10)
        assert ok == (mc >= 1e-4)


def test_no_self_collision_tests(orc):
    """A single robot whose own spheres overlap (adjacent links) is valid in
    free space: only robot-obstacle and robot-robot pairs count."""
    scene = synth.planar_pair_scene(0)
    one = synth.Scene([scene.robots[0]], np.zeros((0, 4), np.float32),
                      np.zeros((0, 15), np.float32))
    o = orc.OracleScene(one)
    ok, mc = o.config_valid([0.0, math.pi, 0.0], 0.0)   # folded arm
    assert ok and mc == np.finfo(float).max


# ----------------------------------------------------------------------------
# edges: interpolation count and verdicts
# ----------------------------------------------------------------------------

def test_edge_npoints_exact_cases(orc):
    scene = synth.planar_pair_scene(0)
    o = orc.OracleScene(scene)
    z = np.zeros(6, np.float32)
    assert o.edge_npoints(z, z, 0.02) == 1                       # zero-length edge
    qb = z.copy(); qb[0], qb[1] = 0.75, 1.0                      # |dq| = 1.25 exactly
    assert o.edge_npoints(z, qb, 0.25) == 5
    assert o.edge_npoints(z, qb, 0.5) == 3                       # ceil(2.5)
    qb = z.copy(); qb[3] = 1e-3
    assert o.edge_npoints(z, qb, 0.02) == 1
    rng = np.random.default_rng(8)
    for _ in range(500):
        qa = rng.uniform(-3, 3, 6).astype(np.float32)
        qb = (qa + rng.normal(0, 0.5, 6)).astype(np.float32)
        n = o.edge_npoints(qa, qb, 0.02)
        L = np.linalg.norm(qb.astype(float) - qa.astype(float))
        # spacing never exceeds the resolution (up to FP32 rounding of L)
        assert n * 0.02 >= L * (1 - 1e-6)
        assert (n - 1) * 0.02 < L * (1 + 1e-6) or n == 1


def test_edge_verdict_vs_dense_bruteforce(orc):
    """Oracle edge verdict at res against 64x denser sampling with the
    closed-form planar pipeline: a collision found at res is found densely
    (the res points are a subset); a valid edge at res with clearance above the
    largest sphere displacement between samples stays valid densely."""
    scene = synth.planar_pair_scene(1)
    o = orc.OracleScene(scene)
    qa, qb = synth.candidate_edges(scene, 60, seed=3)
    res = 0.02
    for e in range(qa.shape[1]):
        ok, mc, fh, n = o.edge_valid(qa[:, e], qb[:, e], res, 0.0)
        a, b = qa[:, e].astype(float), qb[:, e].astype(float)
        nf = 64 * n
        clear = [_planar_min_clearance(scene, a + (k / nf) * (b - a)) for k in range(nf + 1)]
        dense_ok = min(clear) >= 0.0
        coarse = min(clear[::64])
        assert mc == pytest.approx(coarse, abs=1e-12)
        if not ok:
            assert not dense_ok
            assert clear[64 * fh] < 0 and all(c >= 0 for c in clear[:64 * fh:64])
        # sphere displacement between coarse samples <= 0.9 m * |dq|/n (lever x angle)
        step = 0.9 * np.abs(b - a).sum() / n
        if ok and mc > step:
            assert dense_ok


def test_edge_early_exit_consistent(orc):
    scene = synth.table_pair_scene(0)
    o = orc.OracleScene(scene)
    qa, qb = synth.candidate_edges(scene, 40, seed=4)
    full = o.validate_edges(qa, qb, 0.02, 1e-4, early_exit=False)
    fast = o.validate_edges(qa, qb, 0.02, 1e-4, early_exit=True)
    np.testing.assert_array_equal(full["valid"], fast["valid"])
    np.testing.assert_array_equal(full["first_hit"], fast["first_hit"])
    assert 0 < full["valid"].sum() < 40


def test_stay_put_robot_constant(orc):
    """An edge where robot 2 stays put: robot 2's spheres are identical at all
    points, so its verdict depends on robot 1 only (Prop. 1: stay-put edges)."""
    scene = synth.table_pair_scene(0)
    o = orc.OracleScene(scene)
    rng = np.random.default_rng(9)
    qa = synth.uniform_configs(scene, 1, rng)[:, 0]
    qb = qa.copy()
    qb[:7] += 0.3
    n = o.edge_npoints(qa, qb, 0.02)
    w0 = o.fk_robot(1, qa[7:].astype(float))
    for k in range(n + 1):
        qk = qa.astype(float) + (k / n) * (qb.astype(float) - qa.astype(float))
        np.testing.assert_array_equal(o.fk_robot(1, qk[7:]), w0)


# ----------------------------------------------------------------------------
# nearest / neighbours
# ----------------------------------------------------------------------------

def _nearest_bruteforce(tree, q, c):
    D = tree.shape[0] - 1
    d = np.linalg.norm(tree[:D].astype(float) - q.astype(float)[:, None], axis=0)
    g = tree[D].astype(float)
    adm = np.nonzero(g + d < c)[0]
    if adm.size == 0:
        return -1
    order = np.lexsort((adm, g[adm], d[adm]))   # last key is primary
    return int(adm[order[0]])


def test_nearest_vs_bruteforce_with_ties(orc):
    D = 14
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree(D, 600, lo, hi, seed=1, dup_frac=0.1)
    qs, cs = synth.nn_queries(D, 300, lo, hi, seed=2, budget_lo=0, budget_hi=25)
    n_empty = 0
    for i in range(qs.shape[1]):
        idx = orc.nearest(tree, qs[:, i], cs[i])[0]
        assert idx == _nearest_bruteforce(tree, qs[:, i], cs[i])
        n_empty += idx < 0
    assert 0 < n_empty < 300
    # exact duplicates: query at a duplicated configuration -> lowest g, then index
    dup = np.nonzero(np.all(tree[:D, :, None] == tree[:D, None, :], axis=0).sum(1) > 1)[0]
    assert dup.size > 0
    for v in dup[:20]:
        q = tree[:D, v].copy()
        same = np.nonzero(np.all(tree[:D] == q[:, None], axis=0))[0]
        g = tree[D, same]
        expect = same[np.lexsort((same, g))[0]]
        assert orc.nearest(tree, q, np.float32(1e9))[0] == expect


def test_nearest_unbounded_is_plain_nn(orc):
    """With c = +inf the filter admits everything: plain nearest neighbour."""
    D = 7
    rng = np.random.default_rng(10)
    tree = np.zeros((D + 1, 2000), np.float32)
    tree[:D] = rng.uniform(-1, 1, (D, 2000))
    tree[D] = rng.uniform(0, 5, 2000)
    kd = cKDTree(tree[:D].T.astype(float))
    for _ in range(200):
        q = rng.uniform(-1, 1, D).astype(np.float32)
        d, i = kd.query(q.astype(float))
        got, bd, _, _ = orc.nearest(tree, q, np.inf)
        assert got == i and bd == pytest.approx(d, abs=1e-12)


def test_nearest_filter_strict(orc):
    tree = np.array([[0.0, 1.0], [0.0, 0.0], [1.0, 0.0]], np.float32)  # D=2, g=(1,0)
    q = np.array([0.0, 0.0], np.float32)
    # vertex 0: g + d = 1 + 0 = 1; vertex 1: 0 + 1 = 1
    assert orc.nearest(tree, q, 1.0)[0] == -1          # strict <: neither admitted
    assert orc.nearest(tree, q, 1.0000001)[0] == 0     # both admitted, 0 is closer
    tree[2, 0] = 1.5
    assert orc.nearest(tree, q, 1.2)[0] == 1           # vertex 0 filtered out


def test_neighbors_vs_kdtree(orc):
    D = 7
    rng = np.random.default_rng(11)
    tree = np.zeros((D + 1, 3000), np.float32)
    tree[:D] = rng.uniform(-2.9, 2.9, (D, 3000))
    kd = cKDTree(tree[:D].T.astype(float))
    for _ in range(100):
        q = rng.uniform(-2.9, 2.9, D).astype(np.float32)
        delta = float(rng.uniform(1.0, 3.0))
        ref = sorted(kd.query_ball_point(q.astype(float), delta))
        got, cnt, _ = orc.neighbors(tree, q, np.float32(delta), k_max=32)
        assert cnt == len(ref)
        assert list(got) == ref[:32]


def test_path_cost(orc):
    rng = np.random.default_rng(12)
    a, b = rng.normal(size=14), rng.normal(size=14)
    ts = np.sort(rng.uniform(0, 1, 10))
    ts[0], ts[-1] = 0.0, 1.0
    path = np.stack([a + t * (b - a) for t in ts]).astype(np.float32)
    L = np.linalg.norm(path[-1].astype(float) - path[0].astype(float))
    assert orc.path_cost(path) == pytest.approx(L, rel=1e-6)   # collinear: no detour
    path = rng.normal(size=(7, 5)).astype(np.float32)
    ref = sum(np.linalg.norm(path[j + 1].astype(float) - path[j].astype(float)) for j in range(6))
    assert orc.path_cost(path) == pytest.approx(ref, rel=1e-14)
    assert orc.path_cost(path[:1]) == 0.0


# ----------------------------------------------------------------------------
# optional self-collision (links at least two apart on one robot)
# ----------------------------------------------------------------------------

def test_self_collision_folded_planar_arm(orc):
    """Hand-derived: the planar arm of the golden file folded as (0, pi, 0)
    puts link 2's first sphere at (-0.4, -0.0375) and link 0's first sphere at
    (-0.4, 0.0375): 0.075 m apart, radii 0.04 + 0.04 -> clearance -0.005.
    Links 0-1 and 1-2 are adjacent and never tested against each other."""
    scene = synth.planar_pair_scene(0)
    one = synth.Scene([scene.robots[0]], np.zeros((0, 4), np.float32),
                      np.zeros((0, 15), np.float32))
    q = [0.0, math.pi, 0.0]
    ok, mc = orc.OracleScene(one, self_collision=True).config_valid(q, 0.0)
    assert not ok and mc == pytest.approx(-0.005, abs=1e-6)
    ok, _ = orc.OracleScene(one, self_collision=False).config_valid(q, 0.0)
    assert ok
    # straight arm: the closest tested pair is link 0's last circle (y = 0.2625)
    # and link 2's first (y = 0.6375), 0.375 apart -> clearance 0.295
    ok, mc = orc.OracleScene(one, self_collision=True).config_valid([0.0, 0.0, 0.0], 0.0)
    assert ok and mc == pytest.approx(0.295, abs=1e-6)
    # an adjacency mask without the (0, 2) pair accepts the folded arm
    rb = dataclasses.replace(scene.robots[0], self_mask=np.zeros(3, np.uint16))
    masked = synth.Scene([rb], one.obs_spheres, one.obs_cuboids)
    ok, mc = orc.OracleScene(masked, self_collision=True).config_valid(q, 0.0)
    assert ok and mc > 1e300  # no pair is tested: the minimum stays at DBL_MAX


@pytest.mark.parametrize("masked", [False, True])
def test_self_collision_allpairs_planar(orc, masked):
    """All-pairs numpy (closed-form planar FK) including the same-robot pairs
    of the adjacency mask agrees with the oracle's minimum and verdict: the
    default mask (links two or more apart) and a 5-link arm's explicit mask
    that pairs links (0, 2), (0, 4), (1, 3) and (2, 4) only."""
    scene = synth.planar_pair_scene(1)
    if masked:
        rng = np.random.default_rng(3)
        arms = []
        for rb in scene.robots:
            arm = synth.planar_arm(rb.base, n_links=5, link_len=0.2)
            arms.append(dataclasses.replace(
                arm, self_mask=np.array([0, 0, 1, 2, 1 | 4], np.uint16)))
        scene = synth.Scene(arms, scene.obs_spheres, scene.obs_cuboids)
        pairs = {(0, 2), (0, 4), (1, 3), (2, 4)}
    o = orc.OracleScene(scene, self_collision=True)
    rng = np.random.default_rng(21)
    n_bad = n_self = 0
    for _ in range(200):
        q = rng.uniform(-math.pi, math.pi, scene.D)
        ref = _planar_min_clearance(scene, q)
        ref_other = ref
        off = 0
        for rb in scene.robots:
            w = planar_closed_form(rb, q[off:off + rb.dof])
            off += rb.dof
            lk = rb.sphere_link
            for a in range(len(w)):
                for b in range(a + 1, len(w)):
                    la, lb = sorted((int(lk[a]), int(lk[b])))
                    if ((la, lb) in pairs) if masked else lb - la >= 2:
                        d = np.linalg.norm(w[a, :3] - w[b, :3]) - w[a, 3] - w[b, 3]
                        ref = min(ref, d)
        ok, mc = o.config_valid(q, 0.0)
        assert mc == pytest.approx(ref, abs=1e-12)
        assert ok == (ref >= 0.0)
        n_bad += not ok
        n_self += ref < 0.0 <= ref_other
    assert n_bad > 0 and n_self > 0


# ----------------------------------------------------------------------------
# work of the paper's two-stage check (Sec. III-E), counted for the roofline
# ----------------------------------------------------------------------------

def _two_link_arm(x, y):
    """Planar 2-link arm (links 0.3 m along +x at q = 0, base at (x, y)) with
    2 spheres of r = 0.02 per link, at 0.075 and 0.225 m along each link."""
    base = np.array([1, 0, 0, x, 0, 1, 0, y, 0, 0, 1, 0], np.float32)
    return synth.planar_arm(base, n_links=2, link_len=0.3, spheres_per_link=2, radius=0.02)


def _units(counts, orc):
    return dict(zip(orc.WORK_UNITS, (int(c) for c in counts)))


def test_method_work_hand_counted_one_arm(orc):
    """One arm at q = (0, 0), one obstacle sphere (0.45, 0.12, 0), r = 0.05;
    the zero-length edge has n = 1, so 2 checkpoints.  By hand: link coarse
    spheres have centres (0.15, 0, 0) and (0.45, 0, 0) and radius 0.075 +
    0.02 + 1e-4 = 0.0951.  Link 1's centre is 0.12 from the obstacle centre
    (< 0.0951 + 0.05): a coarse hit; link 0's is 0.323 away: none.  The fine
    spheres of link 1, at (0.375, 0, 0) and (0.525, 0, 0), are 0.1415 from it
    (> 0.02 + 0.05): the edge is free.  Per checkpoint: 2 joints, 2 coarse
    centres, 2 coarse sphere tests, then link 1's 2 fine centres and 2 fine
    sphere tests."""
    sc = synth.Scene([_two_link_arm(0.0, 0.0)], np.array([[0.45, 0.12, 0.0, 0.05]], np.float32),
                     np.zeros((0, 15), np.float32))
    o = orc.OracleScene(sc)
    q = np.zeros((2, 1), np.float32)
    counts, valid = o.method_work(q, q, 0.02, 0.0)
    assert valid.tolist() == [1]
    assert _units(counts, orc) == dict(checkpoints=2, joints=4, coarse_points=4, coarse_sphere=4,
                                       coarse_cuboid=0, coarse_pair=0, fine_points=4,
                                       fine_sphere=4, fine_cuboid=0, fine_pair=0)
    # moving the obstacle out of every coarse sphere leaves stage 1 only
    sc.obs_spheres[0, :2] = (0.45, 0.5)
    counts, valid = orc.OracleScene(sc).method_work(q, q, 0.02, 0.0)
    assert valid.tolist() == [1]
    assert _units(counts, orc)["fine_points"] == 0 and _units(counts, orc)["fine_sphere"] == 0
    assert _units(counts, orc)["coarse_sphere"] == 4


def test_method_work_hand_counted_two_arms(orc):
    """Arms at y = 0 and y = 0.15 (both along +x) and the obstacle of the
    one-arm case.  By hand, per checkpoint: 4 links, 4 coarse centres, 4
    coarse sphere tests (hits: link 1 of both arms, 0.12 and 0.03 away), 4
    coarse pair tests (hits: link 0 with link 0 and link 1 with link 1, 0.15
    apart < 2 x 0.0951; the crossed pairs are 0.335 apart).  Every link has a
    hit: 8 fine centres; fine sphere tests 2 + 2 (the two links 1); fine pair
    tests 2 x 2 for each of the two hit pairs = 8.  Closest fine distances:
    pairs 0.15 (> 0.04), arm 2's link 1 to the obstacle 0.0808 (> 0.07): free.
    A cuboid far from both arms adds 4 coarse box tests and nothing else."""
    far_box = np.zeros((1, 15), np.float32)
    far_box[0, :6] = (0.0, -1.0, 0.0, 0.05, 0.05, 0.05)
    far_box[0, 6:] = np.eye(3, dtype=np.float32).ravel()
    sc = synth.Scene([_two_link_arm(0.0, 0.0), _two_link_arm(0.0, 0.15)],
                     np.array([[0.45, 0.12, 0.0, 0.05]], np.float32), far_box)
    o = orc.OracleScene(sc)
    q = np.zeros((4, 1), np.float32)
    counts, valid = o.method_work(q, q, 0.02, 0.0)
    assert valid.tolist() == [1]
    assert _units(counts, orc) == dict(checkpoints=2, joints=8, coarse_points=8, coarse_sphere=8,
                                       coarse_cuboid=8, coarse_pair=8, fine_points=16,
                                       fine_sphere=8, fine_cuboid=0, fine_pair=16)
    # a 0.1 rad edge of the first joint: n = ceil(0.1 / 0.02) = 5, 6 checkpoints
    qb = q.copy()
    qb[0, 0] = 0.1
    counts, _ = o.method_work(q, qb, 0.02, 0.0)
    u = _units(counts, orc)
    assert u["checkpoints"] == 6 and u["joints"] == 24 and u["coarse_points"] == 24
    assert u["coarse_pair"] == 24 and u["coarse_sphere"] == 24 and u["coarse_cuboid"] == 24


@pytest.mark.parametrize("make,self_collision", [(lambda: synth.planar_pair_scene(0), False),
                                                 (lambda: synth.planar_pair_scene(0), True),
                                                 (lambda: synth.table_pair_scene(0), False)])
def test_method_work_verdicts_equal_all_pairs(orc, make, self_collision):
    """The two-stage check decides exactly what the all-pairs definition
    decides (each coarse sphere encloses its link's fine spheres), and the
    early-exit count never exceeds the full count; on free edges both agree."""
    sc = make()
    o = orc.OracleScene(sc, self_collision=self_collision)
    qa, qb = synth.candidate_edges(sc, 60, seed=23, step_hi=1.5)
    ref = o.validate_edges(qa, qb, 0.02, 1e-4)
    full, v_full = o.method_work(qa, qb, 0.02, 1e-4)
    early, v_early = o.method_work(qa, qb, 0.02, 1e-4, early_exit=True)
    np.testing.assert_array_equal(v_full, ref["valid"])
    np.testing.assert_array_equal(v_early, ref["valid"])
    assert 0 < ref["valid"].sum() < 60
    assert (early <= full).all() and early[0] < full[0]
    free = np.nonzero(ref["valid"])[0]
    f_full, _ = o.method_work(qa[:, free], qb[:, free], 0.02, 1e-4)
    f_early, _ = o.method_work(qa[:, free], qb[:, free], 0.02, 1e-4, early_exit=True)
    np.testing.assert_array_equal(f_full, f_early)
    u = _units(f_full, orc)
    assert u["checkpoints"] == int((ref["npoints"][free] + 1).sum())
    assert u["joints"] == u["checkpoints"] * sc.D
    n_obs = len(sc.obs_spheres) + len(sc.obs_cuboids)
    assert u["coarse_sphere"] + u["coarse_cuboid"] == u["coarse_points"] * n_obs
    assert u["fine_points"] <= u["checkpoints"] * sum(r.n_spheres for r in sc.robots)
