"""Seeded synthetic workloads: robots, obstacle scenes, candidate edges, trees.

This module produces *inputs* only.  It holds no forward kinematics, no
collision test, no nearest-neighbour rule and no cost computation, so the
FP64 oracle and the CUDA path can both draw from it without sharing any of
the method's arithmetic.

The paper evaluates on Franka/Fetch benchmark scenes (Sec. V-A) that are not
available here; the scenes below stand in for them with the same structure:
serial arms approximated by sphere sets (Sec. III-E), several arms sharing a
cluttered workspace (Sec. III-A), composite configurations that concatenate
the per-robot joint vectors (Sec. III-A).

Conventions shared by every consumer
------------------------------------
* Robot ``i`` is a serial chain of ``dof`` revolute joints with standard DH
  rows ``(a, alpha, d, theta_offset)``.  Frame ``F_j'`` is the frame of joint
  ``j`` after its rotation ``Rz(theta_j + theta_offset_j)``; link ``j``'s
  collision spheres are expressed in ``F_j'``.  The next frame is
  ``F_j' * Tz(d_j) * Tx(a_j) * Rx(alpha_j)``.
* ``base`` is a row-major 3x4 pose ``[R | t]`` of the robot's first frame.
* Obstacle spheres are rows ``(cx, cy, cz, r)``.  Cuboids are rows
  ``(cx, cy, cz, hx, hy, hz, R00..R22)`` with ``R`` row-major whose columns
  are the box axes in the world frame.
* A composite configuration of dimension ``D = sum(dof)`` concatenates the
  robots' joint vectors in robot order.  Batches of configurations are SoA
  ``float32[D, n]``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Iterator, List, Optional

import numpy as np

# Config ids used to derive seeds; a workload is named by what it is.
PLANAR_PAIR = 1      # 2 planar 3-link arms, 6-DOF composite, 10 circles
TABLE_PAIR = 2       # 2 spatial 7-DOF arms over a table, 32 cuboids + 32 spheres
GRID4 = 3            # 4 spatial 7-DOF arms around a 1.5 m cube, 128 obstacles
BATCHED = 4          # heterogeneous problems: 2..8 arms, 16..256 obstacles
SERVING = 5          # Poisson request stream over BATCHED-style problems


def rng_for(config_id: int, idx: int, salt: int = 0) -> np.random.Generator:
    """Independent PCG64 stream for (config, problem index, purpose)."""
    return np.random.default_rng([int(config_id), int(idx), int(salt)])


@dataclasses.dataclass
class Robot:
    dof: int
    dh: np.ndarray           # float32 [dof, 4]  (a, alpha, d, theta_offset)
    q_lo: np.ndarray         # float32 [dof]
    q_hi: np.ndarray         # float32 [dof]
    sphere_link: np.ndarray  # int32 [S], non-decreasing link index
    sphere_xyzr: np.ndarray  # float32 [S, 4] in the link's frame F_j'
    base: np.ndarray         # float32 [12] row-major 3x4
    # uint16 [dof] or None: bit i of row j (i < j) pairs links i and j for
    # self-collision tests; None pairs every link two or more apart
    self_mask: Optional[np.ndarray] = None

    @property
    def n_spheres(self) -> int:
        return int(self.sphere_link.shape[0])


@dataclasses.dataclass
class Scene:
    robots: List[Robot]
    obs_spheres: np.ndarray  # float32 [n, 4]
    obs_cuboids: np.ndarray  # float32 [n, 15]
    name: str = ""

    @property
    def K(self) -> int:
        return len(self.robots)

    @property
    def D(self) -> int:
        return int(sum(r.dof for r in self.robots))

    @property
    def q_lo(self) -> np.ndarray:
        return np.concatenate([r.q_lo for r in self.robots]).astype(np.float32)

    @property
    def q_hi(self) -> np.ndarray:
        return np.concatenate([r.q_hi for r in self.robots]).astype(np.float32)

    @property
    def dof_offsets(self) -> List[int]:
        out, acc = [], 0
        for r in self.robots:
            out.append(acc)
            acc += r.dof
        return out


# ----------------------------------------------------------------------------
# small geometric helpers used only to *place* things (no method arithmetic)
# ----------------------------------------------------------------------------

def _yaw_base(x: float, y: float, z: float, yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([c, -s, 0.0, x,
                     s, c, 0.0, y,
                     0.0, 0.0, 1.0, z], dtype=np.float32)


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    qv = rng.standard_normal(4)
    qv /= np.linalg.norm(qv)
    w, x, y, z = qv
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def _spheres_along_links(dh: np.ndarray, per_link: List[int],
                         radii: np.ndarray) -> tuple:
    """Spheres spaced evenly on the segment from F_j' origin to (a_j, 0, d_j)."""
    links, xyzr, k = [], [], 0
    for j, cnt in enumerate(per_link):
        a, d = float(dh[j, 0]), float(dh[j, 2])
        for m in range(cnt):
            f = (m + 0.5) / cnt
            links.append(j)
            xyzr.append((f * a, 0.0, f * d, float(radii[k])))
            k += 1
    return (np.asarray(links, dtype=np.int32),
            np.asarray(xyzr, dtype=np.float32).reshape(-1, 4))


def planar_arm(base: np.ndarray, n_links: int = 3, link_len: float = 0.3,
               spheres_per_link: int = 4, radius: float = 0.04) -> Robot:
    """Planar arm in the z=0 plane: DH rows with alpha = d = 0."""
    dh = np.zeros((n_links, 4), dtype=np.float32)
    dh[:, 0] = link_len
    per = [spheres_per_link] * n_links
    links, xyzr = _spheres_along_links(
        dh, per, np.full(n_links * spheres_per_link, radius))
    lo = np.full(n_links, -math.pi, dtype=np.float32)
    return Robot(n_links, dh, lo, -lo, links, xyzr, base.astype(np.float32))


def spatial_arm(rng: np.random.Generator, base: np.ndarray) -> Robot:
    """Synthetic 7-DOF arm: a~U[0,0.08], d~U[0.05,0.3], alpha=+-pi/2,
    60 spheres (4 links x 9 + 3 links x 8) with r~U[0.03,0.08]."""
    dof = 7
    dh = np.zeros((dof, 4), dtype=np.float32)
    dh[:, 0] = rng.uniform(0.0, 0.08, dof)
    dh[:, 1] = np.where(rng.random(dof) < 0.5, -math.pi / 2, math.pi / 2)
    dh[:, 2] = rng.uniform(0.05, 0.3, dof)
    per = [9, 9, 9, 9, 8, 8, 8]
    radii = rng.uniform(0.03, 0.08, sum(per))
    links, xyzr = _spheres_along_links(dh, per, radii)
    lo = np.full(dof, -2.9, dtype=np.float32)
    return Robot(dof, dh, lo, -lo, links, xyzr, base.astype(np.float32))


def _cuboid_row(c, h, R) -> np.ndarray:
    return np.concatenate([np.asarray(c, float), np.asarray(h, float),
                           np.asarray(R, float).reshape(9)]).astype(np.float32)


def _clutter(rng: np.random.Generator, n_sph: int, n_cub: int,
             lo, hi, bases=(), keep_out: float = 0.25) -> tuple:
    """Random spheres (r~U[0.03,0.1]) and rotated cuboids (half extents
    ~U[0.02,0.1]) with centres uniform in the box [lo, hi].  An obstacle whose
    bounding sphere comes closer than ``keep_out`` to a robot base origin is
    redrawn, so that no arm is in collision for every configuration."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    origins = [np.array([b[3], b[7], b[11]], float) for b in bases]

    def clear_of_bases(c, bound):
        return all(np.linalg.norm(c - o) - bound >= keep_out for o in origins)

    sph = np.zeros((n_sph, 4), dtype=np.float32)
    i = 0
    while i < n_sph:
        c, r = rng.uniform(lo, hi), rng.uniform(0.03, 0.1)
        if clear_of_bases(c, r):
            sph[i, :3], sph[i, 3] = c, r
            i += 1
    cub = np.zeros((n_cub, 15), dtype=np.float32)
    i = 0
    while i < n_cub:
        c, h, R = rng.uniform(lo, hi), rng.uniform(0.02, 0.1, 3), _random_rotation(rng)
        if clear_of_bases(c, float(np.linalg.norm(h))):
            cub[i] = _cuboid_row(c, h, R)
            i += 1
    return sph, cub


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def planar_pair_scene(seed: int = 0) -> Scene:
    """2 planar 3-link arms (links 0.3 m, 4 circles/link r=0.04) with bases at
    (-0.4,0) and (+0.4,0) pointing +y, 10 circle obstacles in [-1,1]^2 with
    r~U[0.05,0.15]; circles closer than 0.1 m to a base are redrawn."""
    rng = rng_for(PLANAR_PAIR, seed)
    bases = [_yaw_base(-0.4, 0.0, 0.0, math.pi / 2),
             _yaw_base(+0.4, 0.0, 0.0, math.pi / 2)]
    robots = [planar_arm(b) for b in bases]
    circles = []
    while len(circles) < 10:
        c = rng.uniform(-1.0, 1.0, 2)
        r = rng.uniform(0.05, 0.15)
        if min(math.hypot(c[0] - b[3], c[1] - b[7]) for b in bases) - r < 0.1:
            continue
        circles.append((c[0], c[1], 0.0, r))
    return Scene(robots, np.asarray(circles, dtype=np.float32),
                 np.zeros((0, 15), dtype=np.float32), "planar_pair")


def table_pair_scene(seed: int = 0) -> Scene:
    """2 synthetic 7-DOF arms at (0,-0.6,0) and (0,+0.6,0) facing each other
    across a table cuboid (centre (0,0,-0.1), half (0.4,0.3,0.08)), plus 31
    random cuboids and 32 spheres in [-0.6,0.6]x[-0.4,0.4]x[0,0.8]."""
    rng = rng_for(TABLE_PAIR, seed)
    robots = [spatial_arm(rng, _yaw_base(0.0, -0.6, 0.0, +math.pi / 2)),
              spatial_arm(rng, _yaw_base(0.0, +0.6, 0.0, -math.pi / 2))]
    sph, cub = _clutter(rng, 32, 31, (-0.6, -0.4, 0.0), (0.6, 0.4, 0.8),
                        [r.base for r in robots])
    table = _cuboid_row((0.0, 0.0, -0.1), (0.4, 0.3, 0.08), np.eye(3))
    cub = np.concatenate([table[None], cub], axis=0)
    return Scene(robots, sph, cub, "table_pair")


def grid4_scene(seed: int = 0) -> Scene:
    """4 synthetic 7-DOF arms at (+-0.75, +-0.75, 0) yawed toward the centre of
    a 1.5 m cube workspace, 64 spheres + 64 cuboids inside the cube."""
    rng = rng_for(GRID4, seed)
    robots = []
    for x, y in ((-0.75, -0.75), (0.75, -0.75), (-0.75, 0.75), (0.75, 0.75)):
        robots.append(spatial_arm(rng, _yaw_base(x, y, 0.0, math.atan2(-y, -x))))
    sph, cub = _clutter(rng, 64, 64, (-0.75, -0.75, 0.0), (0.75, 0.75, 1.5),
                        [r.base for r in robots])
    return Scene(robots, sph, cub, "grid4")


def batched_scene(idx: int, config_id: int = BATCHED) -> Scene:
    """One of the heterogeneous batched problems: K~U{2..8} synthetic 7-DOF
    arms on a circle of radius 0.9 m facing its centre, 16..256 obstacles
    (half spheres, half cuboids) inside radius 0.6 m, z in [0, 0.8]."""
    rng = rng_for(config_id, idx)
    K = int(rng.integers(2, 9))
    n_obs = int(rng.integers(16, 257))
    robots = []
    phase = rng.uniform(0, 2 * math.pi)
    for k in range(K):
        ang = phase + 2 * math.pi * k / K
        x, y = 0.9 * math.cos(ang), 0.9 * math.sin(ang)
        robots.append(spatial_arm(rng, _yaw_base(x, y, 0.0, ang + math.pi)))
    n_s = n_obs // 2
    sph, cub = _clutter(rng, n_s, n_obs - n_s, (-0.6, -0.6, 0.0), (0.6, 0.6, 0.8),
                        [r.base for r in robots])
    return Scene(robots, sph, cub, f"batched_{idx}")


# ----------------------------------------------------------------------------
# configurations, edges, trees, queries
# ----------------------------------------------------------------------------

def uniform_configs(scene: Scene, n: int, rng: np.random.Generator) -> np.ndarray:
    """float32 [D, n] uniform in the joint limits."""
    lo, hi = scene.q_lo.astype(float), scene.q_hi.astype(float)
    return rng.uniform(lo[:, None], hi[:, None], (scene.D, n)).astype(np.float32)


def candidate_edges(scene: Scene, n_edges: int, seed: int = 0,
                    stay_prob: float = 0.25, step_lo: float = 0.05,
                    step_hi: float = 1.0, salt: int = 7) -> tuple:
    """Candidate composite edges as a planner proposes them: q_a uniform in the
    limits; each robot either stays put (probability ``stay_prob``) or moves by
    ``delta_i * u`` with ``u`` a uniform unit direction in its joint space and
    ``delta_i ~ U[step_lo, step_hi]`` rad; q_b is clipped to the limits.
    Returns float32 SoA arrays ``qa, qb`` of shape [D, n_edges]."""
    rng = rng_for(0, seed, salt)
    qa = uniform_configs(scene, n_edges, rng)
    qb = qa.astype(np.float64).copy()
    for r, off in zip(scene.robots, scene.dof_offsets):
        u = rng.standard_normal((r.dof, n_edges))
        u /= np.linalg.norm(u, axis=0, keepdims=True)
        step = rng.uniform(step_lo, step_hi, n_edges)
        move = rng.random(n_edges) >= stay_prob
        qb[off:off + r.dof] += u * (step * move)[None, :]
    qb = np.clip(qb, scene.q_lo[:, None], scene.q_hi[:, None]).astype(np.float32)
    return qa, qb


def config_stream(scene: Scene, seed: int, salt: int = 11,
                  chunk: int = 256) -> Iterator[np.ndarray]:
    """Endless stream of uniform configurations (float32 [D]) for rejection
    sampling of start/goal states by whichever checker the caller uses."""
    rng = rng_for(0, seed, salt)
    while True:
        block = uniform_configs(scene, chunk, rng)
        for i in range(chunk):
            yield block[:, i].copy()


def first_accepted(stream: Iterator[np.ndarray],
                   accept: Callable[[np.ndarray], bool],
                   max_tries: int = 100000) -> Optional[np.ndarray]:
    for _ in range(max_tries):
        q = next(stream)
        if accept(q):
            return q
    return None


def random_tree(D: int, n: int, lo: np.ndarray, hi: np.ndarray, seed: int = 0,
                dup_frac: float = 0.02, step_lo: float = 0.05,
                step_hi: float = 0.5) -> np.ndarray:
    """Synthetic state-cost tree ``float32 [D+1, n]`` (row D holds g): vertex 0
    is the root with g = 0; vertex i extends a uniformly chosen earlier vertex
    by a random step and gets g = g_parent + step.  A fraction ``dup_frac`` of
    vertices duplicates an earlier vertex's configuration (with either the same
    or a different g) to exercise tie-breaking."""
    rng = rng_for(0, seed, 23)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    q = np.zeros((D, n))
    g = np.zeros(n)
    q[:, 0] = rng.uniform(lo, hi)
    for i in range(1, n):
        p = int(rng.integers(0, i))
        if rng.random() < dup_frac:
            q[:, i] = q[:, p]
            g[i] = g[p] if rng.random() < 0.5 else g[p] + rng.uniform(0.0, 0.3)
            continue
        u = rng.standard_normal(D)
        u /= np.linalg.norm(u)
        step = rng.uniform(step_lo, step_hi)
        q[:, i] = np.clip(q[:, p] + step * u, lo, hi)
        g[i] = g[p] + step
    out = np.zeros((D + 1, n), dtype=np.float32)
    out[:D] = q
    out[D] = g
    return out


def random_tree_fast(D: int, n: int, lo: np.ndarray, hi: np.ndarray,
                     seed: int = 0) -> np.ndarray:
    """Large synthetic tree without the sequential parent walk: configurations
    uniform in the box and g uniform in [0, 2 * box diagonal].  Used where the
    tree is only a scan target (throughput runs)."""
    rng = rng_for(0, seed, 29)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    out = np.zeros((D + 1, n), dtype=np.float32)
    out[:D] = rng.uniform(lo[:, None], hi[:, None], (D, n))
    diag = float(np.sqrt(np.sum((hi - lo) ** 2)))
    out[D] = rng.uniform(0.0, 2.0 * diag, n)
    out[D, 0] = 0.0
    return out


def nn_queries(D: int, n: int, lo: np.ndarray, hi: np.ndarray, seed: int = 0,
               budget_lo: float = 0.0, budget_hi: float = 10.0) -> tuple:
    """Query configurations float32 [D, n] uniform in the box and budgets
    float32 [n] uniform in [budget_lo, budget_hi]; low budgets produce empty
    admissible sets, high ones admit most of the tree."""
    rng = rng_for(0, seed, 31)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    qs = rng.uniform(lo[:, None], hi[:, None], (D, n)).astype(np.float32)
    c = rng.uniform(budget_lo, budget_hi, n).astype(np.float32)
    return qs, c


def poisson_arrivals(rate: float, n: int, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = rng_for(SERVING, seed, int(rate))
    return np.cumsum(rng.exponential(1.0 / rate, n))
