"""Plain FP64 CPU oracle for MR. POP's motion validation and nearest queries.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path in ``paper_2609_30644_gb300`` and never imports it.

The arithmetic lives in ``mrpop_oracle.c`` (plain C, double precision, no
culling or reordering); this module compiles it with gcc on first use and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrpop_oracle.c")
_SRC_PLANNER = os.path.join(_HERE, "mrpop_ref_planner.c")
_HDR = os.path.join(_HERE, "mrpop_oracle.h")
_LIB = os.path.join(_HERE, f"liboracle.{platform.machine()}.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no fp contraction)."""
    newest = max(os.path.getmtime(f) for f in (_SRC, _SRC_PLANNER, _HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-Wall", "-Wextra", "-o", tmp, _SRC, _SRC_PLANNER, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [
        ("K", C.c_int32),
        ("dof", C.c_void_p),
        ("dh", C.c_void_p),
        ("n_spheres", C.c_void_p),
        ("sphere_link", C.c_void_p),
        ("sphere_xyzr", C.c_void_p),
        ("base", C.c_void_p),
        ("n_obs_spheres", C.c_int32),
        ("obs_spheres", C.c_void_p),
        ("n_obs_cuboids", C.c_int32),
        ("obs_cuboids", C.c_void_p),
        ("self_collision", C.c_int32),
        ("self_mask", C.c_void_p),
    ]


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        i32, i64, f32, f64, vp = C.c_int32, C.c_int64, C.c_float, C.c_double, C.c_void_p
        pd = C.POINTER(C.c_double)
        sig = {
            "orc_fk_robot": (None, [vp, i32, vp, vp]),
            "orc_link_frames": (None, [vp, i32, vp, vp]),
            "orc_sphere_sphere_clearance": (f64, [vp, f64, vp, f64]),
            "orc_sphere_cuboid_clearance": (f64, [vp, f64, vp]),
            "orc_config_valid": (i32, [vp, vp, f64, pd]),
            "orc_edge_npoints": (i32, [vp, vp, i64, i32, f32]),
            "orc_edge_valid": (i32, [vp, vp, vp, i64, f32, f64, i32, vp, vp, vp]),
            "orc_validate_edges": (None, [vp, vp, vp, i64, i64, i64, f32, f64, i32,
                                          vp, vp, vp, vp]),
            "orc_nearest": (i64, [vp, i64, i64, i32, vp, f32, pd, pd, pd]),
            "orc_neighbors": (i64, [vp, i64, i64, i32, vp, f32, i64, vp, pd]),
            "orc_path_cost": (f64, [vp, i64, i32]),
            "orc_path_valid": (i32, [vp, vp, i64, f32, f64, vp]),
            "orc_edge_method_work": (i32, [vp, vp, vp, i64, f32, f64, i32, vp]),
            "orc_method_work_edges": (None, [vp, vp, vp, i64, i64, i64, f32, f64, i32, vp, vp]),
            "orc_plan": (i32, [vp, vp, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, i64, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# Units counted by OracleScene.method_work, in the order of the C enum.
WORK_UNITS = ("checkpoints", "joints", "coarse_points", "coarse_sphere", "coarse_cuboid",
              "coarse_pair", "fine_points", "fine_sphere", "fine_cuboid", "fine_pair")


class OracleScene:
    """Holds contiguous float32/int32 copies of a synth.Scene for the C oracle."""

    def __init__(self, scene, self_collision: bool = False):
        rs = scene.robots
        self.K = len(rs)
        self.D = int(sum(r.dof for r in rs))
        self.dof = np.ascontiguousarray([r.dof for r in rs], dtype=np.int32)
        self.dh = np.ascontiguousarray(np.concatenate([r.dh for r in rs]), dtype=np.float32)
        self.n_spheres = np.ascontiguousarray([r.n_spheres for r in rs], dtype=np.int32)
        self.sphere_link = np.ascontiguousarray(
            np.concatenate([r.sphere_link for r in rs]), dtype=np.int32)
        self.sphere_xyzr = np.ascontiguousarray(
            np.concatenate([r.sphere_xyzr for r in rs]), dtype=np.float32)
        self.base = np.ascontiguousarray(np.stack([r.base for r in rs]), dtype=np.float32)
        self.obs_spheres = np.ascontiguousarray(scene.obs_spheres, dtype=np.float32).reshape(-1, 4)
        self.obs_cuboids = np.ascontiguousarray(scene.obs_cuboids, dtype=np.float32).reshape(-1, 15)
        if self.obs_spheres.size == 0:
            self.obs_spheres = np.zeros((1, 4), dtype=np.float32)
            n_os = 0
        else:
            n_os = self.obs_spheres.shape[0]
        if self.obs_cuboids.size == 0:
            self.obs_cuboids = np.zeros((1, 15), dtype=np.float32)
            n_oc = 0
        else:
            n_oc = self.obs_cuboids.shape[0]
        self.n_sph_per = [r.n_spheres for r in rs]
        # adjacency masks (bit i of row j pairs links i < j); robots without
        # one take every pair two or more links apart
        masks = [getattr(r, "self_mask", None) for r in rs]
        self.self_mask = None
        if any(m is not None for m in masks):
            rows = []
            for r, m in zip(rs, masks):
                rows.append(np.asarray(m, dtype=np.uint16) if m is not None else np.array(
                    [(1 << (j - 1)) - 1 if j >= 2 else 0 for j in range(r.dof)], dtype=np.uint16))
            self.self_mask = np.ascontiguousarray(np.concatenate(rows), dtype=np.uint16)
        self._s = _Scene(self.K, _p(self.dof), _p(self.dh), _p(self.n_spheres),
                         _p(self.sphere_link), _p(self.sphere_xyzr), _p(self.base),
                         n_os, _p(self.obs_spheres), n_oc, _p(self.obs_cuboids),
                         int(bool(self_collision)),
                         _p(self.self_mask) if self.self_mask is not None else None)

    @property
    def ptr(self):
        return C.byref(self._s)

    # --- kinematics --------------------------------------------------------
    def fk_robot(self, k: int, q) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros((self.n_sph_per[k], 4), dtype=np.float64)
        _load().orc_fk_robot(self.ptr, k, _p(q), _p(out))
        return out

    def link_frames(self, k: int, q) -> np.ndarray:
        q = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros((int(self.dof[k]), 4, 4), dtype=np.float64)
        _load().orc_link_frames(self.ptr, k, _p(q), _p(out))
        return out

    def fk(self, q) -> np.ndarray:
        """World spheres [sum S, 4] of every robot at composite q [D]."""
        q = np.asarray(q, dtype=np.float64)
        outs, o = [], 0
        for k in range(self.K):
            d = int(self.dof[k])
            outs.append(self.fk_robot(k, q[o:o + d]))
            o += d
        return np.concatenate(outs)

    # --- validity ----------------------------------------------------------
    def config_valid(self, q, margin: float = 0.0) -> tuple:
        q = np.ascontiguousarray(q, dtype=np.float64)
        mc = C.c_double()
        ok = _load().orc_config_valid(self.ptr, _p(q), margin, C.byref(mc))
        return bool(ok), mc.value

    def edge_npoints(self, qa, qb, res: float) -> int:
        qa = np.ascontiguousarray(qa, dtype=np.float32)
        qb = np.ascontiguousarray(qb, dtype=np.float32)
        return int(_load().orc_edge_npoints(_p(qa), _p(qb), 1, qa.shape[0], res))

    def edge_valid(self, qa, qb, res: float, margin: float = 0.0,
                   early_exit: bool = False) -> tuple:
        qa = np.ascontiguousarray(qa, dtype=np.float32)
        qb = np.ascontiguousarray(qb, dtype=np.float32)
        mc, fh, npt = C.c_double(), C.c_int32(), C.c_int32()
        ok = _load().orc_edge_valid(self.ptr, _p(qa), _p(qb), 1, res, margin,
                                    int(early_exit), C.byref(mc), C.byref(fh), C.byref(npt))
        return bool(ok), mc.value, fh.value, npt.value

    def validate_edges(self, qa, qb, res: float, margin: float = 0.0,
                       early_exit: bool = False, e0: int = 0,
                       n: Optional[int] = None) -> dict:
        """SoA qa, qb float32 [D, E] -> dict of valid/min_clear/first_hit/npoints."""
        qa = np.ascontiguousarray(qa, dtype=np.float32)
        qb = np.ascontiguousarray(qb, dtype=np.float32)
        ld = qa.shape[1]
        n = ld - e0 if n is None else n
        valid = np.zeros(n, dtype=np.uint8)
        mc = np.zeros(n, dtype=np.float64)
        fh = np.zeros(n, dtype=np.int32)
        npt = np.zeros(n, dtype=np.int32)
        _load().orc_validate_edges(self.ptr, _p(qa), _p(qb), ld, e0, n, res, margin,
                                   int(early_exit), _p(valid), _p(mc), _p(fh), _p(npt))
        return {"valid": valid, "min_clear": mc, "first_hit": fh, "npoints": npt}

    def method_work(self, qa, qb, res: float, margin: float = 0.0,
                    early_exit: bool = False) -> tuple:
        """Work units of the paper's two-stage check (Sec. III-E) over the SoA
        edges qa, qb float32 [D, E], summed over the edges (see WORK_UNITS),
        and each edge's verdict."""
        qa = np.ascontiguousarray(qa, dtype=np.float32)
        qb = np.ascontiguousarray(qb, dtype=np.float32)
        n = qa.shape[1]
        counts = np.zeros(len(WORK_UNITS), dtype=np.int64)
        valid = np.zeros(n, dtype=np.uint8)
        _load().orc_method_work_edges(self.ptr, _p(qa), _p(qb), n, 0, n, res, margin,
                                      int(early_exit), _p(counts), _p(valid))
        return counts, valid

    def path_valid(self, path, res: float, margin: float = 0.0) -> tuple:
        path = np.ascontiguousarray(path, dtype=np.float32)
        bad = C.c_int64()
        ok = _load().orc_path_valid(self.ptr, _p(path), path.shape[0], res, margin,
                                    C.byref(bad))
        return bool(ok), bad.value


def sphere_sphere_clearance(c1, r1, c2, r2) -> float:
    a = np.ascontiguousarray(c1, dtype=np.float64)
    b = np.ascontiguousarray(c2, dtype=np.float64)
    return _load().orc_sphere_sphere_clearance(_p(a), float(r1), _p(b), float(r2))


def sphere_cuboid_clearance(c, r, cuboid) -> float:
    a = np.ascontiguousarray(c, dtype=np.float64)
    cb = np.ascontiguousarray(cuboid, dtype=np.float32)
    return _load().orc_sphere_cuboid_clearance(_p(a), float(r), _p(cb))


def nearest(tree, q, c, n_vertices: Optional[int] = None) -> tuple:
    """Returns (idx, best_d, second_d, filter_gap)."""
    tree = np.ascontiguousarray(tree, dtype=np.float32)
    q = np.ascontiguousarray(q, dtype=np.float32)
    D = tree.shape[0] - 1
    N = tree.shape[1] if n_vertices is None else n_vertices
    bd, sd, gp = C.c_double(), C.c_double(), C.c_double()
    idx = _load().orc_nearest(_p(tree), N, tree.shape[1], D, _p(q), float(c),
                              C.byref(bd), C.byref(sd), C.byref(gp))
    return int(idx), bd.value, sd.value, gp.value


def neighbors(tree, q, delta, k_max: int, n_vertices: Optional[int] = None,
              dims: Optional[int] = None) -> tuple:
    """Returns (indices[:min(count,k_max)], count, gap).  ``dims`` defaults to
    the tree's configuration rows (all rows but the last)."""
    tree = np.ascontiguousarray(tree, dtype=np.float32)
    q = np.ascontiguousarray(q, dtype=np.float32)
    D = tree.shape[0] - 1 if dims is None else dims
    N = tree.shape[1] if n_vertices is None else n_vertices
    out = np.zeros(max(k_max, 1), dtype=np.int64)
    gp = C.c_double()
    cnt = _load().orc_neighbors(_p(tree), N, tree.shape[1], D, _p(q), float(delta),
                                k_max, _p(out), C.byref(gp))
    return out[:min(cnt, k_max)].copy(), int(cnt), gp.value


def path_cost(path) -> float:
    path = np.ascontiguousarray(path, dtype=np.float32)
    return float(_load().orc_path_cost(_p(path), path.shape[0], path.shape[1]))


class _PlanParams(C.Structure):
    _fields_ = [("resolution", C.c_double), ("margin", C.c_double), ("delta", C.c_double),
                ("n_per_round", C.c_int32), ("max_iters", C.c_int64),
                ("iter_budget", C.c_int64), ("time_budget_s", C.c_double),
                ("round_budget", C.c_int64), ("target_cost", C.c_double),
                ("seed", C.c_uint64)]


def plan_reference(scene, start, goal, *, resolution: float = 0.02, margin: float = 1e-4,
                   delta: float = 1.0, n_per_round: int = 64, max_iters: int = 4096,
                   iter_budget: int = 0, time_budget_s: float = 0.0,
                   round_budget: int = 0, target_cost: float = -1.0, seed: int = 0, self_collision: bool = False,
                   path_cap: int = 1 << 16, trace_cap: int = 1024) -> dict:
    """The FP64 reference planner (Alg. 1/2, sequential) on a synth.Scene.
    Returns {status, path [M, D] float64 or None, cost, times, costs,
    trace_iters, iterations}; status 0 = solved, 1 = no solution, -1 = error."""
    o = OracleScene(scene, self_collision=self_collision)
    lo = np.ascontiguousarray(np.concatenate([r.q_lo for r in scene.robots]), dtype=np.float32)
    hi = np.ascontiguousarray(np.concatenate([r.q_hi for r in scene.robots]), dtype=np.float32)
    st = np.ascontiguousarray(start, dtype=np.float64)
    gl = np.ascontiguousarray(goal, dtype=np.float64)
    pp = _PlanParams(resolution, margin, delta, n_per_round, max_iters, iter_budget,
                     time_budget_s, round_budget, target_cost, seed)
    path = np.zeros((path_cap, o.D), dtype=np.float64)
    tt = np.zeros(trace_cap, dtype=np.float64)
    tc = np.zeros(trace_cap, dtype=np.float64)
    ti = np.zeros(trace_cap, dtype=np.int64)
    plen, cost, ntr, its = C.c_int64(), C.c_double(), C.c_int64(), C.c_int64()
    status = _load().orc_plan(o.ptr, _p(lo), _p(hi), _p(st), _p(gl), C.byref(pp), _p(path),
                              path_cap, C.byref(plen), C.byref(cost), _p(tt), _p(tc), _p(ti),
                              trace_cap, C.byref(ntr), C.byref(its))
    n = min(ntr.value, trace_cap)
    return {"status": int(status),
            "path": path[:plen.value].copy() if status == 0 and plen.value <= path_cap else None,
            "cost": cost.value, "times": tt[:n].copy(), "costs": tc[:n].copy(),
            "trace_iters": ti[:n].copy(), "iterations": its.value}
