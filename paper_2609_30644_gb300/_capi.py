"""ctypes binding of libmrpop.so with the C ABI's names.

Argument marshalling only: tensors must already live on the right device with
the right dtype and layout; this module checks that and passes raw pointers
and the current torch stream to the library.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libmrpop.so")

# Every symbol declared in include/mrpop.h.
EXPORTS = (
    "mrpop_last_error",
    "mrpop_create_problem",
    "mrpop_destroy_problem",
    "mrpop_problem_dims",
    "mrpop_fk",
    "mrpop_validate_edges",
    "mrpop_validate_edges_ex",
    "mrpop_edge_clearance",
    "mrpop_validate_work",
    "mrpop_autotune",
    "mrpop_set_launch",
    "mrpop_nearest",
    "mrpop_nearest_ex",
    "mrpop_nearest_noalloc",
    "mrpop_nearest_work",
    "mrpop_neighbors",
    "mrpop_path_cost",
    "mrpop_plan",
    "mrpop_plan_batch",
    "mrpop_plan_result",
    "mrpop_plan_trace",
    "mrpop_plan_history",
    "mrpop_server_create",
    "mrpop_server_submit",
    "mrpop_server_poll",
    "mrpop_server_stats",
    "mrpop_server_destroy",
    "mrpop_fp32_peak",
    "mrpop_planner_nearest_pass",
    "mrpop_planner_neighbors_pass",
    "mrpop_plan_batch_ex",
    "mrpop_set_persistent_limits",
    "mrpop_set_launch_ex",
    "mrpop_get_launch",
    "mrpop_autotune_cache_save",
    "mrpop_autotune_cache_load",
    "mrpop_autotune_cache_clear",
    "mrpop_nearest_autotune",
    "mrpop_neighbors_autotune",
    "mrpop_server_cancel",
    "mrpop_server_inject",
    "mrpop_scratch_stats",
    "mrpop_plan_batch_phase_stats",
)

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ECAPACITY", 5: "ETIMEOUT",
          6: "ENOSOLUTION", 7: "EBUSY", 8: "ECANCELLED"}


class MrpopError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mrpop {STATUS.get(status, status)}: {msg}")
        self.status = status


class _Robot(C.Structure):
    _fields_ = [("dof", C.c_int32), ("n_spheres", C.c_int32), ("dh", C.c_void_p),
                ("q_lo", C.c_void_p), ("q_hi", C.c_void_p), ("sphere_link", C.c_void_p),
                ("sphere_xyzr", C.c_void_p), ("base", C.c_float * 12),
                ("self_mask", C.c_void_p)]


class _Obstacles(C.Structure):
    _fields_ = [("n_spheres", C.c_int32), ("spheres", C.c_void_p),
                ("n_cuboids", C.c_int32), ("cuboids", C.c_void_p)]


class _Config(C.Structure):
    _fields_ = [("resolution", C.c_float), ("margin", C.c_float), ("delta", C.c_float),
                ("n_per_round", C.c_int32), ("tree_cap", C.c_int64),
                ("roadmap_cap", C.c_int64), ("max_iters", C.c_int64), ("seed", C.c_uint64),
                ("self_collision", C.c_int32)]


def _load() -> C.CDLL:
    if not os.path.exists(library_path):
        raise ImportError(
            f"{library_path} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a). "
            "There is no CPU fallback.")
    L = C.CDLL(library_path)
    vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    sig = {
        "mrpop_last_error": (C.c_char_p, []),
        "mrpop_create_problem": (i32, [vp, i32, vp, vp, vp, vp, vp]),
        "mrpop_destroy_problem": (i32, [vp]),
        "mrpop_problem_dims": (i32, [vp, vp, vp, vp]),
        "mrpop_fk": (i32, [vp, vp, i64, vp, vp]),
        "mrpop_validate_edges": (i32, [vp, vp, vp, i64, vp, vp]),
        "mrpop_validate_edges_ex": (i32, [vp, vp, vp, i64, vp, vp, vp, vp]),
        "mrpop_edge_clearance": (i32, [vp, vp, vp, i64, vp, vp]),
        "mrpop_validate_work": (i32, [vp, vp, vp, i64, vp, vp]),
        "mrpop_autotune": (i32, [vp, vp, vp, i64, vp, vp, vp, vp]),
        "mrpop_set_launch": (i32, [vp, i32, i32, i32]),
        "mrpop_nearest": (i32, [vp, i64, i64, i32, vp, vp, i64, vp, vp]),
        "mrpop_nearest_ex": (i32, [vp, i64, i64, i32, vp, vp, i64, i32, vp, vp]),
        "mrpop_nearest_noalloc": (i32, [vp, i64, i64, i32, vp, vp, i64, vp, vp]),
        "mrpop_nearest_work": (i32, [vp, i64, i64, i32, vp, vp, i64, vp, vp]),
        "mrpop_neighbors": (i32, [vp, i64, i64, i32, vp, i64, f32, i64, vp, vp, vp]),
        "mrpop_path_cost": (i32, [vp, i64, i32, vp, vp]),
        "mrpop_plan": (i32, [vp, C.c_double, vp, i64, vp, vp]),
        "mrpop_plan_trace": (i32, [vp, vp, vp, i64, vp, vp]),
        "mrpop_plan_batch": (i32, [vp, i32, C.c_double, i64, vp, vp]),
        "mrpop_plan_result": (i32, [vp, vp, i64, vp, vp]),
        "mrpop_plan_history": (i32, [vp, i64, vp, i64, vp, vp]),
        "mrpop_server_create": (i32, [i32, i64, vp]),
        "mrpop_server_submit": (i32, [vp, vp, C.c_double, i64, C.c_double, vp]),
        "mrpop_server_poll": (i32, [vp, i64, vp, vp, vp]),
        "mrpop_server_stats": (i32, [vp, vp]),
        "mrpop_server_destroy": (i32, [vp]),
        "mrpop_fp32_peak": (i32, [i32, i32, vp, vp]),
        "mrpop_planner_nearest_pass": (i32, [vp, i64, i64, i32, vp, vp, i32, i32, vp, vp]),
        "mrpop_planner_neighbors_pass": (i32, [vp, i64, i64, i32, vp, i64, f32, vp, vp, vp]),
        "mrpop_plan_batch_ex": (i32, [vp, i32, C.c_double, i64, vp, vp, i32]),
        "mrpop_set_persistent_limits": (i32, [i32, i64]),
        "mrpop_set_launch_ex": (i32, [vp, i32, i32, i32, i32]),
        "mrpop_get_launch": (i32, [vp, vp]),
        "mrpop_autotune_cache_save": (i32, [C.c_char_p]),
        "mrpop_autotune_cache_load": (i32, [C.c_char_p]),
        "mrpop_autotune_cache_clear": (i32, []),
        "mrpop_nearest_autotune": (i32, [vp, i64, i64, i32, vp, vp, i64, i32, vp, vp, vp, vp]),
        "mrpop_neighbors_autotune": (i32, [vp, i64, i64, i32, vp, i64, f32, i64, vp, vp, vp, vp,
                                           vp]),
        "mrpop_server_cancel": (i32, [vp, i64]),
        "mrpop_server_inject": (i32, [vp, i32, i64]),
        "mrpop_scratch_stats": (i32, [i32, vp]),
        "mrpop_plan_batch_phase_stats": (i32, [vp, vp, vp]),
    }
    for name in EXPORTS:
        fn = getattr(L, name)
        fn.restype, fn.argtypes = sig[name]
    return L


lib = _load()


def _check(status: int) -> None:
    if status != 0:
        raise MrpopError(status, lib.mrpop_last_error().decode())


def _stream(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dptr(t: Optional[torch.Tensor], dtype: torch.dtype, name: str) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


class Problem:
    """Owns an ``mrpop_problem`` handle built from a ``synth.Scene``-like
    object (robots with dh/q_lo/q_hi/sphere_link/sphere_xyzr/base, and
    obs_spheres/obs_cuboids) on the current CUDA device."""

    def __init__(self, scene, resolution: float = 0.02, margin: float = 0.0,
                 delta: float = 1.0, n_per_round: int = 64, tree_cap: int = 1 << 16,
                 roadmap_cap: int = 1 << 14, max_iters: int = 4096, seed: int = 0,
                 start: Optional[Sequence[float]] = None,
                 goal: Optional[Sequence[float]] = None, self_collision: bool = False):
        keep = []
        robots = (_Robot * len(scene.robots))()
        for i, r in enumerate(scene.robots):
            arrs = [_host(r.dh, np.float32), _host(r.q_lo, np.float32),
                    _host(r.q_hi, np.float32), _host(r.sphere_link, np.int32),
                    _host(r.sphere_xyzr, np.float32)]
            keep += arrs
            robots[i].dof = int(r.dof)
            robots[i].n_spheres = int(len(r.sphere_link))
            robots[i].dh, robots[i].q_lo, robots[i].q_hi = (a.ctypes.data for a in arrs[:3])
            robots[i].sphere_link, robots[i].sphere_xyzr = arrs[3].ctypes.data, arrs[4].ctypes.data
            for j, v in enumerate(np.asarray(r.base, dtype=np.float32).reshape(12)):
                robots[i].base[j] = float(v)
            sm = getattr(r, "self_mask", None)
            if sm is not None:
                sm = _host(sm, np.uint16)
                keep.append(sm)
                robots[i].self_mask = sm.ctypes.data
        osph = _host(np.asarray(scene.obs_spheres).reshape(-1, 4), np.float32)
        ocub = _host(np.asarray(scene.obs_cuboids).reshape(-1, 15), np.float32)
        keep += [osph, ocub]
        obs = _Obstacles(osph.shape[0], osph.ctypes.data if osph.size else None,
                         ocub.shape[0], ocub.ctypes.data if ocub.size else None)
        cfg = _Config(resolution, margin, delta, n_per_round, tree_cap, roadmap_cap,
                      max_iters, seed, int(bool(self_collision)))
        st = _host(start, np.float32) if start is not None else None
        gl = _host(goal, np.float32) if goal is not None else None
        keep += [a for a in (st, gl) if a is not None]
        h = C.c_void_p()
        _check(lib.mrpop_create_problem(robots, len(scene.robots), C.byref(obs),
                                        st.ctypes.data if st is not None else None,
                                        gl.ctypes.data if gl is not None else None,
                                        C.byref(cfg), C.byref(h)))
        self._h = h
        D, K, S = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib.mrpop_problem_dims(h, C.byref(D), C.byref(K), C.byref(S)))
        self.D, self.K, self.S = D.value, K.value, S.value
        self.resolution, self.margin = resolution, margin

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise ValueError("problem destroyed")
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib.mrpop_destroy_problem(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _edges(p: Problem, qa: torch.Tensor, qb: torch.Tensor) -> int:
    if qa.shape != qb.shape or qa.dim() != 2 or qa.shape[0] != p.D:
        raise ValueError(f"qa, qb must both be [D={p.D}, n]")
    return int(qa.shape[1])


def fk(p: Problem, q: torch.Tensor, out: Optional[torch.Tensor] = None,
       stream=None) -> torch.Tensor:
    """World sphere centres [3, S, n] of configurations q [D, n]."""
    n = int(q.shape[1])
    if out is None:
        out = torch.empty((3, p.S, n), dtype=torch.float32, device=q.device)
    _check(lib.mrpop_fk(p.handle, _dptr(q, torch.float32, "q"), n,
                        _dptr(out, torch.float32, "out"), _stream(stream)))
    return out


def validate_edges(p: Problem, qa: torch.Tensor, qb: torch.Tensor,
                   valid: Optional[torch.Tensor] = None, length: Optional[torch.Tensor] = None,
                   npoints: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    n = _edges(p, qa, qb)
    if valid is None:
        valid = torch.empty(n, dtype=torch.uint8, device=qa.device)
    _check(lib.mrpop_validate_edges_ex(
        p.handle, _dptr(qa, torch.float32, "qa"), _dptr(qb, torch.float32, "qb"), n,
        _dptr(valid, torch.uint8, "valid"), _dptr(length, torch.float32, "length"),
        _dptr(npoints, torch.int32, "npoints"), _stream(stream)))
    return valid


def edge_clearance(p: Problem, qa: torch.Tensor, qb: torch.Tensor,
                   out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    n = _edges(p, qa, qb)
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=qa.device)
    _check(lib.mrpop_edge_clearance(p.handle, _dptr(qa, torch.float32, "qa"),
                                    _dptr(qb, torch.float32, "qb"), n,
                                    _dptr(out, torch.float32, "min_clear"), _stream(stream)))
    return out


def validate_work(p: Problem, qa: torch.Tensor, qb: torch.Tensor, stream=None) -> torch.Tensor:
    n = _edges(p, qa, qb)
    out = torch.zeros(12, dtype=torch.int64, device=qa.device)   # MRPOP_WORK_COUNTERS
    _check(lib.mrpop_validate_work(p.handle, _dptr(qa, torch.float32, "qa"),
                                   _dptr(qb, torch.float32, "qb"), n,
                                   _dptr(out, torch.int64, "counters"), _stream(stream)))
    return out


def autotune(p: Problem, qa: torch.Tensor, qb: torch.Tensor, stream=None) -> tuple:
    """Tunes p's validation launch on these edges: (warps, order, fine_stage, ms)."""
    n = _edges(p, qa, qb)
    valid = torch.empty(n, dtype=torch.uint8, device=qa.device)
    cfg = np.zeros(3, dtype=np.int32)
    ms = C.c_float()
    _check(lib.mrpop_autotune(p.handle, _dptr(qa, torch.float32, "qa"),
                              _dptr(qb, torch.float32, "qb"), n, valid.data_ptr(),
                              cfg.ctypes.data, C.byref(ms), _stream(stream)))
    return int(cfg[0]), int(cfg[1]), int(cfg[2]), ms.value


def set_launch(p: Problem, warps_per_block: int, order: int, fine_stage: int = 0,
               registers: int = 0) -> None:
    _check(lib.mrpop_set_launch_ex(p.handle, int(warps_per_block), int(order), int(fine_stage),
                                   int(registers)))


def get_launch(p: Problem) -> tuple:
    """(warps per block, order, fine stage, register budget) of p's validation."""
    out = (C.c_int32 * 4)()
    _check(lib.mrpop_get_launch(p.handle, out))
    return tuple(int(v) for v in out)


def autotune_cache_save(path: str) -> None:
    _check(lib.mrpop_autotune_cache_save(os.fsencode(path)))


def autotune_cache_load(path: str) -> None:
    _check(lib.mrpop_autotune_cache_load(os.fsencode(path)))


def autotune_cache_clear() -> None:
    _check(lib.mrpop_autotune_cache_clear())


def nearest_autotune(tree: torch.Tensor, queries: torch.Tensor, budgets: torch.Tensor,
                     filter: int = 0, stream=None) -> tuple:
    """Tunes the budget-ordered NEAREST's slice waves for this shape; returns
    (indices, waves, ms per call)."""
    dim, ld = int(tree.shape[0]) - 1, int(tree.shape[1])
    Q = int(queries.shape[1])
    out = torch.empty(Q, dtype=torch.int64, device=queries.device)
    w, ms = C.c_int32(), C.c_float()
    _check(lib.mrpop_nearest_autotune(_dptr(tree, torch.float32, "tree"), ld, ld, dim,
                                      _dptr(queries, torch.float32, "queries"),
                                      _dptr(budgets, torch.float32, "budgets"), Q, int(filter),
                                      _dptr(out, torch.int64, "out_idx"), C.byref(w),
                                      C.byref(ms), _stream(stream)))
    return out, w.value, ms.value


def neighbors_autotune(tree: torch.Tensor, queries: torch.Tensor, delta: float, k_max: int,
                       dim: Optional[int] = None, stream=None) -> tuple:
    """Tunes NEIGHBORS's vertex ranges for this shape; returns (indices,
    counts, warps per SM, ms per call)."""
    dim = int(queries.shape[0]) if dim is None else int(dim)
    ld = int(tree.shape[1])
    Q = int(queries.shape[1])
    idx = torch.empty((Q, max(k_max, 1)), dtype=torch.int64, device=queries.device)
    cnt = torch.empty(Q, dtype=torch.int64, device=queries.device)
    t, ms = C.c_int32(), C.c_float()
    _check(lib.mrpop_neighbors_autotune(_dptr(tree, torch.float32, "tree"), ld, ld, dim,
                                        _dptr(queries, torch.float32, "queries"), Q,
                                        float(delta), int(k_max),
                                        _dptr(idx, torch.int64, "out_idx"),
                                        _dptr(cnt, torch.int64, "out_cnt"), C.byref(t),
                                        C.byref(ms), _stream(stream)))
    return idx[:, :k_max], cnt, t.value, ms.value


NEAREST_FILTER_FP32 = 0     # MRPOP_NEAREST_FILTER_FP32 (the default)
NEAREST_FILTER_TENSOR = 1   # MRPOP_NEAREST_FILTER_TENSOR


def nearest(tree: torch.Tensor, queries: torch.Tensor, budgets: torch.Tensor,
            n_vertices: Optional[int] = None, out: Optional[torch.Tensor] = None,
            stream=None, filter: int = NEAREST_FILTER_FP32) -> torch.Tensor:
    """tree [dim+1, ld] (row dim = g), queries [dim, Q], budgets [Q] -> int64 [Q].
    filter picks the large-batch expansion filter (FP32 FMA or tensor cores);
    the indices do not depend on it."""
    dim = int(tree.shape[0]) - 1
    ld = int(tree.shape[1])
    N = ld if n_vertices is None else int(n_vertices)
    Q = int(queries.shape[1])
    if queries.shape[0] != dim or budgets.shape != (Q,):
        raise ValueError("queries must be [dim, Q] and budgets [Q]")
    if out is None:
        out = torch.empty(Q, dtype=torch.int64, device=queries.device)
    _check(lib.mrpop_nearest_ex(_dptr(tree, torch.float32, "tree"), N, ld, dim,
                                _dptr(queries, torch.float32, "queries"),
                                _dptr(budgets, torch.float32, "budgets"), Q, int(filter),
                                _dptr(out, torch.int64, "out_idx"), _stream(stream)))
    return out


ROADMAP_DEGREE_CAP = 64    # MRPOP_ROADMAP_DEGREE_CAP


def planner_nearest_pass(tree: torch.Tensor, queries: torch.Tensor, budgets: torch.Tensor,
                         pass_: int = 0, n_vertices: Optional[int] = None,
                         stream=None) -> torch.Tensor:
    """One pass of the planner's own NEAREST kernel (test hook): tree [dim+1,
    ld], queries [dim, Q <= 256], budgets [Q] -> int64 [Q]."""
    dim, ld = int(tree.shape[0]) - 1, int(tree.shape[1])
    N = ld if n_vertices is None else int(n_vertices)
    Q = int(queries.shape[1])
    out = torch.empty(Q, dtype=torch.int64, device=queries.device)
    _check(lib.mrpop_planner_nearest_pass(_dptr(tree, torch.float32, "tree"), N, ld, dim,
                                          _dptr(queries, torch.float32, "queries"),
                                          _dptr(budgets, torch.float32, "budgets"), Q,
                                          int(pass_), _dptr(out, torch.int64, "out_idx"),
                                          _stream(stream)))
    return out


def planner_neighbors_pass(V: torch.Tensor, queries: torch.Tensor, delta: float,
                           n_vertices: Optional[int] = None, stream=None):
    """One pass of the planner's roadmap NEIGHBORS kernel (test hook): V [dof,
    ld], queries [dof, Q] -> (int64 [Q, 64], int64 [Q])."""
    dof, ld = int(V.shape[0]), int(V.shape[1])
    N = ld if n_vertices is None else int(n_vertices)
    Q = int(queries.shape[1])
    idx = torch.empty((Q, ROADMAP_DEGREE_CAP), dtype=torch.int64, device=queries.device)
    cnt = torch.empty(Q, dtype=torch.int64, device=queries.device)
    _check(lib.mrpop_planner_neighbors_pass(_dptr(V, torch.float32, "V"), N, ld, dof,
                                            _dptr(queries, torch.float32, "queries"), Q,
                                            float(delta), _dptr(idx, torch.int64, "out_idx"),
                                            _dptr(cnt, torch.int64, "out_cnt"), _stream(stream)))
    return idx, cnt


def nearest_work(tree: torch.Tensor, queries: torch.Tensor, budgets: torch.Tensor,
                 n_vertices: Optional[int] = None, stream=None) -> int:
    """(query, vertex) pairs nearest() evaluates for these inputs."""
    dim, ld = int(tree.shape[0]) - 1, int(tree.shape[1])
    N = ld if n_vertices is None else int(n_vertices)
    Q = int(queries.shape[1])
    out = C.c_int64()
    _check(lib.mrpop_nearest_work(_dptr(tree, torch.float32, "tree"), N, ld, dim,
                                  _dptr(queries, torch.float32, "queries"),
                                  _dptr(budgets, torch.float32, "budgets"), Q, C.byref(out),
                                  _stream(stream)))
    return out.value


def neighbors(tree: torch.Tensor, queries: torch.Tensor, delta: float, k_max: int,
              dim: Optional[int] = None, n_vertices: Optional[int] = None,
              stream=None) -> tuple:
    """Radius query: returns (idx [Q, k_max] int64 with -1 padding, count [Q])."""
    dim = int(queries.shape[0]) if dim is None else dim
    ld = int(tree.shape[1])
    N = ld if n_vertices is None else int(n_vertices)
    Q = int(queries.shape[1])
    idx = torch.empty((Q, k_max), dtype=torch.int64, device=queries.device)
    cnt = torch.empty(Q, dtype=torch.int64, device=queries.device)
    _check(lib.mrpop_neighbors(_dptr(tree, torch.float32, "tree"), N, ld, dim,
                               _dptr(queries, torch.float32, "queries"), Q, float(delta),
                               k_max, _dptr(idx, torch.int64, "out_idx") if k_max else None,
                               _dptr(cnt, torch.int64, "out_cnt"), _stream(stream)))
    return idx, cnt


def path_cost(path: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """C(sigma) of a path [M, dim] -> float64 tensor [1] on the device."""
    M, dim = int(path.shape[0]), int(path.shape[1])
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=path.device)
    _check(lib.mrpop_path_cost(_dptr(path, torch.float32, "path"), M, dim,
                               _dptr(out, torch.float64, "cost"), _stream(stream)))
    return out


def fp32_peak(packed: bool = False, iters: int = 32768, stream=None) -> float:
    """Measured FP32 FMA throughput of the current device (TFLOP/s)."""
    out = C.c_double()
    _check(lib.mrpop_fp32_peak(int(bool(packed)), int(iters), C.byref(out), _stream(stream)))
    return out.value


def plan(p: Problem, time_budget_s: float, path_cap: int = 1 << 16) -> tuple:
    """Runs the planner on p for time_budget_s seconds.  Returns (path
    float32 [M, D] or None, cost); cost is +inf when no path was found."""
    buf = np.zeros((path_cap, p.D), dtype=np.float32)
    n, cost = C.c_int64(), C.c_double()
    st = lib.mrpop_plan(p.handle, float(time_budget_s), buf.ctypes.data, path_cap,
                        C.byref(n), C.byref(cost))
    if st == 6:  # MRPOP_ENOSOLUTION
        return None, float("inf")
    _check(st)
    return buf[:n.value].copy(), cost.value


def plan_history(p: Problem, index: int, path_cap: int = 1 << 16) -> tuple:
    """(path float32 [M, D], cost) of the index-th accepted incumbent."""
    buf = np.zeros((path_cap, p.D), dtype=np.float32)
    n, cost = C.c_int64(), C.c_double()
    _check(lib.mrpop_plan_history(p.handle, int(index), buf.ctypes.data, path_cap, C.byref(n),
                                  C.byref(cost)))
    return buf[:n.value].copy(), cost.value


def plan_trace(p: Problem) -> tuple:
    """(times, costs, iterations) of the incumbent history."""
    n, it = C.c_int64(), C.c_int64()
    _check(lib.mrpop_plan_trace(p.handle, None, None, 0, C.byref(n), C.byref(it)))
    t = np.zeros(max(n.value, 1))
    c = np.zeros(max(n.value, 1))
    _check(lib.mrpop_plan_trace(p.handle, t.ctypes.data, c.ctypes.data, n.value, None, None))
    return t[:n.value], c[:n.value], it.value


BATCH_PERSISTENT = 0   # MRPOP_BATCH_PERSISTENT (mrpop_plan_batch)
BATCH_STEPPED = 1      # MRPOP_BATCH_STEPPED


def plan_batch(problems, time_budget_s: float, max_steps: int = 0, targets=None,
               form: int = BATCH_PERSISTENT) -> np.ndarray:
    """Plans all problems at once (one persistent launch, or the stepped
    form); returns their int32 statuses."""
    n = len(problems)
    hs = (C.c_void_p * n)(*[p.handle.value for p in problems])
    st = np.zeros(n, dtype=np.int32)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.float64)
    _check(lib.mrpop_plan_batch_ex(hs, n, float(time_budget_s), int(max_steps),
                                   None if tg is None else tg.ctypes.data, st.ctypes.data,
                                   int(form)))
    return st


PLAN_PHASE_NAMES = ("start", "roadmap_sample", "roadmap_candidate_check", "roadmap_append",
                    "roadmap_neighbors", "roadmap_candidate_edges", "roadmap_edge_check",
                    "roadmap_link_bfs", "search_sample", "nearest_own_tree", "direction_oracle",
                    "extension_check", "insert", "nearest_other_tree", "connection_prep",
                    "connection_check", "solution", "res4_recheck", "accept",
                    "phase_transitions")


def plan_batch_phase_stats() -> dict:
    """Where the last persistent launch's CTA time went: {phase: (ns, chunks)},
    plus 'ctas' and 'wall_ns'."""
    n = len(PLAN_PHASE_NAMES)
    ns, ch, cw = (C.c_int64 * n)(), (C.c_int64 * n)(), (C.c_int64 * 2)()
    _check(lib.mrpop_plan_batch_phase_stats(ns, ch, cw))
    out = {k: (int(ns[i]), int(ch[i])) for i, k in enumerate(PLAN_PHASE_NAMES)}
    out["ctas"], out["wall_ns"] = int(cw[0]), int(cw[1])
    return out


def set_persistent_limits(ctas: int = 0, idle_polls: int = 0) -> None:
    """Process-wide limits of the persistent launch (tests, diagnostics)."""
    _check(lib.mrpop_set_persistent_limits(int(ctas), int(idle_polls)))


def plan_result(p: Problem, path_cap: int = 1 << 16) -> tuple:
    """(path float32 [M, D] or None, cost) of the best path found so far."""
    buf = np.zeros((path_cap, p.D), dtype=np.float32)
    n, cost = C.c_int64(), C.c_double()
    st = lib.mrpop_plan_result(p.handle, buf.ctypes.data, path_cap, C.byref(n), C.byref(cost))
    if st == 6:
        return None, float("inf")
    _check(st)
    return buf[:n.value].copy(), cost.value


FAULT_ADMIT_ENOMEM = 1   # MRPOP_FAULT_ADMIT_ENOMEM
FAULT_STALL_MS = 2       # MRPOP_FAULT_STALL_MS


class Server:
    """Continuous-batching planning server (mrpop_server_*)."""

    def __init__(self, max_slots: int = 64, device_mem_budget: int = 0):
        h = C.c_void_p()
        _check(lib.mrpop_server_create(int(max_slots), int(device_mem_budget), C.byref(h)))
        self._h = h

    def submit(self, p: Problem, budget_s: float, max_steps: int = 0,
               target_cost: float = float("nan")) -> int:
        t = C.c_int64()
        _check(lib.mrpop_server_submit(self._h, p.handle, float(budget_s), int(max_steps),
                                       float(target_cost), C.byref(t)))
        return t.value

    def poll(self, ticket: int) -> tuple:
        """(state, times[4], cost); raises MrpopError for a failed request."""
        st = C.c_int32()
        times = np.zeros(4)
        cost = C.c_double()
        _check(lib.mrpop_server_poll(self._h, int(ticket), C.byref(st), times.ctypes.data,
                                     C.byref(cost)))
        return st.value, times, cost.value

    def poll_status(self, ticket: int) -> tuple:
        """(state, times[4], cost, status): like poll, with a failed or
        cancelled request's status returned instead of raised."""
        st = C.c_int32()
        times = np.zeros(4)
        cost = C.c_double()
        status = lib.mrpop_server_poll(self._h, int(ticket), C.byref(st), times.ctypes.data,
                                       C.byref(cost))
        if status == 1:   # EINVAL: unknown ticket
            _check(status)
        return st.value, times, cost.value, int(status)

    def cancel(self, ticket: int) -> None:
        _check(lib.mrpop_server_cancel(self._h, int(ticket)))

    def inject(self, fault: int, count: int) -> None:
        """Host-side fault injection (FAULT_ADMIT_ENOMEM, FAULT_STALL_MS)."""
        _check(lib.mrpop_server_inject(self._h, int(fault), int(count)))

    def stats(self) -> dict:
        v = np.zeros(6, dtype=np.int64)
        _check(lib.mrpop_server_stats(self._h, v.ctypes.data))
        return dict(zip(("admitted", "completed", "peak_active", "peak_mem", "mem_budget",
                         "queued"), (int(x) for x in v)))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            lib.mrpop_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
