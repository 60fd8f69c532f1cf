"""GB300 (sm_103a) motion validation and nearest-neighbour library for MR. POP.

This package is a thin binding over the C ABI in ``include/mrpop.h``
(``libmrpop.so``, built in-tree by ``build.py``).  Every function here only
marshals arguments (torch tensors -> device pointers, torch streams -> raw
``cudaStream_t``); all computation runs in the library's CUDA kernels.  There
is no CPU fallback: the first use of an operation loads ``libmrpop.so`` and
raises ImportError if it has not been built.  The submodules ``synth`` (input
generators) and ``build`` import without the library.
"""
from __future__ import annotations

_OPS = ("MrpopError", "Problem", "edge_clearance", "fk", "lib", "library_path", "nearest",
        "neighbors", "path_cost", "validate_edges", "validate_work", "EXPORTS", "plan", "plan_trace",
        "plan_batch", "plan_result", "Server", "autotune", "set_launch",
        "plan_history", "fp32_peak", "nearest_work", "NEAREST_FILTER_FP32",
        "NEAREST_FILTER_TENSOR", "planner_nearest_pass", "planner_neighbors_pass",
        "ROADMAP_DEGREE_CAP", "BATCH_PERSISTENT", "BATCH_STEPPED", "set_persistent_limits",
        "get_launch", "autotune_cache_save", "autotune_cache_load", "autotune_cache_clear",
        "nearest_autotune", "neighbors_autotune", "FAULT_ADMIT_ENOMEM", "FAULT_STALL_MS",
        "plan_batch_phase_stats", "PLAN_PHASE_NAMES")


def __getattr__(name):
    if name in _OPS:
        from . import _capi
        return getattr(_capi, name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")


def __dir__():
    return sorted(list(globals()) + list(_OPS))
