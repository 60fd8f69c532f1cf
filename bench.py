#!/usr/bin/env python3
"""Throughput of the MR. POP motion-validation hot path on one GB300.

Workload (2 synthetic 7-DOF arms facing each other over a table, 32 cuboids +
32 spheres, composite 14-DOF; edge resolution 0.02 rad, contact margin 1e-4 m):
one step is one pass of the whole hot path over one batch of synthetic input:

  1. mrpop_validate_edges   65,536 candidate composite edges (interpolation,
                            per-robot FK to spheres, sphere-vs-obstacle and
                            robot-vs-robot tests, early exit)
  2. mrpop_nearest          65,536 cost-filtered NEAREST queries (one per
                            candidate edge) over a 16,384-vertex state-cost tree
  3. mrpop_neighbors        1,024 radius queries (delta = 1.2 rad, k_max = 32)
                            over a 4,096-vertex 7-DOF per-robot roadmap
  4. mrpop_path_cost        cost of a 65,537-vertex composite path

The parts are independent: the timed step runs 1 on the main stream, 2 on a
second and 3 + 4 on a third, and ends when all have; each kernel's own time
(for the rooflines) comes from the same steps run one part after another.

metric: edge checks/s = 65,536 / step time (device time, CUDA events, inputs
resident in HBM, L2 flushed between steps).  All data are synthetic.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; every rank validates its own
batch (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

E_EDGES = 65536
NN_TREE = 16384
NN_QUERIES = 65536
RM_VERTS = 4096
RM_QUERIES = 1024
RM_DELTA = 1.2
RM_KMAX = 32
PATH_M = 65537
RES = 0.02
MARGIN = 1e-4
METRIC = "edge checks/sec"
UNIT = "edges/s"
WORKLOAD = "table_pair_14dof_65536_edges"

# FP32 arithmetic per counted unit (FMA = 2 flops; compares and the
# transcendental sincosf excluded), matching the kernel's formulas.
FLOPS_PER = {
    "joint_transform": 51,      # interpolate, add offset, F = T Rz, T = F Tz Tx Rx
    "bound_test": 10,           # |c - c_o|^2 vs (r + r_o + m)^2
    "sphere_obstacle_test": 11,
    "cuboid_test": 31,          # R^T (c - c_b), clamp excess, squared norm
    "box_bound_test": 31,       # the same box distance for a tile bound
    "pair_test": 11,
    "point_transform": 18,      # R p + t
    "tile_bound": 390,          # centroid and max radius of 32 coarse centres
}


def tile_level_flops(cnt) -> float:
    """The part of algorithmic_flops spent on the kernel's own tile level (its
    bounds and the tests against them), which the paper's method does not have."""
    c = [int(x) for x in cnt]
    return (c[8] * FLOPS_PER["bound_test"] + c[9] * FLOPS_PER["tile_bound"]
            + c[11] * FLOPS_PER["box_bound_test"])


def algorithmic_flops(cnt) -> float:
    c = [int(x) for x in cnt]
    return (c[1] * FLOPS_PER["joint_transform"]
            + (c[2] + c[3]) * FLOPS_PER["bound_test"]
            + c[4] * FLOPS_PER["sphere_obstacle_test"]
            + c[5] * FLOPS_PER["cuboid_test"]
            + c[6] * FLOPS_PER["pair_test"]
            + c[7] * FLOPS_PER["point_transform"]
            + c[8] * FLOPS_PER["bound_test"]
            + c[9] * FLOPS_PER["tile_bound"]
            + (c[10] + c[11]) * FLOPS_PER["box_bound_test"])


# The same FP32 weights per unit of the paper's two-stage check (Sec. III-E),
# whose units the oracle counts (oracle.WORK_UNITS): FK, one coarse sphere per
# link tested against every obstacle and every other robot's link, then the
# fine spheres of the links a coarse test hit.
METHOD_FLOPS_PER = {
    "joints": 51,           # a joint transform, as above
    "coarse_points": 18,    # R p + t
    "coarse_sphere": 11,    # |c - c_o|^2 vs (r + r_o + m)^2
    "coarse_cuboid": 31,    # R^T (c - c_b), clamp excess, squared norm
    "coarse_pair": 11,
    "fine_points": 18,
    "fine_sphere": 11,
    "fine_cuboid": 31,
    "fine_pair": 11,
}
METHOD_SAMPLE = 1024


def make_inputs(rank: int):
    """Seeded synthetic inputs of one step (numpy, host)."""
    import numpy as np

    from paper_2609_30644_gb300 import synth
    scene = synth.table_pair_scene(0)
    qa, qb = synth.candidate_edges(scene, E_EDGES, seed=rank)
    D = scene.D
    lo, hi = scene.q_lo, scene.q_hi
    tree = synth.random_tree_fast(D, NN_TREE, lo, hi, seed=100 + rank)
    qs, cs = synth.nn_queries(D, NN_QUERIES, lo, hi, seed=200 + rank,
                              budget_lo=10.0, budget_hi=40.0)
    r0 = scene.robots[0]
    roadmap = synth.random_tree_fast(r0.dof, RM_VERTS, r0.q_lo, r0.q_hi, seed=300 + rank)
    rq, _ = synth.nn_queries(r0.dof, RM_QUERIES, r0.q_lo, r0.q_hi, seed=400 + rank)
    rng = np.random.default_rng(500 + rank)
    path = np.ascontiguousarray(
        rng.uniform(lo, hi, (PATH_M, D)).astype(np.float32))
    return scene, dict(qa=qa, qb=qb, tree=tree, qs=qs, cs=cs, roadmap=roadmap, rq=rq, path=path)


# ---------------------------------------------------------------------------
# CPU oracle leg (the oracle as it stands, on the host cores)
# ---------------------------------------------------------------------------

_WORKER_CACHE = {}


def _oracle_chunk(args):
    """Worker: runs the oracle over one slice of the sampled step and returns
    the time of the oracle calls alone (inputs are generated once per worker
    process, outside the timing)."""
    rank, e_idx, q_idx, r_idx, path_len = args
    import numpy as np

    import oracle
    if rank not in _WORKER_CACHE:
        scene, x = make_inputs(rank)
        _WORKER_CACHE[rank] = (oracle.OracleScene(scene), x)
    o, x = _WORKER_CACHE[rank]
    t0 = time.perf_counter()
    qa = np.ascontiguousarray(x["qa"][:, e_idx])
    qb = np.ascontiguousarray(x["qb"][:, e_idx])
    o.validate_edges(qa, qb, RES, MARGIN, early_exit=True)
    for i in q_idx:
        oracle.nearest(x["tree"], x["qs"][:, i], x["cs"][i])
    for i in r_idx:
        oracle.neighbors(x["roadmap"], x["rq"][:, i], RM_DELTA, RM_KMAX)
    if path_len > 1:
        oracle.path_cost(x["path"][:path_len])
    return time.perf_counter() - t0


def oracle_sample(n_edges: int, workers: int, rank: int = 0):
    """Times the oracle on a bounded sample of the step with the same
    per-edge composition (1 nearest query per edge, 1 radius query per 64
    edges, path vertices = edges + 1), spread over ``workers`` processes."""
    import multiprocessing as mpr

    import numpy as np
    stride = max(1, E_EDGES // n_edges)
    e_all = np.arange(0, stride * n_edges, stride)[:n_edges]
    q_all = e_all.copy()
    r_all = np.arange(0, RM_QUERIES, max(1, RM_QUERIES // max(1, n_edges // 64)))[:max(1, n_edges // 64)]
    chunks = []
    for w in range(workers):
        chunks.append((rank, e_all[w::workers], q_all[w::workers], r_all[w::workers],
                       (n_edges + 1) if w == 0 else 0))
    ctx = mpr.get_context("spawn")
    import oracle
    oracle.build()
    with ctx.Pool(workers) as pool:
        # warm every worker (input generation), then time the slices; the
        # slices run concurrently, one per process, so the step takes as long
        # as the slowest slice
        pool.map(_oracle_chunk, [(rank, e_all[:1], q_all[:1], r_all[:1], 2)] * (4 * workers),
                 chunksize=1)
        times = pool.map(_oracle_chunk, chunks, chunksize=1)
    wall = max(times)
    return n_edges / wall, wall


def oracle_method_flops(scene, qa, qb, early_exit: bool):
    """CPU-leg part of the roofline: the oracle's count of the paper's
    two-stage check (Sec. III-E) over a stride sample of METHOD_SAMPLE edges
    of a batch (host SoA [D, E]), weighted per unit by METHOD_FLOPS_PER.
    Returns (flops per edge, units, edges sampled, seconds)."""
    import numpy as np

    import oracle
    E = qa.shape[1]
    idx = np.arange(0, E, max(1, E // METHOD_SAMPLE))[:METHOD_SAMPLE]
    t0 = time.perf_counter()
    counts, _ = oracle.OracleScene(scene).method_work(
        np.ascontiguousarray(qa[:, idx]), np.ascontiguousarray(qb[:, idx]), RES, MARGIN,
        early_exit=early_exit)
    units = dict(zip(oracle.WORK_UNITS, (int(c) for c in counts)))
    flops = sum(units[k] * w for k, w in METHOD_FLOPS_PER.items())
    return flops / len(idx), units, len(idx), time.perf_counter() - t0


def run_reference(args) -> None:
    """--impl reference: the FP64 oracle (this method's only reference
    implementation) timed on the host cores, on the same workload and metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    workers = os.cpu_count() or 1
    n = max(64, 16 * workers)
    vals = []
    for _ in range(args.warmup):
        oracle_sample(min(n, 64), workers)
    walls = []
    for _ in range(args.steps):
        v, w = oracle_sample(n, workers)
        vals.append(v)
        walls.append(w)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * statistics.median(walls), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "edges_per_step_sample": n, "res_rad": RES,
                   "margin_m": MARGIN},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": f"{n} edges (+{n} nearest queries over {NN_TREE} vertices, "
                                   f"{max(1, n // 64)} radius queries, {n + 1}-vertex path "
                                   f"cost) of the {E_EDGES}-edge batch per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200", "-f", self.path]
            if self.uuid:
                cmd.insert(1, f"--id={self.uuid}")
            self.proc = subprocess.Popen(cmd, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx),
                       reasons=sorted(reasons), samples=len(sm))
        try:
            os.unlink(self.path)
        except Exception:
            pass
        return out


# ---------------------------------------------------------------------------
# planner leg: problems solved per second to 1.1x best cost, plain vs batched
# ---------------------------------------------------------------------------
PLAN_PROBLEMS = 256     # the batched workload: 256 problems of 2-8 arms
PLAIN_SAMPLE = 16       # problems the one-at-a-time planner and the references run
BATCHED_BUDGET_S = 10.0
PLAN_BUDGET_S = 1.5
PLAN_DELTA = 2.5
LONG_FACTOR = 10   # best-cost runs (GPU batched, CPU reference) get 10x the budget


def plan_problems(mp, synth, n: int):
    """Heterogeneous batched-workload problems (2..8 synthetic 7-DOF arms,
    16..256 obstacles).  Start and goal are drawn uniformly and accepted when
    the library's clearance is above 2 mm; scenes without such a pair in 10,240
    draws are skipped."""
    import numpy as np
    import torch
    out = []
    idx = 0
    while len(out) < n and idx < 4 * n:
        sc = synth.batched_scene(idx)
        stream = synth.config_stream(sc, idx)
        found = []
        with mp.Problem(sc) as tmp:
            for _ in range(40):
                qs = np.stack([next(stream) for _ in range(256)], axis=1)
                qd = torch.from_numpy(qs).cuda()
                c = mp.edge_clearance(tmp, qd, qd).cpu().numpy()
                found += [qs[:, i].copy() for i in np.nonzero(c > 2e-3)[0]]
                if len(found) >= 2:
                    break
        if len(found) >= 2:
            out.append((idx, sc, found[0], found[1]))
        idx += 1
    return out


def _ref_plan_worker(args):
    """Worker: the FP64 reference planner (oracle side) on one planner-leg
    problem, rebuilt from its scene index, with the GPU planner's parameters."""
    idx, qs, qg, budget = args
    import oracle as orc
    from paper_2609_30644_gb300 import synth
    r = orc.plan_reference(synth.batched_scene(idx), qs, qg, resolution=RES, margin=MARGIN,
                           delta=PLAN_DELTA, n_per_round=64, max_iters=4096,
                           time_budget_s=budget, seed=idx)
    return r["times"], r["costs"], r["iterations"], r["status"]


def run_reference_planner(entries, budget: float):
    """The reference planner over the leg's problems, one process per problem
    on the host cores (spawn pool, started after the GPU legs finished)."""
    import multiprocessing as mpr
    import oracle
    oracle.build()
    workers = min(len(entries), os.cpu_count() or 1)
    jobs = [(idx, qs.astype("float64"), qg.astype("float64"), budget)
            for idx, _, qs, qg in entries]
    t0 = time.perf_counter()
    with mpr.get_context("spawn").Pool(workers) as pool:
        out = pool.map(_ref_plan_worker, jobs, chunksize=1)
    return out, workers, time.perf_counter() - t0


def run_planner_leg(mp, synth, n_problems: int = PLAN_PROBLEMS, plain_sample: int = PLAIN_SAMPLE,
                    batched_budget: float = PLAN_BUDGET_S):
    """Plain (one problem at a time, on the first plain_sample problems: its
    throughput does not depend on how many follow) against batched (all
    n_problems at once, batched_budget of wall time); the FP64 reference and a
    long batched run on the same sample supply best-cost candidates."""
    import numpy as np

    def make(entry):
        idx, sc, qs, qg = entry
        return mp.Problem(sc, resolution=RES, margin=MARGIN, delta=PLAN_DELTA, n_per_round=64,
                          tree_cap=1 << 15, roadmap_cap=1 << 13, max_iters=4096, seed=idx,
                          start=qs, goal=qg)

    entries = plan_problems(mp, synth, n_problems)
    sample = entries[:plain_sample]
    traces = {"plain": [], "batched": []}
    for e in sample:                                   # one problem at a time
        p = make(e)
        mp.plan(p, PLAN_BUDGET_S)
        traces["plain"].append(mp.plan_trace(p)[:2])
        p.close()
    probs = [make(e) for e in entries]                 # all problems at once
    t0 = time.perf_counter()
    mp.plan_batch(probs, batched_budget)               # one persistent launch
    batched_wall = time.perf_counter() - t0
    phases = mp.plan_batch_phase_stats()
    traces["batched"] = [mp.plan_trace(p)[:2] for p in probs]
    for p in probs:
        p.close()
    probs = [make(e) for e in entries]                 # the stepped batch form
    t0 = time.perf_counter()
    mp.plan_batch(probs, batched_budget, form=mp.BATCH_STEPPED)
    stepped_wall = time.perf_counter() - t0
    traces["batched_stepped"] = [mp.plan_trace(p)[:2] for p in probs]
    for p in probs:
        p.close()
    # a long batched run that only supplies best-cost candidates
    probs = [make(e) for e in sample]
    mp.plan_batch(probs, LONG_FACTOR * PLAN_BUDGET_S)
    long_final = [mp.plan_trace(p)[1] for p in probs]
    long_final = [c[-1] if len(c) else np.inf for c in long_final]
    for p in probs:
        p.close()
    # CPU baseline: the FP64 reference planner on the same problems (it cannot
    # finish a first roadmap on most of them within the GPU's budget)
    ref_out, ref_workers, ref_wall = run_reference_planner(sample, LONG_FACTOR * PLAN_BUDGET_S)
    traces["cpu_reference"] = [(np.asarray(t), np.asarray(c)) for t, c, _, _ in ref_out]
    kinds = ("plain", "batched", "batched_stepped", "cpu_reference")
    final = lambda c: c[-1] if len(c) else np.inf
    best = np.minimum(np.array([final(c) for t, c in traces["batched"]]),
                      np.array([final(c) for t, c in traces["batched_stepped"]]))
    m = len(sample)
    for cand in ([final(c) for t, c in traces["plain"]], [final(c) for t, c in traces["cpu_reference"]],
                 long_final):
        best[:m] = np.minimum(best[:m], cand)
    res = {"problems": len(entries), "plain_sample": m, "budget_s": PLAN_BUDGET_S,
           "batched_budget_s": batched_budget,
           "robots": [int(e[1].K) for e in entries], "batched_wall_s": batched_wall,
           "batched_stepped_wall_s": stepped_wall,
           "batched_form": "one persistent launch (mrpop_plan_batch)",
           "batched_stepped_form": "a captured graph per step (mrpop_plan_batch_ex, stepped)",
           "best_cost_from": (f"minimum final cost over the plain and both batched runs, a "
                              f"{LONG_FACTOR}x-budget batched run and the FP64 reference "
                              f"(the last three on the first {m} problems)")}
    for k in kinds:
        reach, ttfs = [], []
        for (t, c), b in zip(traces[k], best):
            hit = np.nonzero(c <= 1.1 * b)[0] if len(c) else []
            reach.append(float(t[hit[0]]) if len(hit) else None)
            if len(t):
                ttfs.append(float(t[0]))
        solved = sum(r is not None for r in reach)
        budget = {"plain": PLAN_BUDGET_S, "batched": batched_budget,
                  "batched_stepped": batched_budget,
                  "cpu_reference": LONG_FACTOR * PLAN_BUDGET_S}[k]
        spent = [r if r is not None else budget for r in reach]
        # plain: problems run back to back; batched: all at once; the CPU
        # reference: back to back on each of its cores (sum / cores)
        wall = (sum(spent) if k == "plain" else max(spent) if k.startswith("batched")
                else sum(spent) / ref_workers)
        res[k] = {"problems": len(reach), "solved_to_1.1x_best": solved, "wall_s": wall,
                  "problems_per_s": solved / wall if wall > 0 else 0.0,
                  "ttfs_p50_s": float(np.percentile(ttfs, 50)) if ttfs else None,
                  "ttfs_p99_s": float(np.percentile(ttfs, 99)) if ttfs else None,
                  "first_solutions": len(ttfs)}
    # The plain planner's time to first solution when all n problems arrive
    # together and it takes them one at a time, moving on at each first
    # solution (or at its budget): problem k waits for the problems before it.
    # Built from the sample's measured first-solution times, cycled over n.
    firsts = [float(t[0]) if len(t) else PLAN_BUDGET_S for t, c in traces["plain"]]
    if firsts:
        queued = np.cumsum([firsts[i % len(firsts)] for i in range(len(entries))])
        res["plain"]["ttfs_queued_p50_s"] = float(np.percentile(queued, 50))
        res["plain"]["ttfs_queued_p99_s"] = float(np.percentile(queued, 99))
        res["plain"]["ttfs_queued"] = (f"{len(entries)} problems submitted together, taken one at "
                                       f"a time to their first solution (measured first-solution "
                                       f"times of the {len(firsts)}-problem sample, cycled)")
    res["cpu_reference"].update({
        "kind": "oracle (FP64 reference planner, Alg. 1/2 sequential)", "cores": ref_workers,
        "budget_s": LONG_FACTOR * PLAN_BUDGET_S,
        "pool_wall_s": ref_wall, "iterations": [int(x[2]) for x in ref_out],
        "statuses": [int(x[3]) for x in ref_out]})
    if res["plain"]["problems_per_s"] > 0:
        res["batched_over_plain"] = res["batched"]["problems_per_s"] / res["plain"]["problems_per_s"]
    # where the persistent launch's CTA time went, by phase kind
    busy = sum(phases[k][0] for k in mp.PLAN_PHASE_NAMES)
    if busy > 0:
        res["batched"]["phase_share"] = {k: round(phases[k][0] / busy, 4)
                                         for k in mp.PLAN_PHASE_NAMES if phases[k][0] > 0}
        res["batched"]["phase_chunks"] = {k: phases[k][1] for k in mp.PLAN_PHASE_NAMES
                                          if phases[k][1] > 0}
        res["batched"]["cta_busy_fraction"] = (busy / (phases["ctas"] * phases["wall_ns"])
                                               if phases["ctas"] and phases["wall_ns"] else None)
    if res["batched_stepped"]["problems_per_s"] > 0:
        res["persistent_over_stepped"] = (res["batched"]["problems_per_s"] /
                                          res["batched_stepped"]["problems_per_s"])
    return res, entries, best


SERVE_RATES = "10,30,100,300,1000"
# resident requests at most (device-memory admission applies below this); with
# first-solution targets at 1000/s, 64 / 128 / 256 slots completed 72 / 107 /
# 140 requests/s, so the GPU has room for more than 64
SERVE_SLOTS = 256
SERVE_REQUESTS = 200


def run_serving_leg(mp, synth, entries, best, rate: float,
                    n_requests: int = SERVE_REQUESTS):
    """Poisson stream of planning requests (the planner leg's problems, cycled)
    into the continuous-batching server.  Each request ends at 1.1x its
    problem's best known cost or after the planner budget.  Reports p50/p99
    time to first solution and to the target, and completed requests/s."""
    import numpy as np
    arrivals = synth.poisson_arrivals(rate, n_requests, seed=7)
    reqs = []
    with mp.Server(max_slots=SERVE_SLOTS) as srv:
        t0 = time.perf_counter()
        for k, ta in enumerate(arrivals):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0005)
            j = k % len(entries)
            idx, sc, qs, qg = entries[j]
            p = mp.Problem(sc, resolution=RES, margin=MARGIN, delta=PLAN_DELTA, n_per_round=64,
                           tree_cap=1 << 15, roadmap_cap=1 << 13, max_iters=4096, seed=idx,
                           start=qs, goal=qg)
            tgt = 1.1 * best[j] if np.isfinite(best[j]) else float("inf")
            reqs.append((p, srv.submit(p, PLAN_BUDGET_S, target_cost=tgt)))
        done = {}
        while len(done) < len(reqs):
            for p, t in reqs:
                if t not in done:
                    st, times, _ = srv.poll(t)
                    if st == 2:
                        done[t] = times
            time.sleep(0.002)
        wall = time.perf_counter() - t0
        stats = srv.stats()
    for p, _ in reqs:
        p.close()
    tt = np.array([done[t] for _, t in reqs])
    first = tt[:, 1][tt[:, 1] >= 0]
    target = tt[:, 2][tt[:, 2] >= 0]
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    return {"rate_per_s": rate, "requests": len(reqs), "wall_s": wall,
            "completed_per_s": len(reqs) / wall, "ttfs_p50_s": pct(first, 50),
            "ttfs_p99_s": pct(first, 99), "to_1.1x_best_p50_s": pct(target, 50),
            "to_1.1x_best_p99_s": pct(target, 99), "reached_1.1x_best": int(len(target)),
            "first_solutions": int(len(first)), "peak_concurrent": stats["peak_active"],
            "max_slots": SERVE_SLOTS}


def kernel_source_sha(kernel_files: str) -> str:
    """sha256 over the kernel's source files ('+'-separated names under csrc/,
    concatenated in that order)."""
    import hashlib
    h = hashlib.sha256()
    for f in kernel_files.split("+"):
        h.update(open(os.path.join(ROOT, "paper_2609_30644_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def profiled_traffic(kernel_files: str, name: str):
    """DRAM bytes per launch of a kernel from the committed ncu summary
    profiles/<name>.txt, when that summary was taken on the current source of
    kernel_files (their sha256 is recorded there); None otherwise."""
    path = os.path.join(ROOT, "profiles", name + ".txt")
    try:
        rec = dict(l.split(":", 1) for l in open(path) if ":" in l and not l.startswith("#"))
        sha = kernel_source_sha(kernel_files)
        if rec.get("source_sha256", "").strip() != sha:
            return None
        return float(rec["dram_bytes_per_launch"])
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_profile_leg(args) -> None:
    """--profile-leg: one kernel's leg of the step alone, for ncu captures of
    a known launch.  validate-free: the free-set construction (one validation
    launch), then W warm-up and K timed launches on the free set;
    validate-mixed: W + K launches on the step's mixed batch; nearest (FP32
    filter) and nearest-tensor: W + K NEAREST calls (one filter launch each).  The validation launch shape is
    --launch (warps per block, order, fine stage, optional register budget).  Prints one JSON line with
    the mean time of the timed launches."""
    import numpy as np
    import torch

    import paper_2609_30644_gb300 as mp
    from paper_2609_30644_gb300 import synth as _synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    scene, x = make_inputs(0)
    stream = torch.cuda.current_stream()
    w, o, f, *r = (int(v) for v in args.launch.split(","))
    with mp.Problem(scene, resolution=RES, margin=MARGIN) as prob:
        mp.set_launch(prob, w, o, f, registers=r[0] if r else 0)
        if args.profile_leg == "validate-free":
            cqa, cqb = _synth.candidate_edges(scene, 3 * E_EDGES, seed=1000)
            cqa_d, cqb_d = torch.from_numpy(cqa).to(dev), torch.from_numpy(cqb).to(dev)
            keep = mp.validate_edges(prob, cqa_d, cqb_d).bool()
            sel = torch.nonzero(keep).flatten()[:E_EDGES]
            qa, qb = cqa_d[:, sel].contiguous(), cqb_d[:, sel].contiguous()
            run = lambda out: mp.validate_edges(prob, qa, qb, out)
            out = torch.empty(E_EDGES, dtype=torch.uint8, device=dev)
        elif args.profile_leg == "validate-mixed":
            qa = torch.from_numpy(x["qa"]).to(dev)
            qb = torch.from_numpy(x["qb"]).to(dev)
            run = lambda out: mp.validate_edges(prob, qa, qb, out)
            out = torch.empty(E_EDGES, dtype=torch.uint8, device=dev)
        else:
            tree = torch.from_numpy(x["tree"]).to(dev)
            qs = torch.from_numpy(x["qs"]).to(dev)
            cs = torch.from_numpy(x["cs"]).to(dev)
            filt = (mp.NEAREST_FILTER_TENSOR if args.profile_leg == "nearest-tensor"
                    else mp.NEAREST_FILTER_FP32)
            run = lambda out: mp.nearest(tree, qs, cs, out=out, filter=filt)
            out = torch.empty(NN_QUERIES, dtype=torch.int64, device=dev)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        for _ in range(args.warmup):
            run(out)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run(out)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    print(json.dumps({"profile_leg": args.profile_leg, "launch": args.launch,
                      "steps": args.steps, "warmup": args.warmup,
                      "ms": statistics.mean(ms) if ms else None}), flush=True)


def run_ours(args) -> None:
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        workers = os.cpu_count() or 1
        n = 256 * workers
        v, wall = oracle_sample(n, workers)
        v1, wall1 = oracle_sample(256, 1)
        cpu = {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"{n} edges (every {E_EDGES // n}th of the batch) with {n} nearest "
                         f"queries over {NN_TREE} vertices, {n // 64} radius queries and a "
                         f"{n + 1}-vertex path cost; {wall:.1f} s wall on {workers} processes",
               "single_core_value": v1,
               "single_core_sample": f"256 edges of the same composition on one process, "
                                     f"{wall1:.1f} s"}

    import numpy as np
    import torch

    import paper_2609_30644_gb300 as mp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2609_30644_gb300 import replicas
    dist = replicas.init("nccl", dev)   # replicas: no collective on the data path

    scene, x = make_inputs(rank)
    prob = mp.Problem(scene, resolution=RES, margin=MARGIN)
    g = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in x.items()}
    valid = torch.empty(E_EDGES, dtype=torch.uint8, device=dev)
    nn_out = torch.empty(NN_QUERIES, dtype=torch.int64, device=dev)
    cost = torch.empty(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(inp, ev=None):
        if ev is not None:
            ev[0].record(stream)
        mp.validate_edges(prob, inp["qa"], inp["qb"], valid)
        if ev is not None:
            ev[1].record(stream)
        mp.nearest(g["tree"], inp["qs"], inp["cs"], out=nn_out)
        if ev is not None:
            ev[2].record(stream)
        idx, cnt = mp.neighbors(g["roadmap"], inp["rq"], RM_DELTA, RM_KMAX, dim=scene.robots[0].dof)
        if ev is not None:
            ev[3].record(stream)
        mp.path_cost(inp["path"], out=cost)
        if ev is not None:
            ev[4].record(stream)
        return idx, cnt

    # The step as it runs in the timed loop: the three independent parts of
    # the path on three streams -- validation on the main stream, NEAREST on
    # a second, NEIGHBORS and path cost on a third -- so that each fills the
    # SMs the others leave idle (their ordering passes, launch gaps and grid
    # tails); the step ends when all three have.  The sequential form above
    # times each kernel on its own for the rooflines.
    s_nn = torch.cuda.Stream(device=dev)
    s_rm = torch.cuda.Stream(device=dev)
    e_fork, e_nn, e_rm = torch.cuda.Event(), torch.cuda.Event(), torch.cuda.Event()

    def step_concurrent(inp):
        e_fork.record(stream)
        s_nn.wait_event(e_fork)
        s_rm.wait_event(e_fork)
        mp.validate_edges(prob, inp["qa"], inp["qb"], valid)
        with torch.cuda.stream(s_nn):
            mp.nearest(g["tree"], inp["qs"], inp["cs"], out=nn_out)
            e_nn.record(s_nn)
        with torch.cuda.stream(s_rm):
            idx, cnt = mp.neighbors(g["roadmap"], inp["rq"], RM_DELTA, RM_KMAX,
                                    dim=scene.robots[0].dof)
            mp.path_cost(inp["path"], out=cost)
            e_rm.record(s_rm)
        return idx, cnt

    def join():
        stream.wait_event(e_nn)
        stream.wait_event(e_rm)

    # launch shapes from the autotuners (validation, NEAREST, NEIGHBORS),
    # then the algorithmic work of the validation launch on this batch (all
    # untimed)
    tuned = mp.autotune(prob, g["qa"], g["qb"])
    tuned_regs = mp.get_launch(prob)[3]
    _, nn_waves, _ = mp.nearest_autotune(g["tree"], g["qs"], g["cs"])
    _, _, nb_target, _ = mp.neighbors_autotune(g["roadmap"], g["rq"], RM_DELTA, RM_KMAX,
                                               dim=scene.robots[0].dof)
    counters = mp.validate_work(prob, g["qa"], g["qb"]).cpu().numpy()
    flops_per_launch = algorithmic_flops(counters)
    # (query, vertex) pairs NEAREST evaluates: vertices whose cost-to-come
    # already exceeds a block's largest budget are never admissible (Alg. 2)
    nn_pairs = mp.nearest_work(g["tree"], g["qs"], g["cs"])

    for _ in range(max(args.warmup, 0)):
        step(g)
        step_concurrent(g)
        join()
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    replicas.barrier(dist)
    torch.cuda.synchronize()
    clocks.start()
    ends = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                       # L2 flush (256 MB > 129 MB L2), untimed
        ends[i][0].record(stream)
        step_concurrent(g)
        join()
        ends[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    # the same steps with the parts one after another, for each kernel's time
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        step(g, evs[i])
    torch.cuda.synchronize()
    replicas.barrier(dist)
    clk = clocks.stop()

    step_ms = [e[0].elapsed_time(e[1]) for e in ends]
    seq_step_ms = [e[0].elapsed_time(e[4]) for e in evs]
    val_ms = [e[0].elapsed_time(e[1]) for e in evs]
    nn_ms = [e[1].elapsed_time(e[2]) for e in evs]
    rm_ms = [e[2].elapsed_time(e[3]) for e in evs]
    pc_ms = [e[3].elapsed_time(e[4]) for e in evs]
    total_ms = replicas.max_over_ranks(dist, float(sum(step_ms)), dev)
    ms_per_step = total_ms / args.steps
    value = world * E_EDGES / (ms_per_step / 1000.0)
    ms_per_step_sequential = statistics.mean(seq_step_ms)

    # ---- end to end through the public API with host buffers -------------
    pin = {k: torch.from_numpy(np.ascontiguousarray(x[k])).pin_memory()
           for k in ("qa", "qb", "qs", "cs", "rq", "path")}
    h_valid = torch.empty(E_EDGES, dtype=torch.uint8).pin_memory()
    h_nn = torch.empty(NN_QUERIES, dtype=torch.int64).pin_memory()
    h_idx = torch.empty((RM_QUERIES, RM_KMAX), dtype=torch.int64).pin_memory()
    h_cnt = torch.empty(RM_QUERIES, dtype=torch.int64).pin_memory()
    h_cost = torch.empty(1, dtype=torch.float64).pin_memory()
    d_in = {k: torch.empty_like(v, device=dev) for k, v in pin.items()}
    h2d = sum(v.numel() * v.element_size() for v in pin.values())
    d2h = sum(t.numel() * t.element_size() for t in (h_valid, h_nn, h_idx, h_cnt, h_cost))

    # One step with its copies overlapped: each of the three parts copies its
    # own inputs in on its own stream, runs, and copies its results back, so
    # every part starts as soon as its inputs have landed and the copies of
    # the others overlap its kernels.  The step ends when all three are done.
    def e2e_step():
        e_fork.record(stream)
        s_nn.wait_event(e_fork)
        s_rm.wait_event(e_fork)
        with torch.cuda.stream(s_nn):
            d_in["qs"].copy_(pin["qs"], non_blocking=True)
            d_in["cs"].copy_(pin["cs"], non_blocking=True)
            mp.nearest(g["tree"], d_in["qs"], d_in["cs"], out=nn_out)
            h_nn.copy_(nn_out, non_blocking=True)
            e_nn.record(s_nn)
        with torch.cuda.stream(s_rm):
            d_in["rq"].copy_(pin["rq"], non_blocking=True)
            d_in["path"].copy_(pin["path"], non_blocking=True)
            idx, cnt = mp.neighbors(g["roadmap"], d_in["rq"], RM_DELTA, RM_KMAX,
                                    dim=scene.robots[0].dof)
            mp.path_cost(d_in["path"], out=cost)
            h_idx.copy_(idx, non_blocking=True)
            h_cnt.copy_(cnt, non_blocking=True)
            h_cost.copy_(cost, non_blocking=True)
            e_rm.record(s_rm)
        d_in["qa"].copy_(pin["qa"], non_blocking=True)
        d_in["qb"].copy_(pin["qb"], non_blocking=True)
        mp.validate_edges(prob, d_in["qa"], d_in["qb"], valid)
        h_valid.copy_(valid, non_blocking=True)
        join()

    for _ in range(max(args.warmup, 1)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_total = replicas.max_over_ranks(dist, float(sum(e2e_ms)), dev)
    e2e_value = world * E_EDGES / (e2e_total / args.steps / 1000.0)

    # sanity: the e2e results equal the resident-input results
    assert torch.equal(h_valid, valid.cpu()) and torch.equal(h_nn, nn_out.cpu())
    step_valid_fraction = float(valid.float().mean().item())  # (valid is reused below)

    # ---- validation on a free edge set (every checkpoint runs to the end) --
    # Seeded candidates of the same generator, of which the first E_EDGES that
    # the kernel accepts form the set (its verdicts are parity-tested against
    # the oracle); early exit cannot skip work here, so this set carries the
    # validation roofline.
    from paper_2609_30644_gb300 import synth as _synth
    cqa, cqb = _synth.candidate_edges(scene, 3 * E_EDGES, seed=1000 + rank)
    cqa_d = torch.from_numpy(cqa).to(dev)
    cqb_d = torch.from_numpy(cqb).to(dev)
    keep = mp.validate_edges(prob, cqa_d, cqb_d).bool()
    sel = torch.nonzero(keep).flatten()[:E_EDGES]
    assert sel.numel() == E_EDGES, "too few free candidates"
    fqa = cqa_d[:, sel].contiguous()
    fqb = cqb_d[:, sel].contiguous()
    del cqa_d, cqb_d
    free_counters = mp.validate_work(prob, fqa, fqb).cpu().numpy()
    free_flops = algorithmic_flops(free_counters)
    for _ in range(max(args.warmup, 0)):
        mp.validate_edges(prob, fqa, fqb, valid)
    torch.cuda.synchronize()
    free_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mp.validate_edges(prob, fqa, fqb, valid)
        b.record(stream)
        b.synchronize()
        free_ms.append(a.elapsed_time(b))
    assert bool(valid.bool().all())

    # ---- the other validation workloads: the planar pair (6-DOF) and the
    # four-arm grid (28-DOF), mixed candidate edges of the same generator, each
    # with its own autotuned launch
    others = {}
    for name, make_scene in (("planar_pair_6dof", lambda: _synth.planar_pair_scene(0)),
                             ("grid4_28dof", lambda: _synth.grid4_scene(0))):
        osc = make_scene()
        oqa, oqb = _synth.candidate_edges(osc, E_EDGES, seed=2000 + rank)
        oqa_d = torch.from_numpy(oqa).to(dev)
        oqb_d = torch.from_numpy(oqb).to(dev)
        ov = torch.empty(E_EDGES, dtype=torch.uint8, device=dev)
        with mp.Problem(osc, resolution=RES, margin=MARGIN) as op:
            otuned = mp.autotune(op, oqa_d, oqb_d)
            oregs = mp.get_launch(op)[3]
            for _ in range(max(args.warmup, 0)):
                mp.validate_edges(op, oqa_d, oqb_d, ov)
            torch.cuda.synchronize()
            oms = []
            for _ in range(args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                mp.validate_edges(op, oqa_d, oqb_d, ov)
                b.record(stream)
                b.synchronize()
                oms.append(a.elapsed_time(b))
        others[name] = {"edges": E_EDGES, "robots": osc.K, "dof": osc.D,
                        "obstacles": f"{len(osc.obs_spheres)} spheres + {len(osc.obs_cuboids)} cuboids",
                        "edge_set": "mixed", "ms": statistics.mean(oms),
                        "edges_per_s": E_EDGES / (statistics.mean(oms) / 1000.0),
                        "valid_fraction": float(ov.float().mean().item()),
                        "validate_launch": {"warps_per_block": otuned[0],
                                            "order": ["strided", "contiguous"][otuned[1]],
                                            "fine_stage": ["union", "reassigned"][otuned[2]],
                                            "registers": ["compact", "wide"][oregs]}}
        del oqa_d, oqb_d

    # ---- CPU leg: the oracle's count of the paper's two-stage check on a
    # 1,024-edge sample of the free set and of the step's mixed batch
    method = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        samp = torch.arange(0, E_EDGES, E_EDGES // METHOD_SAMPLE, device=dev)[:METHOD_SAMPLE]
        f_fpe, f_units, f_n, f_s = oracle_method_flops(
            scene, fqa[:, samp].cpu().numpy(), fqb[:, samp].cpu().numpy(), early_exit=False)
        m_fpe, m_units, m_n, m_s = oracle_method_flops(scene, x["qa"], x["qb"], early_exit=True)
        method = {"free": (f_fpe, f_units, f_n, f_s), "mixed": (m_fpe, m_units, m_n, m_s)}

    # ---- NEAREST with the tensor-core filter (an option beside the default
    # FP32 filter; same indices), timed alone on the step's inputs
    nn_tc_out = torch.empty_like(nn_out)
    for _ in range(max(args.warmup, 0)):
        mp.nearest(g["tree"], g["qs"], g["cs"], out=nn_tc_out, filter=mp.NEAREST_FILTER_TENSOR)
    torch.cuda.synchronize()
    nn_tc_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mp.nearest(g["tree"], g["qs"], g["cs"], out=nn_tc_out, filter=mp.NEAREST_FILTER_TENSOR)
        b.record(stream)
        b.synchronize()
        nn_tc_ms.append(a.elapsed_time(b))
    assert torch.equal(nn_tc_out, nn_out), "the NEAREST filters disagree"

    # ---- measured FP32 FMA rate (roofline denominator) ---------------------
    fma_scalar = mp.fp32_peak(False)
    fma_packed = mp.fp32_peak(True)

    planner = serving = None
    if rank == 0 and not args.no_planner:
        from paper_2609_30644_gb300 import synth as _synth
        planner, entries, best = run_planner_leg(
            mp, _synth, args.planner_problems,
            min(args.planner_problems, args.plain_sample), args.batched_budget)
        serving = [run_serving_leg(mp, _synth, entries, best, float(r), args.serving_requests)
                   for r in args.serving_rates.split(",")]
        serving = serving[0] if len(serving) == 1 else serving

    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        peaks = measured_peaks()
        sm_max = float(peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0)
        derived_tflops = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
        peak_tflops = max(fma_scalar, fma_packed)
        peak_source = (f"measured FMA-chain rate (scalar {fma_scalar:.1f}, packed f32x2 "
                       f"{fma_packed:.1f} TFLOP/s; derived {props.multi_processor_count} SMs x "
                       f"128 lanes x 2 x {sm_max:.0f} MHz = {derived_tflops:.1f}) (of measured)")
        val_avg_s = statistics.mean(val_ms) / 1000.0
        achieved = flops_per_launch / val_avg_s / 1e12
        free_avg_s = statistics.mean(free_ms) / 1000.0
        free_achieved = free_flops / free_avg_s / 1e12
        # NEAREST (the step's default FP32 filter): per (query, vertex) pair the
        # budget ordering keeps, the expansion filter runs D fused
        # multiply-adds (2 D flops) on the FMA pipe, against the FP32 peak.
        # The definition's own count (D subtractions and D multiply-adds, 3 D
        # flops per pair) is given beside it.  The time is that of the whole
        # NEAREST call (ordering, seeding, filter, reduce), so the rates are
        # lower bounds for the filter kernel alone.
        # The tensor-core option: the same filter as one contraction over D +
        # 2 terms (coordinates and the two squared norms) per pair, mma.sync
        # with FP16 operands up to D + 2 = 16, TF32 above; FP16's dense peak
        # equals bf16's (the measured GEMM rate), TF32's is that rate times
        # the nominal dense TF32 / bf16 ratio (1.1 / 2.25 PFLOP/s).
        bf16_peak = float(peaks.get("bf16_tflops") or 1900.0)
        nn_f16 = scene.D + 2 <= 16
        nn_tc_kernel = f"nearest_tc16_kernel<{scene.D}>" if nn_f16 else f"nearest_tc_kernel<{scene.D}>"
        nn_kernel = f"nearest_f32_kernel<{scene.D}>"
        tc_peak = bf16_peak if nn_f16 else bf16_peak * 1.1 / 2.25
        nn_s = statistics.mean(nn_ms) / 1000.0
        nn_tc_s = statistics.mean(nn_tc_ms) / 1000.0
        nn_f32_flops = float(nn_pairs) * 2 * scene.D
        nn_tc_flops = float(nn_pairs) * 2 * (scene.D + 2)
        # the definition's work per (query, vertex) pair: D differences and D
        # squares added up (3D), the cost-to-come added and the budget compared
        nn_flops = float(nn_pairs) * (3 * scene.D + 2)
        nn_all_flops = float(NN_QUERIES) * NN_TREE * (3 * scene.D + 2)
        # HBM side of the same launches: each input is read once, each output
        # written once (algorithmic bytes)
        hbm_peak = float(peaks.get("hbm_gbs") or 6658.3)
        nn_bytes = 4.0 * (scene.D + 1) * NN_TREE + 4.0 * (scene.D + 1) * NN_QUERIES + 8.0 * NN_QUERIES
        val_bytes = 2 * 4.0 * scene.D * E_EDGES + E_EDGES
        hbm = {}
        for k, b, ms_ in (("nearest", nn_bytes, statistics.mean(nn_ms)),
                          ("validate_mixed", val_bytes, statistics.mean(val_ms))):
            gbs = b / (ms_ / 1000.0) / 1e9
            hbm[k] = {"bytes_per_launch": b, "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                      "frac": gbs / hbm_peak}
        # Validation on the free set (no early exit), two counts of its work:
        #  * method: the paper's two-stage check (Sec. III-E) as the oracle
        #    counts it on a 1,024-edge sample (FK, a coarse sphere per link
        #    against every obstacle and every other robot's link, fine tests on
        #    coarse hits), scaled to the launch -- the algorithmic work;
        #  * kernel: what this kernel evaluates by its own counters, whose tile
        #    level (bounds over 32 checkpoints, tests against them) culls most
        #    of the method's coarse tests; its share is shown apart.
        free_tile = tile_level_flops(free_counters)
        roofline_validate = {
            "bound": "alu", "kernel": "validate_kernel",
            "edge_set": "free (65,536 accepted edges, no early exit)",
            "peak": peak_tflops, "unit": "TFLOP/s", "peak_source": peak_source,
            "ms": statistics.mean(free_ms), "edges_per_s": E_EDGES / free_avg_s,
            "traffic": profiled_traffic("validate.cu+validate_body.cuh",
                                        "validate_kernel_table_pair_free"),
            "kernel_flops_per_launch": free_flops,
            "kernel_achieved": free_achieved, "kernel_frac": free_achieved / peak_tflops,
            "kernel_tile_level_flops": free_tile,
            "kernel_tile_level_share": free_tile / free_flops if free_flops else None,
            "kernel_frac_without_tile_level":
                (free_flops - free_tile) / free_avg_s / 1e12 / peak_tflops}
        if method is not None:
            f_fpe, f_units, f_n, f_s = method["free"]
            m_fpe, m_units, m_n, m_s = method["mixed"]
            method_flops = f_fpe * E_EDGES
            roofline_validate.update({
                "achieved": method_flops / free_avg_s / 1e12,
                "frac": method_flops / free_avg_s / 1e12 / peak_tflops,
                "flops_per_launch": method_flops,
                "count": "method (oracle two-stage count, Sec. III-E)",
                "method_flops": method_flops,
                "method_frac": method_flops / free_avg_s / 1e12 / peak_tflops,
                "method_flops_per_edge": f_fpe,
                "method_units_sample": f_units,
                "method_sample": f"{f_n} edges (every {E_EDGES // f_n}th of the free set), "
                                 f"counted by the FP64 oracle in {f_s:.1f} s",
                "method_flops_per_edge_mixed_early_exit": m_fpe,
                "method_units_mixed_sample": m_units})
        else:
            roofline_validate.update({
                "achieved": free_achieved, "frac": free_achieved / peak_tflops,
                "flops_per_launch": free_flops,
                "count": "kernel counters (the oracle's method count runs in the CPU leg, "
                         "which was skipped)"})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "edges": E_EDGES, "robots": 2, "dof": scene.D,
                       "obstacles": "32 cuboids + 32 spheres", "res_rad": RES,
                       "margin_m": MARGIN, "nearest": f"{NN_QUERIES} queries x {NN_TREE} vertices",
                       "neighbors": f"{RM_QUERIES} queries x {RM_VERTS} vertices, 7-DOF",
                       "path_vertices": PATH_M, "l2": "flushed between steps (256 MB write)",
                       "streams": ("validation, NEAREST, and NEIGHBORS + path cost on three "
                                   "streams in the timed step; kernel times and shares from "
                                   "the same steps run one part after another"),
                       "nearest_filter": "FP32 FMA expansion filter, exact FP32 decision",
                       "validate_launch": {"warps_per_block": tuned[0],
                                           "order": ["strided", "contiguous"][tuned[1]],
                                           "fine_stage": ["union", "reassigned"][tuned[2]],
                                           "registers": ["compact", "wide"][tuned_regs],
                                           "autotune_ms": tuned[3]},
                       "nearest_launch": {"slice_waves": nn_waves},
                       "neighbors_launch": {"warps_per_sm": nb_target},
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline_nearest": {
                "bound": "alu", "kernel": nn_kernel, "filter": "FP32 FMA (default)",
                "achieved": nn_f32_flops / nn_s / 1e12, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": nn_f32_flops / nn_s / 1e12 / peak_tflops,
                "traffic": profiled_traffic("nearest.cu", "nearest_f32_kernel_table_pair"),
                "peak_source": peak_source,
                "flops_per_launch": nn_f32_flops,
                "pairs_evaluated": int(nn_pairs),
                "pairs_all": NN_QUERIES * NN_TREE,
                "ms": statistics.mean(nn_ms),
                "definition_rate_tflops": nn_flops / nn_s / 1e12,
                "definition_frac_of_fp32": nn_flops / nn_s / 1e12 / peak_tflops,
                "all_pairs_definition_rate_tflops": nn_all_flops / nn_s / 1e12,
                "share_of_step": statistics.mean(nn_ms) / ms_per_step_sequential},
            "roofline_nearest_tensor": {
                "bound": "tensor", "kernel": nn_tc_kernel,
                "filter": "tensor cores (option; not in the step)",
                "achieved": nn_tc_flops / nn_tc_s / 1e12, "peak": tc_peak, "unit": "TFLOP/s",
                "frac": nn_tc_flops / nn_tc_s / 1e12 / tc_peak,
                "traffic": profiled_traffic("nearest.cu", nn_tc_kernel.split("<")[0] + "_table_pair"),
                "peak_source": (f"FP16 dense = measured bf16 GEMM {bf16_peak:.1f} TFLOP/s "
                                "(of measured)" if nn_f16 else
                                f"TF32 dense = measured bf16 GEMM {bf16_peak:.1f} TFLOP/s x "
                                "1.1 / 2.25 (of measured)"),
                "flops_per_launch": nn_tc_flops, "ms": statistics.mean(nn_tc_ms),
                "queries_per_s": NN_QUERIES / nn_tc_s},
            "roofline_validate": roofline_validate,
            "roofline_validate_mixed": {"bound": "alu", "kernel": "validate_kernel",
                                        "edge_set": "mixed (the step's batch)",
                                        "achieved": achieved, "peak": peak_tflops,
                                        "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                                        "traffic": profiled_traffic("validate.cu+validate_body.cuh",
                                                                    "validate_kernel_table_pair"),
                                        "peak_source": peak_source,
                                        "flops_per_launch": flops_per_launch,
                                        "share_of_step": statistics.mean(val_ms) / ms_per_step_sequential},
            "roofline_hbm": hbm,
            "ms_per_step_sequential": ms_per_step_sequential,
            "kernel_ms": {"validate": statistics.mean(val_ms), "nearest": statistics.mean(nn_ms),
                          "neighbors": statistics.mean(rm_ms), "path_cost": statistics.mean(pc_ms)},
            "valid_fraction": step_valid_fraction,
            "work_counters": [int(c) for c in counters],
            "nearest_queries_per_s": NN_QUERIES / (statistics.mean(nn_ms) / 1000.0),
            "wall_s_timed_loop": t_wall,
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            # per step: validate; NEAREST = setup (+ g range), histogram (+
            # scan), scatter, seeding (+ cuts) and the FP32 filter kernel (+
            # reduce); neighbors over vertex ranges + the ordered merge; path
            # cost + its sum
            "gpu_launches": 10 * args.steps,
            "cpu_baseline": cpu,
            "planner": planner,
            "serving": serving,
        }
        # the headline roofline: edge validation on the free set, where early
        # exit cannot skip work
        line["roofline"] = line["roofline_validate"]
        line["other_workloads"] = others
        line = {k: line[k] for k in ["metric", "value", "unit", "n_gpus", "steps", "warmup",
                                     "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
                                     "dtype", "data", "config", "roofline"]
                + [k for k in line if k not in ("metric", "value", "unit", "n_gpus", "steps",
                                                 "warmup", "ms_per_step", "higher_is_better",
                                                 "scaling", "vs_baseline", "dtype", "data",
                                                 "config", "roofline")]}
        print(json.dumps(line), flush=True)
    prob.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-planner", action="store_true",
                    help="skip the plain-vs-batched planner leg (problems/s to 1.1x best)")
    ap.add_argument("--planner-problems", type=int, default=PLAN_PROBLEMS,
                    help="problems planned at once in the batched planner leg (256: the "
                         "batched workload of 2-8 arms)")
    ap.add_argument("--plain-sample", type=int, default=PLAIN_SAMPLE,
                    help="problems the plain planner and the CPU reference run, one at a time")
    ap.add_argument("--batched-budget", type=float, default=BATCHED_BUDGET_S,
                    help="wall-clock budget of the batched planner run (s)")
    ap.add_argument("--serving-rates", default=SERVE_RATES,
                    help="comma-separated Poisson arrival rates of the serving leg (1/s)")
    ap.add_argument("--serving-requests", type=int, default=SERVE_REQUESTS,
                    help="requests per serving rate")
    ap.add_argument("--profile-leg", choices=["validate-free", "validate-mixed", "nearest",
                                              "nearest-tensor"],
                    default=None, help="run one kernel's leg alone (for ncu captures)")
    ap.add_argument("--launch", default="4,0,0",
                    help="validation launch of --profile-leg: warps per block, order, fine "
                         "stage[, register budget]")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_leg:
        run_profile_leg(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
