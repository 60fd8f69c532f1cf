"""Continuous-batching server (mrpop_server_*): requests that arrive while
others run are admitted as slots and device memory free up, their work
overlaps on the device, and each result is the same alone and in the mix."""
import time

import numpy as np
import pytest
import torch

from paper_2609_30644_gb300 import synth
from test_gpu_planner import RES, _check_path, _start_goal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    import paper_2609_30644_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return m


@pytest.fixture(scope="module")
def cases(orc):
    out = []
    for seed in (0, 2, 3):
        scene = synth.planar_pair_scene(seed)
        qs, qg, o = _start_goal(orc, scene, seed)
        out.append((seed, scene, qs, qg, o))
    return out


def _make(mp, case):
    seed, scene, qs, qg, _ = case
    return mp.Problem(scene, resolution=RES, margin=1e-4, delta=0.8, n_per_round=64,
                      tree_cap=1 << 15, roadmap_cap=1 << 13, max_iters=4096, seed=seed,
                      start=qs, goal=qg)


def _wait(server, tickets, timeout=60.0):
    t0 = time.time()
    res = {}
    while len(res) < len(tickets):
        assert time.time() - t0 < timeout, "requests did not finish"
        for t in tickets:
            if t not in res:
                st, times, cost = server.poll(t)
                if st == 2:
                    res[t] = (times, cost)
        time.sleep(0.005)
    return res


def test_serving_result_same_alone_and_in_mix(mp, orc, cases):
    steps = 400   # long enough that every later arrival joins a running batch
    alone = []
    for c in cases:
        p = _make(mp, c)
        mp.plan_batch([p], 60.0, max_steps=steps)
        alone.append(mp.plan_result(p))
        p.close()
    probs = [_make(mp, c) for c in cases]
    with mp.Server(max_slots=8) as srv:
        tickets = []
        for p in probs:
            tickets.append(srv.submit(p, 60.0, max_steps=steps))
            time.sleep(0.002)      # staggered arrivals: later ones join a running batch
        _wait(srv, tickets)
        st = srv.stats()
    assert st["completed"] == len(cases) and st["peak_active"] >= 2
    for p, (path_a, cost_a), c in zip(probs, alone, cases):
        path_m, cost_m = mp.plan_result(p)
        assert path_a is not None
        np.testing.assert_array_equal(path_a, path_m)
        assert cost_a == cost_m
        _check_path(orc, c[4], path_m, cost_m, c[2], c[3])
        p.close()


def test_serving_memory_admission(mp, cases):
    """A 1-byte budget admits a request only when nothing else runs."""
    probs = [_make(mp, c) for c in cases]
    with mp.Server(max_slots=8, device_mem_budget=1) as srv:
        tickets = [srv.submit(p, 30.0, max_steps=5) for p in probs]
        _wait(srv, tickets)
        st = srv.stats()
    assert st["peak_active"] == 1 and st["completed"] == len(cases)
    for p in probs:
        p.close()


def test_serving_poisson_stream_first_solutions(mp, orc, cases):
    """A Poisson stream (50 requests/s) of first-solution requests: every
    request completes with an oracle-valid path; admission, first solution
    and completion times are ordered."""
    arrivals = synth.poisson_arrivals(50.0, 12, seed=1)
    probs, tickets = [], []
    with mp.Server(max_slots=16) as srv:
        t0 = time.time()
        for k, ta in enumerate(arrivals):
            while time.time() - t0 < ta:
                time.sleep(0.001)
            p = _make(mp, cases[k % len(cases)])
            probs.append((p, cases[k % len(cases)]))
            tickets.append(srv.submit(p, 5.0, target_cost=float("inf")))
        res = _wait(srv, tickets)
    ttfs = []
    for t, (p, c) in zip(tickets, probs):
        times, cost = res[t]
        assert 0 <= times[0] <= times[1] <= times[3]
        ttfs.append(times[1])
        path, cost2 = mp.plan_result(p)
        assert cost2 == cost
        _check_path(orc, c[4], path, cost, c[2], c[3])
        p.close()
    assert np.percentile(ttfs, 99) < 5.0
