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


# ----------------------------------------------------------------------------
# failure paths (host-side injection; nothing faults on the GPU)
# ----------------------------------------------------------------------------

def _wait_all(server, tickets, timeout=60.0):
    t0 = time.time()
    out = {}
    while len(out) < len(tickets):
        assert time.time() - t0 < timeout, "requests did not finish"
        for t in tickets:
            if t not in out:
                st, times, cost, status = server.poll_status(t)
                if st == 2:
                    out[t] = (times, cost, status)
        time.sleep(0.005)
    return out


def test_serving_cancel_queued_and_running(mp, orc, cases):
    """With one slot, a request cancelled while queued never runs and one
    cancelled while running ends after the iteration in flight; both report
    MRPOP_ECANCELLED, a later request runs normally, cancelling a finished
    request changes nothing and an unknown ticket is refused."""
    ps = [_make(mp, c) for c in cases]
    with mp.Server(max_slots=1) as srv:
        t_run = srv.submit(ps[0], 30.0)
        t_queued = srv.submit(ps[1], 30.0)
        t0 = time.time()
        while srv.poll_status(t_run)[0] != 1:
            assert time.time() - t0 < 30.0
            time.sleep(0.002)
        srv.cancel(t_queued)
        srv.cancel(t_run)
        t_next = srv.submit(ps[2], 5.0, target_cost=float("inf"))
        res = _wait_all(srv, [t_run, t_queued, t_next])
        assert res[t_queued][2] == 8 and res[t_queued][0][0] < 0    # never admitted
        assert res[t_run][2] == 8 and res[t_run][0][0] >= 0         # admitted, then cancelled
        assert res[t_run][0][3] < 10.0                               # long before its budget
        assert res[t_next][2] == 0 and np.isfinite(res[t_next][1])
        srv.cancel(t_next)                                           # already done: no change
        assert srv.poll_status(t_next)[3] == 0
        with pytest.raises(mp.MrpopError):
            srv.cancel(10 ** 9)
    path, cost = mp.plan_result(ps[2])
    _check_path(orc, cases[2][4], path, cost, cases[2][2], cases[2][3])
    for p in ps:
        p.close()


def test_serving_refused_allocation_at_admission(mp, orc, cases):
    """An admission whose device allocation is refused (injected on the
    host) finishes with MRPOP_ENOMEM; the server carries on, the other
    requests find oracle-valid paths, and the refused problem can be
    submitted again."""
    ps = [_make(mp, c) for c in cases]
    with mp.Server(max_slots=4) as srv:
        srv.inject(mp.FAULT_ADMIT_ENOMEM, 1)
        ts = [srv.submit(p, 5.0, target_cost=float("inf")) for p in ps]
        res = _wait_all(srv, ts)
        assert [res[t][2] for t in ts] == [2, 0, 0]       # arrival order: the first is refused
        t_again = srv.submit(ps[0], 5.0, target_cost=float("inf"))
        assert _wait_all(srv, [t_again])[t_again][2] == 0
        assert srv.stats()["queued"] == 0
    for p, c in zip(ps, cases):
        path, cost = mp.plan_result(p)
        _check_path(orc, c[4], path, cost, c[2], c[3])
        p.close()


def test_serving_stalled_loop_and_idle_producer(mp, orc, cases):
    """An injected 400 ms stall of the server loop leaves submit, poll and
    cancel responsive (the loop holds no lock while stalled); a producer that
    then pauses finds the server idle, and requests submitted before and
    after the pause all complete."""
    ps = [_make(mp, c) for c in cases]
    with mp.Server(max_slots=8) as srv:
        srv.inject(mp.FAULT_STALL_MS, 400)
        time.sleep(0.05)                                   # the loop is now stalled
        t0 = time.time()
        t_a = srv.submit(ps[0], 5.0, target_cost=float("inf"))
        worst = time.time() - t0
        for _ in range(10):
            t1 = time.time()
            srv.poll_status(t_a)
            worst = max(worst, time.time() - t1)
        assert worst < 0.05, worst
        assert _wait_all(srv, [t_a])[t_a][2] == 0
        time.sleep(0.3)                                    # the producer pauses
        st = srv.stats()
        assert st["queued"] == 0 and st["completed"] == 1
        ts = [srv.submit(p, 5.0, target_cost=float("inf")) for p in ps[1:]]
        res = _wait_all(srv, ts)
        assert all(res[t][2] == 0 for t in ts)
    for p, c in zip(ps, cases):
        path, cost = mp.plan_result(p)
        _check_path(orc, c[4], path, cost, c[2], c[3])
        p.close()
