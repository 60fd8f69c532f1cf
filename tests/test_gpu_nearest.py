"""GPU parity of NEAREST (cost-filtered), NEIGHBORS (radius) and path cost
against the FP64 oracle, through the C ABI.

Indices must match exactly, ties included (key: distance, then g, then
index).  The one allowance is a genuine FP32/FP64 near-tie: when the oracle's
best and runner-up distances, or some vertex's filter value g + d and the
budget c, are within 1e-5 relative, the GPU must still return a vertex that
is admissible and as close as the oracle's best within that tolerance.
"""
import numpy as np
import pytest
import torch

from paper_2609_30644_gb300 import synth

pytestmark = pytest.mark.gpu
REL = 1e-5


@pytest.fixture(scope="module")
def mp():
    import paper_2609_30644_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_nearest(orc, tree, qs, cs, got, N=None, sample=None):
    D = tree.shape[0] - 1
    N = tree.shape[1] if N is None else N
    idxs = range(qs.shape[1]) if sample is None else sample
    n_tie = 0
    for i in idxs:
        ref, bd, sd, gap = orc.nearest(tree, qs[:, i], cs[i], n_vertices=N)
        if got[i] == ref:
            continue
        scale = max(1.0, abs(float(cs[i])))
        near_tie = (np.isfinite(sd) and sd - bd <= REL * max(bd, 1e-30)) or gap <= REL * scale
        assert near_tie, (i, got[i], ref, bd, sd, gap)
        n_tie += 1
        if got[i] >= 0:
            v = tree[:D, got[i]].astype(float)
            d = np.linalg.norm(v - qs[:, i].astype(float))
            assert tree[D, got[i]] + d < cs[i] + REL * scale
            assert d <= bd * (1 + REL) + 1e-12 or ref < 0
    return n_tie


@pytest.mark.parametrize("D,N,Q", [(14, 3000, 500), (28, 2000, 200), (6, 5000, 300),
                                   (7, 777, 129), (3, 1000, 64), (64, 600, 40), (21, 1, 16)])
def test_nearest_parity(mp, orc, D, N, Q):
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree(D, N, lo, hi, seed=D, dup_frac=0.05)
    qs, cs = synth.nn_queries(D, Q, lo, hi, seed=D + 1, budget_lo=0.0, budget_hi=20.0)
    got = mp.nearest(_dev(tree), _dev(qs), _dev(cs)).cpu().numpy()
    ties = _check_nearest(orc, tree, qs, cs, got)
    assert ties <= max(2, Q // 50)
    assert (got >= -1).all() and (got < N).all()


def test_nearest_exact_ties(mp, orc):
    """Queries placed exactly on duplicated vertices: the tie must go to the
    lowest g, then the lowest index (Sec. III-D), bit-exactly."""
    D = 14
    rng = np.random.default_rng(5)
    base = rng.uniform(-2, 2, (D, 50)).astype(np.float32)
    tree = np.zeros((D + 1, 400), np.float32)
    for j in range(400):
        tree[:D, j] = base[:, j % 50]
        tree[D, j] = np.float32([0.5, 0.25, 0.25, 1.0][(j // 50) % 4])
    qs = np.ascontiguousarray(base[:, :50])
    cs = np.full(50, 100.0, np.float32)
    got = mp.nearest(_dev(tree), _dev(qs), _dev(cs)).cpu().numpy()
    for i in range(50):
        assert got[i] == orc.nearest(tree, qs[:, i], cs[i])[0]
        assert got[i] == 50 + i      # g = 0.25 first appears at block 1


def test_nearest_empty_and_filtered(mp, orc):
    D = 7
    lo, hi = -np.ones(D), np.ones(D)
    tree = synth.random_tree(D, 500, lo, hi, seed=3)
    qs, _ = synth.nn_queries(D, 64, lo, hi, seed=4)
    cs = np.zeros(64, np.float32)                     # nothing admissible
    got = mp.nearest(_dev(tree), _dev(qs), _dev(cs)).cpu().numpy()
    assert (got == -1).all()
    empty = torch.empty((D + 1, 0), dtype=torch.float32, device="cuda")
    got = mp.nearest(empty, _dev(qs), _dev(np.full(64, 1e9, np.float32))).cpu().numpy()
    assert (got == -1).all()


def test_nearest_split_tree_few_queries(mp, orc):
    """Few queries over a large tree: the tree is split across blocks and the
    partial minima are reduced; also ld > n_vertices."""
    D = 14
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    N, ld = 200_000, 200_064
    tree = np.zeros((D + 1, ld), np.float32)
    tree[:, :N] = synth.random_tree_fast(D, N, lo, hi, seed=9)
    tree[:, N:] = -7.0                                 # must never be read
    qs, cs = synth.nn_queries(D, 5, lo, hi, seed=10, budget_lo=5, budget_hi=30)
    got = mp.nearest(_dev(tree), _dev(qs), _dev(cs), n_vertices=N).cpu().numpy()
    _check_nearest(orc, tree, qs, cs, got, N=N)


FILTERS = (0, 1)   # NEAREST_FILTER_FP32 (default), NEAREST_FILTER_TENSOR


def test_nearest_full_size_sampled(mp, orc):
    """65,536 queries against a 16,384-vertex 14-D tree (the benchmark's
    launch configuration), 200 sampled queries re-checked by the oracle, for
    both large-batch filters, which must also agree index for index."""
    D = 14
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree_fast(D, 16384, lo, hi, seed=1)
    qs, cs = synth.nn_queries(D, 65536, lo, hi, seed=2, budget_lo=10, budget_hi=40)
    got = mp.nearest(_dev(tree), _dev(qs), _dev(cs)).cpu().numpy()
    tc = mp.nearest(_dev(tree), _dev(qs), _dev(cs), filter=1).cpu().numpy()
    np.testing.assert_array_equal(got, tc)
    sample = np.random.default_rng(0).choice(65536, 200, replace=False)
    _check_nearest(orc, tree, qs, cs, got, sample=sample)


def test_nearest_large_tree_sampled(mp, orc):
    """A tree past the size whose cost-to-come range the ordering's setup
    block finds alone (131,072 vertices; larger trees take a separate range
    pass), with a ragged vertex count and a ragged last query block: sampled
    queries against the oracle, both large-batch filters index for index."""
    D, N, Q = 7, 140_001, 2_500
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree_fast(D, N, lo, hi, seed=21)
    qs, cs = synth.nn_queries(D, Q, lo, hi, seed=22, budget_lo=2.0, budget_hi=30.0)
    got = mp.nearest(_dev(tree), _dev(qs), _dev(cs)).cpu().numpy()
    tc = mp.nearest(_dev(tree), _dev(qs), _dev(cs), filter=1).cpu().numpy()
    np.testing.assert_array_equal(got, tc)
    sample = np.concatenate([np.arange(Q - 60, Q), np.random.default_rng(3).choice(Q, 60, replace=False)])
    _check_nearest(orc, tree, qs, cs, got, sample=sample)


@pytest.mark.parametrize("D,N,Q,k_max", [(7, 3000, 200, 32), (14, 1000, 64, 8), (6, 65, 33, 100),
                                         (3, 10, 5, 0)])
def test_neighbors_parity(mp, orc, D, N, Q, k_max):
    rng = np.random.default_rng(D)
    tree = np.zeros((D + 1, N), np.float32)
    tree[:D] = rng.uniform(-2.9, 2.9, (D, N))
    tree[D] = rng.uniform(0, 5, N)
    qs = rng.uniform(-2.9, 2.9, (D, Q)).astype(np.float32)
    delta = np.float32(1.2 * np.sqrt(D))
    idx, cnt = mp.neighbors(_dev(tree), _dev(qs), float(delta), k_max)
    idx, cnt = idx.cpu().numpy(), cnt.cpu().numpy()
    for i in range(Q):
        ref, rc, gap = orc.neighbors(tree, qs[:, i], delta, k_max)
        if gap > REL * delta:
            assert cnt[i] == rc
            np.testing.assert_array_equal(idx[i, :len(ref)], ref)
        else:
            assert abs(int(cnt[i]) - rc) <= 2
        row = idx[i, :min(int(cnt[i]), k_max)]
        assert (np.diff(row) > 0).all()
        assert (idx[i, min(int(cnt[i]), k_max):] == -1).all()


def test_path_cost_parity(mp, orc):
    rng = np.random.default_rng(7)
    for M, D in [(2, 14), (17, 6), (65537, 14), (1, 28)]:
        path = rng.uniform(-2.9, 2.9, (M, D)).astype(np.float32)
        got = float(mp.path_cost(_dev(path)).cpu().numpy()[0])
        ref = orc.path_cost(path)
        assert got == pytest.approx(ref, rel=1e-6, abs=1e-12)


@pytest.mark.parametrize("filt", FILTERS)
@pytest.mark.parametrize("D,N,Q", [(14, 3000, 4096), (28, 2000, 2048), (6, 5000, 3000),
                                   (3, 700, 2500), (7, 257, 2049), (21, 1501, 2100),
                                   (14, 1001, 2300)])
def test_nearest_query_blocked_parity(mp, orc, D, N, Q, filt):
    """Batches of >= 2048 queries take the budget-ordered path (FP32 or
    tensor-core expansion filter + exact re-check); sampled queries against
    the oracle, duplicates in the tree for ties, and the whole batch against
    the small-batch kernel (called in chunks of < 2048 queries), which must
    agree index for index."""
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree(D, N, lo, hi, seed=100 + D, dup_frac=0.1)
    qs, cs = synth.nn_queries(D, Q, lo, hi, seed=200 + D, budget_lo=0.0, budget_hi=25.0)
    qs[:, :64] = tree[:D, :64]            # queries exactly on (duplicated) vertices
    big = mp.nearest(_dev(tree), _dev(qs), _dev(cs), filter=filt).cpu().numpy()
    small = np.concatenate([
        mp.nearest(_dev(tree), _dev(np.ascontiguousarray(qs[:, i:i + 1000])),
                   _dev(cs[i:i + 1000])).cpu().numpy() for i in range(0, Q, 1000)])
    np.testing.assert_array_equal(big, small)
    sample = np.concatenate([np.arange(64), np.random.default_rng(D).choice(Q, 200, replace=False)])
    _check_nearest(orc, tree, qs, cs, big, sample=sample)


def test_nearest_work_counts(mp, orc):
    """Pairs the budget-ordered pass evaluates: all of them for unbounded
    budgets or small batches, none when every budget is below every cost
    (and then nothing is admissible), and in between for mixed budgets; the
    results of the mixed case still match the oracle on a sample."""
    D, N, Q = 7, 3000, 4096
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree(D, N, lo, hi, seed=9, dup_frac=0.05)
    qs, _ = synth.nn_queries(D, Q, lo, hi, seed=10)
    t, q = _dev(tree), _dev(qs)
    big = torch.full((Q,), 1e30, dtype=torch.float32, device="cuda")
    assert mp.nearest_work(t, q, big) == Q * N
    assert mp.nearest_work(t, q[:, :100].contiguous(), big[:100]) == 100 * N
    low = torch.full((Q,), float(tree[D].min()) * 0.5 - 1.0, dtype=torch.float32, device="cuda")
    assert mp.nearest_work(t, q, low) == 0
    assert (mp.nearest(t, q, low).cpu().numpy() == -1).all()
    cs = np.random.default_rng(11).uniform(0.0, float(tree[D].max()), Q).astype(np.float32)
    pairs = mp.nearest_work(t, q, _dev(cs))
    assert 0 < pairs < Q * N
    got = mp.nearest(t, q, _dev(cs)).cpu().numpy()
    _check_nearest(orc, tree, qs, cs, got, sample=np.arange(0, Q, 37))


@pytest.mark.parametrize("filt", FILTERS)
@pytest.mark.parametrize("D,case", [(D, c) for D in (14, 21)
                                    for c in ("offset", "tiny", "huge", "nan", "colossal")]
                         + [(14, "scaled_down"), (14, "scaled_up"), (7, "scaled_down")])
def test_nearest_filter_range(mp, orc, D, case, filt):
    """Both filters' error bounds are relative to |q|^2 + |x|^2: a box far
    from the origin (large norms, small distances) must stay exact.  The
    FP16 tensor filter (D <= 14) scales the batch by a power of two taken
    from its largest magnitude: boxes shrunk by 1e-12 or grown by 1e15 must
    stay exact, as must a single tiny or huge coordinate.  For the FP32 and
    TF32 filters a nonzero coordinate below 2^-60 or above 2^60 turns the
    filter off; a NaN does so for all.  A query coordinate of 3e38, shared
    with its own vertex, makes -2 q overflow: the exact check must still see
    the query itself (distance 0 to that vertex).  Results must equal the
    small-batch kernel's and the oracle's."""
    N, Q = 1500, 2048
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree(D, N, lo, hi, seed=31 + D, dup_frac=0.05)
    qs, cs = synth.nn_queries(D, Q, lo, hi, seed=32 + D, budget_lo=0.0, budget_hi=25.0)
    qs[:, :32] = tree[:D, :32]
    if case == "offset":
        tree[:D] += np.float32(1000.0)
        qs += np.float32(1000.0)
    elif case == "tiny":
        qs[3, 5] = np.float32(1e-25)
    elif case == "huge":
        tree[2, 7] = np.float32(2.0 ** 61)
    elif case == "nan":
        tree[4, 11] = np.nan
    elif case == "colossal":
        qs[2, 9] = tree[2, 9] = np.float32(3e38)  # query 9 is vertex 9
        cs[9] = np.float32(tree[D, 9]) + np.float32(1.0)  # and vertex 9 is admissible
    else:
        # every coordinate, the costs and the budgets scaled alike: the
        # nearest vertex is the same, distances scale by f
        f = np.float32(1e-12 if case == "scaled_down" else 1e15)
        tree *= f
        qs *= f
        cs *= f
    big = mp.nearest(_dev(tree), _dev(qs), _dev(cs), filter=filt).cpu().numpy()
    if case == "colossal":
        assert big[9] == 9, big[9]
    small = np.concatenate([
        mp.nearest(_dev(tree), _dev(np.ascontiguousarray(qs[:, i:i + 1000])),
                   _dev(cs[i:i + 1000])).cpu().numpy() for i in range(0, Q, 1000)])
    np.testing.assert_array_equal(big, small)
    sample = np.concatenate([np.arange(40), np.random.default_rng(7).choice(Q, 120, replace=False)])
    _check_nearest(orc, tree, qs, cs, big, sample=sample)


def test_nearest_and_neighbors_tuned_launches_same_results(mp, orc, tmp_path):
    """The autotuners' knobs (NEAREST's slice waves, NEIGHBORS's vertex-range
    target) change the launch, never the result: every candidate, forced
    through the tuned-launch cache (saved, edited and loaded back), returns
    the same indices as the default launch."""
    D = 14
    lo, hi = -2.9 * np.ones(D), 2.9 * np.ones(D)
    tree = synth.random_tree(D, 4000, lo, hi, seed=81, dup_frac=0.05)
    qs, cs = synth.nn_queries(D, 3000, lo, hi, seed=82, budget_lo=0.0, budget_hi=25.0)
    t, q, c = _dev(tree), _dev(qs), _dev(cs)
    mp.autotune_cache_clear()
    ref = mp.nearest(t, q, c).cpu().numpy()
    got, waves, ms = mp.nearest_autotune(t, q, c)
    assert waves in (2, 4, 8) and ms > 0
    np.testing.assert_array_equal(got.cpu().numpy(), ref)
    rq = np.ascontiguousarray(qs[:7, :256])
    rtree = np.ascontiguousarray(tree[:8])
    rref, rcnt = mp.neighbors(_dev(rtree), _dev(rq), 2.0, 32, dim=7)
    ridx, rc2, target, _ = mp.neighbors_autotune(_dev(rtree), _dev(rq), 2.0, 32, dim=7)
    assert target in (14, 54, 216)
    np.testing.assert_array_equal(ridx.cpu().numpy(), rref.cpu().numpy())
    np.testing.assert_array_equal(rc2.cpu().numpy(), rcnt.cpu().numpy())
    path = tmp_path / "tuned.txt"
    mp.autotune_cache_save(str(path))
    lines = [l for l in path.read_text().splitlines() if l and not l.startswith("#")]
    nkey = [l.split(" = ")[0] for l in lines if l.startswith("nearest ")]
    bkey = [l.split(" = ")[0] for l in lines if l.startswith("neighbors ")]
    assert len(nkey) == 1 and len(bkey) == 1
    for wv, tg in ((2, 14), (8, 216), (4, 54)):
        path.write_text(f"{nkey[0]} = {wv}\n{bkey[0]} = {tg}\n")
        mp.autotune_cache_load(str(path))
        np.testing.assert_array_equal(mp.nearest(t, q, c).cpu().numpy(), ref)
        i2, c2 = mp.neighbors(_dev(rtree), _dev(rq), 2.0, 32, dim=7)
        np.testing.assert_array_equal(i2.cpu().numpy(), rref.cpu().numpy())
        np.testing.assert_array_equal(c2.cpu().numpy(), rcnt.cpu().numpy())
    _check_nearest(orc, tree, qs, cs, ref, sample=np.arange(0, 3000, 97))
    mp.autotune_cache_clear()
