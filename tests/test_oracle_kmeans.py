"""Pins of the oracle's K-means slotting (subproblem 3, Sec. 5) against what
fixes each step independently of the oracle's own code:

* features: the dense co-occurrence matrix (sum over orders of n_o n_o^T -
  diag(n_o), n_o the order's SKU counts) times the sign matrix, exact integer
  square roots (math.isqrt) and truncation toward zero;
* Lloyd rounds: scikit-learn's Lloyd K-means on separated blobs gives the same
  final assignment; on any data the result is a fixed point (every row at its
  nearest centroid, ties to the lowest; every non-empty centroid within 1/2 of
  its members' mean); hand-sized cases for the rounding of negative means and
  for empty clusters;
* K-means++: hand-computed picks on a three-point case, distinct seeds on
  distinct points, and pick frequencies proportional to D^2 over many draws;
* placement: a bijection onto the first n_sku aisle-major locations with the
  clusters in weight order, each contiguous, and SKUs by frequency inside."""
import math

import numpy as np
import pytest

import oracle
import wh_gen

D, SK = oracle.KM_DIM, oracle.KM_SKETCH


def trunc_div(a: int, b: int) -> int:
    q = abs(a) // b
    return q if a >= 0 else -q


def dense_features(order_off, line_sku, n_sku, signs, fw):
    counts = np.zeros((len(order_off) - 1, n_sku), np.int64)
    for o in range(len(order_off) - 1):
        for s in line_sku[order_off[o]:order_off[o + 1]]:
            counts[o, s] += 1
    C = counts.T @ counts - np.diag(counts.sum(axis=0))
    co = C @ signs[:, :SK].astype(np.int64)
    freq = counts.sum(axis=0)
    x = np.zeros((n_sku, D), np.int64)
    for s in range(n_sku):
        n = math.isqrt(int((co[s] ** 2).sum()))
        if n > 0:
            x[s, :SK] = [trunc_div(int(c) * oracle.KM_SCALE, n) for c in co[s]]
        x[s, SK] = fw * int(freq[s]).bit_length()
    return x, freq


def test_features_match_dense_cooccurrence():
    rng = np.random.default_rng(1)
    n_sku = 40
    sizes = rng.integers(1, 9, 120)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    lines = rng.integers(0, n_sku, int(off[-1])).astype(np.int32)   # repeats inside an order allowed
    signs = wh_gen.gen_signs(2, (n_sku, D))
    for fw in (0, 7, 256):
        x, freq = oracle.kmeans_features(off, lines, n_sku, signs, fw)
        wx, wf = dense_features(off, lines, n_sku, signs, fw)
        assert np.array_equal(freq, wf)
        assert np.array_equal(x, wx)
    assert np.abs(x[:, :SK]).max() <= oracle.KM_SCALE


def test_features_hand_case():
    # orders {0, 1}, {0, 1, 2}, {3}: SKU 0 co-occurs with 1 twice and 2 once
    off = np.array([0, 2, 5, 6], np.int32)
    lines = np.array([0, 1, 0, 1, 2, 3], np.int32)
    signs = np.ones((4, D), np.int8)
    signs[2] = -1
    x, freq = oracle.kmeans_features(off, lines, 4, signs, 3)
    assert freq.tolist() == [2, 2, 1, 1]
    # co_0 = 2 * s1 + s2 = (1, ..., 1): n = isqrt(31) = 5, x = 1024 // 5 = 204
    assert (x[0, :SK] == 204).all() and x[0, SK] == 3 * 2
    assert (x[2, :SK] == 2048 // 11).all()         # co_2 = s0 + s1 = 2 per dim, n = isqrt(124) = 11
    assert (x[3, :SK] == 0).all() and x[3, SK] == 3  # alone in its order


def blobs(seed, k, per, spread=20):
    rng = np.random.default_rng(seed)
    centres = rng.integers(-900, 900, (k, D))
    x = np.concatenate([c + rng.integers(-spread, spread + 1, (per, D)) for c in centres]).astype(np.int32)
    return x, np.repeat(np.arange(k), per)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lloyd_matches_sklearn_on_blobs(seed):
    sk = pytest.importorskip("sklearn.cluster")
    x, truth = blobs(seed, 6, 40)
    rng = np.random.default_rng(seed + 10)
    # one starting point in every blob, in a random order: the clusters stay
    # separated, so the rounding of the centroids cannot move a point
    init = x[rng.permutation(6) * 40 + rng.integers(0, 40, 6)]
    cent, assign = oracle.kmeans_lloyd(x, init, 25)
    km = sk.KMeans(n_clusters=6, init=init.astype(np.float64), n_init=1, max_iter=25, tol=0.0,
                   algorithm="lloyd").fit(x.astype(np.float64))
    assert np.array_equal(assign, km.predict(x.astype(np.float64)))
    assert np.abs(cent - km.cluster_centers_).max() <= 0.5 + 1e-9
    assert len(set(zip(truth.tolist(), assign.tolist()))) == 6     # the blobs recovered


def nearest_bruteforce(x, cent):
    d = ((x[:, None, :].astype(np.int64) - cent[None, :, :].astype(np.int64)) ** 2).sum(axis=2)
    return d.argmin(axis=1)          # first minimum: the lowest cluster on ties


def test_lloyd_fixed_point_on_real_features():
    inst = wh_gen.midsize_cat(seed=6, n_plans=1)
    signs = wh_gen.gen_signs(3, (inst.n_sku, D))
    x, _ = oracle.kmeans_features(inst.order_off, inst.line_sku, inst.n_sku, signs, 64)
    rng = np.random.default_rng(0)
    cent, assign = oracle.kmeans_lloyd(x, x[rng.choice(inst.n_sku, 32, replace=False)], 200)
    assert np.array_equal(assign, nearest_bruteforce(x, cent))
    for c in range(32):
        m = x[assign == c]
        if len(m):
            assert np.abs(cent[c] - m.mean(axis=0)).max() <= 0.5


def test_lloyd_rounding_and_empty_cluster():
    x = np.zeros((3, D), np.int32)
    x[:, 0] = [-3, -2, 0]             # one cluster: mean -5/3 -> -2 (nearest integer)
    x[:, 1] = [1, 2, 2]               # mean 5/3 -> 2
    x[:, 2] = [-1, -2, 0]             # mean -1 exactly
    x[:, 3] = [-1, 0, 0]              # mean -1/3 -> 0
    x[:, 4] = [-2, -1, 0]             # mean -1
    init = np.stack([x[0], np.full(D, 5000, np.int32)])   # the second centroid attracts nothing
    cent, assign = oracle.kmeans_lloyd(x, init, 1)
    assert assign.tolist() == [0, 0, 0]
    assert cent[0, :5].tolist() == [-2, 2, -1, 0, -1]
    assert (cent[1] == 5000).all()
    y = np.zeros((2, D), np.int32)
    y[:, 0] = [-3, 0]                 # mean -3/2: halves go up, to -1
    cent, _ = oracle.kmeans_lloyd(y, y[:1], 1)
    assert cent[0, 0] == -1


def test_kmeans_pp_hand_case():
    x = np.zeros((3, D), np.int32)
    x[:, 0] = [0, 10, 100]            # D^2 from point 0: 0, 100, 10000; total 10,100
    u = np.array([3, 50, 7], np.uint64)
    assert oracle.kmeans_pp_init(x, 2, u).tolist() == [0, 1]       # 3 mod 3 = 0; 50 < 100
    u = np.array([0, 100, 0], np.uint64)
    assert oracle.kmeans_pp_init(x, 2, u).tolist() == [0, 2]       # the running sum 100 does not exceed 100
    u = np.array([0, 10100 + 99, 5], np.uint64)
    assert oracle.kmeans_pp_init(x, 3, u).tolist() == [0, 1, 2]    # only point 2 has D > 0 left


def test_kmeans_pp_distinct_and_proportional():
    x, _ = blobs(5, 4, 10, spread=3)
    rng = np.random.default_rng(1)
    for _ in range(20):
        u = rng.integers(0, 2 ** 63, 8, dtype=np.uint64)
        seeds = oracle.kmeans_pp_init(x, 8, u)
        assert len(set(seeds.tolist())) == 8
    # second pick ~ D^2 from the first point
    x = np.zeros((4, D), np.int32)
    x[:, 0] = [0, 1, 2, 3]            # D^2 = 0, 1, 4, 9 from point 0
    picks = [oracle.kmeans_pp_init(x, 2, np.array([0, int(v)], np.uint64))[1]
             for v in rng.integers(0, 2 ** 40, 4000)]
    freq = np.bincount(picks, minlength=4) / 4000
    assert freq[0] == 0
    assert np.allclose(freq[1:], np.array([1, 4, 9]) / 14, atol=0.03)


@pytest.mark.parametrize("fw,k", [(64, 16), (0, 8), (256, 40)])
def test_placement_follows_its_definition(fw, k):
    inst = wh_gen.midsize_cat(seed=8, n_plans=1)
    lay = inst.layout
    signs = wh_gen.gen_signs(4, (inst.n_sku, D))
    u = np.array([wh_gen.stream_word(9, 3, i) for i in range(k)], np.uint64)
    x, seeds, cent, assign, smap = oracle.kmeans_slotting(lay, inst.order_off, inst.line_sku, inst.n_sku, signs,
                                                          fw, k, 10, u=u)
    freq = np.bincount(inst.line_sku, minlength=inst.n_sku)
    assert np.array_equal(seeds, oracle.kmeans_pp_init(x, k, u))
    c0 = x[seeds]
    c_want, a_want = oracle.kmeans_lloyd(x, c0, 10)
    assert np.array_equal(cent, c_want) and np.array_equal(assign, a_want)
    L = lay.slots_per_side
    r_of_loc = {}
    for r in range(inst.n_sku):
        a, q = divmod(r, 2 * L)
        r_of_loc[(a * 2 + q % 2) * L + q // 2] = r
    rank = np.array([r_of_loc[int(l)] for l in smap])            # KeyError unless in the first n_sku
    assert len(set(rank.tolist())) == inst.n_sku                  # a bijection
    order = np.argsort(rank)
    w = np.bincount(assign, weights=freq, minlength=k)
    seq = assign[order]
    blocks = [seq[0]] + [c for p, c in zip(seq[:-1], seq[1:]) if c != p]
    assert len(blocks) == len(set(blocks))                         # every cluster contiguous
    wb = [(w[c], -c) for c in blocks]
    assert wb == sorted(wb, reverse=True)                          # heavier first, ties lower id
    for c in blocks:
        members = order[seq == c]
        keys = [(-freq[s], s) for s in members]
        assert keys == sorted(keys)                                # more picks first, ties lower id


def test_given_init_and_errors():
    inst = wh_gen.midsize_cat(seed=8, n_plans=1)
    signs = wh_gen.gen_signs(4, (inst.n_sku, D))
    init = np.arange(0, 800, 100, dtype=np.int32)
    x, seeds, cent, assign, smap = oracle.kmeans_slotting(inst.layout, inst.order_off, inst.line_sku, inst.n_sku,
                                                          signs, 32, 8, 5, init=init)
    assert np.array_equal(seeds, init)
    with pytest.raises(ValueError):
        oracle.kmeans_slotting(wh_gen.Layout(2, 10), inst.order_off, inst.line_sku, inst.n_sku, signs, 32, 8, 5,
                               init=init)                          # more SKUs than locations
    with pytest.raises(ValueError):
        oracle.kmeans_slotting(inst.layout, inst.order_off, inst.line_sku, inst.n_sku, signs, 257, 8, 5, init=init)
