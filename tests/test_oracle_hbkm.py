"""The oracle's hierarchical balanced k-means (Sec. 4.1, Def. 2, Algorithm 2)
pinned to hand-worked traces, to plain Lloyd's k-means (the penalty-free
single split), to the exact balance a dominant penalty forces, and to the
invariants of Def. 3's hubs."""
import numpy as np

import oracle
from paper_2506_15986_gb300 import synth

# eight points on a line (second coordinate 0); keys pick ids 1 and 2 as the
# root split's initial centroids (smallest keys 10, 20), then 7 and 4 inside
# {4, 5, 6, 7} (keys 30, 70)
X8 = np.array([[0, 0], [1, 0], [2, 0], [3, 0], [10, 0], [11, 0], [12, 0], [13, 0]], np.float32)
K8 = np.array([50, 10, 20, 60, 70, 80, 90, 30], np.uint32)


def test_hand_trace_two_levels_no_penalty():
    # level 1 from centroids 1, 2: it 1 puts {0,1} / {2..7} (means 0.5, 8.5),
    # it 2 puts {0..3} / {4..7} (means 1.5, 11.5).  Level 2: {0..3} from
    # centroids x1, x2 -> {0,1} / {2,3}; {4..7} from x7 = 13, x4 = 10 ->
    # child 0 = {6,7}, child 1 = {4,5}.  Every member sits 0.25 from its
    # centroid, so each hub is its cluster's smaller id.
    lab, cent, hubs, sizes = oracle.hbkm(X8, 2, 2, 0.0, 2, K8)
    assert lab.tolist() == [0, 0, 1, 1, 3, 3, 2, 2]
    assert cent.tolist() == [[0.5, 0], [2.5, 0], [12.5, 0], [10.5, 0]]
    assert hubs.tolist() == [0, 2, 6, 4]
    assert sizes.tolist() == [2, 2, 2, 2]


def test_hand_trace_penalty():
    # one split, lambda = 1: mean 6.5, sigma^2 = 210 / 8 = 26.25, m = 4,
    # lam = 26.25 / 4 = 6.5625; penalty of child j = lam * (2 (c_j - 4) + 1).
    # From centroids 1 and 2 the visit in id order gives
    #   x0: costs 1-45.9375 | 4-45.9375          -> 0  (c = 1, 0)
    #   x1: 0-32.8125 | 1-45.9375                -> 1  (1, 1)
    #   x2: 1-32.8125 | 0-32.8125                -> 1  (1, 2)
    #   x3: 4-32.8125 | 1-19.6875                -> 0  (2, 2)
    #   x4: 81-19.6875 | 64-19.6875              -> 1  (2, 3)
    #   x5: 100-19.6875 | 81-6.5625              -> 1  (2, 4)
    #   x6: 121-19.6875 | 100+6.5625             -> 0  (3, 4)
    #   x7: 144-6.5625 | 121+6.5625              -> 1  (3, 5)
    # centroids 15/3 = 5 and 37/5; hubs: 3 (distance 4) and 4 (distance 6.76)
    lab, cent, hubs, sizes = oracle.hbkm(X8, 2, 1, 1.0, 1, K8)
    assert lab.tolist() == [0, 1, 1, 0, 1, 1, 0, 1]
    assert cent[0].tolist() == [5.0, 0.0]
    assert cent[1].tolist() == [np.float32(37) / np.float32(5), 0.0]
    assert hubs.tolist() == [3, 4] and sizes.tolist() == [3, 5]


def test_dominant_penalty_balances_every_split():
    # with the penalty dominating the distances, the visit always picks a
    # smallest child: every split's children differ in size by at most one
    rng = np.random.default_rng(3)
    x = rng.standard_normal((1003, 5)).astype(np.float32)
    keys = synth.hbkm_keys(1003, seed=4)
    k, levels = 3, 3
    lab, cent, hubs, sizes = oracle.hbkm(x, k, levels, 1e12, 2, keys)
    assert sizes.sum() == 1003
    for lvl in range(1, levels + 1):
        part = np.bincount(lab // k ** (levels - lvl), minlength=k ** lvl)
        parent = part.reshape(-1, k)
        assert (parent.max(1) - parent.min(1) <= 1).all(), (lvl, parent)


def test_no_penalty_single_split_is_lloyd():
    # lambda = 0 and one level: T iterations of nearest-centroid assignment and
    # mean update from the same starting rows, as in or_kmeans
    rng = np.random.default_rng(9)
    centres = np.array([[0, 0, 0], [40, 0, 0], [0, 40, 0], [0, 0, 40], [40, 40, 40]], np.float64)
    lab0 = rng.integers(0, 5, 600)
    x = (centres[lab0] + 6.0 * rng.standard_normal((600, 3))).astype(np.float32)
    keys = synth.hbkm_keys(600, seed=1)
    lab, cent, hubs, sizes = oracle.hbkm(x, 5, 1, 0.0, 6, keys)
    init = np.lexsort((np.arange(600), keys))[:5].astype(np.int32)
    c64, a64, _ = oracle.kmeans(x, 5, init, 6)
    assert np.array_equal(lab, a64)
    np.testing.assert_allclose(cent, c64, rtol=1e-5, atol=1e-4)


def test_invariants_partition_means_and_hubs():
    w = synth.shift_f32(n=3000, nq=1, n_train=0)
    x = w["base"]
    keys = synth.hbkm_keys(3000, seed=2)
    k, levels = 4, 2
    lab, cent, hubs, sizes = oracle.hbkm(x, k, levels, 1.0, 4, keys)
    assert lab.min() >= 0 and lab.max() < k ** levels
    assert np.array_equal(np.bincount(lab, minlength=k ** levels), sizes)
    xd = x.astype(np.float64)
    for c in range(k ** levels):
        mem = np.where(lab == c)[0]
        if len(mem) == 0:
            assert hubs[c] == -1
            continue
        np.testing.assert_allclose(cent[c], xd[mem].mean(0), rtol=1e-4, atol=1e-4)
        d = ((xd[mem] - cent[c].astype(np.float64)) ** 2).sum(1)
        assert lab[hubs[c]] == c
        assert d[mem == hubs[c]][0] <= d.min() * (1 + 1e-5) + 1e-6
    # balance: the penalty shrinks the spread of sizes against lambda = 0
    _, _, _, s0 = oracle.hbkm(x, k, levels, 0.0, 4, keys)
    assert sizes.std() < s0.std()


def test_fewer_rows_than_clusters():
    # 5 rows into 3 x 3 clusters: the root split takes all three starts; a
    # child with fewer than 3 members leaves the rest of its children empty
    x = np.array([[0], [1], [2], [10], [20]], np.float32)
    keys = np.array([4, 3, 2, 1, 0], np.uint32)
    lab, cent, hubs, sizes = oracle.hbkm(x, 3, 2, 0.0, 3, keys)
    assert sizes.sum() == 5 and (hubs[sizes == 0] == -1).all()
    assert all(lab[h] == c for c, h in enumerate(hubs) if h >= 0)
