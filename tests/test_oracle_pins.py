"""Hand-worked pins for the oracle's small helpers (CPU only).

* ``oracle.rerank``: the exact re-scoring of a final pool (the precision line's
  rerank step): (distance, id) order with ties to the smaller id, -1 slots
  skipped, (-1, +inf) padding, and the inner-product sign (distance = -<x, q>).
* ``oracle.recall_at_k``: recall@k = |R ∩ R'| / k averaged over queries
  (Sec. 2.1, Problem 1 and the recall definition that follows it), on rows
  with known hit counts, -1 padding and k below the row width.
* ``oracle.pruned_row``: one node's relative-neighbourhood pruning of its
  exact K nearest (Sec. 2.1, Def. 1, with the pruning rule of the graph
  builder), on the four-point case worked by hand for ``or_build_graph``, and
  with alpha > 1, where fewer candidates are dominated.
"""
import numpy as np
import pytest

import oracle

# ---- rerank ----------------------------------------------------------------

# ids 0..4 at (0,0) (1,0) (0,1) (3,4) (-1,0)
_X = np.array([[0, 0], [1, 0], [0, 1], [3, 4], [-1, 0]], np.float64)


def test_rerank_l2_ties_padding_and_empty_rows():
    q = np.array([[0, 0], [1, 1], [0, 0]], np.float64)
    pool = np.array([[3, -1, 1, 2, 4],     # squared L2 25, -, 1, 1, 1
                     [0, 3, -1, -1, -1],   # to (1,1): 2, 13
                     [-1, -1, -1, -1, -1]], np.int32)
    ids, d = oracle.rerank(_X, pool, q, 3)
    # the three-way tie at distance 1 goes to the smaller ids, 3 (25) drops out
    assert ids.tolist() == [[1, 2, 4], [0, 3, -1], [-1, -1, -1]]
    assert d[0].tolist() == [1.0, 1.0, 1.0]
    assert d[1, :2].tolist() == [2.0, 13.0] and np.isinf(d[1, 2])
    assert np.isinf(d[2]).all()


def test_rerank_inner_product_sign_and_ties():
    q = np.array([[1, 2], [1, 1]], np.float64)
    pool = np.array([[4, 1, 3, 2],   # -<x,q> for q=(1,2): +1, -1, -11, -2
                     [2, 1, 4, -1]], np.int32)  # for q=(1,1): -1, -1, +1
    ids, d = oracle.rerank(_X, pool, q, 3, metric=oracle.IP)
    # the largest inner product first: a reversed sign would put id 4 first
    assert ids[0].tolist() == [3, 2, 1]
    assert d[0].tolist() == [-11.0, -2.0, -1.0]
    # ids 1 and 2 tie at -1: the smaller id first
    assert ids[1].tolist() == [1, 2, 4]
    assert d[1].tolist() == [-1.0, -1.0, 1.0]


def test_rerank_keeps_the_pool_order_free():
    # the result depends on the pool's set, not its order
    q = np.array([[0.2, 0.3]], np.float64)
    rng = np.random.default_rng(0)
    pool = np.array([[0, 1, 2, 3, 4]], np.int32)
    a = oracle.rerank(_X, pool, q, 5)
    b = oracle.rerank(_X, pool[:, rng.permutation(5)], q, 5)
    assert a[0].tolist() == b[0].tolist()
    # squared L2 0.13, 0.73, 0.53, 21.53, 1.53
    assert a[0][0].tolist() == [0, 2, 1, 4, 3]


# ---- recall@k --------------------------------------------------------------

def test_recall_hand_counts():
    found = np.array([[1, 2, 3, 9],
                      [5, -1, -1, -1],
                      [0, -1, -1, -1]], np.int32)
    truth = np.array([[3, 2, 7, 1],
                      [5, 6, 7, 8],
                      [0, 1, 2, 3]], np.int32)
    # k = 1: {1}&{3}=0, {5}&{5}=1, {0}&{0}=1 -> 2 / 3
    assert oracle.recall_at_k(found, truth, 1) == pytest.approx(2 / 3)
    # k = 2: {1,2}&{3,2}=1, {5}&{5,6}=1, {0}&{0,1}=1 -> 3 / 6
    assert oracle.recall_at_k(found, truth, 2) == pytest.approx(3 / 6)
    # k = 4: {1,2,3,9}&{3,2,7,1}=3, 1, 1 -> 5 / 12
    assert oracle.recall_at_k(found, truth, 4) == pytest.approx(5 / 12)


def test_recall_padding_is_never_a_hit():
    # -1 on both sides (fewer results than k, or fewer true neighbours) is no hit
    found = np.array([[4, -1, -1]], np.int32)
    truth = np.array([[4, -1, -1]], np.int32)
    assert oracle.recall_at_k(found, truth, 3) == pytest.approx(1 / 3)
    # an id found twice counts once
    found = np.array([[4, 4, -1]], np.int32)
    truth = np.array([[4, 5, 6]], np.int32)
    assert oracle.recall_at_k(found, truth, 3) == pytest.approx(1 / 3)


def test_recall_only_looks_at_the_first_k_columns():
    found = np.array([[7, 8, 1, 2]], np.int32)
    truth = np.array([[1, 2, 7, 8]], np.int32)
    assert oracle.recall_at_k(found, truth, 2) == 0.0
    assert oracle.recall_at_k(found, truth, 4) == 1.0


# ---- pruned_row ------------------------------------------------------------

_P = np.array([[0, 0], [1, 0], [2, 0.1], [0, 1.5]], np.float32)


def test_pruned_row_hand_case_alpha_one():
    # the case worked by hand for or_build_graph (alpha = 1):
    # node 0 -> [1, 3], node 1 -> [0, 2], node 2 -> [1], node 3 -> [0]
    assert [oracle.pruned_row(_P, p, 3, 3) for p in range(4)] == [[1, 3], [0, 2], [1], [0]]


def test_pruned_row_degree_cut():
    # R = 1 keeps the nearest candidate only
    assert [oracle.pruned_row(_P, p, 3, 1) for p in range(4)] == [[1], [0], [1], [0]]


def test_pruned_row_alpha_above_one():
    # alpha = 4, squared distances d(0,1)=1, d(0,2)=4.01, d(0,3)=2.25,
    # d(1,2)=1.01, d(1,3)=3.25, d(2,3)=5.96; c is dropped when a kept s has
    # 4 d(s,c) <= d(p,c):
    # node 0: 1 kept; 3 kept (13 > 2.25); 2 kept (4.04 > 4.01, 23.84 > 4.01)
    # node 1: 0 kept; 2 kept (16.04 > 1.01); 3 kept (9 > 3.25, 23.84 > 3.25)
    # node 2: 1 kept; 0 dropped (4 <= 4.01); 3 kept (13 > 5.96)
    # node 3: 0 kept; 1 kept (4 > 3.25); 2 dropped (4.04 <= 5.96)
    rows = [oracle.pruned_row(_P, p, 3, 3, alpha=4.0) for p in range(4)]
    assert rows == [[1, 3, 2], [0, 2, 3], [1, 3], [0, 1]]
    # the builder applies the same rule with the same alpha
    g, _ = oracle.build_graph(_P, K=3, R=3, alpha=4.0)
    assert [r[r >= 0].tolist() for r in g] == rows
