"""Pins for the oracle's exact k-NN and graph search (CPU only).

The search is pinned by hand-traced toy graphs (tests/golden/toy_graphs.json),
by the special case L >= N on a connected graph (the search must then return
the exact k-NN), and by invariants; the exact k-NN is pinned by a hand-computed
case and by torch.cdist in float64 (a library routine)."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2506_15986_gb300 import synth


def _load_cases(golden_dir):
    with open(os.path.join(golden_dir, "toy_graphs.json")) as f:
        return json.load(f)["cases"]


def _f(v):
    return math.inf if v == "inf" else float(v)


def test_toy_graphs_hand_traced(golden_dir):
    for c in _load_cases(golden_dir):
        pts = np.asarray(c["points"], np.float32)
        adj = np.asarray(c["adjacency"], np.int32)
        q = np.asarray([c["query"]], np.float64)
        ids, d, ev, hp = oracle.search(pts, adj, q, c["entry"], c["L"], c["k"], W=c["W"])
        assert ids[0].tolist() == c["ids"], c["name"]
        assert [float(x) for x in d[0]] == [_f(x) for x in c["dists"]], c["name"]
        assert int(ev[0]) == c["evals"], c["name"]
        assert int(hp[0]) == c["hops"], c["name"]


def test_knn_hand_case():
    # points on a line; query 2.5: distances 6.25, 2.25, 0.25, 0.25, 2.25
    base = np.array([[0], [1], [2], [3], [4]], np.float32)
    ids, d = oracle.knn(base, np.array([[2.5]]), 4)
    assert ids[0].tolist() == [2, 3, 1, 4]  # ties broken by smaller id
    assert d[0].tolist() == [0.25, 0.25, 2.25, 2.25]
    ids, d = oracle.knn(base, np.array([[2.5]]), 7)  # k > n pads
    assert ids[0].tolist()[5:] == [-1, -1] and math.isinf(d[0][6])
    # inner product: delta = -<q, x>
    ids, d = oracle.knn(base, np.array([[1.0]]), 2, metric=oracle.IP)
    assert ids[0].tolist() == [4, 3] and d[0].tolist() == [-4.0, -3.0]


def test_knn_matches_torch_cdist():
    rng = np.random.default_rng(7)
    base = rng.standard_normal((700, 24)).astype(np.float32)
    q = rng.standard_normal((40, 24))
    ids, d = oracle.knn(base, q, 10)
    D = torch.cdist(torch.from_numpy(q), torch.from_numpy(base.astype(np.float64))) ** 2
    tv, ti = torch.topk(D, 10, largest=False, sorted=True)
    assert np.array_equal(ids, ti.numpy().astype(np.int32))
    np.testing.assert_allclose(d, tv.numpy(), rtol=1e-12, atol=1e-12)
    # IP against a float64 matmul
    ids, d = oracle.knn(base, q, 5, metric=oracle.IP)
    S = torch.from_numpy(q) @ torch.from_numpy(base.astype(np.float64)).T
    tv, ti = torch.topk(S, 5, largest=True, sorted=True)
    assert np.array_equal(ids, ti.numpy().astype(np.int32))
    np.testing.assert_allclose(-d, tv.numpy(), rtol=1e-12)


def test_knn_u8_exact_integers():
    w = synth.small_u8(n=600, nq=8)
    ids, d = oracle.knn(w["base"], w["queries"].astype(np.float64), 10)
    diff = w["base"][None].astype(np.int64) - w["queries"][:, None].astype(np.int64)
    full = (diff * diff).sum(-1)
    for i in range(8):
        order = np.lexsort((np.arange(600), full[i]))[:10]
        assert ids[i].tolist() == order.tolist()
        assert d[i].tolist() == full[i][order].astype(np.float64).tolist()


def _connected_graph(n, d, seed):
    rng = np.random.default_rng(seed)
    base = rng.integers(0, 256, (n, d)).astype(np.uint8)
    g, _ = oracle.build_graph(base, K=16, R=8)
    return base, g


def test_search_full_pool_is_exact_knn():
    # Special case: with L >= N on a graph where every node is reachable from
    # the entry, every node is evaluated and the pool is the exact top-L.
    base, g = _connected_graph(300, 16, 3)
    rng = np.random.default_rng(4)
    q = rng.integers(0, 256, (25, 16)).astype(np.float64)
    med = oracle.medoid(base)
    ids, d, ev, hp = oracle.search(base, g, q, med, 300, 10)
    tid, td = oracle.knn(base, q, 10)
    assert np.array_equal(ids, tid)
    assert np.array_equal(d, td)
    assert (ev == 300).all()  # each node evaluated exactly once
    assert (hp == 300).all()  # and expanded exactly once


def test_search_invariants():
    w = synth.small_u8(n=2000, nq=30)
    g, _ = oracle.build_graph(w["base"], K=32, R=16)
    med = oracle.medoid(w["base"])
    q = w["queries"].astype(np.float64)
    for W in (1, 2, 4):
        ids, d, ev, hp = oracle.search(w["base"], g, q, med, 40, 10, W=W)
        for i in range(len(q)):
            keys = list(zip(d[i].tolist(), ids[i].tolist()))
            assert keys == sorted(keys)                      # sorted by (dist, id)
            assert len(set(ids[i].tolist())) == 10           # unique
            assert ((ids[i] >= 0) & (ids[i] < 2000)).all()
            x = w["base"][ids[i]].astype(np.int64) - w["queries"][i].astype(np.int64)
            assert d[i].tolist() == (x * x).sum(1).astype(np.float64).tolist()
            assert hp[i] <= ev[i] <= 2000
            assert ev[i] >= 40                               # pool filled before stop


def test_search_recall_grows_with_L():
    # Greedy search is not monotone in L query by query, but on unclustered
    # data and a repaired (fully reachable) graph the mean recall@10 grows
    # with the pool and reaches the exact answer once L covers the graph.
    rng = np.random.default_rng(11)
    base = rng.integers(0, 256, (3000, 32)).astype(np.uint8)
    g, _ = oracle.build_graph(base, K=32, R=16)
    med = oracle.medoid(base)
    q = rng.integers(0, 256, (60, 32)).astype(np.float64)
    tid, _ = oracle.knn(base, q, 10)
    r = [oracle.recall_at_k(oracle.search(base, g, q, med, L, 10)[0], tid, 10)
         for L in (10, 40, 160, 3000)]
    assert r[0] <= r[1] <= r[2] <= r[3] and r[2] > 0.9 and r[3] == 1.0


def test_per_query_L_and_k():
    w = synth.small_u8(n=1500, nq=12)
    g, _ = oracle.build_graph(w["base"], K=32, R=16)
    med = oracle.medoid(w["base"])
    q = w["queries"].astype(np.float64)
    Ls = np.array([16, 32, 64, 10, 20, 30, 40, 50, 60, 70, 80, 90], np.int32)
    ks = np.array([1, 10, 5, 10, 3, 7, 10, 2, 8, 9, 10, 4], np.int32)
    ids, d, ev, hp = oracle.search(w["base"], g, q, med, 0, 0, Ls=Ls, ks=ks)
    for i in range(12):
        a, b, e, h = oracle.search(w["base"], g, q[i:i + 1], med, int(Ls[i]), int(ks[i]))
        assert ids[i, :ks[i]].tolist() == a[0].tolist()
        assert (ids[i, ks[i]:] == -1).all()
        assert ev[i] == e[0] and hp[i] == h[0]


def test_label_mode_counters(golden_dir):
    c = [x for x in _load_cases(golden_dir) if x["name"] == "chain8_W1"][0]
    pts = np.asarray(c["points"], np.float32)
    adj = np.asarray(c["adjacency"], np.int32)
    q = np.asarray([c["query"]], np.float64)
    # target 5 is evaluated in the 5th expansion step (see the trace): 6 evals
    _, _, ev, hp = oracle.search(pts, adj, q, 0, 3, 1, targets=[5])
    assert (ev[0], hp[0]) == (6, 5)
    # entry == target: counted before any expansion
    _, _, ev, hp = oracle.search(pts, adj, q, 5, 3, 1, targets=[5])
    assert (ev[0], hp[0]) == (1, 0)
    # unreachable target
    adj2 = adj.copy()
    adj2[6] = [5, -1]  # node 7 loses its only in-edge
    _, _, ev, hp = oracle.search(pts, adj2, q, 0, 3, 1, targets=[7])
    assert ev[0] == oracle.INT32_MAX and hp[0] == oracle.INT32_MAX


def test_seed_sets():
    # a seed set generalises the single entry: one seed equals the scalar
    # entry; unused slots (-1) and repeated seeds change nothing; every
    # distinct seed is evaluated once and starts in the pool
    rng = np.random.default_rng(11)
    base = rng.standard_normal((400, 6)).astype(np.float32)
    g, _ = oracle.build_graph(base, K=16, R=8)
    q = rng.standard_normal((12, 6))
    med = oracle.medoid(base)
    a = oracle.search(base, g, q, med, 24, 5, W=2)
    b = oracle.search(base, g, q, np.full((12, 3), [med, -1, med], np.int32), 24, 5, W=2)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    # two seeds on a chain 0-1-2-...-7 (points x_i = i), query at 7.2: seeds 0
    # and 5 are evaluated first; the walk from 5 reaches 6 and 7 while the
    # pool (L = 2) drops everything behind
    pts = np.zeros((8, 2), np.float32)
    pts[:, 0] = np.arange(8)
    adj = np.full((8, 2), -1, np.int32)
    for i in range(8):
        nb = [j for j in (i - 1, i + 1) if 0 <= j < 8]
        adj[i, :len(nb)] = nb
    ids, d, ev, hp = oracle.search(pts, adj, np.array([[7.2, 0.0]]), np.array([[0, 5]], np.int32), 2, 2)
    # step 1 expands 5 (closer): evaluates 4, 6; pool [6, 5]; step 2 expands 6:
    # evaluates 7; pool [7, 6]; step 3 expands 7: nothing new; step 4 expands
    # 6 was done -> stop.  evals = 2 seeds + 4, 6, 7 = 5; hops = 3
    assert ids[0].tolist() == [7, 6]
    assert np.allclose(d[0], [0.2 ** 2, 1.2 ** 2])
    assert (int(ev[0]), int(hp[0])) == (5, 3)
    # more seeds than the pool holds: every seed is evaluated (and visited),
    # the pool keeps the L best.  Seeds 0, 2, 4, 6 with L = 2 and the query at
    # 7.2: evaluated 0, 2, 4, 6, pool [6, 4]; expand 6: evaluates 5 and 7,
    # pool [7, 6]; expand 7: nothing new; 6 is done -> stop.  evals = 4 + 2,
    # hops = 2; node 1 and 3 never enter
    ids, d, ev, hp = oracle.search(pts, adj, np.array([[7.2, 0.0]]), np.array([[0, 2, 4, 6]], np.int32), 2, 2)
    assert ids[0].tolist() == [7, 6]
    assert (int(ev[0]), int(hp[0])) == (6, 2)
    # L >= N on a connected graph: exact k-NN from any seed set
    ids, d, _, _ = oracle.search(base, g, q, np.array([[med, 3, 77]] * 12, np.int32), 400, 5)
    tid, td = oracle.knn(base, q, 5)
    assert np.array_equal(ids, tid)


def test_ip_search_with_full_pool_is_exact_mips():
    # maximum inner product: with L >= N on a connected graph every node is
    # evaluated, so the result is the exact top-k by inner product (largest
    # first), which oracle.knn gives and a float64 matmul pins
    rng = np.random.default_rng(21)
    x = rng.standard_normal((300, 16))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x = x.astype(np.float32)
    g, _ = oracle.build_graph(x, K=24, R=12)
    q = rng.standard_normal((20, 16))
    ids, d, ev, hp = oracle.search(x, g, q, 0, 300, 10, metric=oracle.IP)
    S = q @ x.astype(np.float64).T
    ref = np.argsort(-S, axis=1, kind="stable")[:, :10]
    assert np.array_equal(ids, ref)
    assert (ev == 300).all()
    np.testing.assert_allclose(-d, np.take_along_axis(S, ref, 1), rtol=1e-12, atol=1e-12)
