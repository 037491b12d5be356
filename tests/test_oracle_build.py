"""Pins for the oracle's offline builders (CPU only): graph builder (Def. 1
with relative-neighbourhood pruning and reachability repair), medoid, k-means,
hub nodes (Def. 3), hub graph (Sec. 4.3) and the label rule (Def. 4)."""
import numpy as np
import pytest

import oracle
from paper_2506_15986_gb300 import synth


def test_rng_prune_hand_case():
    # p0=(0,0) p1=(1,0) p2=(2,0.1) p3=(0,1.5); worked by hand:
    # node 0: candidates 1 (1), 3 (2.25), 2 (4.01); keep 1; keep 3 since
    #   d(1,3)=3.25 > 2.25; drop 2 since d(1,2)=1.01 <= 4.01      -> [1, 3]
    # node 1: 0 (1), 2 (1.01), 3 (3.25); keep 0; keep 2 (4.01 > 1.01);
    #   drop 3 (d(0,3)=2.25 <= 3.25)                               -> [0, 2]
    # node 2: 1 (1.01), 0 (4.01), 3 (5.96); keep 1; drop 0, 3      -> [1]
    # node 3: 0 (2.25), 1 (3.25), 2 (5.96); keep 0; drop 1, 2      -> [0]
    pts = np.array([[0, 0], [1, 0], [2, 0.1], [0, 1.5]], np.float32)
    g, added = oracle.build_graph(pts, K=3, R=3)
    assert g.tolist() == [[1, 3, -1], [0, 2, -1], [1, -1, -1], [0, -1, -1]]
    assert added == 0
    # mean (0.75, 0.4): squared distances 0.7225, 0.2225, 1.6525, 1.7725
    assert oracle.medoid(pts) == 1


def test_repair_hand_case():
    # 1-D points 0,1,3,7 with K=1: rows 0->1, 1->0, 2->1, 3->2; the medoid
    # (mean 2.75) is node 2, which reaches {2,1,0}; node 3 is unreachable and
    # gets the edge from the nearest reachable node with a free slot: node 2.
    pts = np.array([[0], [1], [3], [7]], np.float32)
    g, added, pre = oracle.build_graph(pts, K=1, R=2, return_pre_repair=True)
    assert pre.tolist() == [[1, -1], [0, -1], [1, -1], [2, -1]]
    assert g.tolist() == [[1, -1], [0, -1], [1, 3], [2, -1]]
    assert added == 1


def _reachable(g, root):
    seen = np.zeros(len(g), bool)
    seen[root] = True
    stack = [root]
    while stack:
        v = stack.pop()
        for u in g[v]:
            if u >= 0 and not seen[u]:
                seen[u] = True
                stack.append(u)
    return seen


def test_graph_properties_random():
    w = synth.small_u8(n=1500, nq=1)
    base = w["base"]
    K, R = 24, 12
    g, added, pre = oracle.build_graph(base, K=K, R=R, return_pre_repair=True)
    med = oracle.medoid(base)
    assert _reachable(g, med).all()
    x = base.astype(np.int64)
    D = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    for p in range(0, 1500, 37):
        # candidates: exact K-NN excluding p, by (dist, id)
        order = [i for i in np.lexsort((np.arange(1500), D[p])) if i != p][:K]
        kept = []
        for c in order:
            if len(kept) == R:
                break
            if all(D[s, c] > D[p, c] for s in kept):
                kept.append(c)
        assert pre[p][pre[p] >= 0].tolist() == kept
        # every pruned candidate before the cut is dominated by a kept one
        row = pre[p][pre[p] >= 0].tolist()
        assert len(set(row)) == len(row) and p not in row
    # repair only appends edges into free slots
    assert ((g != pre) <= (pre < 0)).all()
    assert int((g != pre).sum()) == added


def test_medoid_matches_numpy():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((500, 12)).astype(np.float32)
    xd = x.astype(np.float64)
    ref = int(np.argmin(((xd - xd.mean(0)) ** 2).sum(1)))
    assert oracle.medoid(x) == ref
    u = synth.small_u8(n=800, nq=1)["base"]
    ud = u.astype(np.float64)
    assert oracle.medoid(u) == int(np.argmin(((ud - ud.mean(0)) ** 2).sum(1)))


def test_kmeans_hand_case():
    # 1-D points 0, 1, 10, 11 from centroids at rows 0 and 1:
    # it 1: assign {0},{1,10,11}: objective 0+0+81+100 = 181; c = 0, 22/3
    # it 2: assign {0,1},{10,11}: 0+1+(8/3)^2+(11/3)^2 = 1+185/9; c = .5, 10.5
    # it 3: objective 4 * 0.25 = 1
    x = np.array([[0], [1], [10], [11]], np.float32)
    c, a, obj = oracle.kmeans(x, 2, [0, 1], 3)
    np.testing.assert_allclose(obj, [181.0, 1.0 + 185.0 / 9.0, 1.0], rtol=1e-15)
    assert c.ravel().tolist() == [0.5, 10.5]
    h, asg = oracle.hubs(x, c)
    # members at equal distance 0.25 from their centroid: smaller id wins
    assert h.tolist() == [0, 2] and asg.tolist() == [0, 0, 1, 1]


def test_kmeans_objective_nonincreasing_and_hubs():
    w = synth.small_u8(n=2000, nq=1)
    x = w["base"]
    init = synth.kmeans_init(2000, 20, seed=3)
    c, a, obj = oracle.kmeans(x, 20, init, 12)
    assert (np.diff(obj) <= 1e-9 * obj[0]).all()
    h, asg = oracle.hubs(x, c)
    xd = x.astype(np.float64)
    for j in range(20):
        mem = np.where(asg == j)[0]
        if len(mem) == 0:
            assert h[j] == -1
            continue
        dd = ((xd[mem] - c[j]) ** 2).sum(1)
        assert h[j] == mem[np.lexsort((mem, dd))[0]]
    # assignment really is the nearest centroid
    D = ((xd[:, None, :] - c[None]) ** 2).sum(-1)
    assert np.array_equal(asg, np.argmin(D, 1))


def test_kmeans_recovers_separated_clusters():
    rng = np.random.default_rng(9)
    centres = np.array([[0, 0], [100, 0], [0, 100]], np.float64)
    lab = np.repeat(np.arange(3), 50)
    x = (centres[lab] + rng.standard_normal((150, 2))).astype(np.float32)
    init = np.array([0, 50, 100], np.int32)
    c, a, obj = oracle.kmeans(x, 3, init, 5)
    assert np.array_equal(a, lab)
    np.testing.assert_allclose(c, [x[lab == j].astype(np.float64).mean(0) for j in range(3)])


def test_kmeans_empty_cluster_reseed():
    # two identical initial rows: every row goes to centroid 0 (ties go to the
    # smaller centroid index), objective 0+0+1+100; centroid 0 moves to the
    # mean 2.75 and the empty centroid 1 onto the farthest row (10)
    x = np.array([[0], [0], [1], [10]], np.float32)
    c, a, obj = oracle.kmeans(x, 2, [0, 1], 1)
    assert c.ravel().tolist() == [2.75, 10.0]
    assert obj.tolist() == [101.0] and a.tolist() == [0, 0, 0, 0]


def test_hub_graph_matches_bruteforce():
    rng = np.random.default_rng(2)
    E = rng.standard_normal((60, 8))
    adj, ent = oracle.hub_graph(E, 5)
    En = E / np.linalg.norm(E, axis=1, keepdims=True)
    C = En @ En.T
    for i in range(60):
        cand = [j for j in range(60) if j != i]
        order = sorted(cand, key=lambda j: (-C[i, j], j))[:5]
        assert adj[i].tolist() == order
    mean_raw = E.mean(0)
    cos_to_mean = (E @ mean_raw) / (np.linalg.norm(E, axis=1) * np.linalg.norm(mean_raw))
    assert ent == int(np.argmax(cos_to_mean))


def test_hub_graph_hand_case():
    # four unit vectors at angles 0, 10, 90, 180 degrees (s = 1): nearest by
    # cosine: 0->1, 1->0, 2->1 (cos 80deg > cos 90deg), 3->2 (cos 90 > cos 170)
    a = np.deg2rad([0, 10, 90, 180])
    E = np.stack([np.cos(a), np.sin(a)], 1)
    adj, ent = oracle.hub_graph(E, 1)
    assert adj.ravel().tolist() == [1, 0, 1, 2]


def test_undirected_hub_graph_hand_case():
    # the four vectors above (s = 1): directed 0->1, 1->0, 2->1, 3->2, so the
    # undirected edges are {0,1}, {1,2}, {2,3}.  Rows by decreasing cosine:
    # 0: [1]; 1: [0 (cos 10deg), 2 (cos 80deg)]; 2: [1 (cos 80deg), 3 (cos 90deg)];
    # 3: [2]; width 3, padded with -1
    a = np.deg2rad([0, 10, 90, 180])
    E = np.stack([np.cos(a), np.sin(a)], 1)
    adj, ent = oracle.hub_graph_undirected(E, 1, 3)
    assert adj.tolist() == [[1, -1, -1], [0, 2, -1], [1, 3, -1], [2, -1, -1]]
    # a cap of one keeps the most similar neighbour only
    adj1, _ = oracle.hub_graph_undirected(E, 1, 1)
    assert adj1.ravel().tolist() == [1, 0, 1, 2]
    assert ent == oracle.hub_graph(E, 1)[1]


def test_undirected_hub_graph_matches_bruteforce():
    # against the definition from a brute-force cosine ranking: v in N(u) iff
    # v is among u's s nearest or u among v's; symmetric without a cap; each
    # capped row is the prefix of the uncapped one
    rng = np.random.default_rng(3)
    E = rng.standard_normal((80, 6))
    s = 4
    En = E / np.linalg.norm(E, axis=1, keepdims=True)
    C = En @ En.T
    top = [sorted([j for j in range(80) if j != i], key=lambda j: (-C[i, j], j))[:s] for i in range(80)]
    full, _ = oracle.hub_graph_undirected(E, s, 80)
    for i in range(80):
        want = {j for j in top[i]} | {j for j in range(80) if i in top[j]}
        row = [j for j in full[i] if j >= 0]
        assert row == sorted(want, key=lambda j: (-C[i, j], j))
        assert all(i in full[j] for j in row)
    capped, _ = oracle.hub_graph_undirected(E, s, 6)
    for i in range(80):
        row = [j for j in full[i] if j >= 0][:6]
        assert [j for j in capped[i] if j >= 0] == row
        assert (capped[i, len(row):] == -1).all()


def test_labels_rule_hand_case():
    I = oracle.INT32_MAX
    # one query, 5 searched hubs (indices 4,0,1,2,3 in the candidate list)
    cand = np.array([[4, 0, 1, 2, 3]])
    evals = np.array([[50, 40, 40, I, 300]])
    hops = np.array([[6, 5, 4, I, 25]])
    mask, best = oracle.labels_from_costs(evals, hops, cand, 6, t_pos=3, t_neg=15)
    # min hops = 4; positive: hops <= 7 -> hubs 4, 0, 1; negative: hops >= 19 or
    # unreached or unsearched -> hubs 3, 2, 5
    assert mask[0].tolist() == [1, 1, -1, -1, 1, -1]
    # best: smallest evals (40, tie) then hops (4 < 5) -> hub 1
    assert best[0] == 1
    mask, _ = oracle.labels_from_costs(evals, np.array([[6, 5, 4, I, 12]]), cand, 6)
    assert mask[0, 3] == 0  # hops 12: neither (7 < 12 < 19)


def test_listed_labels_hand_case():
    # the hand case above, labels per listed hub: cand [4, 0, 1, 2, 3] with
    # hops [6, 5, 4, unreached, 25] -> +1 +1 +1 -1 -1 (hub 5 is not listed: a
    # negative wherever the labels are used)
    I = oracle.INT32_MAX
    cand = np.array([[4, 0, 1, 2, 3], [0, 1, 2, 3, 4]])
    evals = np.array([[50, 40, 40, I, 300], [I, I, I, I, I]])
    hops = np.array([[6, 5, 4, I, 25], [I, I, I, I, I]])
    lab, best = oracle.labels_listed(evals, hops, cand)
    assert lab.tolist() == [[1, 1, 1, -1, -1], [-1, -1, -1, -1, -1]]
    assert best.tolist() == [1, -1]
    lab, _ = oracle.labels_listed(evals[:1], np.array([[6, 5, 4, I, 12]]), cand[:1])
    assert lab[0].tolist() == [1, 1, 1, -1, 0]


def test_listed_labels_expand_to_the_dense_rule():
    # listing each query's searched hubs with their labels, every other hub a
    # negative, is the dense label matrix of labels_from_costs
    rng = np.random.default_rng(4)
    nq, M, H = 60, 7, 20
    cand = np.stack([rng.choice(H, M, replace=False) for _ in range(nq)])
    hops = rng.integers(0, 30, (nq, M))
    hops[rng.random((nq, M)) < 0.2] = oracle.INT32_MAX
    hops[5] = oracle.INT32_MAX  # a query that reached nothing
    evals = np.where(hops < oracle.INT32_MAX, hops * 10 + rng.integers(0, 10, (nq, M)), oracle.INT32_MAX)
    for tp, tn in ((3, 15), (1, 5), (0, 1)):
        lab, best = oracle.labels_listed(evals, hops, cand, tp, tn)
        dense = np.full((nq, H), -1, np.int8)
        np.put_along_axis(dense, cand, lab, axis=1)
        ref, ref_best = oracle.labels_from_costs(evals, hops, cand, H, tp, tn)
        assert np.array_equal(dense, ref)
        assert np.array_equal(best, ref_best)


def test_hub_costs_match_individual_searches():
    rng = np.random.default_rng(1)
    base = rng.integers(0, 256, (400, 16)).astype(np.uint8)
    g, _ = oracle.build_graph(base, K=16, R=8)
    q = rng.integers(0, 256, (6, 16)).astype(np.float64)
    t, _ = oracle.knn(base, q, 1)
    hubs = np.array([0, 17, 99, 250], np.int32)
    ev, hp = oracle.hub_costs(base, g, q, hubs, t[:, 0], 32)
    for i in range(6):
        for j in range(4):
            _, _, e, h = oracle.search(base, g, q[i:i + 1], hubs[j], 32, 1, targets=[t[i, 0]])
            assert (ev[i, j], hp[i, j]) == (e[0], h[0])
    # a hub that is the target itself costs one evaluation and no hop
    ev2, hp2 = oracle.hub_costs(base, g, q[:1], np.array([t[0, 0]]), t[:1, 0], 32)
    assert (ev2[0, 0], hp2[0, 0]) == (1, 0)
