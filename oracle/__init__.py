"""CPU oracle for the GATE-style graph-ANNS query path (arXiv 2506.15986).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2506_15986_gb300``) and never imports it.

The search, exact k-NN, graph builder, medoid, k-means, hub and hub-graph
routines are plain C (``oracle.c``, compiled here with gcc, double-precision
arithmetic); the entry-model training routines are plain numpy in float64
(``train.py``).  Each function cites the passage of the paper it follows.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = None

U8, F32, F64 = 0, 1, 2
L2, IP = 0, 1
INT32_MAX = 2**31 - 1


def _lib_path() -> str:
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    return os.path.join(_HERE, f"liboracle_{tag}.so")


def build() -> str:
    """Compile oracle.c into a shared library (gcc, -O2, OpenMP)."""
    path = _lib_path()
    if not os.path.exists(path):
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC,
             "-o", tmp, "-lm"])
        os.replace(tmp, path)
    return path


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build())
        p, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.or_knn.argtypes = [p, i64, i32, i32, i32, p, i64, i32, p, p, p, i32]
        lib.or_knn.restype = i32
        lib.or_search.argtypes = [p, i64, i32, i32, i32, p, i32, p, i64, p, i32, i32,
                                  i32, p, p, i32, i32, p, p, p, p, p, i32]
        lib.or_search.restype = i32
        lib.or_medoid.argtypes = [p, i64, i32, i32]
        lib.or_medoid.restype = ctypes.c_int32
        lib.or_build_graph.argtypes = [p, i64, i32, i32, i32, i32, dbl,
                                       ctypes.c_int32, p, p, i32]
        lib.or_build_graph.restype = i64
        lib.or_kmeans.argtypes = [p, i64, i32, i32, i32, p, i32, p, p, p, i32]
        lib.or_kmeans.restype = i32
        lib.or_hubs.argtypes = [p, i64, i32, i32, p, i32, p, p, i32]
        lib.or_hubs.restype = i32
        lib.or_hbkm.argtypes = [p, i64, i32, i32, i32, dbl, i32, p, p, p, p, p]
        lib.or_hbkm.restype = i32
        lib.or_topo_tokens.argtypes = [p, i64, i32, p, i32, p, i32, i32, i32, p, p]
        lib.or_topo_tokens.restype = i32
        lib.or_hub_graph.argtypes = [p, i32, i32, i32, p, p]
        lib.or_hub_graph.restype = i32
        lib.or_num_threads.argtypes = []
        lib.or_num_threads.restype = i32
        _LIB = lib
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _base(x):
    x = np.ascontiguousarray(x)
    if x.dtype == np.uint8:
        return x, U8
    if x.dtype == np.float32:
        return x, F32
    if x.dtype == np.float64:
        return x, F64
    raise TypeError("base rows must be uint8, float32 or float64")


def num_threads() -> int:
    return int(_lib().or_num_threads())


def _threads(t):
    return num_threads() if t is None else int(t)


def knn(base, queries, k, metric=L2, exclude=None, threads=None):
    """Exact k nearest neighbours by (delta, id); delta in float64.

    Sec. 2.1, Problem 1 and the recall@k definition (R = exact top-k)."""
    base, dt = _base(base)
    q = np.ascontiguousarray(queries, dtype=np.float64)
    nq, d = q.shape
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    ex = None if exclude is None else np.ascontiguousarray(exclude, np.int32)
    rc = _lib().or_knn(_ptr(base), base.shape[0], d, dt, metric, _ptr(q), nq, k,
                       _ptr(ex), _ptr(ids), _ptr(dists), _threads(threads))
    if rc:
        raise RuntimeError(f"or_knn failed ({rc})")
    return ids, dists


def search(base, graph, queries, entries, L, k, metric=L2, W=1, Ls=None,
           ks=None, targets=None, threads=None):
    """Greedy best-first graph search (Sec. 2.1, Algorithm 1), sorted-pool form.

    entries: one node per query (scalar or [nq]) or a seed set per query
    ([nq, m], -1 = unused slot, at least one node): the initial pool holds
    every distinct seed, each evaluated once.
    Returns (ids [nq, kstride], dists float64, evals, hops); kstride = max k.
    With ``targets`` the search stops once the target id has been evaluated
    and reports the counters at that step (label mode, Sec. 4.2 Def. 4);
    counters are INT32_MAX when the target is never evaluated."""
    base, dt = _base(base)
    g = np.ascontiguousarray(graph, np.int32)
    q = np.ascontiguousarray(queries, dtype=np.float64)
    nq, d = q.shape
    e = np.asarray(entries, np.int32)
    m = e.shape[1] if e.ndim == 2 else 1
    ent = np.ascontiguousarray(np.broadcast_to(e, (nq, m) if e.ndim == 2 else (nq,)))
    Ls_a = None if Ls is None else np.ascontiguousarray(Ls, np.int32)
    ks_a = None if ks is None else np.ascontiguousarray(ks, np.int32)
    kstride = int(ks_a.max()) if ks_a is not None and nq else int(k)
    tg = None if targets is None else np.ascontiguousarray(targets, np.int32)
    ids = np.empty((nq, kstride), np.int32)
    dists = np.empty((nq, kstride), np.float64)
    ev = np.empty(nq, np.int32)
    hp = np.empty(nq, np.int32)
    rc = _lib().or_search(_ptr(base), base.shape[0], d, dt, metric, _ptr(g),
                          g.shape[1], _ptr(q), nq, _ptr(ent), int(m), int(L), int(k),
                          _ptr(Ls_a), _ptr(ks_a), kstride, int(W), _ptr(tg),
                          _ptr(ids), _ptr(dists), _ptr(ev), _ptr(hp),
                          _threads(threads))
    if rc:
        raise RuntimeError(f"or_search failed ({rc})")
    return ids, dists, ev, hp


def medoid(base) -> int:
    """Navigating node: argmin_i ||x_i - mean||^2 (Sec. 2.1, NSG)."""
    base, dt = _base(base)
    return int(_lib().or_medoid(_ptr(base), base.shape[0], base.shape[1], dt))


def build_graph(base, K=64, R=32, alpha=1.0, root=None, threads=None,
                return_pre_repair=False):
    """Exact K-NN candidates + relative-neighbourhood pruning + reachability
    repair from ``root`` (default: the medoid).  Sec. 2.1, Def. 1."""
    base, dt = _base(base)
    n, d = base.shape
    if root is None:
        root = medoid(base)
    g = np.empty((n, R), np.int32)
    pre = np.empty((n, R), np.int32) if return_pre_repair else None
    rc = _lib().or_build_graph(_ptr(base), n, d, dt, int(K), int(R), float(alpha),
                               int(root), _ptr(g), _ptr(pre), _threads(threads))
    if rc < 0:
        raise RuntimeError(f"or_build_graph failed ({-rc})")
    if return_pre_repair:
        return g, int(rc), pre
    return g, int(rc)


def kmeans(x, k, init, iters, threads=None):
    """Lloyd's k-means (flat stand-in for Algorithm 2). Returns
    (centroids float64 [k, d], assignment of the last iteration, objective[T])."""
    x, dt = _base(x)
    m, d = x.shape
    init = np.ascontiguousarray(init, np.int32)
    cent = np.empty((k, d), np.float64)
    asg = np.empty(m, np.int32)
    obj = np.empty(max(iters, 1), np.float64)
    rc = _lib().or_kmeans(_ptr(x), m, d, dt, int(k), _ptr(init), int(iters),
                          _ptr(cent), _ptr(asg), _ptr(obj), _threads(threads))
    if rc:
        raise RuntimeError(f"or_kmeans failed ({rc})")
    return cent, asg, obj[:iters]


def hubs(base, centroids, threads=None):
    """Hub nodes (Sec. 4.1, Def. 3). Returns (hub ids [k], assignment [n])."""
    base, dt = _base(base)
    n, d = base.shape
    c = np.ascontiguousarray(centroids, np.float64)
    k = c.shape[0]
    h = np.empty(k, np.int32)
    a = np.empty(n, np.int32)
    rc = _lib().or_hubs(_ptr(base), n, d, dt, _ptr(c), k, _ptr(h), _ptr(a),
                        _threads(threads))
    if rc:
        raise RuntimeError(f"or_hubs failed ({rc})")
    return h, a


def hbkm(x, k, levels, lam, T, keys):
    """Hierarchical balanced k-means (Sec. 4.1, Def. 2, Algorithm 2) and the
    hub of every final cluster (Def. 3), float32 as or_hbkm states.  keys:
    one uint32 per row, the seeded draw that picks each split's initial
    centroids.  Returns (label [n], centroids float32 [k^levels, d],
    hubs [k^levels] (-1 = empty), sizes [k^levels])."""
    x = np.ascontiguousarray(x, np.float32)
    n, d = x.shape
    keys = np.ascontiguousarray(keys, np.uint32)
    assert keys.shape == (n,)
    nc = int(k) ** int(levels)
    label = np.empty(n, np.int32)
    cent = np.empty((nc, d), np.float32)
    hubs = np.empty(nc, np.int32)
    sizes = np.empty(nc, np.int64)
    rc = _lib().or_hbkm(_ptr(x), n, d, int(k), int(levels), float(lam), int(T), _ptr(keys),
                        _ptr(label), _ptr(cent), _ptr(hubs), _ptr(sizes))
    if rc:
        raise RuntimeError(f"or_hbkm failed ({rc})")
    return label, cent, hubs, sizes


TOKEN_DIM = 8


def topo_tokens(base, graph, hubs, h, max_nodes=4096):
    """Per-hop topology tokens of each hub from the guided subgraph walk
    (Sec. 4.2), float32 as or_topo_tokens states.  Returns (tokens
    float32 [H, h+1, 8], subgraph sizes [H])."""
    x = np.ascontiguousarray(base, np.float32)
    n, d = x.shape
    g = np.ascontiguousarray(graph, np.int32)
    hubs = np.ascontiguousarray(hubs, np.int32)
    H = len(hubs)
    tok = np.empty((H, h + 1, TOKEN_DIM), np.float32)
    nodes = np.empty(H, np.int32)
    rc = _lib().or_topo_tokens(_ptr(x), n, d, _ptr(g), g.shape[1], _ptr(hubs), H, int(h), int(max_nodes),
                               _ptr(tok), _ptr(nodes))
    if rc:
        raise RuntimeError(f"or_topo_tokens failed ({rc})")
    return tok, nodes


def hub_graph(emb, s):
    """High-tier hub graph (Sec. 4.3): s most cosine-similar hubs per hub.
    Returns (adjacency [H, s], entry hub)."""
    e = np.ascontiguousarray(emb, np.float64)
    H, dim = e.shape
    adj = np.empty((H, s), np.int32)
    ent = np.zeros(1, np.int32)
    rc = _lib().or_hub_graph(_ptr(e), H, dim, int(s), _ptr(adj), _ptr(ent))
    if rc:
        raise RuntimeError(f"or_hub_graph failed ({rc})")
    return adj, int(ent[0])


def hub_graph_undirected(emb, s, max_degree):
    """Undirected reading of the high-tier hub graph (Sec. 4.3): hubs u and v
    are linked when v is among u's s most cosine-similar hubs or u among v's
    (the directed lists of ``hub_graph``).  Row i holds i's neighbours in
    decreasing cosine (float64, ties to the smaller index), at most
    max_degree of them, padded with -1.  Returns (adjacency [H, max_degree],
    entry hub)."""
    adj, ent = hub_graph(emb, s)
    e = np.asarray(emb, np.float64)
    en = e / np.linalg.norm(e, axis=1, keepdims=True)
    H = len(e)
    nbrs = [set() for _ in range(H)]
    for i in range(H):
        for j in adj[i]:
            nbrs[i].add(int(j))
            nbrs[int(j)].add(i)
    out = np.full((H, max_degree), -1, np.int32)
    for i in range(H):
        lst = sorted(nbrs[i], key=lambda j: (-float(en[i] @ en[j]), j))[:max_degree]
        out[i, :len(lst)] = lst
    return out, ent


def recall_at_k(found_ids, truth_ids, k):
    """recall@k = |R ∩ R'| / k averaged over queries (Sec. 2.1, Eq. recall)."""
    f = np.asarray(found_ids)[:, :k]
    t = np.asarray(truth_ids)[:, :k]
    hits = 0
    for a, b in zip(f, t):
        hits += len(set(a[a >= 0].tolist()) & set(b[b >= 0].tolist()))
    return hits / (k * len(f)) if len(f) else 0.0


def hub_costs(base, graph, queries, hub_nodes, targets, L, cand=None, W=1,
              metric=L2, threads=None):
    """Per (query, hub) search cost for label generation (Sec. 4.2, Def. 4).

    For query i and hub index h in cand[i] (default: every hub), run the
    search of ``search`` from node hub_nodes[h] in label mode with target
    targets[i] (the query's exact nearest neighbour) and pool size L.
    Returns (evals, hops) of shape [nq, M]; INT32_MAX where never reached."""
    q = np.ascontiguousarray(queries, np.float64)
    nq = q.shape[0]
    hub_nodes = np.asarray(hub_nodes, np.int32)
    if cand is None:
        cand = np.broadcast_to(np.arange(len(hub_nodes), dtype=np.int32),
                               (nq, len(hub_nodes)))
    cand = np.asarray(cand, np.int32)
    M = cand.shape[1]
    qq = np.repeat(q, M, axis=0)
    ent = hub_nodes[cand.reshape(-1)]
    tg = np.repeat(np.asarray(targets, np.int32), M)
    _, _, ev, hp = search(base, graph, qq, ent, L, 1, metric=metric, W=W,
                          targets=tg, threads=threads)
    return ev.reshape(nq, M), hp.reshape(nq, M)


def labels_from_costs(evals, hops, cand, n_hubs, t_pos=3, t_neg=15):
    """Label rule (Sec. 4.2, Def. 4 and the per-query assignment that follows
    it; t_pos = 3 and t_neg = 15 from Sec. 5.1), read per query over hubs:

    * best hub = argmin over searched hubs of (evals, hops, hub index);
    * m = min hops over searched hubs that reached the target;
    * positive (+1): reached with hops <= m + t_pos;
    * negative (-1): hops >= m + t_neg, never reached, or not searched;
    * otherwise 0 (left out of the loss).
    Returns (mask int8 [nq, n_hubs], best int32 [nq], -1 when none reached)."""
    evals = np.asarray(evals, np.int64)
    hops = np.asarray(hops, np.int64)
    cand = np.asarray(cand, np.int64)
    nq, M = cand.shape
    mask = np.full((nq, n_hubs), -1, np.int8)
    best = np.full(nq, -1, np.int32)
    for i in range(nq):
        reached = hops[i] < INT32_MAX
        if not reached.any():
            continue
        m = hops[i][reached].min()
        order = sorted(range(M), key=lambda j: (evals[i, j], hops[i, j], cand[i, j]))
        best[i] = cand[i, order[0]]
        for j in range(M):
            h = cand[i, j]
            if not reached[j]:
                mask[i, h] = -1
            elif hops[i, j] <= m + t_pos:
                mask[i, h] = 1
            elif hops[i, j] >= m + t_neg:
                mask[i, h] = -1
            else:
                mask[i, h] = 0
    return mask, best


def labels_listed(evals, hops, cand, t_pos=3, t_neg=15):
    """The label rule of ``labels_from_costs`` written per listed hub: for
    query i, the label of its searched hub cand[i, j] (+1, -1 or 0, the same
    rule), so that a hub not listed for a query is a negative (it was never
    searched from that query).  Returns (labels int8 [nq, M], best int32 [nq]).
    Sec. 4.2, Def. 4 and the per-query assignment after it."""
    evals = np.asarray(evals, np.int64)
    hops = np.asarray(hops, np.int64)
    cand = np.asarray(cand, np.int64)
    nq, M = cand.shape
    lab = np.full((nq, M), -1, np.int8)
    best = np.full(nq, -1, np.int32)
    for i in range(nq):
        reached = [j for j in range(M) if hops[i, j] < INT32_MAX]
        if not reached:
            continue
        m = min(hops[i, j] for j in reached)
        best[i] = cand[i, min(reached, key=lambda j: (evals[i, j], hops[i, j], cand[i, j]))]
        for j in reached:
            if hops[i, j] <= m + t_pos:
                lab[i, j] = 1
            elif hops[i, j] < m + t_neg:
                lab[i, j] = 0
    return lab, best


def merge_answers(ids_list, dists_list, k):
    """Answer of a base-partitioned search: per query, the k smallest
    (distance, id) pairs of the union of the shards' answers (Sec. 2.1,
    Problem 1's order; -1 entries are empty), padded with (-1, +inf).
    ids_list / dists_list: one [nq, k_s] array per shard, ids global.
    Returns (ids int32 [nq, k], dists float64 [nq, k])."""
    nq = len(ids_list[0])
    ids = np.full((nq, k), -1, np.int32)
    dists = np.full((nq, k), np.inf)
    for i in range(nq):
        pairs = sorted((float(d[i, j]), int(a[i, j])) for a, d in zip(ids_list, dists_list)
                       for j in range(a.shape[1]) if a[i, j] >= 0)[:k]
        for j, (dv, iv) in enumerate(pairs):
            ids[i, j], dists[i, j] = iv, dv
    return ids, dists


def pruned_row(base, p, K, R, alpha=1.0):
    """Steps 1-2 of the graph builder (Sec. 2.1, Def. 1) for the single node p:
    its K exact nearest other nodes by (dist, id), then relative-neighbourhood
    pruning in that order (c kept unless a kept s has alpha*d(s,c) <= d(p,c)),
    at most R kept.  Distances in float64."""
    b = np.asarray(base)
    x = b.astype(np.float64) if b.dtype != np.float64 else b
    ids, dists = knn(b, x[p:p + 1], K, exclude=[p])
    kept = []
    for c, dpc in zip(ids[0].tolist(), dists[0].tolist()):
        if c < 0 or len(kept) == R:
            break
        if all(alpha * float(((x[s] - x[c]) ** 2).sum()) > dpc for s in kept):
            kept.append(c)
    return kept


def rerank(base_exact, pool_ids, queries, k, metric=L2):
    """Exact re-scoring of a final pool: the ids of each row of pool_ids
    (-1 = empty) ordered by (float64 distance to the exact rows, id); the first
    k are returned with their distances ((-1, +inf) padding)."""
    x = np.asarray(base_exact, np.float64)
    q = np.asarray(queries, np.float64)
    nq = q.shape[0]
    ids = np.full((nq, k), -1, np.int32)
    dists = np.full((nq, k), np.inf)
    for i in range(nq):
        p = [int(v) for v in pool_ids[i] if v >= 0]
        if not p:
            continue
        diff = x[p] - q[i]
        d = (diff * diff).sum(1) if metric == L2 else -(x[p] @ q[i])
        order = sorted(range(len(p)), key=lambda j: (d[j], p[j]))[:k]
        ids[i, :len(order)] = [p[j] for j in order]
        dists[i, :len(order)] = [d[j] for j in order]
    return ids, dists


def quantize_i8s(x):
    """int8 codes with one scale per row, as the precision line's int8
    storage reads: in fp32, scale = max_j |x_j| / 127 and code_j = x_j / scale
    rounded half to even, clipped to [-127, 127]; an all-zero row gets scale 0
    and zero codes.  Returns (codes int8 [n, d], scales float32 [n])."""
    x = np.ascontiguousarray(x, np.float32)
    scale = (np.abs(x).max(axis=1) / np.float32(127)).astype(np.float32)
    safe = np.where(scale > 0, scale, np.float32(1)).astype(np.float32)
    q = np.rint(x / safe[:, None])
    q = np.clip(q, -127, 127)
    q[scale == 0] = 0
    return q.astype(np.int8), scale


def dequantize_i8s(codes, scales):
    """The rows int8 storage stands for, x_j = scale * code_j, exact in
    float64 (a 24-bit by 8-bit product)."""
    return np.asarray(codes, np.float64) * np.asarray(scales, np.float64)[:, None]
