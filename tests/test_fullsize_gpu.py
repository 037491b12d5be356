"""Search parity at the bench's full size and launch configuration: the shifted
1M x 128 fp32 workload (10,000 queries, graph exact 64-NN + RNG prune R = 32
built on the GPU), W = 4, L = 93, the tuned sizes of the headline (no shared
visited table, 8-row gather rounds, 4-lane distance teams, default spill
table), the batch on three streams at once as the bench's lanes run it.

The lanes must agree bit for bit; sampled queries are recomputed one by one
by the float64 oracle on the same graph, entries and (L, W) and must meet the
fp32 bar: >= 99.9 % of (query, rank) ids equal, distances of equal ids within
1e-5 relative, and recall@10 against the GPU's exact ground truth within
0.001 of the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2506_15986_gb300 import ann, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
DEV = torch.device("cuda:0")

N, NQ, R, L, W, K = 1_000_000, 10_000, 32, 93, 4, 10


@pytest.fixture(scope="module")
def full():
    w = synth.shift_f32(n=N, nq=NQ, n_train=0)
    base = torch.from_numpy(w["base"]).to(DEV)
    graph = torch.empty((N, R), dtype=torch.int32, device=DEV)
    med, _ = ann.ann_build_graph(base, N, 128, ann.F32, 64, R, 1.0, graph)
    q = torch.from_numpy(w["queries"]).to(DEV)
    gt = torch.empty((NQ, K), dtype=torch.int32, device=DEV)
    gd = torch.empty((NQ, K), dtype=torch.float32, device=DEV)
    ann.ann_knn(base, N, 128, ann.F32, ann.L2, q, NQ, K, gt, gd)
    h = ann.ann_index_create(base, graph, med, ann.F32, ann.L2)
    yield dict(w=w, base=base, graph=graph.cpu().numpy(), med=med, q=q, gt=gt.cpu().numpy(), h=h)
    ann.ann_free_index(h)


def _lanes(full, entries, m, gather=1, l2=False, extra=0, stage_rows=8):
    flags = (ann.SEARCH_VISITED_L2 if l2 else 0) | extra
    p = ann.search_params(K, L, W=W, hash_bits=-1, stage_rows=stage_rows, team=4, n_entries=m, gather=gather,
                          spill_bits=12 if l2 else 0, flags=flags)
    streams = [torch.cuda.Stream(device=DEV) for _ in range(3)]
    outs = []
    torch.cuda.synchronize()
    for s in streams:
        with torch.cuda.stream(s):
            ids = torch.empty((NQ, K), dtype=torch.int32, device=DEV)
            dd = torch.empty((NQ, K), dtype=torch.float32, device=DEV)
            st = torch.empty((NQ, 2), dtype=torch.int32, device=DEV)
        ann.ann_search_batch(full["h"], full["q"], NQ, entries, p, ids, dd, st, s)
        outs.append((ids, dd, st))
    torch.cuda.synchronize()
    assert ann.ann_sync_status(full["h"]) == ann.OK
    res = [tuple(t.cpu().numpy() for t in o) for o in outs]
    for r in res[1:]:
        for a, b in zip(res[0], r):
            assert np.array_equal(a, b)  # the lanes agree bit for bit
    return res[0]


def _recall(ids, gt):
    return np.mean([len(set(a) & set(b)) / K for a, b in zip(ids, gt)])


@pytest.mark.parametrize("seeds,gather,l2,extra,stage_rows", [
    (0, 1, False, 0, 8), (2, 1, False, 0, 8), (0, 4, True, 0, 8),
    (1, 1, True, ann.SEARCH_GROUP_ENTRIES, 8)])
def test_full_size_sampled_parity(full, seeds, gather, l2, extra, stage_rows):
    # l2: the tuned headline's 2^12-slot first-level visited tables kept
    # resident in L2 (ANN_SEARCH_VISITED_L2); extra: the work order grouped
    # by entry (ANN_SEARCH_GROUP_ENTRIES)
    rng = np.random.default_rng(11 + seeds)
    if seeds:
        ent_np = rng.integers(0, N, size=(NQ, seeds)).astype(np.int32)
        ent = torch.from_numpy(ent_np if seeds > 1 else ent_np[:, 0].copy()).to(DEV)
    else:
        ent_np, ent = None, None
    ids, dd, st = _lanes(full, ent, seeds if seeds > 1 else 0, gather, l2, extra, stage_rows)
    sample = np.sort(rng.choice(NQ, 200, replace=False))
    q64 = full["w"]["queries"][sample].astype(np.float64)
    e = full["med"] if ent_np is None else (ent_np[sample] if seeds > 1 else ent_np[sample, 0])
    oi, od, oe, oh = oracle.search(full["w"]["base"], full["graph"], q64, e, L, K, W=W)
    gi, gd = ids[sample], dd[sample].astype(np.float64)
    same = gi == oi
    assert same.mean() >= 0.999, same.mean()
    assert (np.abs(gd[same] - od[same]) <= 1e-5 * np.maximum(od[same], 1e-30)).all()
    assert abs(_recall(gi, full["gt"][sample]) - _recall(oi, full["gt"][sample])) <= 0.001
    assert (st[sample, 0] == oe).mean() >= 0.99 and (st[sample, 1] == oh).mean() >= 0.99


def _other(gen, R, metric, L, W, tuned, nq, seeds):
    """Build a million-row workload, run its bench configuration on three
    lanes and compare 100 sampled queries with the oracle."""
    w = gen()
    x = w["base"]
    n, d = x.shape
    base = torch.from_numpy(x).to(DEV)
    graph = torch.empty((n, R), dtype=torch.int32, device=DEV)
    med, _ = ann.ann_build_graph(base, n, d, ann.F32, 64, R, 1.0, graph)
    qn = w["queries"][:nq]
    q = torch.from_numpy(np.ascontiguousarray(qn)).to(DEV)
    h = ann.ann_index_create(base, graph, med, ann.F32, metric)
    try:
        rng = np.random.default_rng(5)
        ent_np = rng.integers(0, n, size=(nq, seeds)).astype(np.int32) if seeds else None
        ent = None if ent_np is None else torch.from_numpy(ent_np).to(DEV)
        p = ann.search_params(K, L, W=W, n_entries=seeds, **tuned)
        outs = []
        torch.cuda.synchronize()
        for s in [torch.cuda.Stream(device=DEV) for _ in range(3)]:
            with torch.cuda.stream(s):
                ids = torch.empty((nq, K), dtype=torch.int32, device=DEV)
                dd = torch.empty((nq, K), dtype=torch.float32, device=DEV)
            ann.ann_search_batch(h, q, nq, ent, p, ids, dd, None, s)
            outs.append((ids, dd))
        torch.cuda.synchronize()
        assert ann.ann_sync_status(h) == ann.OK
        res = [(a.cpu().numpy(), b.cpu().numpy()) for a, b in outs]
    finally:
        ann.ann_free_index(h)
    for r in res[1:]:
        assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])
    sample = np.sort(rng.choice(nq, 100, replace=False))
    e = med if ent_np is None else ent_np[sample]
    oi, od, _, _ = oracle.search(x, graph.cpu().numpy(), qn[sample].astype(np.float64), e, L, K, W=W,
                                 metric=oracle.IP if metric == ann.IP else oracle.L2)
    gi, gd = res[0][0][sample], res[0][1][sample].astype(np.float64)
    same = gi == oi
    assert same.mean() >= 0.999, same.mean()
    scale = np.maximum(np.abs(od[same]), 1e-30) if metric == ann.L2 else \
        np.linalg.norm(x[gi[same]], axis=1) * np.linalg.norm(qn[sample], axis=1)[np.nonzero(same)[0]]
    assert (np.abs(gd[same] - od[same]) <= 1e-5 * scale).all()


def test_full_size_ip_config():
    # 1M x 200 unit vectors, maximum inner product, out-of-distribution
    # queries; L = 1,088 (recall 0.95), the bench's tuned sizes, 2-node seeds
    _other(lambda: synth.ip_f32(n=1_000_000, nq=10_000, n_train=0), 32, ann.IP, 1088, 4,
           dict(hash_bits=-1, stage_rows=4, team=8, spill_bits=16), 10_000, 2)


def test_full_size_960d_config():
    # 1M x 960 fp32 (3.84 GB), R = 48, W = 2, L = 224, 1,000 queries, medoid
    _other(lambda: synth.highdim_f32(n=1_000_000, nq=1_000), 48, ann.L2, 224, 2,
           dict(hash_bits=-1, stage_rows=4, team=16, spill_bits=16), 1_000, 0)
