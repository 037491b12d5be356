"""GPU offline builders against the oracle: exact k-NN (ground truth of
recall@k), the medoid, and the proximity graph (K-NN + relative-neighbourhood
pruning + reachability repair).  uint8 data: bit-exact; fp32 data: the
agreement bars of the search tests."""
import numpy as np
import pytest

import oracle
from paper_2506_15986_gb300 import ann, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

DEV = torch.device("cuda:0")


def _knn_gpu(base, q, k, metric=ann.L2, exclude_self=False):
    db = torch.from_numpy(base).to(DEV)
    dq = db if exclude_self else torch.from_numpy(q).to(DEV)
    ids = torch.empty((len(q), k), dtype=torch.int32, device=DEV)
    dists = torch.empty((len(q), k), dtype=torch.int32 if base.dtype == np.uint8 else torch.float32,
                        device=DEV)
    dt = ann.U8 if base.dtype == np.uint8 else ann.F32
    ann.ann_knn(db, len(base), base.shape[1], dt, metric, dq, len(q), k, ids, dists, exclude_self)
    return ids.cpu().numpy(), dists.cpu().numpy()


def _graph_gpu(base, K, R, alpha=1.0):
    db = torch.from_numpy(base).to(DEV)
    g = torch.empty((len(base), R), dtype=torch.int32, device=DEV)
    dt = ann.U8 if base.dtype == np.uint8 else ann.F32
    med, rep = ann.ann_build_graph(db, len(base), base.shape[1], dt, K, R, alpha, g)
    return g.cpu().numpy(), med, rep


def test_knn_u8_bit_exact():
    w = synth.small_u8()
    ids, d = _knn_gpu(w["base"], w["queries"], 10)
    oi, od = oracle.knn(w["base"], w["queries"].astype(np.float64), 10)
    assert np.array_equal(ids, oi) and np.array_equal(d, od.astype(np.int32))


def test_knn_u8_self_excluded_k64():
    w = synth.small_u8(n=3000, nq=1)
    base = w["base"]
    ids, d = _knn_gpu(base, base, 64, exclude_self=True)
    oi, od = oracle.knn(base, base.astype(np.float64), 64, exclude=np.arange(3000))
    assert np.array_equal(ids, oi) and np.array_equal(d, od.astype(np.int32))


def test_knn_f32_l2_and_ip():
    w = synth.shift_f32(n=30000, nq=500, n_train=0)
    ids, d = _knn_gpu(w["base"], w["queries"], 10)
    oi, od = oracle.knn(w["base"], w["queries"].astype(np.float64), 10)
    assert (ids == oi).mean() >= 0.999
    ok = ids == oi
    assert (np.abs(d - od)[ok] / od[ok]).max() <= 1e-5
    v = synth.ip_f32(n=20000, nq=300)
    ids, d = _knn_gpu(v["base"], v["queries"], 10, metric=ann.IP)
    oi, od = oracle.knn(v["base"], v["queries"].astype(np.float64), 10, metric=oracle.IP)
    assert (ids == oi).mean() >= 0.999
    ok = ids == oi
    assert np.abs(d - od)[ok].max() <= 1e-5


def test_medoid_u8_exact_and_f32_within_tolerance():
    w = synth.small_u8()
    db = torch.from_numpy(w["base"]).to(DEV)
    assert ann.ann_medoid(db, 10000, 128, ann.U8) == oracle.medoid(w["base"])
    f = synth.shift_f32(n=50000, nq=1, n_train=0)["base"]
    m = ann.ann_medoid(torch.from_numpy(f).to(DEV), len(f), 128, ann.F32)
    x = f.astype(np.float64)
    dd = ((x - x.mean(0)) ** 2).sum(1)
    assert dd[m] <= dd.min() * (1 + 1e-5)


def test_graph_u8_bit_exact_with_repair():
    w = synth.small_u8()
    g, med, rep = _graph_gpu(w["base"], 64, 32)
    og, orep = oracle.build_graph(w["base"], K=64, R=32)
    assert med == oracle.medoid(w["base"])
    assert rep == orep and rep > 0
    assert np.array_equal(g, og)


def test_graph_f32_agreement():
    w = synth.shift_f32(n=20000, nq=1, n_train=0)
    g, med, rep = _graph_gpu(w["base"], 64, 32)
    og, orep = oracle.build_graph(w["base"], K=64, R=32)
    same_rows = (g == og).all(1).mean()
    assert same_rows >= 0.99, same_rows
    # every node reachable from the medoid
    seen = np.zeros(len(g), bool)
    seen[med] = True
    st = [med]
    while st:
        v = st.pop()
        for u in g[v]:
            if u >= 0 and not seen[u]:
                seen[u] = True
                st.append(u)
    assert seen.all()


def test_insertion_graph_builder():
    # insertion by search: a seed of 15,000 rows built exactly, 45,000 more
    # inserted in batches of 15,000; the graph is valid and reachable, and a
    # search on it reaches the exact graph's recall
    from gpu_util import search
    w = synth.shift_f32(n=60000, nq=500, n_train=0)
    x = torch.from_numpy(w["base"]).to(DEV)
    n, d = w["base"].shape
    g_in = torch.empty((n, 32), dtype=torch.int32, device=DEV)
    g_ex = torch.empty((n, 32), dtype=torch.int32, device=DEV)
    med_i, _ = ann.ann_build_graph_insert(x, n, d, ann.F32, 64, 32, 1.0, 15000, 15000, g_in)
    med_e, _ = ann.ann_build_graph(x, n, d, ann.F32, 64, 32, 1.0, g_ex)
    assert med_i == med_e  # the navigating node does not depend on the edges
    gi = g_in.cpu().numpy()
    assert ((gi >= -1) & (gi < n)).all() and (gi != np.arange(n)[:, None]).all()
    assert all(len(set(r[r >= 0])) == (r >= 0).sum() for r in gi[::97])  # no repeated edge
    seen = np.zeros(n, bool)
    seen[med_i] = True
    front = np.array([med_i])
    while len(front):
        nxt = gi[front].ravel()
        nxt = np.unique(nxt[nxt >= 0])
        nxt = nxt[~seen[nxt]]
        seen[nxt] = True
        front = nxt
    assert seen.all()
    q = w["queries"]
    truth, _ = oracle.knn(w["base"], q.astype(np.float64), 10)
    rec = []
    for g, med in ((g_in, med_i), (g_ex, med_e)):
        h = ann.ann_index_create(x, g, med, ann.F32, ann.L2)
        try:
            ids, *_ = search(h, q, 10, 64, W=2)
        finally:
            ann.ann_free_index(h)
        rec.append(np.mean([len(np.intersect1d(a, b)) / 10 for a, b in zip(ids, truth)]))
    assert rec[0] >= rec[1] - 0.02, rec
    with pytest.raises(ann.AnnError):
        ann.ann_build_graph_insert(x, n, d, ann.F32, 64, 48, 1.0, 15000, 15000, g_in)  # R > 32
