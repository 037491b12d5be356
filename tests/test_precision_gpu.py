"""Precision line: reduced-precision (FP16 / BF16) storage searched with FP32
accumulation, then the exact FP32 rerank of the final pool (ANN_SEARCH_RERANK),
against the oracle run on the same rounded rows and re-scored in float64.

Bars: the traversal over rounded rows follows the fp32 agreement bar of the
search tests (>= 99.9 % equal ids, 1e-5 relative distances); after the rerank
the answer is the exact fp32 answer: ids within the same bar, distances 1e-5
relative to the float64 distances of the fp32 rows."""
import numpy as np
import pytest

import oracle
from paper_2506_15986_gb300 import ann, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
DEV = torch.device("cuda:0")


def _bf16(x):
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def case():
    w = synth.shift_f32(n=20000, nq=300, n_train=0)
    g, _ = oracle.build_graph(w["base"], K=64, R=32)
    return dict(w, graph=g, medoid=oracle.medoid(w["base"]))


def _index(case, storage):
    base = case["base"]
    if storage == "f16":
        stored = base.astype(np.float16)
        rows = stored.astype(np.float32)
        h = ann.ann_index_create(stored, case["graph"], case["medoid"], ann.F16, ann.L2, base_f32=base)
    else:
        rows = _bf16(base)
        stored = torch.from_numpy(base).to(torch.bfloat16)  # round to nearest even
        d = ann.ann_index_desc(n=len(base), dim=128, degree=32, dtype=ann.BF16, metric=ann.L2,
                               base=stored.data_ptr(), graph=case["graph"].ctypes.data,
                               medoid=int(case["medoid"]), base_f32=base.ctypes.data)
        import ctypes
        hh = ctypes.c_void_p()
        assert ann.load_library().ann_index_create(ctypes.byref(d), 0, ctypes.byref(hh)) == ann.OK
        h = hh.value
    return h, rows


def _run(h, q, L, k, flags):
    dq = torch.from_numpy(q).to(DEV)
    ids = torch.empty((len(q), k), dtype=torch.int32, device=DEV)
    dd = torch.empty((len(q), k), dtype=torch.float32, device=DEV)
    ann.ann_search_batch(h, dq, len(q), None, ann.search_params(k, L, flags=flags), ids, dd)
    assert ann.ann_sync_status(h) == ann.OK
    return ids.cpu().numpy(), dd.cpu().numpy()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_reduced_storage_and_exact_rerank(case, storage):
    h, rows = _index(case, storage)
    try:
        q = case["queries"]
        L, k = 96, 10
        ids, d = _run(h, q, L, k, 0)
        pool, pd, _, _ = oracle.search(rows, case["graph"], q.astype(np.float64), case["medoid"], L, L)
        assert (ids == pool[:, :k]).mean() >= 0.999
        ok = ids == pool[:, :k]
        assert (np.abs(d - pd[:, :k])[ok] / pd[:, :k][ok]).max() <= 1e-5
        rid, rd = _run(h, q, L, k, ann.SEARCH_RERANK)
        oid, od = oracle.rerank(case["base"], pool, q, k)
        assert (rid == oid).mean() >= 0.999
        ok = rid == oid
        assert (np.abs(rd - od)[ok] / od[ok]).max() <= 1e-5
        # the rerank can only move results closer to the exact answer
        truth, _ = oracle.knn(case["base"], q.astype(np.float64), k)
        assert oracle.recall_at_k(rid, truth, k) >= oracle.recall_at_k(ids, truth, k) - 1e-9
    finally:
        ann.ann_free_index(h)


def test_rerank_needs_the_fp32_copy(case):
    h = ann.ann_index_create(case["base"].astype(np.float16), case["graph"], case["medoid"], ann.F16,
                             ann.L2)
    try:
        with pytest.raises(ann.AnnError) as e:
            _run(h, case["queries"][:4], 32, 10, ann.SEARCH_RERANK)
        assert e.value.status == ann.ERR_UNSUPPORTED
    finally:
        ann.ann_free_index(h)
