"""Precision line: reduced-precision (FP16 / BF16 / int8 with a per-row scale)
storage searched with FP32 accumulation, then the exact FP32 rerank of the
final pool (ANN_SEARCH_RERANK), against the oracle run on the same rounded
rows and re-scored in float64.  The int8 codes and scales themselves are
bit-exact against the oracle's quantiser.

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
    elif storage == "i8s":
        n, d = base.shape
        packed = _quantize(base)
        rows = oracle.dequantize_i8s(*oracle.quantize_i8s(base))
        h = ann.ann_index_create(packed, case["graph"], case["medoid"], ann.I8S, ann.L2, base_f32=base,
                                 n=n, dim=d, degree=case["graph"].shape[1])
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


def _quantize(base):
    """Packed int8 rows from ann_quantize_i8s, checked byte for byte against
    the oracle's codes and scales."""
    n, d = base.shape
    rb = ann.ann_i8s_row_bytes(d)
    assert rb == 16 + (d + 15) // 16 * 16
    packed = torch.full((n, rb), 0xAB, dtype=torch.uint8, device=DEV)
    ann.ann_quantize_i8s(torch.from_numpy(base).to(DEV), n, d, packed)
    torch.cuda.synchronize()
    pk = packed.cpu().numpy()
    codes, scales = oracle.quantize_i8s(base)
    assert np.array_equal(pk[:, :4].copy().view(np.uint32)[:, 0], scales.view(np.uint32))
    assert (pk[:, 4:16] == 0).all() and (pk[:, 16 + d:] == 0).all()
    assert np.array_equal(pk[:, 16:16 + d].copy().view(np.int8), codes)
    return packed


def _run(h, q, L, k, flags):
    dq = torch.from_numpy(q).to(DEV)
    ids = torch.empty((len(q), k), dtype=torch.int32, device=DEV)
    dd = torch.empty((len(q), k), dtype=torch.float32, device=DEV)
    ann.ann_search_batch(h, dq, len(q), None, ann.search_params(k, L, flags=flags), ids, dd)
    assert ann.ann_sync_status(h) == ann.OK
    return ids.cpu().numpy(), dd.cpu().numpy()


@pytest.mark.parametrize("storage", ["f16", "bf16", "i8s"])
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


def test_i8s_inner_product_and_ragged_dim():
    # unit rows, maximum inner product; dim 200 leaves a partly used last
    # 16-code chunk (zero codes against a zero-extended query)
    w = synth.ip_f32(n=12000, nq=200)
    base = w["base"]
    g, _ = oracle.build_graph(base, K=48, R=32)
    med = oracle.medoid(base)
    packed = _quantize(base)
    h = ann.ann_index_create(packed, g, med, ann.I8S, ann.IP, n=len(base), dim=base.shape[1], degree=32)
    try:
        q = w["queries"]
        ids, d = _run(h, q, 64, 10, 0)
    finally:
        ann.ann_free_index(h)
    rows = oracle.dequantize_i8s(*oracle.quantize_i8s(base))
    oi, od, _, _ = oracle.search(rows, g, q.astype(np.float64), med, 64, 10, metric=oracle.IP)
    assert (ids == oi).mean() >= 0.999
    ok = ids == oi
    scale = np.linalg.norm(q.astype(np.float64), axis=1)[:, None].repeat(10, 1)  # |x| <= 1
    assert (np.abs(d.astype(np.float64) - od)[ok] / scale[ok]).max() <= 1e-5
