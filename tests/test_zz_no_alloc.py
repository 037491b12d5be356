"""The allocation-free entry selection, checked against the regular one.

ann_select_entry_noalloc serves callers that cannot let the library allocate
device memory (a process that reserved all of HBM up front, a latency-bound
loop, a host callback); it keeps its scratch in a static per-device array.
Here it must give the same entries and query embeddings as
ann_select_entry in its exhaustive mode, on two calls in a row (the second
call reuses the array the first one left behind), and refuse a batch larger
than the array holds.  This file is collected last so that a failure here
never hides the other tests, and it builds everything it needs itself."""
import numpy as np
import pytest

from paper_2506_15986_gb300 import _build, ann, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def index_with_model():
    _build.build()
    w = synth.shift_f32(n=3000, nq=900, n_train=0)
    base = w["base"]
    rng = np.random.default_rng(0)
    graph = np.stack([rng.choice(3000, 16, replace=False) for _ in range(3000)]).astype(np.int32)
    h = ann.ann_index_create(base, graph, 0, ann.F32, ann.L2)
    H = 200
    W1, b1, W2, b2, E = synth.model_init(128, H, seed=7)
    hub_nodes = rng.choice(3000, H, replace=False).astype(np.int32)
    ann.ann_set_entry_model(h, 128, W1, b1, W2, b2, hub_nodes, E, 8)
    yield h, torch.from_numpy(w["queries"]).to(DEV)
    ann.ann_free_index(h)


def test_noalloc_matches_regular_path_twice(index_with_model):
    h, q = index_with_model
    nq = q.shape[0]
    ref_e = torch.empty(nq, dtype=torch.int32, device=DEV)
    ref_q = torch.empty((nq, 64), dtype=torch.float32, device=DEV)
    ann.ann_select_entry(h, q, nq, ann.ENTRY_LEARNED_EXHAUSTIVE, 32, ref_e, ref_q)
    assert ann.ann_sync_status(h) == ann.OK
    for _ in range(2):
        e = torch.full((nq,), -5, dtype=torch.int32, device=DEV)
        qh = torch.zeros((nq, 64), dtype=torch.float32, device=DEV)
        ann.ann_select_entry_noalloc(h, q, nq, e, qh)
        assert ann.ann_sync_status(h) == ann.OK
        assert torch.equal(e, ref_e)
        # same kernels on the same inputs: within the FP32 level the other
        # entry tests allow (they are in fact identical)
        assert float((qh - ref_q).abs().max()) <= 1e-6


def test_noalloc_rejects_batches_beyond_its_scratch(index_with_model):
    h, q = index_with_model
    cap = ann.ann_select_entry_noalloc_max_queries()
    assert cap == (16 << 20) // 136 - 4
    out = torch.empty(1, dtype=torch.int32, device=DEV)
    with pytest.raises(ann.AnnError) as err:
        ann.ann_select_entry_noalloc(h, q, cap + 1, out)  # refused before any launch
    assert err.value.status == ann.ERR_CAPACITY


def test_noalloc_at_its_largest_batch(index_with_model):
    # the three scratch regions at the largest accepted batch, each padded to
    # 256 bytes, must still fit: compare with the regular path there
    h, q = index_with_model
    cap = ann.ann_select_entry_noalloc_max_queries()
    reps = (cap + q.shape[0] - 1) // q.shape[0]
    big = q.repeat(reps, 1)[:cap].contiguous()
    ref_e = torch.empty(cap, dtype=torch.int32, device=DEV)
    ann.ann_select_entry(h, big, cap, ann.ENTRY_LEARNED_EXHAUSTIVE, 32, ref_e)
    e = torch.full((cap,), -5, dtype=torch.int32, device=DEV)
    qh = torch.zeros((cap, 64), dtype=torch.float32, device=DEV)
    ann.ann_select_entry_noalloc(h, big, cap, e, qh)
    assert ann.ann_sync_status(h) == ann.OK
    assert torch.equal(e, ref_e)
    # row i of the batch repeats query i mod nq: the last rows' embeddings
    # equal those of the rows they repeat
    n0 = q.shape[0]
    rows = torch.arange(cap - n0, cap, device=DEV) % n0
    assert torch.equal(qh[cap - n0:cap], qh[rows])


def test_noalloc_on_a_uint8_index():
    w = synth.small_u8(n=2000, nq=300)
    rng = np.random.default_rng(3)
    graph = np.stack([rng.choice(2000, 16, replace=False) for _ in range(2000)]).astype(np.int32)
    h = ann.ann_index_create(w["base"], graph, 0, ann.U8, ann.L2)
    try:
        H = 64
        W1, b1, W2, b2, E = synth.model_init(128, H, seed=9)
        ann.ann_set_entry_model(h, 128, W1, b1, W2, b2, rng.choice(2000, H, replace=False).astype(np.int32), E, 8)
        q = torch.from_numpy(w["queries"]).to(DEV)
        nq = q.shape[0]
        ref_e = torch.empty(nq, dtype=torch.int32, device=DEV)
        ann.ann_select_entry(h, q, nq, ann.ENTRY_LEARNED_EXHAUSTIVE, 32, ref_e)
        for _ in range(2):
            e = torch.full((nq,), -5, dtype=torch.int32, device=DEV)
            ann.ann_select_entry_noalloc(h, q, nq, e)
            assert ann.ann_sync_status(h) == ann.OK
            assert torch.equal(e, ref_e)
    finally:
        ann.ann_free_index(h)
