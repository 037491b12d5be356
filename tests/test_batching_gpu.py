"""Batching line on the GPU: one persistent launch over queries with mixed k
and L (k in {1, 10, 100}, L uniform in [max(32, k), 512], as in the 10M batch
workload), a CUDA-graph plan of entry selection + search, and the autotuner,
whose knobs must leave results unchanged."""
import numpy as np
import pytest

import oracle
from paper_2506_15986_gb300 import ann, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def case():
    w = synth.shift_f32(n=15000, nq=600, n_train=0)
    g, _ = oracle.build_graph(w["base"], K=48, R=32)
    med = oracle.medoid(w["base"])
    h = ann.ann_index_create(w["base"], g, med, ann.F32, ann.L2)
    rng = np.random.default_rng(4)
    k = rng.choice(np.array([1, 10, 100], np.int32), size=600)
    lo = np.maximum(32, k)
    L = (lo + np.floor(rng.random(600) * (513 - lo))).astype(np.int32)
    yield dict(w, graph=g, medoid=med, h=h, k=k.astype(np.int32), L=L)
    ann.ann_free_index(h)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_mixed_k_and_L_in_one_launch(case):
    q = case["queries"]
    nq = len(q)
    ids = torch.empty((nq, 100), dtype=torch.int32, device=DEV)
    dd = torch.empty((nq, 100), dtype=torch.float32, device=DEV)
    st = torch.empty((nq, 2), dtype=torch.int32, device=DEV)
    dk, dL, dq = _t(case["k"]), _t(case["L"]), _t(q)  # kept alive until the launch completes
    p = ann.search_params(100, 512, d_k=dk, d_L=dL)
    ann.ann_search_batch(case["h"], dq, nq, None, p, ids, dd, st)
    assert ann.ann_sync_status(case["h"]) == ann.OK
    oi, od, oe, oh = oracle.search(case["base"], case["graph"], q.astype(np.float64), case["medoid"],
                                   0, 0, Ls=case["L"], ks=case["k"])
    gi = ids.cpu().numpy()
    valid = np.arange(100)[None, :] < case["k"][:, None]
    assert ((gi == oi) | ~valid).all(1).mean() >= 0.99
    assert (gi[valid] == oi[valid]).mean() >= 0.999
    assert (gi[~valid] == -1).all()
    s = st.cpu().numpy()
    assert (s[:, 0] == oe).mean() >= 0.99 and (s[:, 1] == oh).mean() >= 0.99


def _model(case):
    H = 128
    W1, b1, W2, b2, E = synth.model_init(128, H, seed=3)
    hub_nodes = np.random.default_rng(8).choice(len(case["base"]), H, replace=False).astype(np.int32)
    ann.ann_set_entry_model(case["h"], 128, W1, b1, W2, b2, hub_nodes, E, 8)


@pytest.mark.parametrize("mode", [ann.ENTRY_MEDOID, ann.ENTRY_LEARNED_NAV, ann.ENTRY_LEARNED_EXHAUSTIVE])
def test_graph_plan_replays_the_batch(case, mode):
    if mode != ann.ENTRY_MEDOID:
        _model(case)
    q = _t(case["queries"])
    nq = q.shape[0]
    p = ann.search_params(10, 64)
    ref_e = torch.empty(nq, dtype=torch.int32, device=DEV)
    ref_i = torch.empty((nq, 10), dtype=torch.int32, device=DEV)
    ref_d = torch.empty((nq, 10), dtype=torch.float32, device=DEV)
    ent = None
    if mode != ann.ENTRY_MEDOID:
        ann.ann_select_entry(case["h"], q, nq, mode, 24, ref_e)
        ent = ref_e
    ann.ann_search_batch(case["h"], q, nq, ent, p, ref_i, ref_d)
    buf = torch.empty(nq, dtype=torch.int32, device=DEV)
    ids = torch.full((nq, 10), -9, dtype=torch.int32, device=DEV)
    dd = torch.zeros((nq, 10), dtype=torch.float32, device=DEV)
    plan = ann.ann_plan_create(case["h"], q, nq, mode, 24, p, buf, ids, dd)
    try:
        for _ in range(2):
            ids.fill_(-9)
            ann.ann_plan_launch(plan)
            torch.cuda.synchronize()
            assert torch.equal(ids, ref_i) and torch.equal(dd, ref_d)
    finally:
        ann.ann_plan_free(plan)
    assert ann.ann_sync_status(case["h"]) == ann.OK


@pytest.mark.parametrize("lanes", [1, 3])
def test_autotune_keeps_results(case, lanes):
    q = _t(case["queries"])
    nq = q.shape[0]
    p = ann.search_params(10, 128)
    ids = torch.empty((nq, 10), dtype=torch.int32, device=DEV)
    dd = torch.empty((nq, 10), dtype=torch.float32, device=DEV)
    ann.ann_search_batch(case["h"], q, nq, None, p, ids, dd)
    ref = ids.clone(), dd.clone()
    ids.fill_(-7)
    best, ms = ann.ann_autotune(case["h"], q, nq, None, p, ids, dd, reps=3, lanes=lanes)
    assert ms > 0 and (best.hash_bits >= 8 or best.hash_bits == -1) and best.stage_rows in (4, 6, 8, 12, 16)
    assert best.gather in (0, 4) and best.flags & ~ann.SEARCH_VISITED_L2 == 0
    assert best.team in (2, 4, 8, 16, 32) and best.spill_bits in (0, 10, 11, 12, 13, 14, 15, 16)
    tuned = ids.clone(), dd.clone()  # the autotuner leaves the chosen combination's results
    ann.ann_search_batch(case["h"], q, nq, None, best, ids, dd)
    torch.cuda.synchronize()
    assert torch.equal(ids, tuned[0]) and torch.equal(dd, tuned[1])
    # the visited-table and gather sizes never change results: equal to a
    # run with the default knobs at the same team size
    same = ann.search_params(10, 128, team=best.team)
    ids2, dd2 = torch.empty_like(ids), torch.empty_like(dd)
    ann.ann_search_batch(case["h"], q, nq, None, same, ids2, dd2)
    torch.cuda.synchronize()
    assert torch.equal(ids, ids2) and torch.equal(dd, dd2)
    # another team size only reorders the FP32 sums: the fp32 parity bar
    a, b = ids.cpu().numpy(), ref[0].cpu().numpy()
    assert (a == b).mean() >= 0.999
    ok = a == b
    da, db = dd.cpu().numpy()[ok].astype(np.float64), ref[1].cpu().numpy()[ok].astype(np.float64)
    assert (np.abs(da - db) <= 1e-5 * np.abs(db)).all()


def test_autotune_rejects_bad_lanes(case):
    q = _t(case["queries"][:8])
    ids = torch.empty((8, 10), dtype=torch.int32, device=DEV)
    dd = torch.empty((8, 10), dtype=torch.float32, device=DEV)
    for bad in (0, 9):
        with pytest.raises(ann.AnnError) as e:
            ann.ann_autotune(case["h"], q, 8, None, ann.search_params(10, 64), ids, dd, lanes=bad)
        assert e.value.status == ann.ERR_INVALID_ARG


def test_concurrent_batches_on_lanes(case):
    # consecutive batches on separate streams overlap on the device; each call
    # takes its own stream-ordered scratch, so the results equal one batch at a
    # time on one stream
    q = case["queries"]
    nq = len(q)
    p = ann.search_params(10, 96)
    halves = [_t(q[: nq // 2]), _t(q[nq // 2:])]
    ref = []
    for dq in halves:
        ids = torch.empty((dq.shape[0], 10), dtype=torch.int32, device=DEV)
        dd = torch.empty((dq.shape[0], 10), dtype=torch.float32, device=DEV)
        ann.ann_search_batch(case["h"], dq, dq.shape[0], None, p, ids, dd)
        torch.cuda.synchronize()
        ref.append((ids.cpu().numpy(), dd.cpu().numpy()))
    lanes = [torch.cuda.Stream(device=DEV) for _ in range(3)]
    outs = []
    for rep in range(4):
        for j, dq in enumerate(halves):
            s = lanes[(2 * rep + j) % 3]
            with torch.cuda.stream(s):
                ids = torch.empty((dq.shape[0], 10), dtype=torch.int32, device=DEV)
                dd = torch.empty((dq.shape[0], 10), dtype=torch.float32, device=DEV)
            ann.ann_search_batch(case["h"], dq, dq.shape[0], None, p, ids, dd, None, s)
            outs.append((j, ids, dd))
    torch.cuda.synchronize()
    assert ann.ann_sync_status(case["h"]) == ann.OK
    for j, ids, dd in outs:
        assert np.array_equal(ids.cpu().numpy(), ref[j][0])
        assert np.array_equal(dd.cpu().numpy(), ref[j][1])
