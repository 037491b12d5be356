"""GPU parity of the batched beam search (Sec. 2.1, Algorithm 1) against the
CPU oracle, through the C ABI.

uint8 data: ids, int32 distances, evaluation and expansion counts bit-exact.
fp32 data: >= 99.9% of (query, rank) ids equal, distances within 1e-5
relative (1e-5 of |x||q| for inner product), recall@10 within 0.001."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2506_15986_gb300 import ann, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import make_index, search  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2506_15986_gb300 import _build
    _build.build()
    ann.load_library()


@pytest.fixture(scope="module")
def c1():
    w = synth.small_u8()
    g, _ = oracle.build_graph(w["base"], K=64, R=32, alpha=1.0)
    med = oracle.medoid(w["base"])
    h = make_index(w["base"], g, med)
    yield dict(w, graph=g, medoid=med, h=h)
    ann.ann_free_index(h)


def _oracle(w, q, L, k, **kw):
    return oracle.search(w["base"], w["graph"], np.asarray(q, np.float64),
                         kw.pop("entries", w["medoid"]), L, k, **kw)


def test_toy_graphs_exact(golden_dir):
    with open(os.path.join(golden_dir, "toy_graphs.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        pts = np.asarray(c["points"], np.float32)
        pad = np.zeros((len(pts), 4), np.float32)
        pad[:, : pts.shape[1]] = pts  # zero padding keeps squared L2 unchanged
        q = np.zeros((1, 4), np.float32)
        q[0, : pts.shape[1]] = c["query"]
        h = make_index(pad, np.asarray(c["adjacency"], np.int32), c["entry"])
        try:
            ids, d, ev, hp, st = search(h, q, c["k"], c["L"], W=c["W"])
        finally:
            ann.ann_free_index(h)
        assert st == ann.OK
        assert ids[0].tolist() == c["ids"], c["name"]
        exp = [math.inf if v == "inf" else float(v) for v in c["dists"]]
        assert d[0].tolist() == exp, c["name"]
        assert (int(ev[0]), int(hp[0])) == (c["evals"], c["hops"]), c["name"]


@pytest.mark.parametrize("L,W", [(64, 1), (16, 1), (128, 1), (64, 2), (512, 2), (10, 1),
                                 (64, 3), (128, 4), (512, 4), (1024, 4), (2048, 2), (4096, 2)])
def test_c1_u8_bit_exact(c1, L, W):
    q = c1["queries"]
    k = min(10, L)
    ids, d, ev, hp, st = search(c1["h"], q, k, L, W=W)
    oi, od, oe, oh = _oracle(c1, q, L, k, W=W)
    assert st == ann.OK
    assert np.array_equal(ids, oi)
    assert np.array_equal(d, od.astype(np.int64).clip(max=2**31 - 1).astype(np.int32))
    assert np.array_equal(ev, oe) and np.array_equal(hp, oh)


@pytest.mark.parametrize("R,W", [(100, 1), (64, 2), (128, 1)])
def test_u8_wide_rows_bit_exact(c1, R, W):
    # unpruned K-NN graphs with up to 128 neighbour slots per step: ragged
    # last slot (R = 100), and steps whose survivors need the 128-key sort
    base = c1["base"][:4000]
    g, _ = oracle.knn(base, base.astype(np.float64), R, exclude=np.arange(len(base), dtype=np.int32))
    med = oracle.medoid(base)
    h = make_index(base, g, med)
    try:
        q = c1["queries"]
        ids, d, ev, hp, st = search(h, q, 10, 96, W=W)
    finally:
        ann.ann_free_index(h)
    oi, od, oe, oh = oracle.search(base, g, q.astype(np.float64), med, 96, 10, W=W)
    assert st == ann.OK
    assert np.array_equal(ids, oi)
    assert np.array_equal(d, od.astype(np.int64).astype(np.int32))
    assert np.array_equal(ev, oe) and np.array_equal(hp, oh)


@pytest.mark.parametrize("team,stage_rows,gather", [(1, 32, 1), (2, 4, 1), (4, 8, 1), (16, 16, 1), (32, 5, 1),
                                                    (4, 8, 4), (8, 5, 4), (2, 12, 4), (32, 16, 4), (4, 1, 4)])
def test_c1_team_sizes_bit_exact(c1, team, stage_rows, gather):
    # every distance team size, gather round size and fetch mode (a bulk copy
    # per row, or TMA tensor gathers of four rows with ragged rounds padded)
    # gives the same exact int32 distances, hence the same search
    q = c1["queries"]
    ids, d, ev, hp, st = search(c1["h"], q, 10, 128, W=2, team=team, stage_rows=stage_rows, gather=gather)
    oi, od, oe, oh = _oracle(c1, q, 128, 10, W=2)
    assert st == ann.OK
    assert np.array_equal(ids, oi) and np.array_equal(ev, oe) and np.array_equal(hp, oh)
    assert np.array_equal(d, od.astype(np.int64).astype(np.int32))


def test_forced_wait_timeout_is_reported_and_recoverable(c1):
    # fault injection: every wait for gathered rows gives up at once.  Each
    # query fails with -1 ids, the call reports a timeout, the copies in
    # flight still land, and the next normal call on the same index is exact.
    q = c1["queries"]
    ids, d, ev, hp, st = search(c1["h"], q, 10, 64, flags=ann.SEARCH_FAULT_WAIT)
    assert st == ann.ERR_TIMEOUT
    assert (ids == -1).all() and (d == 2**31 - 1).all()
    ids, d, ev, hp, st = search(c1["h"], q, 10, 64)
    oi, od, oe, oh = _oracle(c1, q, 64, 10)
    assert st == ann.OK
    assert np.array_equal(ids, oi) and np.array_equal(ev, oe) and np.array_equal(hp, oh)


@pytest.mark.parametrize("L,spill_bits,hash_bits", [(128, 0, 8), (512, 10, 8), (128, 0, -1), (512, 10, -1)])
def test_c1_spill_to_global_table_stays_exact(c1, L, spill_bits, hash_bits):
    # hash_bits=8: 192 shared slots, far fewer than the evaluations, so the
    # exact global spill table carries most of the visited set; with
    # spill_bits=10 at L=512 most queries pass 768 evaluations and move on to
    # the second, 4x larger table
    q = c1["queries"]
    ids, d, ev, hp, st = search(c1["h"], q, 10, L, hash_bits=hash_bits, spill_bits=spill_bits)
    oi, od, oe, oh = _oracle(c1, q, L, 10)
    assert st == ann.OK
    assert (oe > 192).mean() > 0.8  # most queries outgrow the shared table
    if spill_bits:
        assert (oe > 768).mean() > 0.5  # ... and the first global one
    assert np.array_equal(ids, oi) and np.array_equal(ev, oe) and np.array_equal(hp, oh)


@pytest.mark.parametrize("spill_bits", [10, 12])
def test_visited_tables_kept_in_l2_change_nothing(c1, spill_bits):
    # ANN_SEARCH_VISITED_L2 only changes where the first-level visited tables
    # live in the cache: the search stays bit-exact
    q = c1["queries"]
    ids, d, ev, hp, st = search(c1["h"], q, 10, 96, W=2, hash_bits=-1, spill_bits=spill_bits,
                                flags=ann.SEARCH_VISITED_L2)
    oi, od, oe, oh = _oracle(c1, q, 96, 10, W=2)
    assert st == ann.OK
    assert np.array_equal(ids, oi) and np.array_equal(ev, oe) and np.array_equal(hp, oh)
    assert np.array_equal(d, od.astype(np.int64).astype(np.int32))


@pytest.mark.parametrize("nq,m,n_hubs", [(20_000, 1, 8), (6_000, 4, 1_500), (1, 1, 1), (5_000, 1, 5_000)])
def test_grouped_work_order_changes_nothing(c1, nq, m, n_hubs):
    # ANN_SEARCH_GROUP_ENTRIES only changes the order in which the teams take
    # the work items (sorted by a hash of the first seed): every item's ids,
    # distances and counters stay bit-exact at its own index.  Batches larger
    # than the sort's 4,096 buckets and 1,024 threads, few and many distinct
    # first seeds, seed sets, per-query k and L.
    rng = np.random.default_rng(nq + m)
    q = np.tile(c1["queries"], (nq // len(c1["queries"]) + 1, 1))[:nq]
    hubs = rng.choice(len(c1["base"]), n_hubs, replace=False)
    seeds = hubs[rng.integers(0, n_hubs, (nq, m))].astype(np.int32)
    if m > 1:
        seeds[:, 1:][rng.random((nq, m - 1)) < 0.3] = -1
    Ls = rng.integers(10, 97, nq).astype(np.int32)
    ks = np.minimum(rng.integers(1, 11, nq), Ls).astype(np.int32)
    ent = seeds if m > 1 else seeds[:, 0]
    ids, d, ev, hp, st = search(c1["h"], q, 10, 96, W=2, entries=ent, ks=ks, Ls=Ls,
                                flags=ann.SEARCH_GROUP_ENTRIES)
    oi, od, oe, oh = oracle.search(c1["base"], c1["graph"], q.astype(np.float64), ent, 0, 0, W=2,
                                   Ls=Ls, ks=ks)
    assert st == ann.OK
    oi_full = np.full((nq, 10), -1, np.int32)
    oi_full[:, : oi.shape[1]] = oi
    assert np.array_equal(ids, oi_full)
    assert np.array_equal(ev, oe) and np.array_equal(hp, oh)
    od_full = np.zeros((nq, 10), np.int64)
    od_full[:, : od.shape[1]] = np.where(np.isfinite(od), od, 0).astype(np.int64)
    valid = oi_full >= 0
    assert np.array_equal(d[valid], od_full[valid].astype(np.int32))


def test_grouped_work_order_with_a_bad_seed(c1):
    # a seed out of range fails its own item only, wherever the sort put it
    q = np.tile(c1["queries"], (30, 1))
    seeds = np.full(len(q), c1["medoid"], np.int32)
    seeds[1234] = len(c1["base"])
    ids, d, ev, hp, st = search(c1["h"], q, 10, 64, entries=seeds, flags=ann.SEARCH_GROUP_ENTRIES)
    assert st == ann.ERR_INVALID_ARG
    assert (ids[1234] == -1).all()
    ok = np.arange(len(q)) != 1234
    oi, od, oe, oh = _oracle(c1, q[ok], 64, 10)
    assert np.array_equal(ids[ok], oi) and np.array_equal(ev[ok], oe)


def test_c1_per_query_entries_k_L(c1):
    rng = np.random.default_rng(3)
    q = c1["queries"]
    nq = len(q)
    entries = rng.integers(0, len(c1["base"]), nq).astype(np.int32)
    Ls = rng.integers(10, 200, nq).astype(np.int32)
    ks = np.minimum(rng.integers(1, 11, nq), Ls).astype(np.int32)
    ids, d, ev, hp, st = search(c1["h"], q, 10, 200, entries=entries, ks=ks, Ls=Ls)
    oi, od, oe, oh = oracle.search(c1["base"], c1["graph"], q.astype(np.float64), entries, 0, 0,
                                   Ls=Ls, ks=ks)
    assert st == ann.OK
    oi_full = np.full((nq, 10), -1, np.int32)
    oi_full[:, : oi.shape[1]] = oi
    assert np.array_equal(ids, oi_full)
    assert np.array_equal(ev, oe) and np.array_equal(hp, oh)


@pytest.mark.parametrize("m,W", [(2, 1), (4, 4), (32, 2)])
def test_c1_seed_sets_bit_exact(c1, m, W):
    # seed sets with unused slots (-1) and repeated seeds: the initial pool
    # holds every distinct seed, evaluated once
    rng = np.random.default_rng(m)
    q = c1["queries"]
    seeds = rng.integers(0, len(c1["base"]), (len(q), m)).astype(np.int32)
    seeds[rng.random(seeds.shape) < 0.3] = -1
    seeds[:, 0] = np.where(seeds[:, 0] < 0, c1["medoid"], seeds[:, 0])
    if m > 1:
        seeds[::3, 1] = seeds[::3, 0]  # a repeated seed
    ids, d, ev, hp, st = search(c1["h"], q, 10, 64, W=W, entries=seeds)
    oi, od, oe, oh = oracle.search(c1["base"], c1["graph"], q.astype(np.float64), seeds, 64, 10, W=W)
    assert st == ann.OK
    assert np.array_equal(ids, oi) and np.array_equal(ev, oe) and np.array_equal(hp, oh)
    assert np.array_equal(d, od.astype(np.int64).astype(np.int32))


def test_c1_label_mode_targets(c1):
    q = c1["queries"][:50]
    t, _ = oracle.knn(c1["base"], q.astype(np.float64), 1)
    rng = np.random.default_rng(5)
    entries = rng.integers(0, len(c1["base"]), 50).astype(np.int32)
    entries[0] = t[0, 0]  # entry is the target: 1 evaluation, 0 expansions
    ids, d, ev, hp, st = search(c1["h"], q, 1, 64, entries=entries, targets=t[:, 0])
    _, _, oe, oh = oracle.search(c1["base"], c1["graph"], q.astype(np.float64), entries, 64, 1,
                                 targets=t[:, 0])
    assert st == ann.OK
    assert np.array_equal(ev, oe) and np.array_equal(hp, oh)
    assert (ev[0], hp[0]) == (1, 0)


def test_empty_batch_and_bad_device_inputs(c1):
    q = c1["queries"]
    ids, d, ev, hp, st = search(c1["h"], q[:0], 10, 64)
    assert ids.shape == (0, 10) and st == ann.OK
    # a per-query L above the launch maximum is reported, never read past
    ids, d, ev, hp, st = search(c1["h"], q[:4], 10, 64, Ls=np.array([64, 65, 64, 64]))
    assert st == ann.ERR_INVALID_ARG
    assert (ids[1] == -1).all() and (ids[0] >= 0).all()
    assert ann.ann_sync_status(c1["h"]) == ann.OK  # cleared by the read
    # host-side parameter checks return before any launch
    for kw in (dict(team=3), dict(team=64), dict(stage_rows=33), dict(W=5), dict(hash_bits=7), dict(hash_bits=-2),
               dict(spill_bits=9), dict(spill_bits=17), dict(flags=16), dict(gather=2),
               dict(entries=np.zeros((4, 33), np.int32))):
        with pytest.raises(ann.AnnError) as e:
            search(c1["h"], q[:4], 10, 64, **kw)
        assert e.value.status == ann.ERR_INVALID_ARG, kw
    # a seed row without any node, or with an id out of range, fails on the device
    for bad in ([-1, -1], [5, len(c1["base"])]):
        ids, d, ev, hp, st = search(c1["h"], q[:1], 10, 64, entries=np.array([bad], np.int32))
        assert st == ann.ERR_INVALID_ARG and (ids == -1).all()


@pytest.fixture(scope="module")
def f32_case():
    w = synth.shift_f32(n=20000, nq=300, n_train=0)
    g, _ = oracle.build_graph(w["base"], K=64, R=32)
    med = oracle.medoid(w["base"])
    h = make_index(w["base"], g, med)
    yield dict(w, graph=g, medoid=med, h=h)
    ann.ann_free_index(h)


def _f32_parity(ids, d, oi, od, truth, scale=None):
    agree = (ids == oi).mean()
    assert agree >= 0.999, agree
    ok = ids == oi
    ref = np.abs(od) if scale is None else scale[:, None].repeat(od.shape[1], 1)
    rel = np.abs(d.astype(np.float64) - od)[ok] / np.maximum(ref[ok], 1e-30)
    assert rel.max() <= 1e-5, rel.max()
    r_gpu = oracle.recall_at_k(ids, truth, 10)
    r_or = oracle.recall_at_k(oi, truth, 10)
    assert abs(r_gpu - r_or) <= 1e-3


@pytest.mark.parametrize("L,W,team,gather", [(32, 1, 0, 0), (64, 1, 0, 0), (128, 2, 0, 0), (128, 2, 2, 0),
                                            (128, 4, 32, 0), (96, 4, 4, 4), (128, 4, 8, 4)])
def test_f32_l2_parity(f32_case, L, W, team, gather):
    q = f32_case["queries"]
    ids, d, ev, hp, st = search(f32_case["h"], q, 10, L, W=W, team=team, gather=gather)
    oi, od, oe, oh = _oracle(f32_case, q, L, 10, W=W)
    truth, _ = oracle.knn(f32_case["base"], q.astype(np.float64), 10)
    assert st == ann.OK
    _f32_parity(ids, d, oi, od, truth)
    assert (ev == oe).mean() >= 0.99 and (hp == oh).mean() >= 0.99


def test_f32_ip_parity():
    w = synth.ip_f32(n=12000, nq=200)
    base = w["base"]
    # graph built on L2 over unit vectors (same order as IP for unit norms)
    g, _ = oracle.build_graph(base, K=48, R=32)
    med = oracle.medoid(base)
    h = make_index(base, g, med, metric=ann.IP)
    try:
        q = w["queries"]
        ids, d, ev, hp, st = search(h, q, 10, 64)
    finally:
        ann.ann_free_index(h)
    oi, od, oe, oh = oracle.search(base, g, q.astype(np.float64), med, 64, 10, metric=oracle.IP)
    truth, _ = oracle.knn(base, q.astype(np.float64), 10, metric=oracle.IP)
    scale = np.linalg.norm(q.astype(np.float64), axis=1)  # |x| = 1
    assert st == ann.OK
    _f32_parity(ids, d, oi, od, truth, scale=scale)


def test_visited_set_outgrows_both_global_tables():
    # points on a line, x_i = i, each node linked to the next 64: a search
    # from node 0 walks the chain and evaluates every node up to a little past
    # the query.  At L = 16 the shared table (1,024 slots) and the first
    # global table (4,096) overflow; the 4x larger one takes up to 12,288
    # keys, so the query at 6,000 still finishes exactly and the one at
    # 14,000 (all 14,000 nodes) fails with a capacity status and -1 ids.
    n, R = 14000, 64
    base = np.zeros((n, 4), np.float32)
    base[:, 0] = np.arange(n)
    nb = np.arange(n)[:, None] + 1 + np.arange(R)[None, :]
    g = np.where(nb < n, nb, -1).astype(np.int32)
    q = np.zeros((3, 4), np.float32)
    q[:, 0] = [2000, 6000, 14000]
    h = make_index(base, g, 0)
    try:
        ids, d, ev, hp, st = search(h, q, 10, 16, hash_bits=10)
    finally:
        ann.ann_free_index(h)
    assert st == ann.ERR_CAPACITY
    oi, od, oe, oh = oracle.search(base, g, q[:2].astype(np.float64), 0, 16, 10)
    assert oe[1] > 3 * 4096 // 4  # past the first global table
    assert np.array_equal(ids[:2], oi) and np.array_equal(ev[:2], oe) and np.array_equal(hp[:2], oh)
    assert np.array_equal(d[:2], od.astype(np.float32))
    assert (ids[2] == -1).all()
