"""Base-partitioned search on the GPU against the oracle.

The merge kernel and the id map are checked bit for bit against
oracle.merge_answers and plain indexing; the whole path (shards of whole
clusters, each with its own GPU-built graph, searched by ann_search_batch,
ids mapped, answers merged) against the oracle's search of the same shard
graphs merged by oracle.merge_answers (uint8 data: bit-exact); and two ranks
that share cuda:0, each holding one shard and exchanging answers over gloo,
against the same path run in one process.  The two ranks' kernels never wait
on each other: the exchange is a host-side all-gather between launches."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_2506_15986_gb300 import ann, shard, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
DEV = torch.device("cuda:0")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sorted_lists(rng, P, nq, k, int_dists):
    ids = np.full((P, nq, k), -1, np.int32)
    d = np.full((P, nq, k), np.inf)
    used = rng.permutation(10 * P * nq * k).astype(np.int32)  # distinct ids across lists
    for p in range(P):
        for i in range(nq):
            n = rng.integers(0, k + 1)  # ragged: some lists shorter than k
            vals = rng.integers(0, 50, n).astype(np.float64) if int_dists else \
                np.round(rng.standard_normal(n), 1)  # many ties
            pid = used[(p * nq + i) * k:(p * nq + i) * k + n]
            o = np.lexsort((pid, vals))
            ids[p, i, :n], d[p, i, :n] = pid[o], vals[o]
    return ids, d


@pytest.mark.parametrize("P,k,int_dists", [(1, 10, True), (3, 10, True), (5, 7, False), (32, 4, False)])
def test_merge_kernel_matches_oracle(P, k, int_dists):
    rng = np.random.default_rng(P * 10 + k)
    nq = 333
    ids, d = _sorted_lists(rng, P, nq, k, int_dists)
    ref_i, ref_d = oracle.merge_answers(list(ids), list(d), k)
    di = torch.from_numpy(ids).to(DEV)
    if int_dists:
        dd = torch.from_numpy(np.where(np.isinf(d), 2**31 - 1, d).astype(np.int32)).to(DEV)
    else:
        dd = torch.from_numpy(d.astype(np.float32)).to(DEV)
    oi = torch.empty((nq, k), dtype=torch.int32, device=DEV)
    od = torch.empty((nq, k), dtype=dd.dtype, device=DEV)
    shard.merge(di, dd, int_dists, oi, od)
    torch.cuda.synchronize()
    assert np.array_equal(oi.cpu().numpy(), ref_i)
    got = od.cpu().numpy().astype(np.float64)
    if int_dists:
        got[got == 2**31 - 1] = np.inf
    assert np.array_equal(got, ref_d.astype(np.float32).astype(np.float64))


def test_map_ids():
    rng = np.random.default_rng(5)
    m = rng.permutation(1000).astype(np.int32)
    loc = rng.integers(-1, 1000, 5000).astype(np.int32)
    loc[7] = 1000  # not a row of the map
    ids = torch.from_numpy(loc.copy()).to(DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    ann.ann_map_ids(ids, len(loc), torch.from_numpy(m).to(DEV), len(m), st)
    torch.cuda.synchronize()
    ref = np.where(loc >= 0, m[np.clip(loc, 0, 999)], -1)
    ref[7] = -1
    assert np.array_equal(ids.cpu().numpy(), ref)
    assert int(st.item()) == 1


def _shards(P, n=9000):
    w = synth.small_u8(n=n, nq=120)
    base = w["base"]
    lab = np.random.default_rng(11).integers(0, 40, n)  # stand-in hub clusters
    _, rows = shard.assign_shards(lab, 40, P)
    return w, rows


def _gpu_partitioned(w, rows, L, k):
    q = torch.from_numpy(w["queries"]).to(DEV)
    nq = q.shape[0]
    P = len(rows)
    all_i = torch.empty((P, nq, k), dtype=torch.int32, device=DEV)
    all_d = torch.empty((P, nq, k), dtype=torch.int32, device=DEV)
    shards = [shard.Shard(w["base"][r], r, ann.U8, ann.L2, K=32, R=16) for r in rows]
    try:
        p = ann.search_params(k, L)
        for s, sh in enumerate(shards):
            sh.search(q, nq, p, all_i[s], all_d[s])
            assert ann.ann_sync_status(sh.h) == ann.OK
        oi = torch.empty((nq, k), dtype=torch.int32, device=DEV)
        od = torch.empty((nq, k), dtype=torch.int32, device=DEV)
        shard.merge(all_i, all_d, True, oi, od)
        torch.cuda.synchronize()
        graphs = [(sh.graph.cpu().numpy(), sh.medoid) for sh in shards]
    finally:
        for sh in shards:
            sh.free()
    return oi.cpu().numpy(), od.cpu().numpy(), graphs


@pytest.mark.parametrize("P", [1, 3])
def test_partitioned_search_bit_exact(P):
    w, rows = _shards(P)
    k, L = 10, 48
    ids, d, graphs = _gpu_partitioned(w, rows, L, k)
    q = w["queries"].astype(np.float64)
    parts_i, parts_d = [], []
    for r, (g, med) in zip(rows, graphs):
        assert med == oracle.medoid(w["base"][r])
        li, ld, _, _ = oracle.search(w["base"][r], g, q, med, L, k)
        parts_i.append(np.where(li >= 0, r[np.maximum(li, 0)], -1))
        parts_d.append(ld)
    ref_i, ref_d = oracle.merge_answers(parts_i, parts_d, k)
    assert np.array_equal(ids, ref_i)
    assert np.array_equal(d, np.where(np.isinf(ref_d), 2**31 - 1, ref_d).astype(np.int32))
    # more shards searched apart: recall against the exact answer stays usable
    gt, _ = oracle.knn(w["base"], q, k)
    assert oracle.recall_at_k(ids, gt, k) > 0.3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch as t
    import torch.distributed as distd
    from paper_2506_15986_gb300 import ann as a, shard as sh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    distd.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t.cuda.set_device(0)  # both ranks share the one GPU
        a.load_library()
        w, rows = _shards(world)
        r = rows[rank]
        q = t.from_numpy(w["queries"]).to("cuda:0")
        nq, k = q.shape[0], 10
        s = sh.Shard(w["base"][r], r, a.U8, a.L2, K=32, R=16)
        try:
            ids = t.empty((nq, k), dtype=t.int32, device="cuda:0")
            d = t.empty((nq, k), dtype=t.int32, device="cuda:0")
            s.search(q, nq, a.search_params(k, 48), ids, d)
            t.cuda.synchronize()
            all_i, all_d = sh.exchange(ids, d)
            oi = t.empty_like(ids)
            od = t.empty_like(d)
            sh.merge(all_i, all_d, True, oi, od)
            t.cuda.synchronize()
            out[rank] = (oi.cpu().numpy(), od.cpu().numpy())
        finally:
            s.free()
    finally:
        distd.destroy_process_group()


def test_two_ranks_on_one_gpu_match_one_process():
    import torch.multiprocessing as mp
    w, rows = _shards(2)
    ids, d, _ = _gpu_partitioned(w, rows, 48, 10)
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        assert np.array_equal(res[rank][0], ids)
        assert np.array_equal(res[rank][1], d)
