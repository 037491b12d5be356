"""Base-partitioned search on the CPU: the shard assignment (whole hub
clusters, balanced rows), the oracle of the merged answer, and the exchange of
answers between two gloo ranks.

Pins of oracle.merge_answers: a hand case with a distance tie and padding,
and the special case that merging each shard's exact k nearest neighbours
gives the exact k nearest neighbours of the whole base set (Sec. 2.1,
Problem 1: the exact answer of a union is the best of the parts' exact
answers)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2506_15986_gb300 import shard, synth  # noqa: E402

torch = pytest.importorskip("torch")
import torch.distributed as distd  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def test_assign_shards_hand_case():
    # cluster sizes 5, 3, 3, 2, 1 (clusters 0..4); P = 2: cluster 0 -> shard 0
    # (5), 1 -> shard 1 (3), 2 -> shard 1 (6), 3 -> shard 0 (7), 4 -> shard 1 (7)
    lab = np.array([0] * 5 + [1] * 3 + [2] * 3 + [3] * 2 + [4])
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(lab))
    shard_of, rows = shard.assign_shards(lab[perm], 5, 2)
    assert shard_of.tolist() == [0, 1, 1, 0, 1]
    assert sorted(np.concatenate(rows).tolist()) == list(range(len(lab)))
    for s in (0, 1):
        assert (shard_of[lab[perm][rows[s]]] == s).all()
        assert (np.diff(rows[s]) > 0).all()
    assert [len(r) for r in rows] == [7, 7]


def test_assign_shards_properties():
    rng = np.random.default_rng(1)
    lab = rng.integers(0, 300, 20_000)
    for P in (1, 2, 3, 8):
        shard_of, rows = shard.assign_shards(lab, 300, P)
        assert sum(len(r) for r in rows) == len(lab)
        assert len(np.unique(np.concatenate(rows))) == len(lab)
        sizes = np.bincount(lab, minlength=300)
        loads = [len(r) for r in rows]
        # greedy largest-first: loads differ by at most the largest cluster
        assert max(loads) - min(loads) <= sizes.max()
        again, _ = shard.assign_shards(lab, 300, P)
        assert np.array_equal(shard_of, again)
    with pytest.raises(ValueError):
        shard.assign_shards(lab, 100, 2)  # labels beyond the cluster count


def test_merge_answers_hand_case():
    a_ids = np.array([[3, 9, -1], [1, 2, 4]])
    a_d = np.array([[0.5, 2.0, np.inf], [1.0, 1.0, 3.0]])
    b_ids = np.array([[7, 8, -1], [5, 6, -1]])
    b_d = np.array([[0.5, 1.0, np.inf], [0.5, 1.0, np.inf]])
    ids, d = oracle.merge_answers([a_ids, b_ids], [a_d, b_d], 4)
    # query 0: (0.5, 3) before (0.5, 7) (tie: smaller id), then 8, then 9
    assert ids[0].tolist() == [3, 7, 8, 9]
    assert d[0].tolist() == [0.5, 0.5, 1.0, 2.0]
    # query 1: 5 (0.5), then the three at 1.0 by id: 1, 2, 6
    assert ids[1].tolist() == [5, 1, 2, 6]
    ids, d = oracle.merge_answers([a_ids[:, :1], b_ids[:, :1]], [a_d[:, :1], b_d[:, :1]], 3)
    assert ids[0].tolist() == [3, 7, -1] and np.isinf(d[0, 2])


def test_merged_exact_shard_answers_are_the_exact_answer():
    w = synth.small_u8(n=3000, nq=40)
    base, q = w["base"], w["queries"].astype(np.float64)
    rng = np.random.default_rng(2)
    lab = rng.integers(0, 12, len(base))
    _, rows = shard.assign_shards(lab, 12, 3)
    k = 10
    parts_i, parts_d = [], []
    for r in rows:
        li, ld = oracle.knn(base[r], q, k)
        parts_i.append(np.where(li >= 0, r[np.maximum(li, 0)], -1))
        parts_d.append(ld)
    ids, d = oracle.merge_answers(parts_i, parts_d, k)
    ref_i, ref_d = oracle.knn(base, q, k)
    assert np.array_equal(ids, ref_i)
    assert np.array_equal(d, ref_d)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    distd.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.small_u8(n=2400, nq=30)
        base, q = w["base"], w["queries"].astype(np.float64)
        lab = np.random.default_rng(3).integers(0, 10, len(base))
        _, rows = shard.assign_shards(lab, 10, world)
        r = rows[rank]
        # this rank's shard: its own graph, searched by the oracle from its medoid
        g, _ = oracle.build_graph(base[r], K=24, R=12)
        li, ld, _, _ = oracle.search(base[r], g, q, oracle.medoid(base[r]), 40, 10)
        gi = torch.from_numpy(np.where(li >= 0, r[np.maximum(li, 0)], -1).astype(np.int32))
        gd = torch.from_numpy(ld.astype(np.float32))
        all_i, all_d = shard.exchange(gi, gd)
        out[rank] = (all_i.numpy(), all_d.numpy())
    finally:
        distd.destroy_process_group()


def test_two_gloo_ranks_exchange_their_shards_answers():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    # both ranks hold every shard's answers, in rank order
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    all_i, all_d = res[0]
    assert all_i.shape == (2, 30, 10)
    w = synth.small_u8(n=2400, nq=30)
    base, q = w["base"], w["queries"].astype(np.float64)
    lab = np.random.default_rng(3).integers(0, 10, len(base))
    _, rows = shard.assign_shards(lab, 10, 2)
    for s in (0, 1):
        assert np.isin(all_i[s][all_i[s] >= 0], rows[s]).all()  # shard s's rows only
    ids, d = oracle.merge_answers(list(all_i), list(all_d.astype(np.float64)), 10)
    # every merged answer is a true distance to a row of the base set
    ok = ids >= 0
    x = base.astype(np.float64)
    for i in range(len(q)):
        di = ((x[ids[i][ok[i]]] - q[i]) ** 2).sum(1)
        assert np.allclose(di, d[i][ok[i]])
    assert (np.diff(d, axis=1) >= 0).all()
