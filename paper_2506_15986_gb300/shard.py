"""Base-partitioned search: the base set split into shards of whole hub
clusters (Sec. 4.1, Def. 3), each shard with its own graph searched apart, and
a query's answer merged from the shards' answers under the (distance, id)
order of Sec. 2.1, Problem 1.

This module is host-side plumbing around libann: which clusters form which
shard, the shard's rows and index, and the exchange of answers between ranks
over torch.distributed.  Every step on the data runs in libann's kernels:
ann_build_graph (the shard's graph), ann_search_batch (the shard's search),
ann_map_ids (shard-local ids to global ids) and ann_merge_shards (the merge).
One rank holds one shard; the exchange is one all-gather of k (id, distance)
pairs per query per shard, the only collective of the path.
"""
from __future__ import annotations

import numpy as np

from . import ann


def assign_shards(cluster_of_row, n_clusters, P):
    """Shards of whole clusters with balanced row counts: clusters in order of
    decreasing size (ties: smaller cluster index) each go to the shard with the
    fewest rows so far (ties: smaller shard index).  Returns (shard of each
    cluster [n_clusters], rows of each shard: P sorted int32 arrays)."""
    lab = np.asarray(cluster_of_row, np.int64)
    if P < 1 or n_clusters < 1 or (lab.size and (lab.min() < 0 or lab.max() >= n_clusters)):
        raise ValueError("bad shard count or cluster labels")
    size = np.bincount(lab, minlength=n_clusters)
    order = sorted(range(n_clusters), key=lambda c: (-size[c], c))
    load = [0] * P
    shard_of = np.empty(n_clusters, np.int32)
    for c in order:
        s = min(range(P), key=lambda p: (load[p], p))
        shard_of[c] = s
        load[s] += int(size[c])
    row_shard = shard_of[lab]
    rows = [np.flatnonzero(row_shard == s).astype(np.int32) for s in range(P)]
    return shard_of, rows


class Shard:
    """One shard's index on one device: its rows (global ids, sorted), the
    graph built over them, their medoid, and the device map local -> global."""

    def __init__(self, base_rows, rows, dtype, metric, K=64, R=32, alpha=1.0, device=0):
        import torch
        self.dev = torch.device("cuda", device)
        self.rows = np.asarray(rows, np.int32)
        n = len(self.rows)
        if n < 2:
            raise ValueError("a shard needs at least two rows")
        x = base_rows if isinstance(base_rows, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(base_rows))
        self.base = x.to(self.dev).contiguous()
        self.dim = self.base.shape[1]
        self.graph = torch.empty((n, R), dtype=torch.int32, device=self.dev)
        self.medoid, self.repairs = ann.ann_build_graph(self.base, n, self.dim, dtype, min(K, n - 1), R, alpha,
                                                        self.graph)
        self.h = ann.ann_index_create(self.base, self.graph, self.medoid, dtype, metric, device=device)
        self.id_map = torch.from_numpy(self.rows).to(self.dev)
        self.int_dists = dtype == ann.U8

    def search(self, queries, nq, params, ids, dists, stream=None):
        """The shard's answers with global ids (asynchronous on stream)."""
        ann.ann_search_batch(self.h, queries, nq, None, params, ids, dists, None, stream)
        ann.ann_map_ids(ids, nq * params.k, self.id_map, len(self.rows), None, stream)

    def free(self):
        if self.h:
            ann.ann_free_index(self.h)
            self.h = None


def exchange(ids, dists, group=None):
    """All-gather of every rank's answers (nq x k ids and distances): returns
    [P, nq, k] tensors in rank order, on the device of the inputs.  With the
    gloo backend the answers travel through host memory; with NCCL they stay
    on the device."""
    import torch
    import torch.distributed as dist
    P = dist.get_world_size(group)
    dev = ids.device
    host = dist.get_backend(group) == "gloo" and dev.type != "cpu"
    src_i, src_d = (ids.cpu(), dists.cpu()) if host else (ids, dists)
    gi = [torch.empty_like(src_i) for _ in range(P)]
    gd = [torch.empty_like(src_d) for _ in range(P)]
    dist.all_gather(gi, src_i.contiguous(), group=group)
    dist.all_gather(gd, src_d.contiguous(), group=group)
    all_i, all_d = torch.stack(gi), torch.stack(gd)
    if host:
        all_i, all_d = all_i.to(dev), all_d.to(dev)
    return all_i, all_d


def merge(all_ids, all_dists, int_dists, out_ids, out_dists, stream=None):
    """k best (distance, id) per query of the P shards' answers (device)."""
    P, nq, k = all_ids.shape
    ann.ann_merge_shards(all_ids.contiguous(), all_dists.contiguous(), P, nq, k, int_dists, out_ids, out_dists,
                         stream)
