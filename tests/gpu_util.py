"""Helpers for the GPU parity tests: run libann through its C ABI on cuda:0."""
import numpy as np
import torch

from paper_2506_15986_gb300 import ann

DEV = torch.device("cuda:0")


def make_index(base, graph, medoid, metric=ann.L2, base_f32=None):
    dt = {np.dtype(np.uint8): ann.U8, np.dtype(np.float32): ann.F32,
          np.dtype(np.float16): ann.F16}[np.asarray(base).dtype]
    return ann.ann_index_create(np.ascontiguousarray(base), np.ascontiguousarray(graph, np.int32),
                                int(medoid), dt, metric, device=0,
                                base_f32=None if base_f32 is None else np.ascontiguousarray(base_f32))


def search(h, queries, k, L, W=1, entries=None, hash_bits=0, ks=None, Ls=None, targets=None,
           u8=None, team=0, stage_rows=0, spill_bits=0, flags=0, gather=0):
    q = torch.from_numpy(np.ascontiguousarray(queries)).to(DEV)
    nq = q.shape[0]
    if u8 is None:
        u8 = q.dtype == torch.uint8
    ids = torch.full((nq, k), -7, dtype=torch.int32, device=DEV)
    dists = torch.full((nq, k), -7, dtype=torch.int32 if u8 else torch.float32, device=DEV)
    stats = torch.full((nq, 2), -7, dtype=torch.int32, device=DEV)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.int32)).to(DEV)
    ent, dk, dL, dt = t(entries), t(ks), t(Ls), t(targets)
    m = 0 if entries is None or np.ndim(entries) == 1 else np.shape(entries)[1]
    p = ann.search_params(k, L, W=W, hash_bits=hash_bits, d_k=dk, d_L=dL, d_target=dt, team=team,
                          stage_rows=stage_rows, spill_bits=spill_bits, flags=flags, n_entries=m, gather=gather)
    ann.ann_search_batch(h, q, nq, ent, p, ids, dists, stats)
    st = ann.ann_sync_status(h)
    return ids.cpu().numpy(), dists.cpu().numpy(), stats[:, 0].cpu().numpy(), \
        stats[:, 1].cpu().numpy(), st


def dense_as_listed(mask):
    """A dense nq x H label matrix (numpy int8) in the trainer's listed form:
    every hub listed for every query.  Returns (cand, labels, M) on cuda:0."""
    nq, H = mask.shape
    cand = torch.arange(H, dtype=torch.int32, device=DEV).repeat(nq, 1).contiguous()
    return cand, torch.from_numpy(np.ascontiguousarray(mask, np.int8)).to(DEV), H
