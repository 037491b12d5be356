"""Thin Python binding of libann's C ABI (``include/ann.h``).

Argument marshalling only: every function here forwards to the entry point of
the same name in ``libann.so`` and raises ``AnnError`` on a non-OK status.
Device buffers are passed as ``torch.Tensor`` (CUDA) or raw integer pointers;
streams as ``torch.cuda.Stream`` or raw ``cudaStream_t`` integers.  There is no
fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libann.so")

# ann_status
OK, ERR_INVALID_ARG, ERR_IO, ERR_FORMAT, ERR_OOM, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_UNSUPPORTED = range(9)
# ann_dtype / ann_metric
U8, F32, F16, BF16, I8S = 0, 1, 2, 3, 4
L2, IP = 0, 1
SEARCH_RERANK, SEARCH_FAULT_WAIT, SEARCH_VISITED_L2, SEARCH_GROUP_ENTRIES = 1, 2, 4, 8
MAX_L, MAX_W, MAX_STEP_CAND, MAX_SEEDS, MAX_ENTRY_HUBS = 4096, 4, 128, 32, 8

_c = ctypes
_p = ctypes.c_void_p


class ann_index_desc(ctypes.Structure):
    _fields_ = [("n", _c.c_int64), ("dim", _c.c_int32), ("degree", _c.c_int32),
                ("dtype", _c.c_int32), ("metric", _c.c_int32), ("base", _p),
                ("graph", _p), ("medoid", _c.c_int32), ("base_f32", _p)]


class ann_search_params(ctypes.Structure):
    _fields_ = [("k", _c.c_int32), ("L", _c.c_int32), ("W", _c.c_int32),
                ("hash_bits", _c.c_int32), ("stage_rows", _c.c_int32), ("team", _c.c_int32),
                ("spill_bits", _c.c_int32), ("n_entries", _c.c_int32),
                ("flags", _c.c_uint32), ("gather", _c.c_int32), ("d_k", _p),
                ("d_L", _p), ("d_target", _p)]


class ann_entry_model_desc(ctypes.Structure):
    _fields_ = [("in_dim", _c.c_int32), ("hidden", _c.c_int32), ("out_dim", _c.c_int32),
                ("W1", _p), ("b1", _p), ("W2", _p), ("b2", _p), ("n_hubs", _c.c_int32),
                ("hub_nodes", _p), ("hub_emb", _p), ("hub_degree", _c.c_int32),
                ("hub_graph", _p), ("hub_entry", _c.c_int32)]


ENTRY_MEDOID, ENTRY_LEARNED_NAV, ENTRY_LEARNED_EXHAUSTIVE = 0, 1, 2


class AnnError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


_LIB = None


def load_library(path: str | None = None):
    """Load libann.so (built by ``_build.build()``); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"libann.so not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    i32, i64 = _c.c_int32, _c.c_int64
    pp = _c.POINTER(_p)
    sig = {
        "ann_status_string": ([i32], _c.c_char_p),
        "ann_index_create": ([_c.POINTER(ann_index_desc), i32, pp], i32),
        "ann_i8s_row_bytes": ([i32], i32),
        "ann_quantize_i8s": ([_p, i64, i32, _p, _p], i32),
        "ann_free_index": ([_p], i32),
        "ann_index_info": ([_p] + [_p] * 8, i32),
        "ann_save_index": ([_p, _c.c_char_p], i32),
        "ann_load_index": ([_c.c_char_p, i32, pp], i32),
        "ann_search_batch": ([_p, _p, i64, _p, _c.POINTER(ann_search_params), _p, _p, _p, _p], i32),
        "ann_sync_status": ([_p, _p], i32),
        "ann_knn": ([_p, i64, i32, i32, i32, _p, i64, i32, i32, _p, _p, _p], i32),
        "ann_medoid": ([_p, i64, i32, i32, _c.POINTER(i32), _p], i32),
        "ann_build_graph": ([_p, i64, i32, i32, i32, i32, _c.c_float, _p, _c.POINTER(i32),
                             _c.POINTER(i64), _p], i32),
        "ann_set_entry_model": ([_p, _c.POINTER(ann_entry_model_desc), _p], i32),
        "ann_get_entry_model": ([_p] + [_p] * 7 + [_c.POINTER(i32)], i32),
        "ann_select_entry": ([_p, _p, i64, i32, i32, _p, _p, _p], i32),
        "ann_set_hub_seeds": ([_p, _p, i32], i32),
        "ann_build_hub_graph": ([_p, i32, i32, _p], i32),
        "ann_select_entries": ([_p, _p, i64, i32, i32, i32, _p, _p, _p], i32),
        "ann_trainer_create": ([i32, i32, i32, _p, _p, _p, _p, _p, i64, _c.c_float, _c.c_float,
                                _c.c_float, _c.c_float, _c.c_float, pp], i32),
        "ann_trainer_free": ([_p], i32),
        "ann_trainer_step": ([_p, _p, _p, i64, _p, _p, i32, i32, _c.POINTER(_c.c_float), _p], i32),
        "ann_trainer_fit": ([_p, _p, i64, _p, _p, i32, _p, i32, _p, _p], i32),
        "ann_trainer_get": ([_p, _p, _p, _p, _p, _p, i32], i32),
        "ann_trainer_attach": ([_p, _p, _p, i32, _p], i32),
        "ann_adam_update": ([_p, _p, _p, _p, i64, i64, _c.c_float, _c.c_float, _c.c_float,
                             _c.c_float, _p], i32),
        "ann_kmeans": ([_p, i64, i32, i32, _p, i64, i32, _p, i32, _p, _p, _p], i32),
        "ann_assign_hubs": ([_p, i64, i32, i32, _p, i32, _p, _p, _p], i32),
        "ann_hbkm": ([_p, i64, i32, i32, i32, _c.c_double, i32, _p, _p, _p, _p, _p], i32),
        "ann_build_graph_insert": ([_p, i64, i32, i32, i32, i32, _c.c_float, i64, i64, _p, _c.POINTER(i32),
                                    _c.POINTER(i64), _p], i32),
        "ann_topo_tokens": ([_p, _p, i32, i32, i32, _p, _p, _p], i32),
        "ann_trainer_set_fusion": ([_p, _p, _p, i32, i32, i32, i32, _p, _p, _p, _p], i32),
        "ann_trainer_get_fusion": ([_p, _p, _p, _p, _p, i32], i32),
        "ann_hub_costs": ([_p, _p, i64, _p, _p, i32, _p, i32, i32, _p, _p, _p], i32),
        "ann_hub_labels": ([_p, _p, _p, i64, i32, i32, i32, _p, _p, _p], i32),
        "ann_map_ids": ([_p, i64, _p, i64, _p, _p], i32),
        "ann_release_l2": ([_p], i32),
        "ann_merge_shards": ([_p, _p, i32, i64, i32, i32, _p, _p, _p], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def status_string(s: int) -> str:
    return load_library().ann_status_string(int(s)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st, where):
    if st != OK:
        raise AnnError(st, where)


def ann_index_create(base, graph, medoid, dtype, metric=L2, device=0, base_f32=None,
                     n=None, dim=None, degree=None):
    """Create an index from host (numpy) or device (torch) arrays; returns a handle."""
    if n is None:
        n, dim = base.shape
        degree = graph.shape[1]
    d = ann_index_desc(n=int(n), dim=int(dim), degree=int(degree), dtype=int(dtype),
                       metric=int(metric), base=_ptr(base), graph=_ptr(graph),
                       medoid=int(medoid), base_f32=_ptr(base_f32))
    h = _p()
    _check(load_library().ann_index_create(ctypes.byref(d), int(device), ctypes.byref(h)),
           "ann_index_create")
    return h.value


def ann_i8s_row_bytes(dim):
    return int(load_library().ann_i8s_row_bytes(int(dim)))


def ann_quantize_i8s(x, n, dim, rows, stream=None):
    """Quantise n fp32 rows (device) into packed int8-with-scale rows (device)."""
    _check(load_library().ann_quantize_i8s(_ptr(x), int(n), int(dim), _ptr(rows), _stream(stream)),
           "ann_quantize_i8s")


def ann_free_index(h):
    _check(load_library().ann_free_index(h), "ann_free_index")


def ann_index_info(h):
    vals = [_c.c_int64()] + [_c.c_int32() for _ in range(7)]
    _check(load_library().ann_index_info(h, *[ctypes.byref(v) for v in vals]), "ann_index_info")
    keys = ["n", "dim", "degree", "dtype", "metric", "medoid", "n_hubs", "has_model"]
    return {k: v.value for k, v in zip(keys, vals)}


def ann_save_index(h, path):
    _check(load_library().ann_save_index(h, os.fsencode(path)), "ann_save_index")


def ann_load_index(path, device=0):
    h = _p()
    _check(load_library().ann_load_index(os.fsencode(path), int(device), ctypes.byref(h)),
           "ann_load_index")
    return h.value


def search_params(k, L, W=1, hash_bits=0, flags=0, d_k=None, d_L=None, d_target=None,
                  stage_rows=0, team=0, spill_bits=0, n_entries=0, gather=0):
    return ann_search_params(k=int(k), L=int(L), W=int(W), hash_bits=int(hash_bits),
                             stage_rows=int(stage_rows), team=int(team), spill_bits=int(spill_bits),
                             n_entries=int(n_entries), gather=int(gather),
                             flags=int(flags), d_k=_ptr(d_k), d_L=_ptr(d_L),
                             d_target=_ptr(d_target))


def ann_search_batch(h, queries, nq, entry, params, ids, dists, stats=None, stream=None):
    """Queue the batched beam search; outputs land in the caller's buffers."""
    _check(load_library().ann_search_batch(h, _ptr(queries), int(nq), _ptr(entry),
                                           ctypes.byref(params), _ptr(ids), _ptr(dists),
                                           _ptr(stats), _stream(stream)),
           "ann_search_batch")


def ann_sync_status(h, stream=None):
    """Synchronise the stream and return the device status (0 = OK)."""
    return int(load_library().ann_sync_status(h, _stream(stream)))


def ann_knn(base, n, dim, dtype, metric, queries, nq, k, ids, dists, exclude_self=False,
            stream=None):
    """Exact k-NN on the GPU (blocking); outputs in the caller's device buffers."""
    _check(load_library().ann_knn(_ptr(base), int(n), int(dim), int(dtype), int(metric),
                                  _ptr(queries), int(nq), int(k), int(bool(exclude_self)),
                                  _ptr(ids), _ptr(dists), _stream(stream)), "ann_knn")


def ann_medoid(base, n, dim, dtype, stream=None) -> int:
    m = _c.c_int32(-1)
    _check(load_library().ann_medoid(_ptr(base), int(n), int(dim), int(dtype), ctypes.byref(m),
                                     _stream(stream)), "ann_medoid")
    return m.value


def ann_build_graph_insert(base, n, dim, dtype, K, R, alpha, n_seed, batch, graph, medoid=-1, stream=None):
    """Build the graph by insertion by search (blocking).  Returns (medoid, repairs)."""
    m = _c.c_int32(int(medoid))
    rep = _c.c_int64(0)
    _check(load_library().ann_build_graph_insert(_ptr(base), int(n), int(dim), int(dtype), int(K), int(R),
                                                 float(alpha), int(n_seed), int(batch), _ptr(graph),
                                                 ctypes.byref(m), ctypes.byref(rep), _stream(stream)),
           "ann_build_graph_insert")
    return m.value, rep.value


def ann_build_graph(base, n, dim, dtype, K, R, alpha, graph, medoid=-1, stream=None):
    """Build the proximity graph on the GPU (blocking).  Returns (medoid, repairs)."""
    m = _c.c_int32(int(medoid))
    rep = _c.c_int64(0)
    _check(load_library().ann_build_graph(_ptr(base), int(n), int(dim), int(dtype), int(K),
                                          int(R), float(alpha), _ptr(graph), ctypes.byref(m),
                                          ctypes.byref(rep), _stream(stream)),
           "ann_build_graph")
    return m.value, rep.value


def ann_set_entry_model(h, in_dim, W1, b1, W2, b2, hub_nodes, hub_emb, hub_degree,
                        hub_graph=None, hub_entry=-1, stream=None):
    """Attach the two-tower entry model (arrays: numpy or torch, host or device)."""
    d = ann_entry_model_desc(in_dim=int(in_dim), hidden=256, out_dim=64, W1=_ptr(W1), b1=_ptr(b1),
                             W2=_ptr(W2), b2=_ptr(b2), n_hubs=int(len(hub_nodes)),
                             hub_nodes=_ptr(hub_nodes), hub_emb=_ptr(hub_emb),
                             hub_degree=int(hub_degree), hub_graph=_ptr(hub_graph),
                             hub_entry=int(hub_entry))
    _check(load_library().ann_set_entry_model(h, ctypes.byref(d), _stream(stream)),
           "ann_set_entry_model")


def ann_get_entry_model(h, W1=None, b1=None, W2=None, b2=None, hub_emb=None, hub_nodes=None,
                        hub_graph=None):
    """Copy the attached model into the given buffers; returns the entry hub."""
    e = _c.c_int32(-1)
    _check(load_library().ann_get_entry_model(h, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2),
                                              _ptr(hub_emb), _ptr(hub_nodes), _ptr(hub_graph),
                                              ctypes.byref(e)), "ann_get_entry_model")
    return e.value


def ann_build_hub_graph(h, s_nn, max_degree=0, stream=None):
    """Rebuild the model's hub graph: directed s_nn nearest (max_degree 0) or
    undirected, at most max_degree neighbours per hub."""
    _check(load_library().ann_build_hub_graph(h, int(s_nn), int(max_degree), _stream(stream)),
           "ann_build_hub_graph")


def ann_set_hub_seeds(h, seeds):
    """Hubs the hub-graph search starts from (int32 hub indices, host or
    device); None or an empty list goes back to the single entry hub."""
    n = 0 if seeds is None else int(len(seeds))
    if n and not hasattr(seeds, "data_ptr"):
        seeds = np.ascontiguousarray(seeds, np.int32)
    _check(load_library().ann_set_hub_seeds(h, _ptr(seeds) if n else None, n), "ann_set_hub_seeds")


def ann_select_entry(h, queries, nq, mode, L_hub, entry_out, qhat_out=None, stream=None):
    """Queue entry selection; node ids land in entry_out (device int32[nq])."""
    _check(load_library().ann_select_entry(h, _ptr(queries), int(nq), int(mode), int(L_hub),
                                           _ptr(entry_out), _ptr(qhat_out), _stream(stream)),
           "ann_select_entry")


def ann_select_entries(h, queries, nq, mode, L_hub, m_seeds, entry_out, qhat_out=None, stream=None):
    """Queue seed-set selection: the m_seeds best hubs' nodes per query land
    in entry_out (device int32[nq, m_seeds], -1 = unused slot)."""
    _check(load_library().ann_select_entries(h, _ptr(queries), int(nq), int(mode), int(L_hub),
                                             int(m_seeds), _ptr(entry_out), _ptr(qhat_out),
                                             _stream(stream)),
           "ann_select_entries")


def ann_trainer_create(in_dim, W1, b1, W2, b2, hub_emb, max_batch, tau=0.07, lr=5e-5,
                       beta1=0.9, beta2=0.999, eps=1e-8, device=0):
    h = _p()
    _check(load_library().ann_trainer_create(int(device), int(in_dim), int(len(hub_emb)),
                                             _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2), _ptr(hub_emb),
                                             int(max_batch), float(tau), float(lr), float(beta1),
                                             float(beta2), float(eps), ctypes.byref(h)),
           "ann_trainer_create")
    return h.value


def ann_trainer_free(t):
    _check(load_library().ann_trainer_free(t), "ann_trainer_free")


def ann_trainer_step(t, queries, rows, nb, cand, labels, M, apply_update=True, stream=None):
    """One step; returns the batch loss (blocking).  cand / labels: M listed
    hubs per query row and their labels (+1, -1, 0); unlisted hubs are
    negatives."""
    loss = _c.c_float(0.0)
    _check(load_library().ann_trainer_step(t, _ptr(queries), _ptr(rows), int(nb), _ptr(cand), _ptr(labels),
                                           int(M), int(bool(apply_update)), ctypes.byref(loss),
                                           _stream(stream)), "ann_trainer_step")
    return loss.value


def ann_trainer_fit(t, queries, nt, cand, labels, M, order, epochs, losses=None, stream=None):
    _check(load_library().ann_trainer_fit(t, _ptr(queries), int(nt), _ptr(cand), _ptr(labels), int(M),
                                          _ptr(order), int(epochs), _ptr(losses), _stream(stream)),
           "ann_trainer_fit")


def ann_trainer_get(t, W1=None, b1=None, W2=None, b2=None, hub_emb=None, gradients=False):
    _check(load_library().ann_trainer_get(t, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2),
                                          _ptr(hub_emb), int(bool(gradients))), "ann_trainer_get")


def ann_trainer_attach(t, h, hub_nodes, hub_degree, stream=None):
    _check(load_library().ann_trainer_attach(t, h, _ptr(hub_nodes), int(hub_degree),
                                             _stream(stream)), "ann_trainer_attach")


def ann_adam_update(params, grads, m, v, n, step, lr, beta1=0.9, beta2=0.999, eps=1e-8,
                    stream=None):
    _check(load_library().ann_adam_update(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(n),
                                          int(step), float(lr), float(beta1), float(beta2),
                                          float(eps), _stream(stream)), "ann_adam_update")


def ann_kmeans(x, n, dim, dtype, sample_rows, k, init, iters, centroids, stream=None):
    """Lloyd's k-means on the sample rows (host int64) from init (host int32);
    returns the objective per iteration."""
    import numpy as np
    sr = np.ascontiguousarray(sample_rows, np.int64)
    ini = np.ascontiguousarray(init, np.int32)
    obj = np.zeros(max(1, int(iters)), np.float64)
    _check(load_library().ann_kmeans(_ptr(x), int(n), int(dim), int(dtype), sr.ctypes.data,
                                     int(len(sr)), int(k), ini.ctypes.data, int(iters),
                                     _ptr(centroids), obj.ctypes.data, _stream(stream)),
           "ann_kmeans")
    return obj[:iters]


def ann_assign_hubs(base, n, dim, dtype, centroids, k, hubs, assign=None, stream=None):
    _check(load_library().ann_assign_hubs(_ptr(base), int(n), int(dim), int(dtype),
                                          _ptr(centroids), int(k), _ptr(hubs), _ptr(assign),
                                          _stream(stream)), "ann_assign_hubs")


def ann_hub_costs(h, queries, nq, targets, cand, M, hub_nodes, L, evals, hops, W=1, stream=None):
    _check(load_library().ann_hub_costs(h, _ptr(queries), int(nq), _ptr(targets), _ptr(cand),
                                        int(M), _ptr(hub_nodes), int(L), int(W), _ptr(evals),
                                        _ptr(hops), _stream(stream)), "ann_hub_costs")


def ann_hub_labels(evals, hops, cand, nq, M, t_pos, t_neg, labels, best=None, stream=None):
    """Label rule per query over its M searched hubs: labels (nq x M int8)
    aligned with cand; unlisted hubs count as negatives."""
    _check(load_library().ann_hub_labels(_ptr(evals), _ptr(hops), _ptr(cand), int(nq), int(M),
                                         int(t_pos), int(t_neg), _ptr(labels), _ptr(best), _stream(stream)),
           "ann_hub_labels")


def ann_release_l2(h):
    """Return persisting L2 lines of ANN_SEARCH_VISITED_L2 searches to normal (blocking)."""
    _check(load_library().ann_release_l2(h), "ann_release_l2")


def ann_map_ids(ids, count, id_map, n_map, status=None, stream=None):
    """Shard-local ids to global ids in place (device int32 arrays)."""
    _check(load_library().ann_map_ids(_ptr(ids), int(count), _ptr(id_map), int(n_map), _ptr(status),
                                      _stream(stream)), "ann_map_ids")


def ann_merge_shards(ids, dists, P, nq, k, int_dists, out_ids, out_dists, stream=None):
    """k best (distance, id) of P sorted answer lists per query (device)."""
    _check(load_library().ann_merge_shards(_ptr(ids), _ptr(dists), int(P), int(nq), int(k), int(bool(int_dists)),
                                           _ptr(out_ids), _ptr(out_dists), _stream(stream)), "ann_merge_shards")


def ann_select_entry_noalloc(h, queries, nq, entry_out, qhat_out=None, stream=None):
    """Exhaustive learned entry selection using the library's static scratch
    (no device allocation); see include/ann.h for its limits."""
    lib = load_library()
    lib.ann_select_entry_noalloc.argtypes = [_p, _p, _c.c_int64, _p, _p, _p]
    lib.ann_select_entry_noalloc.restype = _c.c_int32
    _check(lib.ann_select_entry_noalloc(h, _ptr(queries), int(nq), _ptr(entry_out),
                                        _ptr(qhat_out), _stream(stream)),
           "ann_select_entry_noalloc")


def ann_plan_create(h, queries, nq, entry_mode, L_hub, params, entry_buf, ids, dists, stats=None):
    """Capture entry selection + search for fixed buffers into a CUDA graph."""
    lib = load_library()
    lib.ann_plan_create.argtypes = [_p, _p, _c.c_int64, _c.c_int32, _c.c_int32,
                                    _c.POINTER(ann_search_params), _p, _p, _p, _p, _c.POINTER(_p)]
    lib.ann_plan_create.restype = _c.c_int32
    out = _p()
    _check(lib.ann_plan_create(h, _ptr(queries), int(nq), int(entry_mode), int(L_hub),
                               ctypes.byref(params), _ptr(entry_buf), _ptr(ids), _ptr(dists),
                               _ptr(stats), ctypes.byref(out)), "ann_plan_create")
    return out.value


def ann_plan_launch(plan, stream=None):
    lib = load_library()
    lib.ann_plan_launch.argtypes = [_p, _p]
    lib.ann_plan_launch.restype = _c.c_int32
    _check(lib.ann_plan_launch(plan, _stream(stream)), "ann_plan_launch")


def ann_plan_free(plan):
    lib = load_library()
    lib.ann_plan_free.argtypes = [_p]
    lib.ann_plan_free.restype = _c.c_int32
    _check(lib.ann_plan_free(plan), "ann_plan_free")


def ann_autotune(h, queries, nq, entry, params, ids, dists, reps=3, stream=None, lanes=1):
    """Returns (best ann_search_params, best ms per batch)."""
    lib = load_library()
    lib.ann_autotune.argtypes = [_p, _p, _c.c_int64, _p, _c.POINTER(ann_search_params), _p, _p,
                                 _c.c_int32, _c.c_int32, _c.POINTER(ann_search_params),
                                 _c.POINTER(_c.c_float), _p]
    lib.ann_autotune.restype = _c.c_int32
    best = ann_search_params()
    ms = _c.c_float(0.0)
    _check(lib.ann_autotune(h, _ptr(queries), int(nq), _ptr(entry), ctypes.byref(params),
                            _ptr(ids), _ptr(dists), int(reps), int(lanes), ctypes.byref(best),
                            ctypes.byref(ms), _stream(stream)), "ann_autotune")
    return best, ms.value


def ann_select_entry_noalloc_max_queries():
    lib = load_library()
    lib.ann_select_entry_noalloc_max_queries.argtypes = []
    lib.ann_select_entry_noalloc_max_queries.restype = _c.c_int64
    return int(lib.ann_select_entry_noalloc_max_queries())


def ann_hbkm(x, n, dim, k, levels, lam, T, keys, hubs_out, centroids_out=None, label_out=None, stream=None):
    """Hierarchical balanced k-means and its hubs (device buffers); blocking."""
    _check(load_library().ann_hbkm(_ptr(x), int(n), int(dim), int(k), int(levels), float(lam), int(T),
                                   _ptr(keys), _ptr(hubs_out), _ptr(centroids_out), _ptr(label_out),
                                   _stream(stream)), "ann_hbkm")


def ann_topo_tokens(h, hubs, H, hops, tokens_out, nodes_out=None, max_nodes=4096, stream=None):
    """Per-hop topology tokens of H hubs (device buffers); blocking."""
    _check(load_library().ann_topo_tokens(h, _ptr(hubs), int(H), int(hops), int(max_nodes), _ptr(tokens_out),
                                          _ptr(nodes_out), _stream(stream)), "ann_topo_tokens")


def ann_trainer_set_fusion(t, hub_vecs, tokens, T, token_dim, heads, head_dim, WQ, WK, WV, WO):
    """Give the trainer the topology-aware hub tower (weights: numpy or device)."""
    import numpy as np
    keep = [np.ascontiguousarray(w, np.float32) if isinstance(w, np.ndarray) else w for w in (WQ, WK, WV, WO)]
    _check(load_library().ann_trainer_set_fusion(t, _ptr(hub_vecs), _ptr(tokens), int(T), int(token_dim),
                                                 int(heads), int(head_dim), *[_ptr(w) for w in keep]),
           "ann_trainer_set_fusion")


def ann_trainer_get_fusion(t, WQ=None, WK=None, WV=None, WO=None, gradients=False):
    _check(load_library().ann_trainer_get_fusion(t, _ptr(WQ), _ptr(WK), _ptr(WV), _ptr(WO), int(bool(gradients))),
           "ann_trainer_get_fusion")
