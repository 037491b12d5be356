#!/usr/bin/env python3
"""Benchmark: QPS at recall@10 = 0.95 on one GB300, learned vs medoid entry,
with distance evaluations per query (shifted-query 1M x 128 fp32 workload).

Setup (untimed, all on the GPU through libann): the synthetic workload, the
proximity graph (exact 64-NN + RNG pruning, R = 32), exact ground truth, 1,024
k-means hubs, label-mode search costs for 100,000 training queries, the label
rule (t_pos = 3, t_neg = 15) and the contrastive training of the two-tower
entry model (Adam, batch 8,192).

One step = one batch of the 10,000 evaluation queries through the public
path: ann_select_entry (query tower, then the hub-graph search or the
exhaustive tensor-core hub scoring, whichever is faster) then ann_search_batch
(W = 2 pool entries expanded per step, visited-table and gather sizes picked by
ann_autotune), at the pool size L* that first reaches recall@10 >= 0.95 in the
L sweep.  `value` is the learned-entry QPS; the medoid-entry numbers (same W,
own L* and tuning) sit beside it in `config`.  Inputs are resident in HBM when the timed region
starts; the base set (512 MB) is larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the CPU oracle's search (this project's reference arm)
on a bounded sample of the same workload on the host cores.  Multi-GPU runs
(torchrun, N > 1) are query-parallel replicas: every rank builds the same
index and searches its own copy of the batch, with no collective on the data
path (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QPS at recall@10=0.95 on 1 GB300, learned vs medoid entry; dist evals/query"
WORKLOAD = ("shift_f32: N=1,000,000 fp32 d=128 base (1,000-component anisotropic Gaussian "
            "mixture, variance spectrum (1+i)^-1), 10,000 shifted/reweighted queries, graph "
            "exact 64-NN + RNG prune (alpha=1) R=32 with reachability repair, k=10, 1,024 "
            "k-means hubs, BF16 query tower 128-256-64 trained on 100,000 labelled queries")
L_SWEEP = [16, 24, 32, 48, 64, 96, 128, 160, 192, 256, 320, 384, 512]
TARGET = 0.95
K_NN = 10
DIM, DEGREE = 128, 32


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000, help="base size")
    ap.add_argument("--nq", type=int, default=10_000)
    ap.add_argument("--n-train", type=int, default=100_000)
    ap.add_argument("--hubs", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--lr", type=float, default=5e-5)
    ap.add_argument("--tau", type=float, default=0.07)
    ap.add_argument("--cand", type=int, default=64, help="hubs searched per training query")
    ap.add_argument("--l-hub", type=int, default=32)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--W", type=int, default=2, help="pool entries expanded per search step")
    ap.add_argument("--no-tune", action="store_true", help="skip ann_autotune at L*")
    ap.add_argument("--fixed-L", type=int, default=0,
                    help="skip the L sweep and run every entry mode at this pool size")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recall(ids, gt):
    hits = 0
    for a, b in zip(ids, gt):
        hits += len(np.intersect1d(a[a >= 0], b))
    return hits / gt.size


def build_workload(args, torch, ann, synth, dev, n_train):
    t0 = time.time()
    w = synth.shift_f32(n=args.n, nq=args.nq, n_train=n_train)
    t_gen = time.time() - t0
    base = torch.from_numpy(w["base"]).to(dev)
    graph = torch.empty((args.n, DEGREE), dtype=torch.int32, device=dev)
    t0 = time.time()
    med, rep = ann.ann_build_graph(base, args.n, DIM, ann.F32, 64, DEGREE, 1.0, graph)
    t_build = time.time() - t0
    q = torch.from_numpy(w["queries"]).to(dev)
    gt = torch.empty((args.nq, K_NN), dtype=torch.int32, device=dev)
    gtd = torch.empty((args.nq, K_NN), dtype=torch.float32, device=dev)
    ann.ann_knn(base, args.n, DIM, ann.F32, ann.L2, q, args.nq, K_NN, gt, gtd)
    h = ann.ann_index_create(base, graph, med, ann.F32, ann.L2, device=dev.index or 0)
    return dict(w=w, base=base, graph=graph, medoid=med, repairs=rep, q=q, gt=gt.cpu().numpy(),
                h=h, t_build=t_build, t_gen=t_gen)


def build_learned(W, args, torch, ann, synth, dev):
    """Hubs, labels and training of the entry model, all through libann."""
    n, H0, M = args.n, args.hubs, args.cand
    times = {}
    t0 = time.time()
    sample = synth.sample_rows(n, min(n, 262_144), seed=synth.SEED_BASE + 10)
    init = synth.kmeans_init(len(sample), H0, seed=synth.SEED_BASE + 11)
    cent = torch.empty((H0, DIM), dtype=torch.float32, device=dev)
    obj = ann.ann_kmeans(W["base"], n, DIM, ann.F32, sample, H0, init, 25, cent)
    hubs = torch.empty(H0, dtype=torch.int32, device=dev)
    ann.ann_assign_hubs(W["base"], n, DIM, ann.F32, cent, H0, hubs)
    hub_np = hubs.cpu().numpy()
    hub_np = hub_np[hub_np >= 0]
    H = len(hub_np)
    hub_nodes = torch.from_numpy(hub_np).to(dev)
    hub_vecs = torch.from_numpy(W["w"]["base"][hub_np]).to(dev)
    times["hubs_s"] = time.time() - t0

    t0 = time.time()
    tq = torch.from_numpy(W["w"]["train"]).to(dev)
    nt = tq.shape[0]
    cand = torch.empty((nt, M), dtype=torch.int32, device=dev)
    cd = torch.empty((nt, M), dtype=torch.float32, device=dev)
    ann.ann_knn(hub_vecs, H, DIM, ann.F32, ann.L2, tq, nt, M, cand, cd)
    tgt = torch.empty((nt, 1), dtype=torch.int32, device=dev)
    td = torch.empty((nt, 1), dtype=torch.float32, device=dev)
    ann.ann_knn(W["base"], n, DIM, ann.F32, ann.L2, tq, nt, 1, tgt, td)
    ev = torch.empty((nt, M), dtype=torch.int32, device=dev)
    hp = torch.empty_like(ev)
    ann.ann_hub_costs(W["h"], tq, nt, tgt, cand, M, hub_nodes, 64, ev, hp)
    mask = torch.empty((nt, H), dtype=torch.int8, device=dev)
    best = torch.empty(nt, dtype=torch.int32, device=dev)
    ann.ann_hub_labels(ev, hp, cand, nt, M, H, 3, 15, mask, best)
    if ann.ann_sync_status(W["h"]) != ann.OK:
        raise RuntimeError("label search reported a device error")
    m = mask.cpu().numpy()
    reached = (hp.cpu().numpy() < 2**31 - 1).mean()
    times["labels_s"] = time.time() - t0

    t0 = time.time()
    W1, b1, W2, b2, E = synth.model_init(DIM, H)
    # hub tower starts at the query tower applied to each hub's own vector
    ann.ann_set_entry_model(W["h"], DIM, W1, b1, W2, b2, hub_np, E, 16)
    E0 = torch.empty((H, 64), dtype=torch.float32, device=dev)
    tmp = torch.empty(H, dtype=torch.int32, device=dev)
    ann.ann_select_entry(W["h"], hub_vecs, H, ann.ENTRY_LEARNED_EXHAUSTIVE, args.l_hub, tmp, E0)
    batch = 8192
    t = ann.ann_trainer_create(DIM, W1, b1, W2, b2, E0, batch, tau=args.tau, lr=args.lr)
    order = torch.from_numpy(np.concatenate(
        synth.train_batches(nt, batch, args.epochs, seed=synth.SEED_BASE + 12))).to(dev)
    spe = (nt + batch - 1) // batch
    losses = torch.zeros(max(1, args.epochs * spe), device=dev)
    ann.ann_trainer_fit(t, tq, nt, mask, order, args.epochs, losses)
    ann.ann_trainer_attach(t, W["h"], hub_nodes, 16)
    ann.ann_trainer_free(t)
    ls = losses.cpu().numpy()
    times["train_s"] = time.time() - t0
    return dict(H=H, kmeans_obj=[float(obj[0]), float(obj[-1])], label_reached=float(reached),
                positives_per_query=float((m > 0).sum(1).mean()),
                negatives_per_query=float((m < 0).sum(1).mean()),
                loss_first=float(ls[:spe].mean()), loss_last=float(ls[-spe:].mean()),
                epochs=args.epochs, lr=args.lr, tau=args.tau, batch=batch, times=times)


class Runner:
    """One step = entry selection (learned modes) + batched search."""

    def __init__(self, W, torch, ann, args, mode):
        self.W, self.torch, self.ann, self.mode, self.args = W, torch, ann, mode, args
        dev = W["q"].device
        nq = W["q"].shape[0]
        self.nq = nq
        self.stream = torch.cuda.current_stream()
        self.ids = torch.empty((nq, K_NN), dtype=torch.int32, device=dev)
        self.dists = torch.empty((nq, K_NN), dtype=torch.float32, device=dev)
        self.stats = torch.empty((nq, 2), dtype=torch.int32, device=dev)
        self.entry = torch.empty(nq, dtype=torch.int32, device=dev)
        self.tuned = {}  # L -> ann_search_params picked by ann_autotune

    def params(self, L):
        return self.tuned.get(L) or self.ann.search_params(K_NN, L, W=self.args.W)

    def autotune(self, L):
        """Pick the visited-table size and gather round size (speed-only knobs)."""
        q = self.W["q"]
        e = self.select(q)
        best, ms = self.ann.ann_autotune(self.W["h"], q, self.nq, e, self.params(L), self.ids,
                                         self.dists, 3, self.stream)
        self.tuned[L] = best
        return {"hash_bits": best.hash_bits, "stage_rows": best.stage_rows, "search_ms": ms}

    def select(self, q):
        if self.mode == "medoid":
            return None
        m = self.ann.ENTRY_LEARNED_NAV if self.mode == "learned" else self.ann.ENTRY_LEARNED_EXHAUSTIVE
        self.ann.ann_select_entry(self.W["h"], q, self.nq, m, self.args.l_hub, self.entry, None,
                                  self.stream)
        return self.entry

    def search(self, q, entry, L, stats=False):
        self.ann.ann_search_batch(self.W["h"], q, self.nq, entry, self.params(L),
                                  self.ids, self.dists, self.stats if stats else None, self.stream)

    def step(self, L, q=None, stats=False):
        q = self.W["q"] if q is None else q
        self.search(q, self.select(q), L, stats)

    def launches(self):
        return {"medoid": 1, "learned": 4, "exhaustive": 3}[self.mode]


def sweep(run, torch, ann, W):
    """recall@10, evals, QPS per L; L* = the smallest swept L with recall@10 >=
    0.95; QPS at exactly 0.95 interpolated between the bracketing L."""
    out = []
    for L in L_SWEEP:
        run.step(L, stats=True)
        if ann.ann_sync_status(W["h"], run.stream) != ann.OK:
            raise RuntimeError("search reported a device error")
        r = recall(run.ids.cpu().numpy(), W["gt"])
        s = run.stats.cpu().numpy()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(run.stream)
        for _ in range(5):
            run.step(L)
        e1.record(run.stream)
        torch.cuda.synchronize()
        out.append(dict(L=L, recall=r, evals=float(s[:, 0].mean()), hops=float(s[:, 1].mean()),
                        qps=run.nq * 5 / (e0.elapsed_time(e1) / 1e3)))
        if len([x for x in out if x["recall"] >= TARGET]) >= 2:
            break
    hit = [x for x in out if x["recall"] >= TARGET]
    Lstar = hit[0]["L"] if hit else out[-1]["L"]
    interp = None
    if out[0]["recall"] >= TARGET:
        interp = out[0]["qps"]
    for a, b in zip(out, out[1:]):
        if a["recall"] < TARGET <= b["recall"]:
            t = (TARGET - a["recall"]) / (b["recall"] - a["recall"])
            interp = a["qps"] + t * (b["qps"] - a["qps"])
    return Lstar, out, interp


def timed(run, torch, ann, args, L, world, dev):
    """The timed region: W warm-up steps, then K steps bracketed by a barrier
    and a device synchronize; per-launch events around the search kernel."""
    for _ in range(args.warmup):
        run.step(L)
    if world > 1:
        import torch.distributed as distd
        distd.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    q = run.W["q"]
    with Clocks(dev.index or 0) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(run.stream)
        for i in range(args.steps):
            e = run.select(q)
            ev[2 * i].record(run.stream)
            run.search(q, e, L)
            ev[2 * i + 1].record(run.stream)
        t1.record(run.stream)
        torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as distd
        distd.barrier()
    total_ms = t0.elapsed_time(t1)
    search_ms = float(np.mean([ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)]))
    if world > 1:
        import torch.distributed as distd
        tt = torch.tensor([total_ms], device=dev)
        distd.all_reduce(tt, op=distd.ReduceOp.MAX)
        total_ms = float(tt.item())
    return total_ms, search_ms, clk.summary()


def end_to_end(run, torch, L, steps):
    """Same metric through the public calls with host buffers: pinned H2D of the
    queries, entry selection + search, D2H of ids and distances, every step."""
    W = run.W
    qh = torch.from_numpy(W["w"]["queries"]).pin_memory()
    ih = torch.empty((run.nq, K_NN), dtype=torch.int32).pin_memory()
    dh = torch.empty((run.nq, K_NN), dtype=torch.float32).pin_memory()
    qd = torch.empty_like(W["q"])
    for i in range(steps + 3):
        if i == 3:
            torch.cuda.synchronize()
            a0 = time.perf_counter()
        qd.copy_(qh, non_blocking=True)
        run.step(L, q=qd)
        ih.copy_(run.ids, non_blocking=True)
        dh.copy_(run.dists, non_blocking=True)
        run.stream.synchronize()
    dt = time.perf_counter() - a0
    return {"value": run.nq * steps / dt, "unit": "queries/s",
            "h2d_bytes_per_step": int(qh.numel() * 4),
            "d2h_bytes_per_step": int(ih.numel() * 4 + dh.numel() * 4)}


def cpu_baseline(W, L, entries=None, target_s=10.0, width=1):
    """The oracle's search on the host cores on a bounded sample of the
    evaluation queries sized to take about target_s seconds."""
    import oracle
    base = W["w"]["base"]
    g = W["graph"].cpu().numpy()
    allq = W["w"]["queries"].astype(np.float64)
    oracle.build()
    ent = np.full(len(allq), W["medoid"], np.int32) if entries is None else entries
    probe = min(len(allq), 4 * oracle.num_threads())
    t = time.perf_counter()
    oracle.search(base, g, allq[:probe], ent[:probe], L, K_NN, W=width)
    per_q = (time.perf_counter() - t) / probe
    m = int(min(len(allq), max(probe, target_s / max(per_q, 1e-9))))
    t = time.perf_counter()
    ids, _, ev, _ = oracle.search(base, g, allq[:m], ent[:m], L, K_NN, W=width)
    dt = time.perf_counter() - t
    return {"value": m / dt, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {m} of the {len(allq)} evaluation queries at L={L}, W={width}, "
                      f"entries as the GPU arm, float64 distances, one query per OpenMP thread "
                      f"({dt:.1f} s)",
            "recall@10_sample": recall(ids, W["gt"][:m]), "evals_per_query": float(ev.mean())}


def run_gpu(args):
    import torch
    from paper_2506_15986_gb300 import _build, ann, synth

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as distd
        distd.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    ann.load_library()
    W = build_workload(args, torch, ann, synth, dev, 0 if args.no_learned else args.n_train)
    learned = None if args.no_learned else build_learned(W, args, torch, ann, synth, dev)

    res = {}
    for mode in (["medoid"] if args.no_learned else ["medoid", "learned", "exhaustive"]):
        run = Runner(W, torch, ann, args, mode)
        if args.fixed_L:
            Lstar, sw, interp = args.fixed_L, [], None
        else:
            Lstar, sw, interp = sweep(run, torch, ann, W)
        tune = None if args.no_tune else run.autotune(Lstar)
        run.step(Lstar, stats=True)
        torch.cuda.synchronize()
        s = run.stats.cpu().numpy().astype(np.int64)
        res[mode] = dict(L=Lstar, sweep=sw, qps_interp=interp, run=run,
                         recall=recall(run.ids.cpu().numpy(), W["gt"]),
                         evals=float(s[:, 0].mean()), hops=float(s[:, 1].mean()),
                         alg_bytes=int((s[:, 0] * DIM * 4 + s[:, 1] * DEGREE * 4).sum() + run.nq * DIM * 4),
                         entries=None if mode == "medoid" else run.entry.cpu().numpy(), tune=tune)
    # a short timing of every mode picks the headline: the faster learned mode
    # (hub-graph search or exhaustive tensor-core hub scoring), medoid without
    # a model; then the headline is timed under the full protocol
    probe = {}
    for mode, r in res.items():
        tm, _, _ = timed(r["run"], torch, ann, argparse.Namespace(warmup=2, steps=20), r["L"], 1, dev)
        probe[mode] = r["run"].nq * 20 / (tm / 1e3)
    learned_modes = [m for m in res if m != "medoid"]
    head = max(learned_modes, key=lambda m: probe[m]) if learned_modes else "medoid"
    R = res[head]
    total_ms, search_ms, clocks = timed(R["run"], torch, ann, args, R["L"], world, dev)
    value = world * R["run"].nq * args.steps / (total_ms / 1e3)
    others = {}
    for mode, r in res.items():
        if mode != head:
            tm, sm, _ = timed(r["run"], torch, ann, args, r["L"], 1, dev)
            others[mode] = dict(qps=r["run"].nq * args.steps / (tm / 1e3), L=r["L"],
                                recall=r["recall"], evals_per_query=r["evals"],
                                hops_per_query=r["hops"], qps_interpolated_at_0_95=r["qps_interp"],
                                search_ms=sm, tuned=r["tune"], sweep=r["sweep"])
    e2e = end_to_end(R["run"], torch, R["L"], max(10, args.steps // 4))
    e2e["value"] *= world
    peak, peak_kind = peaks()
    achieved = R["alg_bytes"] / (search_ms / 1e3) / 1e9
    out = None
    if rank == 0:
        cpu = None if args.no_cpu else cpu_baseline(W, R["L"], R["entries"], width=args.W)
        cfg = {"workload": WORKLOAD, "n": args.n, "nq": args.nq, "entry": head, "L": R["L"],
               "k": K_NN, "recall@10": R["recall"], "evals_per_query": R["evals"],
               "hops_per_query": R["hops"], "qps_interpolated_at_0.95": R["qps_interp"],
               "W": args.W, "tuned": R["tune"],
               "sweep": R["sweep"], "other_entry_modes": others, "l_hub": args.l_hub,
               "l2": "inputs larger than L2 (512 MB base), no flush",
               "graph_build_s": W["t_build"], "repairs": W["repairs"], "learned": learned,
               "parallelism": f"replicas{world}"}
        if "medoid" in others:
            med = others["medoid"]
            cfg["learned_vs_medoid"] = {
                "qps_ratio": value / world / med["qps"],
                "evals_ratio": R["evals"] / med["evals_per_query"]}
        out = {
            "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "beam_search_kernel<F32,L2>",
                         "peak_kind": f"{peak_kind} copy bandwidth",
                         "alg_bytes_per_launch": R["alg_bytes"], "launch_ms": search_ms},
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": args.steps * R["run"].launches(),
        }
        print(json.dumps(out), flush=True)
    ann.ann_free_index(W["h"])
    if world > 1:
        import torch.distributed as distd
        distd.destroy_process_group()
    return out


def run_reference(args):
    """The CPU oracle's search as the reference arm (rank 0 only), medoid entry,
    at the pool size L* the GPU sweep finds for the same workload."""
    rank, world, local = dist_env()
    if rank != 0:
        return None
    import torch
    from paper_2506_15986_gb300 import _build, ann, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    W = build_workload(args, torch, ann, synth, dev, 0)
    run = Runner(W, torch, ann, args, "medoid")
    Lstar = sweep(run, torch, ann, W)[0]
    for _ in range(args.warmup):
        cpu_baseline(W, Lstar, target_s=2.0, width=args.W)
    per = [cpu_baseline(W, Lstar, target_s=20.0, width=args.W) for _ in range(args.steps)]
    v = float(np.mean([c["value"] for c in per]))
    cpu = dict(per[-1])
    cpu["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * args.nq / v, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "entry": "medoid", "L": Lstar, "k": K_NN,
                      "recall@10": cpu["recall@10_sample"],
                      "evals_per_query": cpu["evals_per_query"]},
           "cpu_baseline": cpu,
           "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    ann.ann_free_index(W["h"])
    return out


def main():
    args = parse()
    if args.impl == "reference":
        args.steps = min(args.steps, 3)  # about 20 s of host CPU per step
        args.warmup = min(args.warmup, 1)
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
