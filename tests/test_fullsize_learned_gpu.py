"""The headline path at full size with a trained entry model, and what the
trained model gains over the medoid entry (the ablation without the learned
entry, Table 3, and the shorter search paths of Sec. 5.2).

Workload: the shifted 1M x 128 fp32 set (10,000 evaluation queries), its GPU
graph (exact 64-NN + RNG prune, R = 32), 1,024 k-means hubs, labels from
label-mode searches of each training query from its 64 nearest hubs
(t_pos = 3, t_neg = 15), and the two-tower model trained through the library
(Adam, lr 5e-5, batch 8,192, 200 epochs) on 30,000 training queries (the
bench trains on 100,000; fewer here to keep the test short).

* Entries: on 200 sampled queries the oracle computes q_hat from the trained
  weights (float64 on the BF16-rounded operands) and picks its own best hub;
  the GPU's choice must score within twice the q_hat difference of the best
  (plus FP32 accumulation), and >= 99 % of choices must be equal.
* Search: the headline launch (L = 93, W = 4, tuned sizes) from those entries
  against the oracle's search on the same graph, entries, L and W, at the
  fp32 bar: >= 99.9 % of (query, rank) ids, distances within 1e-5 relative,
  recall@10 within 0.001, evaluation and expansion counts equal for >= 99 %.
* Gain: over an L sweep, the learned entry reaches recall@10 >= 0.95 with
  fewer distance evaluations per query than the medoid entry does.
* Hub-graph search (the paper's entry path) on the undirected hub graph the
  bench uses: its choices against the oracle's walk over the oracle's graph on
  200 sampled queries, and its entries' evaluation cost against the
  exhaustive argmax's at the same pool size."""
import numpy as np
import pytest

import oracle
from oracle import train as ot
from paper_2506_15986_gb300 import ann, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
DEV = torch.device("cuda:0")

N, NQ, NT, R, K, HUBS, M_CAND, EPOCHS = 1_000_000, 10_000, 30_000, 32, 10, 1024, 64, 200
L_HEAD, W = 93, 4


@pytest.fixture(scope="module")
def learned():
    w = synth.shift_f32(n=N, nq=NQ, n_train=NT)
    base = torch.from_numpy(w["base"]).to(DEV)
    graph = torch.empty((N, R), dtype=torch.int32, device=DEV)
    med, _ = ann.ann_build_graph(base, N, 128, ann.F32, 64, R, 1.0, graph)
    q = torch.from_numpy(w["queries"]).to(DEV)
    gt = torch.empty((NQ, K), dtype=torch.int32, device=DEV)
    gd = torch.empty((NQ, K), dtype=torch.float32, device=DEV)
    ann.ann_knn(base, N, 128, ann.F32, ann.L2, q, NQ, K, gt, gd)
    h = ann.ann_index_create(base, graph, med, ann.F32, ann.L2)
    # hubs: flat k-means on a sample, then the row nearest each centroid
    sample = synth.sample_rows(N, 262_144, seed=synth.SEED_BASE + 10)
    init = synth.kmeans_init(len(sample), HUBS, seed=synth.SEED_BASE + 11)
    cent = torch.empty((HUBS, 128), dtype=torch.float32, device=DEV)
    ann.ann_kmeans(base, N, 128, ann.F32, sample, HUBS, init, 25, cent)
    hubs = torch.empty(HUBS, dtype=torch.int32, device=DEV)
    ann.ann_assign_hubs(base, N, 128, ann.F32, cent, HUBS, hubs)
    hub_np = hubs.cpu().numpy()
    hub_np = hub_np[hub_np >= 0]
    H = len(hub_np)
    hub_nodes = torch.from_numpy(hub_np).to(DEV)
    hub_vecs = torch.from_numpy(w["base"][hub_np]).to(DEV)
    # labels: each training query searched from its 64 nearest hubs
    tq = torch.from_numpy(w["train"]).to(DEV)
    cand = torch.empty((NT, M_CAND), dtype=torch.int32, device=DEV)
    cd = torch.empty((NT, M_CAND), dtype=torch.float32, device=DEV)
    ann.ann_knn(hub_vecs, H, 128, ann.F32, ann.L2, tq, NT, M_CAND, cand, cd)
    tgt = torch.empty((NT, 1), dtype=torch.int32, device=DEV)
    td = torch.empty((NT, 1), dtype=torch.float32, device=DEV)
    ann.ann_knn(base, N, 128, ann.F32, ann.L2, tq, NT, 1, tgt, td)
    ev = torch.empty((NT, M_CAND), dtype=torch.int32, device=DEV)
    hp = torch.empty_like(ev)
    ann.ann_hub_costs(h, tq, NT, tgt, cand, M_CAND, hub_nodes, 64, ev, hp)
    labels = torch.empty((NT, M_CAND), dtype=torch.int8, device=DEV)
    ann.ann_hub_labels(ev, hp, cand, NT, M_CAND, 3, 15, labels)
    assert ann.ann_sync_status(h) == ann.OK
    # the model: hub tower starts at the query tower of each hub's own vector
    W1, b1, W2, b2, E = synth.model_init(128, H)
    ann.ann_set_entry_model(h, 128, W1, b1, W2, b2, hub_np, E, 16)
    E0 = torch.empty((H, 64), dtype=torch.float32, device=DEV)
    tmp = torch.empty(H, dtype=torch.int32, device=DEV)
    ann.ann_select_entry(h, hub_vecs, H, ann.ENTRY_LEARNED_EXHAUSTIVE, 32, tmp, E0)
    t = ann.ann_trainer_create(128, W1, b1, W2, b2, E0, 8192, tau=0.07, lr=5e-5)
    try:
        order = torch.from_numpy(np.concatenate(
            synth.train_batches(NT, 8192, EPOCHS, seed=synth.SEED_BASE + 12))).to(DEV)
        ann.ann_trainer_fit(t, tq, NT, cand, labels, M_CAND, order, EPOCHS)
        ann.ann_trainer_attach(t, h, hub_nodes, 16)
    finally:
        ann.ann_trainer_free(t)
    ent = torch.empty(NQ, dtype=torch.int32, device=DEV)
    qh = torch.empty((NQ, 64), dtype=torch.float32, device=DEV)
    ann.ann_select_entry(h, q, NQ, ann.ENTRY_LEARNED_EXHAUSTIVE, 32, ent, qh)
    assert ann.ann_sync_status(h) == ann.OK
    model = dict(W1=np.zeros((128, 256), np.float32), b1=np.zeros(256, np.float32),
                 W2=np.zeros((256, 64), np.float32), b2=np.zeros(64, np.float32),
                 E=np.zeros((H, 64), np.float32), nodes=np.zeros(H, np.int32))
    ann.ann_get_entry_model(h, model["W1"], model["b1"], model["W2"], model["b2"], model["E"], model["nodes"])
    yield dict(w=w, graph=graph.cpu().numpy(), med=med, q=q, gt=gt.cpu().numpy(), h=h, ent=ent,
               ent_np=ent.cpu().numpy(), qh=qh.cpu().numpy(), model=model)
    ann.ann_free_index(h)


def _search(s, entries, L, stats=True):
    p = ann.search_params(K, L, W=W, hash_bits=-1, stage_rows=8, team=4)
    ids = torch.empty((NQ, K), dtype=torch.int32, device=DEV)
    dd = torch.empty((NQ, K), dtype=torch.float32, device=DEV)
    st = torch.empty((NQ, 2), dtype=torch.int32, device=DEV)
    ann.ann_search_batch(s["h"], s["q"], NQ, entries, p, ids, dd, st)
    assert ann.ann_sync_status(s["h"]) == ann.OK
    return ids.cpu().numpy(), dd.cpu().numpy(), st.cpu().numpy()


def _recall(ids, gt):
    return np.mean([len(set(a[a >= 0]) & set(b)) / K for a, b in zip(ids, gt)])


def test_learned_entries_match_the_oracle(learned):
    m = learned["model"]
    rng = np.random.default_rng(21)
    sample = np.sort(rng.choice(NQ, 200, replace=False))
    bf = ot.bf16_round
    qo, _ = ot.tower_forward(bf(learned["w"]["queries"][sample]), bf(m["W1"]), m["b1"].astype(np.float64),
                             bf(m["W2"]), m["b2"].astype(np.float64), round_hidden=bf)
    En = m["E"].astype(np.float64) / np.linalg.norm(m["E"].astype(np.float64), axis=1, keepdims=True)
    Eb = bf(En)
    S = bf(qo) @ Eb.T
    hub_of = {int(v): i for i, v in enumerate(m["nodes"])}
    chosen = np.array([hub_of[int(e)] for e in learned["ent_np"][sample]])
    best, got = S.max(1), S[np.arange(len(S)), chosen]
    dq = np.linalg.norm(bf(learned["qh"][sample]) - bf(qo), axis=1) * np.linalg.norm(Eb, axis=1).max()
    assert (best - got <= 2 * dq + 1e-5).all(), (best - got - 2 * dq).max()
    assert (chosen == S.argmax(1)).mean() >= 0.99


def test_headline_search_from_learned_entries_matches_the_oracle(learned):
    ids, dd, st = _search(learned, learned["ent"], L_HEAD)
    rng = np.random.default_rng(22)
    sample = np.sort(rng.choice(NQ, 200, replace=False))
    q64 = learned["w"]["queries"][sample].astype(np.float64)
    oi, od, oe, oh = oracle.search(learned["w"]["base"], learned["graph"], q64, learned["ent_np"][sample],
                                   L_HEAD, K, W=W)
    gi, gd = ids[sample], dd[sample].astype(np.float64)
    same = gi == oi
    assert same.mean() >= 0.999, same.mean()
    assert (np.abs(gd[same] - od[same]) <= 1e-5 * np.maximum(od[same], 1e-30)).all()
    gt = learned["gt"][sample]
    assert abs(_recall(gi, gt) - _recall(oi, gt)) <= 0.001
    assert (st[sample, 0] == oe).mean() >= 0.99 and (st[sample, 1] == oh).mean() >= 0.99


def test_trained_entry_needs_fewer_evaluations_than_the_medoid(learned):
    def first_at_target(entries):
        for L in (48, 64, 80, 96, 112, 128, 160, 192, 224, 256, 320):
            ids, _, st = _search(learned, entries, L)
            r = _recall(ids, learned["gt"])
            if r >= 0.95:
                return L, r, float(st[:, 0].mean()), float(st[:, 1].mean())
        raise AssertionError("recall 0.95 not reached")

    Ll, rl, el, hl = first_at_target(learned["ent"])
    Lm, rm, em, hm = first_at_target(None)
    print(f"learned: L={Ll} recall={rl:.4f} evals={el:.0f} hops={hl:.1f}; "
          f"medoid: L={Lm} recall={rm:.4f} evals={em:.0f} hops={hm:.1f}")
    # at equal recall (the first swept L reaching 0.95) the trained entry
    # needs fewer distance evaluations and fewer expansions
    assert el < em and hl < hm
    assert el <= 0.8 * em  # a clear gain, not noise: the bench measures 0.48x


def test_hub_graph_search_on_the_undirected_graph(learned):
    # the paper's entry path with the trained model at full size: the hub
    # graph rebuilt undirected (each hub's 8 most similar hubs and the hubs
    # that list it, at most 16, as the bench uses it), the walk at L_hub = 32.
    # On 200 sampled queries the oracle walks its own graph of the trained
    # embeddings from its own q_hat; then the walk's entries cost the search
    # about what the exhaustive argmax's do
    h, m = learned["h"], learned["model"]
    ann.ann_build_hub_graph(h, 8, 16)
    ent = torch.empty(NQ, dtype=torch.int32, device=DEV)
    ann.ann_select_entry(h, learned["q"], NQ, ann.ENTRY_LEARNED_NAV, 32, ent)
    assert ann.ann_sync_status(h) == ann.OK
    ent_np = ent.cpu().numpy()
    rng = np.random.default_rng(23)
    sample = np.sort(rng.choice(NQ, 200, replace=False))
    bf = ot.bf16_round
    qo, _ = ot.tower_forward(bf(learned["w"]["queries"][sample]), bf(m["W1"]), m["b1"].astype(np.float64),
                             bf(m["W2"]), m["b2"].astype(np.float64), round_hidden=bf)
    En = m["E"].astype(np.float64) / np.linalg.norm(m["E"].astype(np.float64), axis=1, keepdims=True)
    Eb = bf(En)
    adj, entry_hub = oracle.hub_graph_undirected(m["E"].astype(np.float64), 8, 16)
    oi, _, _, _ = oracle.search(Eb.astype(np.float32), adj, qo, entry_hub, 32, 1, metric=oracle.IP)
    hub_of = {int(v): i for i, v in enumerate(m["nodes"])}
    chosen = np.array([hub_of[int(e)] for e in ent_np[sample]])
    assert (chosen == oi[:, 0]).mean() >= 0.98
    S = qo @ Eb.T
    r = np.arange(len(S))
    assert S[r, oi[:, 0]].mean() - S[r, chosen].mean() <= 1e-4
    # the same pool size for both entries: the walk's entries need at most 5 %
    # more evaluations than the exhaustive argmax's (the bench measures 1 %)
    _, _, st_nav = _search(learned, ent, 96)
    _, _, st_exh = _search(learned, learned["ent"], 96)
    assert st_nav[:, 0].mean() <= 1.05 * st_exh[:, 0].mean(), (st_nav[:, 0].mean(), st_exh[:, 0].mean())
