"""GPU hub extraction and label generation against the oracle.

Label-mode search costs and the label rule are integer work: bit-exact on
uint8 data.  k-means runs its assignment in fp32 (the oracle in float64), so
near-ties may send a row to another centroid: per-iteration objectives within
1e-4 relative; hubs of the same centroids within 99% agreement."""
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
def c1():
    w = synth.small_u8()
    g, _ = oracle.build_graph(w["base"], K=64, R=32)
    med = oracle.medoid(w["base"])
    h = ann.ann_index_create(w["base"], g, med, ann.U8, ann.L2)
    yield dict(w, graph=g, medoid=med, h=h)
    ann.ann_free_index(h)


def test_hub_costs_and_labels_bit_exact(c1):
    base = c1["base"]
    q = c1["queries"]
    t, _ = oracle.knn(base, q.astype(np.float64), 1)
    rng = np.random.default_rng(0)
    hub_nodes = rng.choice(len(base), 50, replace=False).astype(np.int32)
    M = 12
    cand = np.stack([rng.choice(50, M, replace=False) for _ in range(len(q))]).astype(np.int32)
    ev_o, hp_o = oracle.hub_costs(base, c1["graph"], q.astype(np.float64), hub_nodes, t[:, 0], 48,
                                  cand=cand)
    dq = torch.from_numpy(q).to(DEV)
    ev = torch.empty((len(q), M), dtype=torch.int32, device=DEV)
    hp = torch.empty_like(ev)
    ann.ann_hub_costs(c1["h"], dq, len(q), torch.from_numpy(t[:, 0].copy()).to(DEV),
                      torch.from_numpy(cand).to(DEV), M, torch.from_numpy(hub_nodes).to(DEV), 48,
                      ev, hp)
    assert ann.ann_sync_status(c1["h"]) == ann.OK
    assert np.array_equal(ev.cpu().numpy(), ev_o) and np.array_equal(hp.cpu().numpy(), hp_o)
    lab_o, best_o = oracle.labels_listed(ev_o, hp_o, cand, t_pos=3, t_neg=15)
    lab = torch.empty((len(q), M), dtype=torch.int8, device=DEV)
    best = torch.empty(len(q), dtype=torch.int32, device=DEV)
    ann.ann_hub_labels(ev, hp, torch.from_numpy(cand).to(DEV), len(q), M, 3, 15, lab, best)
    torch.cuda.synchronize()
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    assert np.array_equal(best.cpu().numpy(), best_o)


def test_label_rule_edge_rows():
    I = 2**31 - 1
    cand = np.array([[4, 0, 1, 2, 3], [0, 1, 2, 3, 4]], np.int32)
    ev = np.array([[50, 40, 40, I, 300], [I, I, I, I, I]], np.int32)
    hp = np.array([[6, 5, 4, I, 12], [I, I, I, I, I]], np.int32)
    lab_o, best_o = oracle.labels_listed(ev, hp, cand)
    t = lambda a: torch.from_numpy(a).to(DEV)
    lab = torch.zeros((2, 5), dtype=torch.int8, device=DEV)
    best = torch.zeros(2, dtype=torch.int32, device=DEV)
    ann.ann_hub_labels(t(ev), t(hp), t(cand), 2, 5, 3, 15, lab, best)
    torch.cuda.synchronize()
    assert np.array_equal(lab.cpu().numpy(), lab_o)
    assert lab_o.tolist() == [[1, 1, 1, -1, 0], [-1, -1, -1, -1, -1]]
    assert best.cpu().numpy().tolist() == best_o.tolist() == [1, -1]


def test_kmeans_and_hubs_against_oracle():
    w = synth.shift_f32(n=20000, nq=1, n_train=0)
    x = w["base"]
    sample = synth.sample_rows(len(x), 8000, seed=5)
    init = synth.kmeans_init(len(sample), 64, seed=6)
    dx = torch.from_numpy(x).to(DEV)
    cent = torch.empty((64, 128), dtype=torch.float32, device=DEV)
    obj = ann.ann_kmeans(dx, len(x), 128, ann.F32, sample, 64, init, 8, cent)
    _, _, obj_o = oracle.kmeans(x[sample], 64, init, 8)
    np.testing.assert_allclose(obj, obj_o, rtol=1e-4)
    assert (np.diff(obj) <= 1e-6 * obj[0]).all()
    c = cent.cpu().numpy()
    hubs = torch.empty(64, dtype=torch.int32, device=DEV)
    ann.ann_assign_hubs(dx, len(x), 128, ann.F32, cent, 64, hubs)
    h_o, _ = oracle.hubs(x, c.astype(np.float64))
    assert (hubs.cpu().numpy() == h_o).mean() >= 0.99
