"""GPU parity of the topology-aware hub tower (NEXT row 3): the per-hop tokens
of the guided subgraph walk (Sec. 4.2) bit for bit against the oracle (both
sides rank and sum in float32 in the same order), and the fusion embedding
(Sec. 4.3, Eq. fusion) inside a training step against the float64 oracle at
the trainer's tolerances (BF16 GEMM operands, FP32 accumulation: gradients by
relative Frobenius error <= 8e-3 and cosine >= 0.99995, the loss within 1e-4,
twice the largest errors measured on a GB300 (2.8e-3 relative Frobenius for
E, WQ and WK, 5e-4 for WV and WO, cosine >= 0.999996, loss 1.1e-5); the
fusion itself runs in FP32: its output within 1e-5 (measured 6e-7))."""
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
from gpu_util import dense_as_listed  # noqa: E402


def _tokens(h_idx, hubs, hops, max_nodes=4096):
    H = len(hubs)
    dh = torch.from_numpy(np.ascontiguousarray(hubs, np.int32)).to(DEV)
    tok = torch.empty((H, hops + 1, 8), dtype=torch.float32, device=DEV)
    nodes = torch.empty(H, dtype=torch.int32, device=DEV)
    ann.ann_topo_tokens(h_idx, dh, H, hops, tok, nodes, max_nodes=max_nodes)
    return tok.cpu().numpy(), nodes.cpu().numpy()


def test_hand_walk_on_gpu():
    x = np.zeros((7, 4), np.float32)
    x[:, 0] = [0, 1, 3, 6, 10, -2, -5]
    g = np.array([[1, 5, 3, 2], [0, 2, -1, -1], [1, 3, 4, -1], [2, 4, -1, -1], [3, 2, -1, -1],
                  [0, 6, -1, -1], [5, 0, -1, -1]], np.int32)
    h = ann.ann_index_create(x, g, 0, ann.F32, ann.L2)
    try:
        tok, nodes = _tokens(h, [0, 3, 6], 2)
    finally:
        ann.ann_free_index(h)
    otok, onodes = oracle.topo_tokens(x, g, [0, 3, 6], 2)
    assert np.array_equal(nodes, onodes) and nodes[0] == 4
    assert np.array_equal(tok.view(np.uint32), otok.view(np.uint32))


@pytest.fixture(scope="module")
def built():
    w = synth.shift_f32(n=6000, nq=1, n_train=0)
    g, _ = oracle.build_graph(w["base"], K=48, R=32)
    h = ann.ann_index_create(w["base"], g, oracle.medoid(w["base"]), ann.F32, ann.L2)
    yield dict(base=w["base"], graph=g, h=h)
    ann.ann_free_index(h)


@pytest.mark.parametrize("hops,max_nodes", [(5, 4096), (3, 3), (8, 50)])
def test_tokens_match_oracle_bit_for_bit(built, hops, max_nodes):
    hubs = np.random.default_rng(1).choice(6000, 300, replace=False).astype(np.int32)
    tok, nodes = _tokens(built["h"], hubs, hops, max_nodes)
    otok, onodes = oracle.topo_tokens(built["base"], built["graph"], hubs, hops, max_nodes=max_nodes)
    assert np.array_equal(nodes, onodes)
    assert np.array_equal(tok.view(np.uint32), otok.view(np.uint32))


def test_tokens_reject_bad_hubs(built):
    for bad in ([-1], [6000]):
        with pytest.raises(ann.AnnError) as e:
            _tokens(built["h"], np.array(bad, np.int32), 3)
        assert e.value.status == ann.ERR_INVALID_ARG


def _fusion_weights(dp, dU, heads, dk, seed=4):
    rng = np.random.default_rng(seed)
    E = heads * dk
    return ((rng.standard_normal((dp, E)) / np.sqrt(dp)).astype(np.float32),
            (rng.standard_normal((dU, E)) / np.sqrt(dU)).astype(np.float32),
            (rng.standard_normal((dU, E)) / np.sqrt(dU)).astype(np.float32),
            (rng.standard_normal((E, 64)) / np.sqrt(E)).astype(np.float32))


def test_fusion_step_matches_oracle():
    rng = np.random.default_rng(0)
    B, D, H, T, dU, heads, dk = 600, 128, 200, 6, 8, 4, 16
    X = rng.standard_normal((B, D)).astype(np.float32)
    W1 = (rng.standard_normal((D, 256)) / np.sqrt(D)).astype(np.float32)
    b1 = (0.1 * rng.standard_normal(256)).astype(np.float32)
    W2 = (rng.standard_normal((256, 64)) / 16).astype(np.float32)
    b2 = (0.1 * rng.standard_normal(64)).astype(np.float32)
    E = (0.5 * rng.standard_normal((H, 64))).astype(np.float32)
    P = rng.standard_normal((H, D)).astype(np.float32)
    U = rng.random((H, T, dU)).astype(np.float32)
    mask = rng.choice(np.array([-1, 0, 1], np.int8), size=(B, H), p=[0.6, 0.3, 0.1])
    WQ, WK, WV, WO = _fusion_weights(D, dU, heads, dk)
    tau = 0.1
    t = ann.ann_trainer_create(D, W1, b1, W2, b2, E, 1024, tau=tau, lr=1e-3)
    try:
        dP, dU_ = torch.from_numpy(P).to(DEV), torch.from_numpy(U).to(DEV)
        ann.ann_trainer_set_fusion(t, dP, dU_, T, dU, heads, dk, WQ, WK, WV, WO)
        rows = torch.arange(B, dtype=torch.int32, device=DEV)
        loss = ann.ann_trainer_step(t, torch.from_numpy(X).to(DEV), rows, B, *dense_as_listed(mask),
                                    apply_update=False)
        Eeff = np.zeros((H, 64), np.float32)
        gE = np.zeros((H, 64), np.float32)
        ann.ann_trainer_get(t, None, None, None, None, Eeff)
        ann.ann_trainer_get(t, None, None, None, None, gE, gradients=True)
        gw = [np.zeros_like(w) for w in (WQ, WK, WV, WO)]
        ann.ann_trainer_get_fusion(t, *gw, gradients=True)
    finally:
        ann.ann_trainer_free(t)
    F, cache = ot.fusion_forward(P.astype(np.float64), U.astype(np.float64), WQ.astype(np.float64),
                                 WK.astype(np.float64), WV.astype(np.float64), WO.astype(np.float64), heads)
    Ee = E.astype(np.float64) + F
    np.testing.assert_allclose(Eeff, Ee, rtol=1e-5, atol=1e-5)
    bf = ot.bf16_round
    ref_loss, ref = ot.loss_and_grads(bf(X), bf(W1), b1.astype(np.float64), bf(W2), b2.astype(np.float64), Ee,
                                      mask, tau)
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    cos = lambda a, b: float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b)))
    assert rel(gE, ref["E"]) <= 8e-3 and cos(gE, ref["E"]) >= 0.99995
    refw = ot.fusion_backward(ref["E"], cache, WO.astype(np.float64))
    for name, g, r in zip(("WQ", "WK", "WV", "WO"), gw, refw):
        assert rel(g, r) <= 8e-3, (name, rel(g, r))
        assert cos(g, r) >= 0.99995, (name, cos(g, r))


def test_fusion_training_lowers_the_loss():
    rng = np.random.default_rng(1)
    B, D, H, T, dU = 1024, 128, 64, 4, 8
    X = rng.standard_normal((4096, D)).astype(np.float32)
    W1, b1, W2, b2, E = synth.model_init(D, H)
    mask = rng.choice(np.array([-1, 0, 1], np.int8), size=(4096, H), p=[0.5, 0.4, 0.1])
    WQ, WK, WV, WO = _fusion_weights(D, dU, 2, 16)
    t = ann.ann_trainer_create(D, W1, b1, W2, b2, E, B, tau=0.1, lr=1e-3)
    try:
        ann.ann_trainer_set_fusion(t, torch.from_numpy(rng.standard_normal((H, D)).astype(np.float32)).to(DEV),
                                   torch.from_numpy(rng.random((H, T, dU)).astype(np.float32)).to(DEV),
                                   T, dU, 2, 16, WQ, WK, WV, WO)
        with pytest.raises(ann.AnnError):  # once per trainer
            ann.ann_trainer_set_fusion(t, torch.zeros((H, D), device=DEV), torch.zeros((H, T, dU), device=DEV),
                                       T, dU, 2, 16, WQ, WK, WV, WO)
        losses = torch.zeros(4 * 10, device=DEV)
        ann.ann_trainer_fit(t, torch.from_numpy(X).to(DEV), 4096, *dense_as_listed(mask), None, 10, losses)
        ls = losses.cpu().numpy()
        w0 = np.zeros_like(WO)
        ann.ann_trainer_get_fusion(t, None, None, None, w0)
    finally:
        ann.ann_trainer_free(t)
    assert ls[-4:].mean() < ls[:4].mean()
    assert not np.array_equal(w0, WO)  # the fusion weights were trained


def test_tokens_and_fusion_reject_bad_sizes(built):
    hubs = torch.zeros(4, dtype=torch.int32, device=DEV)
    tok = torch.empty((4, 10, 8), dtype=torch.float32, device=DEV)
    for H, hops, max_nodes in ((0, 3, 64), (4, 0, 64), (4, 65, 64), (4, 3, 0), (4, 3, 8193)):
        with pytest.raises(ann.AnnError) as e:
            ann.ann_topo_tokens(built["h"], hubs, H, hops, tok, max_nodes=max_nodes)
        assert e.value.status == ann.ERR_INVALID_ARG
    W1, b1, W2, b2, E = synth.model_init(128, 8)
    t = ann.ann_trainer_create(128, W1, b1, W2, b2, E, 64)
    try:
        P = torch.zeros((8, 128), device=DEV)
        U = torch.zeros((8, 4, 8), device=DEV)
        for T, dU, heads, dk in ((0, 8, 2, 16), (4, 0, 2, 16), (4, 8, 0, 16), (4, 8, 17, 16)):
            WQ, WK, WV, WO = _fusion_weights(128, max(dU, 1), max(heads, 1), dk)
            with pytest.raises(ann.AnnError) as e:
                ann.ann_trainer_set_fusion(t, P, U, T, dU, heads, dk, WQ, WK, WV, WO)
            assert e.value.status == ann.ERR_INVALID_ARG
    finally:
        ann.ann_trainer_free(t)
