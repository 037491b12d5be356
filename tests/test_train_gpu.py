"""GPU training kernels against the float64 oracle (Sec. 4.3 Eq. loss, Adam).

Tolerance: every GEMM of a step takes BF16 operands (about 2^-9 relative
rounding each) with FP32 accumulation, and the backward pass chains up to
four such GEMMs whose intermediate operands (the logit gradients, dq_hat, the
hidden layer's gradient) are rounded again, which the oracle fed the same
BF16-rounded inputs does not do.  Measured on a GB300 over batches of 700,
3,000 and 8,192 rows (three seeds each): relative Frobenius error 2.0e-3 to
4.0e-3 per parameter, cosine >= 0.99999, loss within 2.5e-5 relative.  The
bars are twice the largest measured error: relative Frobenius <= 8e-3,
cosine >= 0.99995, loss within 1e-4 relative.  Adam is elementwise fp32
against float64: 1e-5 relative."""
import numpy as np
import pytest

from oracle import train as ot
from paper_2506_15986_gb300 import ann

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
DEV = torch.device("cuda:0")
from gpu_util import dense_as_listed  # noqa: E402


def _problem(B=700, D=128, H=200, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B + 50, D)).astype(np.float32)
    W1 = (rng.standard_normal((D, 256)) / np.sqrt(D)).astype(np.float32)
    b1 = (0.1 * rng.standard_normal(256)).astype(np.float32)
    W2 = (rng.standard_normal((256, 64)) / 16).astype(np.float32)
    b2 = (0.1 * rng.standard_normal(64)).astype(np.float32)
    E = rng.standard_normal((H, 64)).astype(np.float32)
    mask = rng.choice(np.array([-1, 0, 1], np.int8), size=(B + 50, H), p=[0.6, 0.3, 0.1])
    mask[3] = 0  # a query without labels
    rows = rng.permutation(B + 50)[:B].astype(np.int32)  # a batch drawn through a row map
    return X, W1, b1, W2, b2, E, mask, rows


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _cos(a, b):
    return float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.mark.parametrize("B", [700, 3000])
def test_gradients_match_oracle(B):
    # B = 3000: the reductions over the batch (dE, dW1, dW2) are split over
    # K ranges whose partial sums add into the output, the last range ragged
    X, W1, b1, W2, b2, E, mask, rows = _problem(B=B)
    tau = 0.1
    t = ann.ann_trainer_create(128, W1, b1, W2, b2, E, 4096, tau=tau, lr=1e-3)
    try:
        dX = torch.from_numpy(X).to(DEV)
        dr = torch.from_numpy(rows).to(DEV)
        loss = ann.ann_trainer_step(t, dX, dr, len(rows), *dense_as_listed(mask), apply_update=False)
        g = {k: np.zeros_like(v) for k, v in dict(W1=W1, b1=b1, W2=W2, b2=b2, E=E).items()}
        ann.ann_trainer_get(t, g["W1"], g["b1"], g["W2"], g["b2"], g["E"], gradients=True)
    finally:
        ann.ann_trainer_free(t)
    bf = ot.bf16_round
    ref_loss, ref = ot.loss_and_grads(bf(X[rows]), bf(W1), b1.astype(np.float64), bf(W2),
                                      b2.astype(np.float64), E.astype(np.float64), mask[rows], tau)
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    for k in ("W1", "b1", "W2", "b2", "E"):
        assert _rel(g[k], ref[k]) <= 8e-3, (k, _rel(g[k], ref[k]))
        assert _cos(g[k], ref[k]) >= 0.99995, (k, _cos(g[k], ref[k]))


def test_adam_update_matches_oracle():
    rng = np.random.default_rng(3)
    n = 5000
    p = rng.standard_normal(n).astype(np.float32)
    m = np.zeros(n, np.float32)
    v = np.zeros(n, np.float32)
    dp, dm, dv = (torch.from_numpy(a.copy()).to(DEV) for a in (p, m, v))
    pr, mr, vr = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 4):
        gr = rng.standard_normal(n).astype(np.float32)
        ann.ann_adam_update(dp, torch.from_numpy(gr).to(DEV), dm, dv, n, step, 1e-2)
        pr, mr, vr = ot.adam_step(pr, gr.astype(np.float64), mr, vr, step, 1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(dp.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(dm.cpu().numpy(), mr, rtol=1e-5, atol=1e-7)


def test_training_lowers_the_loss_and_attaches():
    X, W1, b1, W2, b2, E, mask, rows = _problem(B=2000, H=64, seed=1)
    # learnable structure: the positive hub of a query is decided by its first coordinates
    lab = (np.abs(X[:, :6]).argmax(1) * 10 + (X[:, 6] > 0)).astype(np.int64) % 64
    mask = np.full((len(X), 64), -1, np.int8)
    mask[np.arange(len(X)), lab] = 1
    t = ann.ann_trainer_create(128, W1, b1, W2, b2, E, 512, tau=0.1, lr=3e-3)
    try:
        dX = torch.from_numpy(X).to(DEV)
        nt = len(X)
        steps = (nt + 511) // 512
        losses = torch.zeros(30 * steps, device=DEV)
        ann.ann_trainer_fit(t, dX, nt, *dense_as_listed(mask), None, 30, losses)
        ls = losses.cpu().numpy()
        assert ls[-steps:].mean() < 0.5 * ls[:steps].mean()
        W = np.zeros_like(W1)
        ann.ann_trainer_get(t, W1=W)
        assert np.isfinite(W).all() and not np.array_equal(W, W1)
    finally:
        ann.ann_trainer_free(t)


def test_listed_labels_train_like_their_dense_matrix():
    # M listed hubs per query (the label search's candidates), every other hub
    # a negative: the same loss and gradients as the dense label matrix that
    # lists all hubs (only the label layout differs)
    X, W1, b1, W2, b2, E, _, rows = _problem(B=900, H=300, seed=4)
    rng = np.random.default_rng(8)
    n, H, M = len(X), 300, 40
    cand = np.stack([rng.choice(H, M, replace=False) for _ in range(n)]).astype(np.int32)
    lab = rng.choice(np.array([-1, 0, 1], np.int8), size=(n, M), p=[0.3, 0.4, 0.3])
    cand[7, 5] = -1  # an empty slot
    dense = np.full((n, H), -1, np.int8)
    for r in range(n):
        ok = cand[r] >= 0
        dense[r, cand[r][ok]] = lab[r][ok]
    out = []
    for labels in ((torch.from_numpy(cand).to(DEV), torch.from_numpy(lab).to(DEV), M), dense_as_listed(dense)):
        t = ann.ann_trainer_create(128, W1, b1, W2, b2, E, 1024, tau=0.1, lr=1e-3)
        try:
            loss = ann.ann_trainer_step(t, torch.from_numpy(X).to(DEV), torch.from_numpy(rows).to(DEV), len(rows),
                                        *labels, apply_update=False)
            gE = np.zeros_like(E)
            ann.ann_trainer_get(t, hub_emb=gE, gradients=True)
        finally:
            ann.ann_trainer_free(t)
        out.append((loss, gE))
    assert out[0][0] == out[1][0]
    # the reductions over the batch may add partial sums in another order
    assert _rel(out[0][1], out[1][1]) <= 1e-5
