"""Entry-model oracle in float64 numpy (TEST INFRASTRUCTURE; see package doc).

The two-tower model of Sec. 2.2 / Sec. 4.3 as this project reads it:

* query tower (Sec. 4.3, Module II, "lightweight MLP with ReLU"):
  q -> Z1 = q W1 + b1 -> A1 = ReLU(Z1) -> Z2 = A1 W2 + b2 -> q_hat = Z2 / ||Z2||
* hub tower: a free embedding table E (one row per hub), e_hat = E / ||E||;
  with the topology-aware variant the hub row is E + F, F the fusion
  embedding of Eq. fusion (Sec. 4.3, Module I) computed from the hub's own
  vector p and its per-hop topology tokens U (fusion_forward below);
* similarity sim(q, v) = q_hat . e_hat_v (cosine, Sec. 2.2);
* loss (Sec. 2.2 Eq. loss and Sec. 4.3 Eq. loss, read per query): with the
  query's positive hubs P and negative hubs N (label mask +1 / -1, 0 = unused),
      L(q) = -(1/|P|) sum_{v in P} log( exp(s_v/tau) / sum_{u in P u N} exp(s_u/tau) )
  and the batch loss is the mean of L(q) over queries with |P| > 0;
* Adam (Sec. 5.1 names Adam; Kingma & Ba's update with bias correction).
"""
from __future__ import annotations

import numpy as np


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    The paper fixes no precision; the tensor-core path takes its GEMM operands
    (queries, weights, the hidden layer, embeddings) in bfloat16, so parity
    tests feed this oracle the same rounded operands."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def tower_forward(X, W1, b1, W2, b2, round_hidden=None):
    """Query tower forward pass; returns (q_hat, cache).  round_hidden, if
    given, is applied to the hidden activations before the second layer."""
    X = np.asarray(X, np.float64)
    Z1 = X @ W1 + b1
    A1 = relu(Z1)
    if round_hidden is not None:
        A1 = round_hidden(A1)
    Z2 = A1 @ W2 + b2
    n = np.sqrt(np.sum(Z2 * Z2, axis=1, keepdims=True))
    Qh = Z2 / n
    return Qh, dict(X=X, Z1=Z1, A1=A1, Z2=Z2, n=n, Qh=Qh)


def normalize_rows(E):
    E = np.asarray(E, np.float64)
    n = np.sqrt(np.sum(E * E, axis=1, keepdims=True))
    return E / n, n


def infonce(Qh, Eh, mask, tau):
    """Multi-positive InfoNCE over each query's labelled hubs.

    Returns (loss, dS) where S = Qh Eh^T / tau and dS = d loss / d S."""
    S = (Qh @ Eh.T) / tau
    pos = mask > 0
    use = mask != 0
    npos = pos.sum(axis=1)
    valid = npos > 0
    nvalid = int(valid.sum())
    dS = np.zeros_like(S)
    if nvalid == 0:
        return 0.0, dS
    Sm = np.where(use, S, -np.inf)
    mx = np.max(np.where(use, S, -np.inf), axis=1, keepdims=True)
    mx = np.where(np.isfinite(mx), mx, 0.0)
    ex = np.where(use, np.exp(Sm - mx), 0.0)
    z = ex.sum(axis=1, keepdims=True)
    lse = np.log(np.where(z > 0, z, 1.0)) + mx
    per_q = np.zeros(S.shape[0])
    safe_np = np.where(valid, npos, 1)
    per_q = -np.sum(np.where(pos, S - lse, 0.0), axis=1) / safe_np
    loss = float(np.sum(per_q[valid]) / nvalid)
    p = ex / np.where(z > 0, z, 1.0)
    dS = (p - pos / safe_np[:, None]) / nvalid
    dS = np.where(valid[:, None] & use, dS, 0.0)
    return loss, dS


def normalize_backward(Y, n, dY):
    """Gradient of y = z / ||z|| given y, ||z|| and dL/dy (row-wise)."""
    return (dY - Y * np.sum(Y * dY, axis=1, keepdims=True)) / n


def loss_and_grads(X, W1, b1, W2, b2, E, mask, tau):
    """Forward, InfoNCE and backward.  Returns (loss, grads dict)."""
    Qh, c = tower_forward(X, W1, b1, W2, b2)
    Eh, En = normalize_rows(E)
    loss, dS = infonce(Qh, Eh, mask, tau)
    dP = dS / tau  # gradient wrt Qh Eh^T
    dQh = dP @ Eh
    dEh = dP.T @ Qh
    dZ2 = normalize_backward(Qh, c["n"], dQh)
    dE = normalize_backward(Eh, En, dEh)
    dW2 = c["A1"].T @ dZ2
    db2 = dZ2.sum(axis=0)
    dA1 = dZ2 @ W2.T
    dZ1 = dA1 * (c["Z1"] > 0)
    dW1 = c["X"].T @ dZ1
    db1 = dZ1.sum(axis=0)
    return loss, dict(W1=dW1, b1=db1, W2=dW2, b2=db2, E=dE, dS=dS, Qh=Qh,
                      Eh=Eh, Z1=c["Z1"], A1=c["A1"], Z2=c["Z2"], dZ2=dZ2,
                      dZ1=dZ1)


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (t >= 1).  Returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def hub_scores_argmax(Qh, Eh):
    """Exhaustive entry choice: argmax_v q_hat . e_hat_v (smaller v on ties),
    with the maximum score."""
    S = np.asarray(Qh, np.float64) @ np.asarray(Eh, np.float64).T
    arg = np.argmax(S, axis=1)  # first maximum = smaller index
    return arg.astype(np.int32), S[np.arange(S.shape[0]), arg]


def fusion_forward(P, U, WQ, WK, WV, WO, heads):
    """Fusion embedding, Sec. 4.3 Eq. fusion: per hub, m = heads attention
    heads of width dk = WQ.shape[1] / heads,
        F = Concat_j softmax((p WQ_j)(U WK_j)^T / sqrt(dk)) (U WV_j)  WO
    with p [dp] the hub's vector and U [T, dU] its topology tokens.
    P [H, dp], U [H, T, dU]; returns (F [H, dF], cache for the backward)."""
    H, T, _ = U.shape
    dk = WQ.shape[1] // heads
    Q = (P @ WQ).reshape(H, heads, dk)
    K = (U @ WK).reshape(H, T, heads, dk)
    V = (U @ WV).reshape(H, T, heads, dk)
    S = np.einsum("hjd,htjd->hjt", Q, K) / np.sqrt(dk)
    S = S - S.max(axis=2, keepdims=True)
    A = np.exp(S)
    A = A / A.sum(axis=2, keepdims=True)
    O = np.einsum("hjt,htjd->hjd", A, V).reshape(H, heads * dk)
    return O @ WO, (P, U, Q, K, V, A, O, dk)


def fusion_backward(dF, cache, WO):
    """Gradients of Eq. fusion's weights from dL/dF (summed over hubs):
    returns (dWQ, dWK, dWV, dWO)."""
    P, U, Q, K, V, A, O, dk = cache
    H, heads, _ = Q.shape
    dWO = O.T @ dF
    dO = (dF @ WO.T).reshape(H, heads, dk)
    dA = np.einsum("hjd,htjd->hjt", dO, V)
    dV = np.einsum("hjt,hjd->htjd", A, dO)
    dS = A * (dA - (A * dA).sum(axis=2, keepdims=True)) / np.sqrt(dk)
    dQ = np.einsum("hjt,htjd->hjd", dS, K).reshape(H, heads * dk)
    dK = np.einsum("hjt,hjd->htjd", dS, Q)
    T = U.shape[1]
    Uf = U.reshape(H * T, -1)
    dWQ = P.T @ dQ
    dWK = Uf.T @ dK.reshape(H * T, heads * dk)
    dWV = Uf.T @ dV.reshape(H * T, heads * dk)
    return dWQ, dWK, dWV, dWO
