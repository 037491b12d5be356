"""Pins for the entry-model oracle (CPU only): forward/backward against torch
float64 autograd (a library routine) and central finite differences, the
InfoNCE loss against its one-positive/one-negative closed form, and Adam's
first step against its closed form."""
import numpy as np
import torch

from oracle import train as ot


def _model(rng, d=12, h=16, e=8, H=10):
    W1 = rng.standard_normal((d, h)) * 0.3
    b1 = rng.standard_normal(h) * 0.1
    W2 = rng.standard_normal((h, e)) * 0.3
    b2 = rng.standard_normal(e) * 0.1
    E = rng.standard_normal((H, e))
    return W1, b1, W2, b2, E


def _mask(rng, B, H):
    m = rng.choice(np.array([-1, 0, 1], np.int8), size=(B, H), p=[0.5, 0.2, 0.3])
    m[0] = 0          # a query with no labelled hub: contributes nothing
    m[1, :] = -1
    m[1, 3] = 1       # exactly one positive
    return m


def test_infonce_closed_form_one_pos_one_neg():
    tau = 0.07
    Qh = np.array([[1.0, 0.0]])
    Eh = np.array([[np.cos(0.3), np.sin(0.3)], [np.cos(1.1), np.sin(1.1)]])
    mask = np.array([[1, -1]], np.int8)
    loss, dS = ot.infonce(Qh, Eh, mask, tau)
    sp, sn = np.cos(0.3), np.cos(1.1)
    assert np.isclose(loss, np.log1p(np.exp((sn - sp) / tau)), rtol=1e-13)
    sig = 1.0 / (1.0 + np.exp(-(sn - sp) / tau))
    # dL/dS with S = s / tau
    np.testing.assert_allclose(dS[0], [-sig, sig], rtol=1e-12)


def test_forward_backward_matches_torch_autograd():
    rng = np.random.default_rng(0)
    W1, b1, W2, b2, E = _model(rng)
    X = rng.standard_normal((7, 12))
    mask = _mask(rng, 7, 10)
    tau = 0.1
    loss, g = ot.loss_and_grads(X, W1, b1, W2, b2, E, mask, tau)

    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True)
         for k, v in dict(W1=W1, b1=b1, W2=W2, b2=b2, E=E).items()}
    Xt = torch.tensor(X, dtype=torch.float64)
    z2 = torch.relu(Xt @ t["W1"] + t["b1"]) @ t["W2"] + t["b2"]
    qh = torch.nn.functional.normalize(z2, dim=1)
    eh = torch.nn.functional.normalize(t["E"], dim=1)
    S = qh @ eh.T / tau
    m = torch.tensor(mask)
    losses = []
    for i in range(7):
        use = m[i] != 0
        pos = m[i] > 0
        if pos.sum() == 0:
            continue
        lse = torch.logsumexp(S[i][use], 0)
        losses.append(-(S[i][pos] - lse).mean())
    L = torch.stack(losses).mean()
    L.backward()
    assert np.isclose(loss, L.item(), rtol=1e-12)
    for k in ("W1", "b1", "W2", "b2", "E"):
        np.testing.assert_allclose(g[k], t[k].grad.numpy(), rtol=1e-9, atol=1e-12)


def test_gradients_central_differences():
    rng = np.random.default_rng(1)
    W1, b1, W2, b2, E = _model(rng, d=6, h=8, e=4, H=5)
    X = rng.standard_normal((5, 6))
    mask = _mask(rng, 5, 5)
    tau = 0.2
    params = dict(W1=W1, b1=b1, W2=W2, b2=b2, E=E)
    _, g = ot.loss_and_grads(X, W1, b1, W2, b2, E, mask, tau)
    h = 1e-6
    for name, p in params.items():
        it = np.nditer(p, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[idx]
            p[idx] = old + h
            lp, _ = ot.loss_and_grads(X, W1, b1, W2, b2, E, mask, tau)
            p[idx] = old - h
            lm, _ = ot.loss_and_grads(X, W1, b1, W2, b2, E, mask, tau)
            p[idx] = old
            num = (lp - lm) / (2 * h)
            assert abs(num - g[name][idx]) <= 1e-6 * max(1.0, abs(num)), (name, idx)


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 5e-5, 1e-8
    p1, m1, v1 = ot.adam_step(p, g, m, v, 1, lr, eps=eps)
    # bias-corrected first step: m_hat = g, v_hat = g^2
    np.testing.assert_allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=1e-14)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_adam_matches_torch():
    rng = np.random.default_rng(4)
    p0 = rng.standard_normal(20)
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(20), np.zeros(20)
    for t in range(1, 6):
        g = rng.standard_normal(20)
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = ot.adam_step(p, g, m, v, t, 1e-2)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12)


def test_hub_argmax_first_maximum():
    Qh = np.array([[1.0, 0.0], [0.0, 1.0]])
    Eh = np.array([[0.5, 0.5], [1.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    arg, s = ot.hub_scores_argmax(Qh, Eh)
    assert arg.tolist() == [1, 3] and s.tolist() == [1.0, 1.0]


def test_bf16_round_ties_and_values():
    # 1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even (1)
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -2.5, 3.0e38], np.float32)
    r = ot.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2**-6 and r[3] == -2.5
    # torch's own bfloat16 conversion (round to nearest even) agrees
    v = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    t = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ot.bf16_round(v), t)
