"""The oracle's topology-aware hub tower (NEXT row 3): the per-hop tokens of
the guided subgraph walk (Sec. 4.2) and the fusion embedding (Sec. 4.3,
Eq. fusion) with its gradients, pinned to a hand-worked walk, the exact
h-hop ball a regular graph gives, torch's multi-head attention (a library
routine), torch autograd and central differences, and the one-token closed
form."""
import numpy as np
import pytest

import oracle
from oracle import train as ot
from paper_2506_15986_gb300 import synth

# seven points on a line, degrees 2..4 (MinDeg 2, MaxDeg 4)
X7 = np.array([[0], [1], [3], [6], [10], [-2], [-5]], np.float32)
G7 = np.array([[1, 5, 3, 2], [0, 2, -1, -1], [1, 3, 4, -1], [2, 4, -1, -1], [3, 2, -1, -1],
               [0, 6, -1, -1], [5, 0, -1, -1]], np.int32)


def test_hand_walk():
    # hub 0, h = 2.  Node 0 ranks 1 (d2 1), 5 (4), 2 (9), 3 (36); x = ceil(2*4/4)
    # = 2: the nearest (1) and the farthest (3, flagged far) join at hop 1.
    # Node 1: x = ceil(2*2/4) = 1, nearest 0 is in.  Node 3: nearest 2 (d2 9)
    # joins at hop 2 with parent 3; hop-2 nodes are not expanded.  Scale
    # s = (1 + 4 + 36 + 9) / 4 = 12.5.
    tok, nodes = oracle.topo_tokens(X7, G7, [0], 2)
    assert nodes.tolist() == [4]
    f = np.float32
    s = f(12.5)
    want = np.array([
        [f(1) / f(4), f(4) / f(4), 0, 0, 0, 0, 0, 1],
        [f(2) / f(4), f(4) / f(8), (f(1) / s + f(36) / s) / f(2), f(36) / s,
         (f(1) / s + f(36) / s) / f(2), f(1) / f(2), f(1) / f(2), 1],
        [f(1) / f(4), f(3) / f(4), f(9) / s, f(9) / s, f(9) / s, 0, 1, 1],
    ], np.float32)
    np.testing.assert_array_equal(tok[0], want)


def _bfs_layers(graph, hub, h):
    layers, seen, front = [[hub]], {hub}, [hub]
    for _ in range(h):
        nxt = []
        for u in front:
            for w in graph[u]:
                if w >= 0 and w not in seen:
                    seen.add(w)
                    nxt.append(w)
        layers.append(nxt)
        front = nxt
    return [len(l) for l in layers]


def test_regular_graph_gives_the_h_hop_ball():
    # MinDeg = MaxDeg: x = deg, every neighbour is sampled (ceil(x/2) nearest
    # and floor(x/2) farthest), so the walk is breadth-first search
    rng = np.random.default_rng(5)
    n, R = 300, 6
    g = np.stack([rng.choice(np.delete(np.arange(n), i), R, replace=False) for i in range(n)]).astype(np.int32)
    x = rng.standard_normal((n, 4)).astype(np.float32)
    hubs = np.array([0, 17, 123], np.int32)
    tok, nodes = oracle.topo_tokens(x, g, hubs, 3)
    for v, hub in enumerate(hubs):
        layers = _bfs_layers(g, int(hub), 3)
        assert nodes[v] == sum(layers)
        np.testing.assert_allclose(tok[v, :, 0] * nodes[v], layers, rtol=1e-6)
        assert (tok[v, :, 1] == 1).all() or (tok[v, :, 0] == 0).any()


def test_invariants_on_a_built_graph():
    w = synth.shift_f32(n=3000, nq=1, n_train=0)
    g, _ = oracle.build_graph(w["base"], K=32, R=16)
    hubs = np.arange(0, 3000, 97, dtype=np.int32)
    h = 4
    tok, nodes = oracle.topo_tokens(w["base"], g, hubs, h, max_nodes=64)
    assert (nodes >= 1).all() and (nodes <= 64).all()
    np.testing.assert_allclose(tok[:, :, 0].sum(1), 1.0, rtol=1e-5)  # every node at one hop
    np.testing.assert_allclose(tok[:, 0, 0] * nodes, 1.0, rtol=1e-6)  # hop 0: the hub alone
    assert (tok[:, 0, 2] == 0).all()
    np.testing.assert_array_equal(tok[:, :, 6], np.tile(np.arange(h + 1) / h, (len(hubs), 1)).astype(np.float32))
    assert (tok[:, :, 7] == 1).all() and (tok[:, :, 5] >= 0).all() and (tok[:, :, 5] <= 1).all()
    assert (tok[:, :, 3] >= tok[:, :, 2]).all()  # max >= mean


def _fusion_case(seed=0, H=6, T=4, dp=10, dU=8, heads=4, dk=4, dF=16):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((H, dp)), rng.standard_normal((H, T, dU)),
            rng.standard_normal((dp, heads * dk)) * 0.5, rng.standard_normal((dU, heads * dk)) * 0.5,
            rng.standard_normal((dU, heads * dk)) * 0.5, rng.standard_normal((heads * dk, dF)) * 0.5, heads)


def test_fusion_equals_torch_multihead_attention():
    torch = pytest.importorskip("torch")
    P, U, WQ, WK, WV, WO, heads = _fusion_case()
    F, _ = ot.fusion_forward(P, U, WQ, WK, WV, WO, heads)
    E = WQ.shape[1]
    mha = torch.nn.MultiheadAttention(E, heads, bias=False, kdim=U.shape[2], vdim=U.shape[2],
                                      batch_first=True, dtype=torch.float64)
    with torch.no_grad():
        mha.q_proj_weight.copy_(torch.eye(E, dtype=torch.float64))  # the query arrives projected
        mha.k_proj_weight.copy_(torch.from_numpy(WK.T))
        mha.v_proj_weight.copy_(torch.from_numpy(WV.T))
        mha.out_proj.weight.copy_(torch.from_numpy(WO.T))
    out, _ = mha(torch.from_numpy(P @ WQ)[:, None, :], torch.from_numpy(U), torch.from_numpy(U),
                 need_weights=False)
    np.testing.assert_allclose(F, out[:, 0].detach().numpy(), rtol=1e-12, atol=1e-12)


def test_fusion_gradients_autograd_and_differences():
    torch = pytest.importorskip("torch")
    P, U, WQ, WK, WV, WO, heads = _fusion_case(1)
    rng = np.random.default_rng(2)
    G = rng.standard_normal((P.shape[0], WO.shape[1]))  # dL/dF of L = sum(G * F)
    F, cache = ot.fusion_forward(P, U, WQ, WK, WV, WO, heads)
    grads = ot.fusion_backward(G, cache, WO)
    ws = [torch.tensor(w, requires_grad=True) for w in (WQ, WK, WV, WO)]
    Pt, Ut = torch.from_numpy(P), torch.from_numpy(U)
    H, T, _ = U.shape
    dk = WQ.shape[1] // heads
    Q = (Pt @ ws[0]).reshape(H, heads, dk)
    K = (Ut @ ws[1]).reshape(H, T, heads, dk)
    V = (Ut @ ws[2]).reshape(H, T, heads, dk)
    A = torch.softmax(torch.einsum("hjd,htjd->hjt", Q, K) / dk ** 0.5, dim=2)
    Ft = torch.einsum("hjt,htjd->hjd", A, V).reshape(H, -1) @ ws[3]
    (Ft * torch.from_numpy(G)).sum().backward()
    for g, w in zip(grads, ws):
        np.testing.assert_allclose(g, w.grad.numpy(), rtol=1e-10, atol=1e-12)
    # central differences on a few entries of each weight
    Ws = [WQ, WK, WV, WO]
    for wi in range(4):
        for idx in [(0, 0), (1, 3), (Ws[wi].shape[0] - 1, Ws[wi].shape[1] - 1)]:
            e = 1e-6
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[wi][idx] += e
            Wm[wi][idx] -= e
            fp = (ot.fusion_forward(P, U, *Wp, heads)[0] * G).sum()
            fm = (ot.fusion_forward(P, U, *Wm, heads)[0] * G).sum()
            assert abs((fp - fm) / (2 * e) - grads[wi][idx]) <= 1e-6 * (1 + abs(grads[wi][idx]))


def test_fusion_single_token_closed_form():
    # one token: the softmax is 1, so F = (U WV) WO whatever WQ and WK are,
    # and their gradients vanish
    P, U, WQ, WK, WV, WO, heads = _fusion_case(3, T=1)
    F, cache = ot.fusion_forward(P, U, WQ, WK, WV, WO, heads)
    np.testing.assert_allclose(F, (U[:, 0] @ WV) @ WO, rtol=1e-12, atol=1e-12)
    dWQ, dWK, dWV, dWO = ot.fusion_backward(np.ones_like(F), cache, WO)
    assert np.abs(dWQ).max() < 1e-12 and np.abs(dWK).max() < 1e-12


def test_size_cap_on_the_hand_walk():
    # the same walk stopped at 3 nodes: hub 0, then 1 and 3 at hop 1; node 2
    # (hop 2) never joins, so the hop-2 token holds only its positional entries
    tok, nodes = oracle.topo_tokens(X7, G7, [0], 2, max_nodes=3)
    assert nodes.tolist() == [3]
    f = np.float32
    np.testing.assert_array_equal(tok[0, 0, :2], [f(1) / f(3), 1])
    np.testing.assert_array_equal(tok[0, 1, :2], [f(2) / f(3), f(4) / f(8)])
    np.testing.assert_array_equal(tok[0, 2], np.array([0, 0, 0, 0, 0, 0, 1, 1], np.float32))
