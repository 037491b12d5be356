"""Pins of the oracle's int8-with-scale quantiser (the precision line's int8
storage) and of its float64-row search path."""
import numpy as np

import oracle


def test_quantize_hand_cases():
    # max |x| = 127 gives scale 1 exactly; -63.5 rounds half to even
    x = np.array([[127.0, -63.5, 31.25, 0.0, -127.0, 2.5, -1.5, 0.5]], np.float32)
    c, s = oracle.quantize_i8s(x)
    assert s.tolist() == [1.0]
    assert c.tolist() == [[127, -64, 31, 0, -127, 2, -2, 0]]
    # max |x| = 254 gives scale 2: 5 / 2 = 2.5 -> 2, 3 / 2 = 1.5 -> 2
    x = np.array([[254.0, 5.0, 3.0, -3.0]], np.float32)
    c, s = oracle.quantize_i8s(x)
    assert s.tolist() == [2.0] and c.tolist() == [[127, 2, 2, -2]]


def test_quantize_zero_row_and_bounds():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((200, 96)).astype(np.float32) * rng.lognormal(0, 2, (200, 1)).astype(np.float32)
    x[5] = 0.0
    c, s = oracle.quantize_i8s(x)
    assert s[5] == 0 and (c[5] == 0).all()
    nz = s > 0
    # the largest |x| of every row maps to +-127
    assert (np.abs(c[nz]).max(axis=1) == 127).all()
    # rounding to nearest: |x - scale * code| <= scale / 2 (plus fp32 slack)
    err = np.abs(x.astype(np.float64) - oracle.dequantize_i8s(c, s))
    assert (err <= s[:, None].astype(np.float64) * (0.5 + 1e-5)).all()


def test_float64_rows_search_like_float32():
    # float64 rows holding float32 values give the float32 search exactly
    rng = np.random.default_rng(3)
    base = rng.standard_normal((600, 8)).astype(np.float32)
    g, _ = oracle.build_graph(base, K=16, R=8)
    q = rng.standard_normal((20, 8))
    med = oracle.medoid(base)
    a = oracle.search(base, g, q, med, 32, 10, W=2)
    b = oracle.search(base.astype(np.float64), g, q, med, 32, 10, W=2)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def test_dequantized_search_is_l_ge_n_exact():
    # the special case L >= N on a connected graph returns the exact k-NN of
    # the dequantised rows
    rng = np.random.default_rng(4)
    x = rng.standard_normal((300, 16)).astype(np.float32)
    c, s = oracle.quantize_i8s(x)
    xd = oracle.dequantize_i8s(c, s)
    g, _ = oracle.build_graph(x, K=16, R=8)
    q = rng.standard_normal((10, 16))
    ids, d, _, _ = oracle.search(xd, g, q, oracle.medoid(x), 300, 10)  # repaired from the medoid
    tid, td = oracle.knn(xd, q, 10)
    assert np.array_equal(ids, tid) and np.allclose(d, td, rtol=0, atol=0)
