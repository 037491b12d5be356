"""Seeded synthetic workloads (inputs only; no search, graph or model arithmetic).

The paper's datasets (Sift10M, Gist1M, Tiny5M, Laion3M, Text2Image10M; Sec. 5.1
Table 1) are not available, so each generator draws a Gaussian-mixture stand-in
with the shape, dtype and query/base relation of one workload.  Every array is
a pure function of (sizes, seed) through numpy's PCG64 generator, so the CUDA
path and the oracle receive identical inputs.  Random numbers that a method
step itself needs (k-means initial rows) are drawn here too and passed in.

Workloads (default sizes; tests pass smaller ones):
  small_u8     10,000 x 128 uint8, 50 isotropic components, centres U[32,224],
               sigma 20, round-half-even and clip to [0,255]; 100 queries from
               the same mixture.
  shift_f32    1,000,000 x 128 fp32, 1,000 components; dimension i carries a
               global scale g_i = (1+i)^-0.5 (descriptor-like data have a low
               intrinsic dimension; with independent equal-variance
               dimensions, RNG-pruned k-NN graphs in 128-d fragment into many
               unreachable nodes), centres g * N(0, I) and per-dimension
               scales g * LogNormal(0, 0.5); queries from the
               same centres moved by a per-component shift N(0, (0.5 sigma)^2)
               and reweighted so that 5% of the components carry 80% of the
               queries; 10,000 evaluation + 100,000 training queries.
  highdim_f32  1,000,000 x 960 fp32, 500 components, x = c + A z64 + 0.1 eps
               (A: 960x64 with N(0, 1/64) entries); queries with a global mean
               shift N(0, 0.5^2 I).
  ip_f32       1,000,000 x 200 unit vectors, 2,000 components
               x = normalise(mu + 0.05 z); queries from a different mixture:
               30% of the centres rotated by one Haar-random rotation, noise
               variance doubled.
  batch_f32    10,000,000 x 96 fp32, 10,000 components N(0, 4^2 I), sigma 1;
               100,000 queries, half in-distribution, half shifted as in
               shift_f32; per-query k uniform on {1, 10, 100} and L uniform
               on the integers [max(32, k), 512].
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20250615


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def _chunks(n, size=1 << 18):
    for s in range(0, n, size):
        yield s, min(n, s + size)


def small_u8(n=10_000, nq=100, d=128, n_comp=50, seed=SEED_BASE + 1):
    rng = _rng(seed)
    centres = rng.uniform(32.0, 224.0, size=(n_comp, d))

    def draw(m):
        comp = rng.integers(0, n_comp, size=m)
        x = centres[comp] + 20.0 * rng.standard_normal((m, d))
        return np.clip(np.rint(x), 0, 255).astype(np.uint8)

    base = draw(n)
    queries = draw(nq)
    return dict(base=base, queries=queries)


def shift_f32(n=1_000_000, nq=10_000, n_train=100_000, d=128, n_comp=1000,
              hot_frac=0.05, hot_mass=0.8, centre_scale=1.0, spectrum=0.5,
              seed=SEED_BASE + 2):
    rng = _rng(seed)
    # global variance spectrum: dimension i has scale (1 + i)^-spectrum, which
    # gives descriptor-like data a low intrinsic dimension (about 18 for 0.5)
    g = (1.0 + np.arange(d)) ** (-spectrum)
    centres = (rng.normal(0.0, centre_scale, size=(n_comp, d)) * g).astype(np.float32)
    scales = (rng.lognormal(0.0, 0.5, size=(n_comp, d)) * g).astype(np.float32)
    shifts = (rng.standard_normal((n_comp, d)) * 0.5 * scales).astype(np.float32)
    n_hot = max(1, int(round(hot_frac * n_comp)))
    hot = rng.permutation(n_comp)[:n_hot]
    p = np.full(n_comp, (1.0 - hot_mass) / max(1, n_comp - n_hot))
    p[hot] = hot_mass / n_hot
    p /= p.sum()

    base = np.empty((n, d), np.float32)
    for s, e in _chunks(n):
        comp = rng.integers(0, n_comp, size=e - s)
        z = rng.standard_normal((e - s, d), dtype=np.float32)
        base[s:e] = centres[comp] + scales[comp] * z

    def queries(m):
        comp = rng.choice(n_comp, size=m, p=p)
        z = rng.standard_normal((m, d), dtype=np.float32)
        return (centres[comp] + shifts[comp] + scales[comp] * z).astype(np.float32)

    q = queries(nq)
    train = queries(n_train) if n_train else np.empty((0, d), np.float32)
    return dict(base=base, queries=q, train=train)


def _spectrum(d, exponent):
    """Global per-dimension scale (1 + i)^-exponent: descriptor-like data with
    a low intrinsic dimension, on which proximity graphs stay navigable."""
    return ((1.0 + np.arange(d)) ** (-exponent)).astype(np.float32)


def highdim_f32(n=1_000_000, nq=1_000, d=960, rank=64, n_comp=500, centre_scale=0.5,
                spectrum=0.5, noise=0.1, seed=SEED_BASE + 3):
    """GIST-shaped rows: a mixture of rank-64 Gaussians plus isotropic noise,
    all under the global spectrum; queries shifted by one global offset."""
    rng = _rng(seed)
    g = _spectrum(d, spectrum)
    centres = (rng.normal(0.0, centre_scale, size=(n_comp, d)) * g).astype(np.float32)
    A = (rng.standard_normal((n_comp, d, rank)) / np.sqrt(rank)).astype(np.float32)
    A *= g[None, :, None]
    comp = rng.integers(0, n_comp, size=n)
    base = np.empty((n, d), np.float32)
    for s, e in _chunks(n, 1 << 15):
        c = comp[s:e]
        zl = rng.standard_normal((e - s, rank), dtype=np.float32)
        eps = rng.standard_normal((e - s, d), dtype=np.float32)
        low = np.einsum("ndr,nr->nd", A[c], zl, optimize=True)
        base[s:e] = centres[c] + low + noise * g * eps
    shift = (rng.normal(0.0, 0.5 * centre_scale, size=d) * g).astype(np.float32)
    qc = rng.integers(0, n_comp, size=nq)
    zl = rng.standard_normal((nq, rank), dtype=np.float32)
    eps = rng.standard_normal((nq, d), dtype=np.float32)
    q = centres[qc] + np.einsum("ndr,nr->nd", A[qc], zl) + noise * g * eps + shift
    return dict(base=base, queries=q.astype(np.float32))


def _normalise(x):
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def ip_f32(n=1_000_000, nq=10_000, n_train=0, d=200, n_comp=2000, noise=0.5, spectrum=0.5,
           rot_frac=0.3, seed=SEED_BASE + 4):
    """Unit rows around normalised centres (von Mises-Fisher-like), all under
    the global spectrum; queries from a different mixture: a Haar rotation of
    30% of the centres and twice the noise variance."""
    rng = _rng(seed)
    g = _spectrum(d, spectrum)
    mu = _normalise(rng.standard_normal((n_comp, d)) * g)
    base = np.empty((n, d), np.float32)
    for s, e in _chunks(n):
        comp = rng.integers(0, n_comp, size=e - s)
        z = rng.standard_normal((e - s, d), dtype=np.float32)
        base[s:e] = _normalise(mu[comp] + noise * g * z)
    # Haar rotation: QR of a Gaussian matrix with the sign fix on R's diagonal
    gm = rng.standard_normal((d, d))
    Qm, Rm = np.linalg.qr(gm)
    Qm = Qm * np.sign(np.diag(Rm))[None, :]
    mu_q = mu.copy()
    rot = rng.permutation(n_comp)[: int(round(rot_frac * n_comp))]
    mu_q[rot] = _normalise(mu[rot] @ Qm.T)

    def queries(m):
        comp = rng.integers(0, n_comp, size=m)
        z = rng.standard_normal((m, d), dtype=np.float32)
        return _normalise(mu_q[comp] + np.sqrt(2.0) * noise * g * z)

    q = queries(nq)
    train = queries(n_train) if n_train else np.empty((0, d), np.float32)
    return dict(base=base, queries=q, train=train)


def batch_f32(n=10_000_000, nq=100_000, n_train=0, d=96, n_comp=10_000, centre_scale=1.0, spectrum=0.5,
              seed=SEED_BASE + 5):
    """The shifted-mixture law of shift_f32 at d = 96 with 10,000 components;
    half of the query stream shifted; per-query k in {1, 10, 100} and L
    uniform in [max(32, k), 512]; training queries from the same law as the
    stream (half shifted), drawn after everything else."""
    rng = _rng(seed)
    g = _spectrum(d, spectrum)
    centres = (rng.normal(0.0, centre_scale, size=(n_comp, d)) * g).astype(np.float32)
    scales = (rng.lognormal(0.0, 0.5, size=(n_comp, d)) * g).astype(np.float32)
    shifts = (0.5 * rng.standard_normal((n_comp, d)) * scales).astype(np.float32)
    base = np.empty((n, d), np.float32)
    for s, e in _chunks(n):
        comp = rng.integers(0, n_comp, size=e - s)
        base[s:e] = centres[comp] + scales[comp] * rng.standard_normal((e - s, d), dtype=np.float32)
    comp = rng.integers(0, n_comp, size=nq)
    q = centres[comp] + scales[comp] * rng.standard_normal((nq, d), dtype=np.float32)
    shifted = np.arange(nq) >= nq // 2
    q[shifted] += shifts[comp[shifted]]
    k = rng.choice(np.array([1, 10, 100], np.int32), size=nq)
    lo = np.maximum(32, k)
    L = (lo + np.floor(rng.random(nq) * (513 - lo))).astype(np.int32)
    train = np.empty((0, d), np.float32)
    if n_train:
        tc = rng.integers(0, n_comp, size=n_train)
        train = centres[tc] + scales[tc] * rng.standard_normal((n_train, d), dtype=np.float32)
        train[n_train // 2:] += shifts[tc[n_train // 2:]]
        train = train.astype(np.float32)
    return dict(base=base, queries=q.astype(np.float32), k=k.astype(np.int32), L=L, train=train)


def kmeans_init(m, k, seed):
    """k distinct row indices of an m-row sample (k-means initial centroids)."""
    return _rng(seed).permutation(m)[:k].astype(np.int32)


def fusion_init(dp, dU, heads, dk, out=64, seed=SEED_BASE + 101):
    """Initial fusion-attention weights (Eq. fusion): WQ [dp, heads*dk],
    WK and WV [dU, heads*dk], WO [heads*dk, out], Glorot-scaled normal draws;
    WO starts small so that the hub rows start near the free embeddings."""
    rng = _rng(seed)
    E = heads * dk
    WQ = rng.standard_normal((dp, E)) / np.sqrt(dp)
    WK = rng.standard_normal((dU, E)) / np.sqrt(dU)
    WV = rng.standard_normal((dU, E)) / np.sqrt(dU)
    WO = 0.1 * rng.standard_normal((E, out)) / np.sqrt(E)
    return tuple(w.astype(np.float32) for w in (WQ, WK, WV, WO))


def hbkm_keys(n, seed):
    """One uniform uint32 key per row: the draw from which hierarchical
    balanced k-means takes each split's initial centroids (the members with
    the smallest keys)."""
    return _rng(seed).integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)


def sample_rows(n, m, seed):
    """m distinct row indices out of n, sorted (k-means training sample)."""
    if m >= n:
        return np.arange(n, dtype=np.int64)
    return np.sort(_rng(seed).choice(n, size=m, replace=False)).astype(np.int64)


def hub_sample(n_hubs, m, seed=SEED_BASE + 102):
    """m distinct hub indices out of n_hubs, in draw order: the random node
    sample that starts the hub-graph search (Algorithm 1's initial set)."""
    return _rng(seed).permutation(n_hubs)[:min(m, n_hubs)].astype(np.int32)


def train_batches(n_train, batch, epochs, seed):
    """Per-epoch random permutations of the training queries."""
    rng = _rng(seed)
    return [rng.permutation(n_train).astype(np.int32) for _ in range(epochs)]


def model_init(in_dim, n_hubs, hidden=256, out=64, seed=SEED_BASE + 100):
    """Initial two-tower parameters: He-normal W1, W2 (zero biases) and
    standard-normal hub embeddings."""
    rng = _rng(seed)
    W1 = (rng.standard_normal((in_dim, hidden)) * np.sqrt(2.0 / in_dim)).astype(np.float32)
    b1 = np.zeros(hidden, np.float32)
    W2 = (rng.standard_normal((hidden, out)) * np.sqrt(2.0 / hidden)).astype(np.float32)
    b2 = np.zeros(out, np.float32)
    E = rng.standard_normal((n_hubs, out)).astype(np.float32)
    return W1, b1, W2, b2, E
