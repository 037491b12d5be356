"""GPU parity of hierarchical balanced k-means (Sec. 4.1, Def. 2, Algorithm 2)
and its hubs (Def. 3) against the oracle.  Both sides decide memberships in
float32 with every operation rounded on its own and the same summation
orders, so labels, centroids and hubs must agree bit for bit; at the bench's
full size (1M x 128, 1,024 hubs) the invariants that hold at any size are
checked instead."""
import numpy as np
import pytest

import oracle
from paper_2506_15986_gb300 import ann, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)
DEV = torch.device("cuda:0")


def _gpu(x, k, levels, lam, T, keys):
    n, d = x.shape
    nc = k ** levels
    dx = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(DEV)
    dk = torch.from_numpy(keys.view(np.int32)).to(DEV)
    hubs = torch.empty(nc, dtype=torch.int32, device=DEV)
    cent = torch.empty((nc, d), dtype=torch.float32, device=DEV)
    lab = torch.empty(n, dtype=torch.int32, device=DEV)
    ann.ann_hbkm(dx, n, d, k, levels, lam, T, dk, hubs, cent, lab)
    return lab.cpu().numpy(), cent.cpu().numpy(), hubs.cpu().numpy()


def _same(x, k, levels, lam, T, keys):
    gl, gc, gh = _gpu(x, k, levels, lam, T, keys)
    ol, oc, oh, osz = oracle.hbkm(x, k, levels, lam, T, keys)
    assert np.array_equal(gl, ol)
    assert np.array_equal(gc.view(np.uint32), oc.view(np.uint32))  # bit for bit
    assert np.array_equal(gh, oh)
    return ol, osz


@pytest.mark.parametrize("k,levels,lam,T", [(4, 3, 1.0, 4), (4, 3, 0.0, 3), (2, 5, 1e12, 2)])
def test_matches_oracle_bit_for_bit(k, levels, lam, T):
    w = synth.shift_f32(n=20011, nq=1, n_train=0)  # ragged: no power of k
    keys = synth.hbkm_keys(20011, seed=7)
    lab, sizes = _same(w["base"], k, levels, lam, T, keys)
    if lam > 1e6:
        part = sizes.reshape(-1, k)
        assert (part.max(1) - part.min(1) <= 1).all()


@pytest.mark.parametrize("n", [9000, 600])
def test_wide_branching(n):
    # k = 32, two levels, 1,024 clusters; at 600 rows the first level's
    # children hold about 19 rows, fewer than k, so second-level children stay
    # empty
    w = synth.shift_f32(n=n, nq=1, n_train=0)
    keys = synth.hbkm_keys(n, seed=8)
    lab, sizes = _same(w["base"], 32, 2, 0.5, 3, keys)
    if n < 32 * 32:
        assert (sizes == 0).any()


def test_fewer_rows_than_clusters():
    x = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [2, 0, 0, 0], [10, 0, 0, 0], [20, 0, 0, 0]], np.float32)
    keys = np.array([4, 3, 2, 1, 0], np.uint32)
    lab, sizes = _same(x, 3, 2, 0.0, 3, keys)
    assert sizes.sum() == 5


def test_invalid_arguments():
    x = torch.zeros((16, 8), dtype=torch.float32, device=DEV)
    keys = torch.zeros(16, dtype=torch.int32, device=DEV)
    hubs = torch.empty(4096, dtype=torch.int32, device=DEV)
    for k, levels, dim, T in ((1, 2, 8, 1), (33, 1, 8, 1), (2, 21, 8, 1), (2, 2, 6, 1), (2, 2, 8, 0)):
        with pytest.raises(ann.AnnError) as e:
            ann.ann_hbkm(x, 16, dim, k, levels, 1.0, T, keys, hubs)
        assert e.value.status == ann.ERR_INVALID_ARG
    with pytest.raises(ann.AnnError):
        ann.ann_hbkm(x, 16, 8, 2, 2, -1.0, 1, keys, hubs)


def test_full_size_invariants():
    # the bench's hub extraction: 1M x 128 rows, k = 32, two levels, T = 10
    w = synth.shift_f32(n=1_000_000, nq=1, n_train=0)
    x = w["base"]
    keys = synth.hbkm_keys(len(x), seed=synth.SEED_BASE + 13)
    lab, cent, hubs = _gpu(x, 32, 2, 1.0, 10, keys)
    sizes = np.bincount(lab, minlength=1024)
    assert sizes.sum() == len(x) and lab.min() >= 0 and lab.max() < 1024
    assert ((hubs >= 0) == (sizes > 0)).all()
    assert (lab[hubs[hubs >= 0]] == np.nonzero(sizes > 0)[0]).all()  # a hub is a member
    # balance: sizes within a factor of the target for almost every cluster
    assert np.mean(np.abs(sizes - len(x) / 1024) <= 0.5 * len(x) / 1024) >= 0.95
    # each centroid is its members' mean; each hub is its member nearest it
    order = np.argsort(lab, kind="stable")
    bounds = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(0)
    for c in rng.choice(np.nonzero(sizes)[0], 64, replace=False):
        mem = order[bounds[c]:bounds[c + 1]]
        xd = x[mem].astype(np.float64)
        np.testing.assert_allclose(cent[c], xd.mean(0), rtol=1e-3, atol=1e-3)
        d = ((xd - cent[c].astype(np.float64)) ** 2).sum(1)
        assert d[mem == hubs[c]][0] <= d.min() * (1 + 1e-4) + 1e-5
