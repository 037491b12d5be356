"""The seeded draws that method steps take as inputs (CPU)."""
import numpy as np

from paper_2506_15986_gb300 import synth


def test_hub_sample_is_a_seeded_set_of_distinct_hubs():
    a = synth.hub_sample(1024, 32)
    assert a.dtype == np.int32 and len(a) == 32 and len(set(a.tolist())) == 32
    assert a.min() >= 0 and a.max() < 1024
    assert np.array_equal(a, synth.hub_sample(1024, 32))          # same seed, same sample
    assert not np.array_equal(a, synth.hub_sample(1024, 32, seed=7))
    assert np.array_equal(synth.hub_sample(1024, 8), a[:8])         # a prefix of one permutation
    assert sorted(synth.hub_sample(5, 32).tolist()) == [0, 1, 2, 3, 4]  # never more than the hubs


def test_kmeans_init_and_sample_rows():
    init = synth.kmeans_init(1000, 50, seed=3)
    assert len(set(init.tolist())) == 50 and init.max() < 1000
    rows = synth.sample_rows(10_000, 500, seed=4)
    assert len(rows) == 500 and (np.diff(rows) > 0).all()
    assert np.array_equal(synth.sample_rows(100, 500, seed=4), np.arange(100))
