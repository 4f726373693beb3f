"""Input generators (CPU): determinism, shapes and the stated distributions."""
import numpy as np

from paper_2603_00326_b300 import datagen as G


def test_trunk_recipe():
    a = G.trunk(n=20000, p=40, seed=5)
    b = G.trunk(n=20000, p=40, seed=5)
    assert a.X.shape == (40, 20000) and a.X.dtype == np.float32 and a.n_classes == 2
    np.testing.assert_array_equal(a.X, b.X)
    np.testing.assert_array_equal(a.y, b.y)
    assert int(a.y.sum()) == 10000  # exactly balanced
    for f in (0, 3, 39):
        mu = 1.0 / np.sqrt(f + 1.0)
        m0 = a.X[f][a.y == 0].mean()
        m1 = a.X[f][a.y == 1].mean()
        assert abs(m0 - mu) < 0.05 and abs(m1 + mu) < 0.05
        assert abs(a.X[f][a.y == 0].std() - 1.0) < 0.05


def test_wide_counts_recipe():
    a = G.wide_counts(n=5000, d=128, seed=7)
    b = G.wide_counts(n=5000, d=128, seed=7)
    np.testing.assert_array_equal(a.X, b.X)
    zero = (a.X == 0).mean()
    assert 0.88 < zero < 0.92
    nz = a.X[a.X != 0]
    assert nz.min() >= 1 and abs(nz.mean() - 3.0 / (1 - np.exp(-3.0))) < 0.1  # zero-truncated Poisson(3)
    assert set(np.unique(a.y)) <= set(range(5))
