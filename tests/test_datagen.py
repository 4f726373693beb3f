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


def test_tree_small_recipe():
    """N(0,1) features; labels = [sum of 4 distinct features > 0] with exactly 5% flipped."""
    a = G.tree_small(n=4000, d=16, seed=11)
    b = G.tree_small(n=4000, d=16, seed=11)
    np.testing.assert_array_equal(a.X, b.X)
    np.testing.assert_array_equal(a.y, b.y)
    assert a.X.shape == (16, 4000) and a.n_classes == 2
    assert abs(a.X.mean()) < 0.02 and abs(a.X.std() - 1.0) < 0.02
    # the rule's four features stand out by their correlation with the label
    corr = np.array([np.corrcoef(a.X[f], a.y)[0, 1] for f in range(16)])
    S = np.sort(np.argsort(-np.abs(corr))[:4])
    assert np.abs(corr[S]).min() > 5 * np.abs(np.delete(corr, S)).max()
    score = np.zeros(4000)
    for f in S:
        score += a.X[f].astype(np.float64)
    assert int(((score > 0).astype(np.uint8) != a.y).sum()) == 200  # exactly 5% flipped


def test_forest_2m_recipe():
    """lognormal(0,1) features; labels = median split of an 8-sparse +-1 score, exactly 10% flipped."""
    a = G.forest_2m(n=20000, d=24, seed=12)
    assert a.X.shape == (24, 20000) and a.X.min() > 0
    lx = np.log(a.X.astype(np.float64))
    assert abs(lx.mean()) < 0.02 and abs(lx.std() - 1.0) < 0.02
    # the median split labels exactly half before the flips; 10% flips keep the mean near 1/2
    assert abs(a.y.mean() - 0.5) < 0.01
    corr = np.array([np.corrcoef(a.X[f], a.y)[0, 1] for f in range(24)])
    assert int((np.abs(corr) > 0.1).sum()) == 8  # eight features carry the signal


def test_root_4m_recipe():
    """Three classes from the argmax of three 4-sparse +-1 scores plus N(0, 0.5^2) noise."""
    a = G.root_4m(n=30000, d=20, seed=13)
    assert a.n_classes == 3 and a.X.shape == (20, 30000)
    frac = np.bincount(a.y, minlength=3) / 30000.0
    assert frac.min() > 0.2 and frac.max() < 0.5
    corr = np.array([[np.corrcoef(a.X[f], a.y == c)[0, 1] for f in range(20)] for c in range(3)])
    assert 4 <= int((np.abs(corr).max(axis=0) > 0.1).sum()) <= 12  # at most 3 x 4 features carry signal


def test_frontier_nodes_recipe():
    """Consecutive chunks of a permutation, each sorted; lognormal(5, 2) sizes summing to n."""
    n, m = 200000, 1024
    idx, off = G.frontier_nodes(n, m, seed=14)
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 1)
    np.testing.assert_array_equal(np.sort(idx), np.arange(n))
    for j in range(m):
        seg = idx[off[j]:off[j + 1]]
        assert np.all(np.diff(seg) > 0)
    # with about 2400 samples a node the rescaled sizes keep the lognormal spread of their logs
    # (smaller means are cut by the rounding and the floor of one sample)
    s2 = G.lognormal_node_sizes(np.random.default_rng(3), 4096, 10 ** 7)
    assert int(s2.sum()) == 10 ** 7 and s2.min() >= 1
    assert abs(np.log(s2).std() - 2.0) < 0.1


def test_bootstrap_indices_recipe():
    """n draws with replacement, sorted, seeded per tree: about 1 - 1/e distinct samples."""
    n = 100000
    a = G.bootstrap_indices(n, 3)
    assert a.shape == (n,) and a.dtype == np.int32 and np.all(np.diff(a) >= 0)
    assert a.min() >= 0 and a.max() < n
    assert abs(len(np.unique(a)) / n - (1 - np.exp(-1))) < 0.01
    np.testing.assert_array_equal(a, G.bootstrap_indices(n, 3))
    assert not np.array_equal(a, G.bootstrap_indices(n, 4))
    assert G.bootstrap_indices(n, 3, n_draws=500).shape == (500,)


def test_random_projections_recipe():
    """nnz = min(cap, d, 1 + Poisson(lam)); distinct sorted features; +-1 signs."""
    rng = np.random.default_rng(15)
    P, d, lam, cap = 20000, 64, 1.5, 4
    pr = G.random_projections(rng, P, d, lam, cap)
    nnz = np.diff(pr.ptr)
    assert nnz.min() >= 1 and nnz.max() == cap
    # P(nnz = k) for k < cap is the Poisson mass at k - 1; the cap collects the tail
    from math import exp, factorial
    for k in range(1, cap):
        p = exp(-lam) * lam ** (k - 1) / factorial(k - 1)
        assert abs((nnz == k).mean() - p) < 4 * np.sqrt(p * (1 - p) / P)
    for p_ in range(0, P, 997):
        f = pr.feat[pr.ptr[p_]:pr.ptr[p_ + 1]]
        assert np.all(np.diff(f) > 0) and f.min() >= 0 and f.max() < d
    assert set(np.unique(pr.sign)) == {-1, 1} and abs(pr.sign.mean()) < 0.02
    narrow = G.random_projections(np.random.default_rng(1), 500, 2, 3.0, 8)
    assert np.diff(narrow.ptr).max() == 2  # never more non-zeros than features


def test_trunk_streamed_equals_trunk():
    """The block-streamed Trunk generator hands over exactly trunk()'s values."""
    n, p = 5000, 150
    ref = G.trunk(n=n, p=p)
    X = np.full((p, n), np.nan, dtype=np.float32)

    def fill(f0, blk):
        X[f0:f0 + blk.shape[0]] = blk

    y = G.trunk_streamed(n, p, fill, workers=3)
    np.testing.assert_array_equal(y, ref.y)
    np.testing.assert_array_equal(X.view(np.uint32), ref.X.view(np.uint32))
