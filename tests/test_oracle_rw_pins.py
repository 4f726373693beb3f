"""Pins of the oracle's random-width histogram (reading R14; the paper's
Section 1 footnote: YDF's bin boundaries sit at random-width intervals).

The boundaries are checked against the order statistics of uniform draws, the
exact grid they live on, exact power-of-two scaling and the splitmix64 stream
they come from; the split search that uses them against exact-rational brute
force and a library bin routine; the threaded search and the tree against the
plain search.  Nothing here needs a GPU.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import brute
from tests.test_oracle_pins import _check_against_brute
from tests.tree_check import route_and_sample

TAG = 0x6A09E667F3BCC908  # first 64 fractional bits of sqrt(2)
MULT = 0xD2B74407B1CE6E93
M64 = (1 << 64) - 1


def test_tag_is_sqrt2_fraction():
    # the stream tag is a nothing-up-my-sleeve number: frac(sqrt(2)) * 2^64
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    frac = Decimal(2).sqrt() - 1
    assert int(frac * (1 << 64)) == TAG


def test_rw_grid_and_stream():
    """On [0, 1] every boundary is (2u+1) 2^-24 for the top 23 bits u of one
    output of the splitmix64 stream at state sm64((key ^ TAG) + p*MULT), and
    the boundaries are those draws in ascending order."""
    for key, p, B in ((0, 0, 256), (123456789, 7, 256), (M64, 1023, 17), (42, 3, 2)):
        t = O.rw_boundaries(key, p, 0.0, 1.0, B).astype(np.float64)
        g = t * 2.0 ** 24
        assert np.all(g == np.round(g)) and np.all(g % 2 == 1) and np.all((g >= 1) & (g < 2 ** 24))
        assert np.all(np.diff(t) >= 0)
        st = O.sm64(((key ^ TAG) + p * MULT) & M64)
        u = []
        for _ in range(B - 1):
            r, st = O.sm64_next(st)
            u.append(r >> 41)
        np.testing.assert_array_equal(g, np.sort(2.0 * np.array(u, dtype=np.float64) + 1.0))


def test_rw_power_of_two_scaling_is_exact():
    base = O.rw_boundaries(99, 5, 0.0, 1.0, 256)
    for k in (-20, -3, 1, 7, 30):
        s = np.float32(2.0 ** k)
        np.testing.assert_array_equal(O.rw_boundaries(99, 5, 0.0, float(s), 256), base * s)


def test_rw_order_statistics():
    """The j-th of B-1 sorted uniforms has mean j/B; pooled draws are uniform;
    streams of neighbouring projections and keys are uncorrelated."""
    B, K = 256, 3000
    F = np.stack([O.rw_boundaries(int(k) * 0x9E3779B97F4A7C15 & M64, 0, 0.0, 1.0, B) for k in range(K)])
    F = F.astype(np.float64)
    mean = F.mean(0)
    np.testing.assert_allclose(mean, np.arange(1, B) / B, atol=0.004)
    pooled = np.sort(F.ravel())
    ecdf = np.arange(1, pooled.size + 1) / pooled.size
    assert np.max(np.abs(ecdf - pooled)) < 0.003  # Kolmogorov-Smirnov distance to U(0, 1)
    F1 = np.stack([O.rw_boundaries(int(k) * 0x9E3779B97F4A7C15 & M64, 1, 0.0, 1.0, B) for k in range(K)])
    for j in (0, 127, 254):
        assert abs(np.corrcoef(F[:, j], F1[:, j])[0, 1]) < 0.09
        assert abs(np.corrcoef(F[:-1, j], F[1:, j])[0, 1]) < 0.09
    # two boundaries of one projection: the single-boundary case is a plain uniform
    one = np.array([O.rw_boundaries(k, 2, 0.0, 1.0, 2)[0] for k in range(K)], dtype=np.float64)
    assert abs(one.mean() - 0.5) < 0.02 and abs(one.var() - 1 / 12) < 0.01


def test_rw_range_and_degenerate():
    for mn, mx in ((-3.0, 4.5), (1e-3, 1e-3 + 1e-7), (-1e30, 1e30), (2.0, 2.0)):
        mn, mx = np.float32(mn), np.float32(mx)
        t = O.rw_boundaries(5, 0, float(mn), float(mx), 256)
        assert np.all(np.diff(t) >= 0)
        assert t[0] >= mn and t[-1] <= np.nextafter(mx, np.float32(np.inf))
    t = O.rw_boundaries(5, 0, 2.0, 2.0, 256)
    assert np.all(t == np.float32(2.0))  # zero range: every boundary at the value, no candidate


def test_rw_histogram_is_upper_bound_count():
    ds = G.tree_small(n=3000, d=12, seed=11)
    rng = np.random.default_rng(3)
    pr = G.random_projections(rng, 6, ds.d, 1.5, 8)
    idx = np.sort(rng.choice(ds.n, 2500, replace=False)).astype(np.int32)
    key = 0xDEADBEEF12345678
    r = O.split_search(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, hist_only=True, want_debug=True,
                       bin_rule=1, bin_key=key)
    e = O.split_search(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, hist_only=True, want_debug=True)
    N = np.bincount(ds.y[idx], minlength=2)
    for p in range(6):
        v = O.project(ds.X, idx, pr.feat[pr.ptr[p]:pr.ptr[p + 1]], pr.sign[pr.ptr[p]:pr.ptr[p + 1]])
        t = O.rw_boundaries(key, p, v.min(), v.max(), 256)
        np.testing.assert_array_equal(r.bounds[p], t)
        b = np.searchsorted(t, v, side="right")  # library routine over the same boundaries
        H = np.zeros((256, 2), dtype=np.int64)
        np.add.at(H, (b, ds.y[idx]), 1)
        np.testing.assert_array_equal(r.hist[p], H)
        np.testing.assert_array_equal(r.hist[p].sum(0), N)
        assert not np.array_equal(r.hist[p], e.hist[p])  # the rule changes the bins
    # the equal-width debug boundaries are R2's
    np.testing.assert_array_equal(e.bounds[0], O.boundaries(e.minmax[0, 0], e.minmax[0, 1], 256))


@pytest.mark.parametrize("seed", range(30))
def test_rw_hist_path_brute_force(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(2, 14))
    d = 4
    C = int(rng.integers(2, 4))
    B = int(rng.choice([2, 3, 4, 8, 16, 64]))
    X = rng.standard_normal((d, 30)).astype(np.float32)
    if seed % 3 == 0:
        X = np.round(X)  # ties
    y = rng.integers(0, C, 30).astype(np.uint8)
    idx = rng.choice(30, n, replace=True).astype(np.int32)
    pr = G.random_projections(rng, 5, d, 1.5, 3)
    key = int(rng.integers(0, 2 ** 63)) * 2 + 1
    r = O.split_search(X, y, C, idx, pr.ptr, pr.feat, pr.sign, n_bins=B, hist_only=True, want_debug=True,
                       bin_rule=1, bin_key=key)
    assert r.path == 0
    cands = []
    for p in range(5):
        f, s = pr.feat[pr.ptr[p]:pr.ptr[p + 1]], pr.sign[pr.ptr[p]:pr.ptr[p + 1]]
        v = O.project(X, idx, f, s)
        t = O.rw_boundaries(key, p, v.min(), v.max(), B)
        for (b, left, g) in brute.hist_path_candidates(v, y[idx], C, t):
            cands.append((p, b, left, g))
    _check_against_brute(r, cands, 5)
    if r.valid:
        t = O.rw_boundaries(key, r.proj, r.minmax[r.proj, 0], r.minmax[r.proj, 1], B)
        assert r.threshold == t[r.cand]


def test_rw_threaded_equals_plain():
    """Each thread's projection sub-range draws the streams of its global
    projection indices, so the threaded search is the plain one."""
    ds = G.tree_small(n=3000, d=12, seed=15)
    rng = np.random.default_rng(2)
    pr = G.random_projections(rng, 29, 12, 1.5, 8)
    idx = G.all_indices(ds.n)
    key = 0x0123456789ABCDEF
    a = O.split_search(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, hist_only=True, bin_rule=1, bin_key=key)
    assert a.valid
    for nt in (2, 5, 29):
        b = O.split_search_mt(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, hist_only=True, n_threads=nt,
                              bin_rule=1, bin_key=key)
        assert (a.valid, a.proj, a.cand, a.n_left) == (b.valid, b.proj, b.cand, b.n_left)
        assert np.float32(a.threshold).tobytes() == np.float32(b.threshold).tobytes()
        assert np.float64(a.gain).tobytes() == np.float64(b.gain).tobytes()


def test_rw_tree_every_node_re_searched():
    """A random-width tree passes the node checker with every node searched
    again from its own key, and differs from the equal-width tree."""
    ds = G.tree_small(n=1500, d=12, seed=71)
    root = G.bootstrap_indices(ds.n, 2, seed=9)
    kw = dict(n_proj=12, lam=1.5, cap=8, n_bins=64, sort_below=200, seed=4, tree_id=2)
    t = O.train_tree(ds.X, ds.y, 2, root, bin_rule=1, **kw)
    assert t.n_nodes > 30 and set(np.unique(t.path)) >= {-1, 0, 1}
    n = route_and_sample(t, ds.X, ds.y, 2, root, check_ids=range(t.n_nodes), bin_rule=1, **kw)
    assert n == int(np.count_nonzero(t.path >= 0))
    e = O.train_tree(ds.X, ds.y, 2, root, **kw)
    assert t.threshold[0] != e.threshold[0] or t.n_nodes != e.n_nodes
    with pytest.raises(AssertionError):  # checked under the wrong rule, the tree fails
        route_and_sample(t, ds.X, ds.y, 2, root, check_ids=[0], bin_rule=0, **kw)
