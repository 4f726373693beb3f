"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test checks the oracle against a published value, a closed form, a
textbook/library routine, an invariant, or exact-rational brute force, so that
a dropped term, a wrong sign or index, or a transposed operand fails one of
them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Random streams
# --------------------------------------------------------------------------

def test_splitmix64_published_vector():
    """splitmix64 from state 1234567: the first five outputs quoted with the
    generator's reference implementation (Vigna's splitmix64.c test vector)."""
    expected = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                4593380528125082431, 16408922859458223821]
    s = 1234567
    got = []
    for _ in range(5):
        r, s = O.sm64_next(s)
        got.append(r)
    assert got == expected


def test_poisson_cdf_matches_closed_form():
    from scipy.stats import poisson
    for lam, cap in [(1.5, 8), (3.0, 16), (0.5, 4)]:
        cdf = O.poisson_cdf(lam, cap)
        ref = poisson.cdf(np.arange(cap - 1), lam)
        np.testing.assert_allclose(cdf, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("lam,cap,d", [(1.5, 8, 64), (3.0, 16, 4096), (1.5, 8, 5)])
def test_sampler_law(lam, cap, d):
    """nnz ~ min(cap, d, 1+Poisson(lam)); features distinct, ascending, uniform;
    signs fair.  Chi-square on many nodes."""
    from scipy.stats import chisquare, poisson
    P = 256
    counts = np.zeros(cap + 1, dtype=np.int64)
    feat_hits = np.zeros(d, dtype=np.int64)
    pos = neg = 0
    for node in range(200):
        nnz, feat, sign = O.sample_node(O.sm64(node), P, d, lam, cap)
        for p in range(P):
            k = nnz[p]
            f = feat[p, :k]
            assert 1 <= k <= min(cap, d)
            assert np.all(np.diff(f) > 0), "features must be distinct and ascending"
            assert f.min() >= 0 and f.max() < d
            feat_hits[f] += 1
            s = sign[p, :k]
            assert set(np.unique(s)).issubset({-1, 1})
            pos += int((s == 1).sum())
            neg += int((s == -1).sum())
            counts[k] += 1
    # law of nnz
    kmax = min(cap, d)
    probs = np.array([poisson.pmf(k - 1, lam) for k in range(1, kmax)])
    probs = np.append(probs, 1.0 - probs.sum())
    obs = counts[1:kmax + 1]
    exp = probs * obs.sum()
    keep = exp > 5
    obs_k = np.append(obs[keep], obs[~keep].sum())
    exp_k = np.append(exp[keep], exp[~keep].sum())
    if exp_k[-1] == 0:
        obs_k, exp_k = obs_k[:-1], exp_k[:-1]
    assert chisquare(obs_k, exp_k).pvalue > 1e-4
    # sign balance
    tot = pos + neg
    assert abs(pos - tot / 2) < 5 * math.sqrt(tot / 4)
    # marginal uniformity of chosen features
    if d <= 64:
        assert chisquare(feat_hits).pvalue > 1e-4


def test_sampler_deterministic_and_key_sensitive():
    a = O.sample_node(123, 16, 50, 1.5, 8)
    b = O.sample_node(123, 16, 50, 1.5, 8)
    c = O.sample_node(124, 16, 50, 1.5, 8)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert not all(np.array_equal(x, y) for x, y in zip(a, c))


def test_floyd_uniform_subsets():
    """Floyd's algorithm draws every k-subset with equal probability: for d=5,
    k=2 (forced by cap=2 and a Poisson draw of >=1) all 10 pairs are equally likely."""
    from scipy.stats import chisquare
    hits = {}
    for node in range(3000):
        nnz, feat, _ = O.sample_node(O.sm64(node * 7 + 1), 8, 5, 50.0, 2)
        for p in range(8):
            assert nnz[p] == 2
            key = tuple(feat[p, :2])
            hits[key] = hits.get(key, 0) + 1
    assert len(hits) == 10
    assert chisquare(np.array(list(hits.values()))).pvalue > 1e-4


# --------------------------------------------------------------------------
# Step 1: apply projection
# --------------------------------------------------------------------------

def test_projection_single_feature_exact_and_signed():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((4, 100)).astype(np.float32)
    idx = np.arange(100, dtype=np.int32)[::-1].copy()
    v = O.project(X, idx, np.array([2]), np.array([1]))
    np.testing.assert_array_equal(v, X[2, idx])
    v = O.project(X, idx, np.array([3]), np.array([-1]))
    np.testing.assert_array_equal(v, -X[3, idx])


def test_projection_never_negative_zero():
    X = np.array([[0.0, -0.0, 1.0], [-0.0, 0.0, -1.0]], dtype=np.float32)
    idx = np.arange(3, dtype=np.int32)
    for signs in ([1, 1], [1, -1], [-1, 1], [-1, -1]):
        v = O.project(X, idx, np.array([0, 1]), np.array(signs))
        assert not np.any(np.signbit(v) & (v == 0)), signs


def test_projection_close_to_exact_sum():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((16, 1000)).astype(np.float32)
    idx = rng.integers(0, 1000, 500).astype(np.int32)
    f = np.array([1, 4, 7, 9, 15])
    s = np.array([1, -1, -1, 1, 1])
    v = O.project(X, idx, f, s)
    exact = (s[:, None] * X[f][:, idx].astype(np.float64)).sum(0)
    scale = np.abs(X[f][:, idx]).sum(0)
    assert np.all(np.abs(v - exact) <= 4 * 2.0 ** -24 * scale + 1e-30)


def test_projection_order_is_ascending_features():
    """Float addition is not associative; the oracle adds in ascending feature
    order starting from +0.  Chosen values make the order visible."""
    X = np.array([[1e8], [1.0], [-1e8]], dtype=np.float32)
    v = O.project(X, np.array([0], np.int32), np.array([0, 1, 2]), np.array([1, 1, 1]))
    # ((0 + 1e8) + 1) + -1e8 = 0 in float (1 is lost), while another order keeps 1
    assert v[0] == np.float32(np.float32(np.float32(1e8) + np.float32(1.0)) - np.float32(1e8))
    assert v[0] == 0.0


# --------------------------------------------------------------------------
# Step 2: equal-width histogram bins
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mn,mx", [(-3.25, 4.0), (0.0, 1.0), (1.0, float(np.nextafter(np.float32(1), np.float32(2)))),
                                   (-1e-30, 1e-30), (5.0, 5.0), (-7.0, -6.9999)])
def test_bin_rule_is_upper_bound(mn, mx):
    mn, mx = np.float32(mn), np.float32(mx)
    t = O.boundaries(mn, mx, 256)
    assert np.all(np.diff(t) >= 0), "boundaries non-decreasing"
    rng = np.random.default_rng(2)
    vs = np.concatenate([t, np.nextafter(t, np.float32(-np.inf)), np.nextafter(t, np.float32(np.inf)),
                         [mn, mx], (mn + (mx - mn) * rng.random(200)).astype(np.float32)]).astype(np.float32)
    vs = vs[(vs >= mn) & (vs <= mx)]
    ref = np.searchsorted(t, vs, side="right")
    got = np.array([O.bin_of(t, float(v)) for v in vs])
    np.testing.assert_array_equal(got, ref)


def test_histogram_counts_sum_to_node():
    ds = G.tree_small(n=3000, d=12, seed=11)
    rng = np.random.default_rng(3)
    pr = G.random_projections(rng, 6, ds.d, 1.5, 8)
    idx = np.sort(rng.choice(ds.n, 2500, replace=False)).astype(np.int32)
    r = O.split_search(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, hist_only=True, want_debug=True)
    N = np.bincount(ds.y[idx], minlength=2)
    for p in range(6):
        assert r.hist[p].sum() == idx.shape[0]
        np.testing.assert_array_equal(r.hist[p].sum(0), N)
        v = O.project(ds.X, idx, pr.feat[pr.ptr[p]:pr.ptr[p + 1]], pr.sign[pr.ptr[p]:pr.ptr[p + 1]])
        assert r.minmax[p, 0] == v.min() and r.minmax[p, 1] == v.max()
        # bins from a library routine over the same boundaries
        t = O.boundaries(v.min(), v.max(), 256)
        b = np.searchsorted(t, v, side="right")
        H = np.zeros((256, 2), dtype=np.int64)
        np.add.at(H, (b, ds.y[idx]), 1)
        np.testing.assert_array_equal(r.hist[p], H)
        assert r.hist[p][0].sum() >= 1 and r.hist[p][255].sum() >= 1  # min in bin 0, max in last


# --------------------------------------------------------------------------
# Step 3: Gini criterion
# --------------------------------------------------------------------------

def test_gini_closed_form_equals_textbook_decrease():
    rng = np.random.default_rng(4)
    for _ in range(300):
        C = int(rng.integers(2, 6))
        N = rng.integers(0, 40, C)
        if N.sum() < 2:
            continue
        L = np.array([rng.integers(0, N[c] + 1) for c in range(C)])
        n, nl = int(N.sum()), int(L.sum())
        Nl, Ll = [int(a) for a in N], [int(a) for a in L]
        if nl == 0 or nl == n:
            continue
        g = O.gini_gain(L, N, n, nl)
        ref = brute.gini(Nl) - Fraction(nl, n) * brute.gini(Ll) \
            - Fraction(n - nl, n) * brute.gini([a - b for a, b in zip(Nl, Ll)])
        assert abs(Fraction(g) - ref) <= Fraction(1, 10 ** 14) * max(ref, Fraction(1, 10 ** 6))


def test_gini_special_cases():
    # balanced binary node split perfectly: decrease = G(parent) = 1/2
    assert O.gini_gain([50, 0], [50, 50], 100, 50) == 0.5
    # C balanced classes split perfectly one vs rest: G(parent) - nR/n G(R)
    C = 4
    g = O.gini_gain([10, 0, 0, 0], [10] * C, 40, 10)
    ref = Fraction(3, 4) - Fraction(30, 40) * Fraction(2, 3)
    assert abs(g - float(ref)) < 1e-15
    # children with the parent's class mix: zero decrease
    assert O.gini_gain([2, 4], [6, 12], 18, 6) == 0.0
    # pure parent: zero decrease for any split
    assert O.gini_gain([3, 0], [9, 0], 9, 3) == 0.0


def test_midpoint_between_neighbours():
    rng = np.random.default_rng(5)
    a = rng.standard_normal(2000).astype(np.float32) * np.float32(10.0) ** rng.integers(-30, 30, 2000).astype(np.float32)
    b = np.where(rng.random(2000) < 0.5, np.nextafter(a, np.float32(np.inf)),
                 a + np.abs(rng.standard_normal(2000)).astype(np.float32)).astype(np.float32)
    for x, z in zip(a, b):
        if not x < z:
            continue
        t = O.midpoint(float(x), float(z))
        assert np.float32(x) < t <= np.float32(z)


# --------------------------------------------------------------------------
# Whole split search: brute force in exact rationals
# --------------------------------------------------------------------------

def _lexi_best(cands):
    """cands: list of (proj, cand, leftset, gain) -> best by (max gain, lowest proj, lowest cand)."""
    best = None
    for c in cands:
        if c[3] <= 0:
            continue
        if best is None or c[3] > best[3]:
            best = c
    return best


def _check_against_brute(r, cands, P):
    best = _lexi_best(cands)
    if best is None:
        assert r.valid == 0
        return
    assert r.valid == 1
    chosen = [c for c in cands if c[0] == r.proj and c[1] == r.cand]
    assert len(chosen) == 1
    if chosen[0][3] != best[3]:
        # only acceptable when the double gains of two different rationals coincide
        assert float(chosen[0][3]) == pytest.approx(float(best[3]), rel=1e-15)
    else:
        # equal rational maxima -> lexicographic rule
        first = min((c for c in cands if c[3] == best[3]), key=lambda c: (c[0], c[1]))
        assert (r.proj, r.cand) == (first[0], first[1])
    assert r.n_left == len(chosen[0][2])
    assert float(r.gain) == pytest.approx(float(chosen[0][3]), rel=1e-14)


@pytest.mark.parametrize("seed", range(40))
def test_sort_path_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 11))
    d = 5
    C = int(rng.integers(2, 4))
    # small integers make ties between values and gains common
    X = rng.integers(-3, 4, (d, 20)).astype(np.float32) * np.float32(0.5)
    y = rng.integers(0, C, 20).astype(np.uint8)
    idx = rng.choice(20, n, replace=True).astype(np.int32)  # repeats allowed (bootstrap)
    pr = G.random_projections(rng, 6, d, 1.5, 3)
    r = O.split_search(X, y, C, idx, pr.ptr, pr.feat, pr.sign, sort_below=1024)
    assert r.path == 1
    cands = []
    for p in range(6):
        f, s = pr.feat[pr.ptr[p]:pr.ptr[p + 1]], pr.sign[pr.ptr[p]:pr.ptr[p + 1]]
        v = O.project(X, idx, f, s)
        for (i, left, g) in brute.sort_path_candidates(v, y[idx], C):
            cands.append((p, i, left, g))
    _check_against_brute(r, cands, 6)
    if r.valid:
        f, s = pr.feat[pr.ptr[r.proj]:pr.ptr[r.proj + 1]], pr.sign[pr.ptr[r.proj]:pr.ptr[r.proj + 1]]
        v = O.project(X, idx, f, s)
        below = v[v < r.threshold]
        above = v[v >= r.threshold]
        assert below.max() < r.threshold <= above.min()


@pytest.mark.parametrize("seed", range(30))
def test_hist_path_brute_force(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 14))
    d = 4
    C = int(rng.integers(2, 4))
    B = int(rng.choice([2, 3, 4, 8, 16]))
    X = rng.standard_normal((d, 30)).astype(np.float32)
    if seed % 3 == 0:
        X = np.round(X)  # ties
    y = rng.integers(0, C, 30).astype(np.uint8)
    idx = rng.choice(30, n, replace=True).astype(np.int32)
    pr = G.random_projections(rng, 5, d, 1.5, 3)
    r = O.split_search(X, y, C, idx, pr.ptr, pr.feat, pr.sign, n_bins=B, hist_only=True, want_debug=True)
    assert r.path == 0
    cands = []
    for p in range(5):
        f, s = pr.feat[pr.ptr[p]:pr.ptr[p + 1]], pr.sign[pr.ptr[p]:pr.ptr[p + 1]]
        v = O.project(X, idx, f, s)
        t = O.boundaries(v.min(), v.max(), B)
        for (b, left, g) in brute.hist_path_candidates(v, y[idx], C, t):
            cands.append((p, b, left, g))
    _check_against_brute(r, cands, 5)
    if r.valid:
        t = O.boundaries(r.minmax[r.proj, 0], r.minmax[r.proj, 1], B)
        assert r.threshold == t[r.cand]


def test_fp64_argmax_rational_audit():
    """Moderate nodes: the oracle's double argmax is a rational argmax (or a
    double tie of rationals) over all candidates of both paths."""
    rng = np.random.default_rng(7)
    for trial in range(6):
        n = 60
        X = rng.standard_normal((6, 200)).astype(np.float32)
        y = rng.integers(0, 3, 200).astype(np.uint8)
        idx = np.sort(rng.choice(200, n, replace=False)).astype(np.int32)
        pr = G.random_projections(rng, 8, 6, 1.5, 4)
        for hist in (False, True):
            r = O.split_search(X, y, 3, idx, pr.ptr, pr.feat, pr.sign, n_bins=32,
                               sort_below=1024, hist_only=hist, want_debug=hist)
            cands = []
            for p in range(8):
                f, s = pr.feat[pr.ptr[p]:pr.ptr[p + 1]], pr.sign[pr.ptr[p]:pr.ptr[p + 1]]
                v = O.project(X, idx, f, s)
                if hist:
                    t = O.boundaries(v.min(), v.max(), 32)
                    cs = brute.hist_path_candidates(v, y[idx], 3, t)
                else:
                    cs = brute.sort_path_candidates(v, y[idx], 3)
                cands += [(p, c[0], c[1], c[2]) for c in cs]
            _check_against_brute(r, cands, 8)


def test_hand_worked_golden():
    kv = {}
    with open(os.path.join(GOLDEN, "hand_split_6.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    X = np.array([[float(t) for t in kv["X0"].split()], [float(t) for t in kv["X1"].split()]],
                 dtype=np.float32)
    y = np.array([int(t) for t in kv["y"].split()], dtype=np.uint8)
    projs = []
    for p in range(3):
        terms = kv[f"proj{p}"].split()
        projs.append(([int(t[1:]) for t in terms], [1 if t[0] == "+" else -1 for t in terms]))
    idx = np.arange(6, dtype=np.int32)

    def csr(ps):
        ptr = np.zeros(len(ps) + 1, np.int32)
        ptr[1:] = np.cumsum([len(f) for f, _ in ps])
        return ptr, np.array(sum([f for f, _ in ps], []), np.int32), np.array(sum([s for _, s in ps], []), np.int8)

    def parse(s):
        t = s.split()
        return {t[i]: t[i + 1] for i in range(0, len(t), 2)}

    def check(r, exp, proj_offset=None):
        if "proj" in exp:
            assert r.proj == int(exp["proj"])
        assert r.cand == int(exp["cand"])
        assert r.threshold == np.float32(float(exp["threshold"]))
        assert Fraction(r.gain) == Fraction(exp["gain"]) or r.gain == pytest.approx(float(Fraction(exp["gain"])), rel=1e-15)
        assert r.n_left == int(exp["n_left"])

    r = O.split_search(X, y, 2, idx, *csr(projs), sort_below=1024)
    check(r, parse(kv["sort.best"]))
    for p in (0, 2):
        r = O.split_search(X, y, 2, idx, *csr([projs[p]]), sort_below=1024)
        check(r, parse(kv[f"sort.p{p}"]))
    r = O.split_search(X, y, 2, idx, *csr(projs), n_bins=4, hist_only=True, want_debug=True)
    check(r, parse(kv["hist4.best"]))
    for p in range(3):
        h = np.array([int(t) for t in kv[f"hist4.p{p}.hist"].split()]).reshape(4, 2)
        np.testing.assert_array_equal(r.hist[p], h)
    for p in (0, 2):
        mm = np.array([float(t) for t in kv[f"hist4.p{p}.minmax"].split()], np.float32)
        np.testing.assert_array_equal(r.minmax[p], mm)


def test_degenerate_nodes():
    X = np.ones((3, 10), dtype=np.float32)
    y = np.array([0, 1] * 5, dtype=np.uint8)
    idx = np.arange(10, dtype=np.int32)
    ptr, f, s = np.array([0, 1, 3], np.int32), np.array([0, 1, 2], np.int32), np.array([1, 1, -1], np.int8)
    for hist in (False, True):
        r = O.split_search(X, y, 2, idx, ptr, f, s, hist_only=hist)
        assert r.valid == 0  # all projected values equal: no split
    # a single sample / empty node
    r = O.split_search(X, y, 2, idx[:1], ptr, f, s)
    assert r.valid == 0
    r = O.split_search(X, y, 2, idx[:0], ptr, f, s)
    assert r.valid == 0
    # pure node: valid splits exist geometrically but all gains are zero
    X2 = np.arange(10, dtype=np.float32)[None, :].repeat(3, 0)
    r = O.split_search(X2, np.zeros(10, np.uint8), 2, idx, ptr, f, s)
    assert r.valid == 0


# --------------------------------------------------------------------------
# Partition and tree invariants
# --------------------------------------------------------------------------

def test_partition_stable_and_consistent():
    ds = G.tree_small(n=5000, d=10, seed=12)
    rng = np.random.default_rng(8)
    idx = np.sort(rng.choice(ds.n, 3000, replace=True)).astype(np.int32)
    pr = G.random_projections(rng, 10, ds.d, 1.5, 8)
    for hist, T in ((True, 0), (False, 100000)):
        r = O.split_search(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, sort_below=T, hist_only=hist)
        assert r.valid
        f, s = pr.feat[pr.ptr[r.proj]:pr.ptr[r.proj + 1]], pr.sign[pr.ptr[r.proj]:pr.ptr[r.proj + 1]]
        out, nl = O.partition(ds.X, idx, f, s, float(r.threshold))
        assert nl == r.n_left
        v = O.project(ds.X, idx, f, s)
        np.testing.assert_array_equal(out[:nl], idx[v < r.threshold])
        np.testing.assert_array_equal(out[nl:], idx[~(v < r.threshold)])
        np.testing.assert_array_equal(np.bincount(ds.y[out[:nl]], minlength=2), r.left_counts)


def _tree_invariants(tr, X, y, C, root_idx, max_depth=-1):
    n_root = root_idx.shape[0]
    assert tr.n_samples[0] == n_root
    leaves = tr.left < 0
    assert tr.n_samples[leaves].sum() == n_root
    for i in range(tr.n_nodes):
        np.testing.assert_array_equal(tr.class_counts[i].sum(), tr.n_samples[i])
        if tr.left[i] >= 0:
            l, r = tr.left[i], tr.right[i]
            assert r == l + 1 and l > i
            assert tr.depth[l] == tr.depth[i] + 1
            np.testing.assert_array_equal(tr.class_counts[l] + tr.class_counts[r], tr.class_counts[i])
            assert tr.gain[i] > 0
            assert tr.n_samples[l] > 0 and tr.n_samples[r] > 0
        else:
            pure = (tr.class_counts[i] > 0).sum() <= 1
            if not pure and (max_depth < 0 or tr.depth[i] < max_depth) and tr.n_samples[i] >= 2:
                assert tr.path[i] in (0, 1)  # searched, found nothing of positive gain
            assert tr.leaf_class[i] == int(np.argmax(tr.class_counts[i]))
    assert np.all(np.diff(tr.depth) >= 0), "breadth-first order"


def test_tree_invariants_and_training_fit():
    ds = G.tree_small(n=2048, d=16, seed=13)
    root = G.all_indices(ds.n)
    tr = O.train_tree(ds.X, ds.y, 2, root, n_proj=16, lam=1.5, cap=8, sort_below=256, seed=5)
    _tree_invariants(tr, ds.X, ds.y, 2, root)
    # grown to purity on distinct points: training data is fitted exactly
    pred = O.predict_tree(tr, ds.X, root[:400])
    np.testing.assert_array_equal(pred, ds.y[:400])
    assert set(np.unique(tr.path)) >= {0, 1}  # both paths used


def test_tree_bootstrap_and_max_depth():
    ds = G.tree_small(n=1500, d=8, seed=14)
    root = G.bootstrap_indices(ds.n, 0, seed=1, n_draws=1500)
    tr = O.train_tree(ds.X, ds.y, 2, root, n_proj=8, lam=1.5, cap=8, sort_below=128, seed=6)
    _tree_invariants(tr, ds.X, ds.y, 2, root)
    tr3 = O.train_tree(ds.X, ds.y, 2, root, n_proj=8, lam=1.5, cap=8, sort_below=128, seed=6, max_depth=3)
    _tree_invariants(tr3, ds.X, ds.y, 2, root, max_depth=3)
    assert tr3.depth.max() <= 3
    # the depth-limited tree is a prefix of the full tree (same keys, same splits)
    k = tr3.n_nodes
    np.testing.assert_array_equal(tr3.threshold[tr3.left >= 0], tr.threshold[:k][tr3.left >= 0])


def test_hist_and_sort_agree_on_aligned_data():
    """When every distinct value sits alone in its own bin, the histogram path
    and the exact path separate the same sets (sanity check, not a pin)."""
    vals = np.arange(8, dtype=np.float32)  # 0..7 with 8 bins of width 7/8
    X = vals[None, :]
    y = np.array([0, 0, 1, 0, 1, 1, 1, 0], np.uint8)
    idx = np.arange(8, dtype=np.int32)
    ptr, f, s = np.array([0, 1], np.int32), np.array([0], np.int32), np.array([1], np.int8)
    rs = O.split_search(X, y, 2, idx, ptr, f, s, sort_below=100)
    rh = O.split_search(X, y, 2, idx, ptr, f, s, n_bins=8, hist_only=True)
    assert rs.n_left == rh.n_left and rs.gain == rh.gain


def test_threaded_split_search_equals_plain():
    """The host-threaded oracle (used to time the CPU baseline on all cores)
    returns the plain split search's result for every thread count."""
    import oracle as O2
    from paper_2603_00326_b300 import datagen as G2
    ds = G2.tree_small(n=3000, d=12, seed=15)
    rng = np.random.default_rng(2)
    pr = G2.random_projections(rng, 29, 12, 1.5, 8)
    idx = G2.all_indices(ds.n)
    for T, ho in ((1024, True), (4000, False)):
        a = O2.split_search(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, sort_below=T, hist_only=ho)
        for nt in (1, 2, 5, 29, 64):
            b = O2.split_search_mt(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, sort_below=T, hist_only=ho,
                                   n_threads=nt)
            assert (a.valid, a.proj, a.cand, a.path, a.n_left) == (b.valid, b.proj, b.cand, b.path, b.n_left)
            assert np.float32(a.threshold).tobytes() == np.float32(b.threshold).tobytes()
            assert np.float64(a.gain).tobytes() == np.float64(b.gain).tobytes()
            np.testing.assert_array_equal(a.left_counts, b.left_counts)
