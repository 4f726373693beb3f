"""Pins of the oracle's entropy criterion (reading R15: information gain, the
criterion of the YDF learner the paper builds on, Section 3 step 3).

The series logarithm against the C library's log and exact multiples of ln 2;
the information gain against scikit-learn's mutual information (a library
routine computing the same quantity from label arrays) and against the
textbook entropy decrease evaluated in 40-digit arithmetic; special cases; the
split search against brute force over every threshold; the threaded search
and a fully re-searched tree against the plain search.  No GPU needed.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests.tree_check import route_and_sample

ENT = 1


def _ulp(x):
    return math.ulp(x) if x != 0 else 5e-324


def test_ln_within_two_ulp_of_libm():
    rng = np.random.default_rng(1)
    xs = np.concatenate([np.arange(1, 5000), rng.integers(1, 2 ** 40, 5000),
                         np.exp(rng.uniform(-700, 700, 3000))])
    worst = 0.0
    for x in xs:
        x = float(x)
        ref = math.log(x)
        got = O.ln(x)
        worst = max(worst, abs(got - ref) / _ulp(ref))
    assert worst <= 2.0, worst
    assert O.ln(1.0) == 0.0


def test_ln_of_powers_of_two_is_k_ln2():
    for k in range(-1000, 1001, 7):
        assert O.ln(2.0 ** k) == k * math.log(2.0)


def test_xlnx_values():
    assert O.xlnx(0) == 0.0 and O.xlnx(1) == 0.0
    for x in (2, 3, 17, 1000, 2 ** 31 - 1):
        assert O.xlnx(x) == pytest.approx(x * math.log(x), rel=1e-15)


def _mp():
    return pytest.importorskip("mpmath")


def _mp_gain(L, N):
    """Textbook entropy decrease H(parent) - nL/n H(L) - nR/n H(R), 40 digits."""
    mpmath = _mp()
    mpmath.mp.dps = 40
    L = [int(c) for c in L]
    N = [int(c) for c in N]

    def H(cnt):
        t = sum(cnt)
        if t == 0:
            return mpmath.mpf(0)
        return -sum(mpmath.mpf(c) / t * mpmath.log(mpmath.mpf(c) / t) for c in cnt if c > 0)
    R = [a - b for a, b in zip(N, L)]
    n, nl = sum(N), sum(L)
    return H(N) - mpmath.mpf(nl) / n * H(L) - mpmath.mpf(n - nl) / n * H(R)


def test_gain_equals_mutual_information_and_textbook():
    mutual_info_score = pytest.importorskip("sklearn.metrics").mutual_info_score
    rng = np.random.default_rng(2)
    for _ in range(300):
        C = int(rng.integers(2, 9))
        n = int(rng.integers(2, 3000))
        y = rng.integers(0, C, n)
        side = (rng.random(n) < rng.uniform(0.05, 0.95)).astype(int)
        if side.min() == side.max():
            side[0] = 1 - side[0]
        N = np.bincount(y, minlength=C)
        L = np.bincount(y[side == 1], minlength=C)
        g = O.entropy_gain(L, N, n, int(L.sum()))
        assert g == pytest.approx(mutual_info_score(y, side), abs=1e-12)
        ref = float(_mp_gain(list(L), list(N)))
        assert abs(g - ref) <= 5e-14  # double evaluation of terms of size ln n


def test_gain_special_cases():
    n = 1000
    # perfect split of a balanced binary node: ln 2
    assert O.entropy_gain([500, 0], [500, 500], n, 500) == pytest.approx(math.log(2), rel=1e-15)
    # left class mix proportional to the node: exactly no information
    assert O.entropy_gain([100, 300, 50], [200, 600, 100], 900, 450) == 0.0
    # pure node: every split carries no information
    assert O.entropy_gain([0, 37], [0, 120], 120, 37) == 0.0
    # gain is symmetric in the two children
    a = O.entropy_gain([30, 10, 5], [50, 60, 20], 130, 45)
    b = O.entropy_gain([20, 50, 15], [50, 60, 20], 130, 85)
    assert a == pytest.approx(b, rel=1e-13)
    # bounded by the parent's entropy: class 0 split off from three classes
    N = [40, 25, 35]
    Hpar = -sum(c / 100 * math.log(c / 100) for c in N)
    g = O.entropy_gain([40, 0, 0], N, 100, 40)
    assert g == pytest.approx(float(_mp_gain([40, 0, 0], N)), abs=1e-15) and 0 < g < Hpar


def _check(r, cands):
    """cands: (proj, cand, left set, mp gain, left counts).  The oracle's pick
    has the largest gain; where mp gains tie, the lowest (proj, cand) unless
    the double values of the tied gains order them otherwise."""
    mpmath = _mp()
    pos = [c for c in cands if c[3] > 1e-30]
    if not pos:
        assert r.valid == 0
        return
    best = max(c[3] for c in pos)
    assert r.valid == 1
    chosen = [c for c in cands if c[0] == r.proj and c[1] == r.cand]
    assert len(chosen) == 1
    ch = chosen[0]
    assert abs(float(ch[3] - best)) <= 1e-13, (float(ch[3]), float(best))
    assert float(r.gain) == pytest.approx(float(ch[3]), rel=1e-12, abs=1e-15)
    ties = sorted((c for c in pos if abs(c[3] - best) < mpmath.mpf(10) ** -30), key=lambda c: (c[0], c[1]))
    first = ties[0]
    if (first[0], first[1]) != (r.proj, r.cand):
        # a tie in exact arithmetic that the fixed double expression orders
        assert O.entropy_gain(first[4], cands[0][5], cands[0][6], int(sum(first[4]))) < r.gain
    assert r.n_left == len(ch[2])


@pytest.mark.parametrize("seed", range(30))
@pytest.mark.parametrize("path", ["sort", "hist"])
def test_entropy_split_brute_force(seed, path):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(2, 14))
    d, C = 4, int(rng.integers(2, 4))
    B = int(rng.choice([2, 3, 8, 16]))
    X = rng.standard_normal((d, 30)).astype(np.float32)
    if seed % 3 == 0:
        X = np.round(X)
    y = rng.integers(0, C, 30).astype(np.uint8)
    idx = rng.choice(30, n, replace=True).astype(np.int32)
    pr = G.random_projections(rng, 5, d, 1.5, 3)
    hist = path == "hist"
    r = O.split_search(X, y, C, idx, pr.ptr, pr.feat, pr.sign, n_bins=B, sort_below=0 if hist else 100,
                       hist_only=hist, want_debug=True, criterion=ENT)
    Nv = np.bincount(y[idx], minlength=C)
    cands = []
    for p in range(5):
        f, s = pr.feat[pr.ptr[p]:pr.ptr[p + 1]], pr.sign[pr.ptr[p]:pr.ptr[p + 1]]
        v = O.project(X, idx, f, s)
        if hist:
            t = O.boundaries(v.min(), v.max(), B)
            splits = [(b, t[b]) for b in range(B - 1)]
            for b, thr in splits:
                left = [j for j in range(n) if v[j] < thr]
                if 0 < len(left) < n:
                    Lc = np.bincount(y[idx][left], minlength=C)
                    cands.append((p, b, frozenset(left), _mp_gain(list(Lc), list(Nv)), Lc, Nv, n))
        else:
            order = sorted(range(n), key=lambda i: (float(v[i]), int(y[idx][i])))
            for i in range(n - 1):
                a, b = float(v[order[i]]), float(v[order[i + 1]])
                if not a < b:
                    continue
                left = [j for j in range(n) if float(v[j]) <= a]
                Lc = np.bincount(y[idx][left], minlength=C)
                cands.append((p, i, frozenset(left), _mp_gain(list(Lc), list(Nv)), Lc, Nv, n))
    _check(r, cands)


def test_entropy_threaded_equals_plain_and_differs_from_gini():
    ds = G.tree_small(n=3000, d=12, seed=15)
    rng = np.random.default_rng(2)
    pr = G.random_projections(rng, 29, 12, 1.5, 8)
    idx = G.all_indices(ds.n)
    for T, ho in ((1024, True), (4000, False)):
        a = O.split_search(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, sort_below=T, hist_only=ho, criterion=ENT)
        assert a.valid
        for nt in (2, 5, 29):
            b = O.split_search_mt(ds.X, ds.y, 2, idx, pr.ptr, pr.feat, pr.sign, sort_below=T, hist_only=ho,
                                  n_threads=nt, criterion=ENT)
            assert (a.valid, a.proj, a.cand, a.n_left) == (b.valid, b.proj, b.cand, b.n_left)
            assert np.float64(a.gain).tobytes() == np.float64(b.gain).tobytes()
        Lc = a.left_counts
        N = np.bincount(ds.y, minlength=2)
        assert a.gain == O.entropy_gain(Lc, N, ds.n, int(Lc.sum()))


def test_entropy_tree_every_node_re_searched():
    ds = G.tree_small(n=1500, d=12, seed=71)
    root = G.bootstrap_indices(ds.n, 2, seed=9)
    kw = dict(n_proj=12, lam=1.5, cap=8, n_bins=64, sort_below=200, seed=4, tree_id=2)
    t = O.train_tree(ds.X, ds.y, 2, root, criterion=ENT, **kw)
    assert t.n_nodes > 30 and set(np.unique(t.path)) >= {-1, 0, 1}
    n = route_and_sample(t, ds.X, ds.y, 2, root, check_ids=range(t.n_nodes), criterion=ENT, **kw)
    assert n == int(np.count_nonzero(t.path >= 0))
    g = O.train_tree(ds.X, ds.y, 2, root, **kw)
    assert not (g.n_nodes == t.n_nodes and np.array_equal(g.threshold, t.threshold))
    with pytest.raises(AssertionError):
        route_and_sample(t, ds.X, ds.y, 2, root, check_ids=range(t.n_nodes), criterion=0, **kw)
