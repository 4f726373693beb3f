"""Exact-rational brute force used to pin the oracle (tests only).

Textbook Gini impurity G(S) = 1 - sum_c p_c^2 and the impurity decrease
G(parent) - |L|/n G(L) - |R|/n G(R), evaluated in fractions.Fraction, over
every threshold that a projection admits.  Independent of the oracle's
closed-form expression.
"""
from fractions import Fraction

import numpy as np


def gini(counts):
    counts = [int(c) for c in counts]
    n = sum(counts)
    if n == 0:
        return Fraction(0)
    return 1 - sum(Fraction(c, n) ** 2 for c in counts)


def decrease(labels_left, labels_right, C):
    L = [0] * C
    R = [0] * C
    for y in labels_left:
        L[y] += 1
    for y in labels_right:
        R[y] += 1
    N = [a + b for a, b in zip(L, R)]
    n = sum(N)
    nl, nr = sum(L), sum(R)
    return gini(N) - Fraction(nl, n) * gini(L) - Fraction(nr, n) * gini(R)


def sort_path_candidates(v, y, C):
    """All exact-split candidates of one projected feature.

    Returns a list of (position i in ascending order, left index set, gain).
    A candidate exists between sorted positions i and i+1 when the values differ.
    """
    v = np.asarray(v, dtype=np.float32)
    order = sorted(range(len(v)), key=lambda i: (float(v[i]), int(y[i])))
    out = []
    for i in range(len(v) - 1):
        a, b = float(v[order[i]]), float(v[order[i + 1]])
        if not a < b:
            continue
        left = [j for j in range(len(v)) if float(v[j]) <= a]
        right = [j for j in range(len(v)) if float(v[j]) > a]
        g = decrease([y[j] for j in left], [y[j] for j in right], C)
        out.append((i, frozenset(left), g))
    return out


def hist_path_candidates(v, y, C, t):
    """Histogram-path candidates: candidate b sends v < t[b] left (t[b] = t_{b+1})."""
    out = []
    n = len(v)
    for b in range(len(t)):
        left = [j for j in range(n) if float(v[j]) < float(t[b])]
        if len(left) == 0 or len(left) == n:
            continue
        right = [j for j in range(n) if not float(v[j]) < float(t[b])]
        g = decrease([y[j] for j in left], [y[j] for j in right], C)
        out.append((b, frozenset(left), g))
    return out
