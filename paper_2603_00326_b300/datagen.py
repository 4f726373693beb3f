"""Seeded synthetic inputs for sparse-oblique split search and tree training.

This module only *creates inputs*: feature matrices, labels, node index
lists, bootstrap draws and (for the split-search calls that take them as an
argument) projection matrices.  It contains none of the split-search
arithmetic: no projection sums, no bins, no Gini, no partition.  Both the CPU
oracle and the CUDA path consume exactly the arrays produced here.

The paper's performance datasets (HIGGS, SUSY, Epsilon, Trunk; Table 1) are
not available offline, so five synthetic workloads shaped like them stand in:

* ``tree_small``    n=8192, d=32, N(0,1), binary labels from 4 features with
                    5% flips, 32 projections/node, tree to purity.
* ``root_4m``       n=4M, d=64, N(0,1), 3 classes from sparse linear scores,
                    256 projections, root split on the histogram path.
* ``frontier_1m``   n=1M, d=128, 4096 nodes with lognormal(5, 2) sizes,
                    64 projections/node, mixed sort / histogram nodes.
* ``forest_2m``     n=2M, d=256, lognormal(0,1) features, 128 bootstrapped
                    trees, 128 projections/node.
* ``wide_counts``   n=500k, d=4096, 90% zeros, Poisson(3) nonzeros, 5 classes.
* ``trunk``         the Trunk generator of the paper's Table 1: p-dimensional
                    Gaussians with class means +mu and -mu, mu_j = 1/sqrt(j),
                    identity covariance, two balanced classes (a "next" workload
                    for the paper's Trunk-100k / 1M scaling rows).

Every generator takes the sizes as arguments, so tests draw the same recipe at
sizes the oracle finishes in seconds.
"""
from __future__ import annotations

import dataclasses
import os
from typing import Optional

import numpy as np

DATA_SEED_BASE = 326000
PROJ_SEED_BASE = 327000


@dataclasses.dataclass
class Dataset:
    """Column-major features ``X[f, i]`` (shape ``[d, n]``, float32) and labels."""

    X: np.ndarray          # float32 [d, n], C-contiguous => column-major by sample
    y: np.ndarray          # uint8 [n]
    n_classes: int
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.X.shape[1])

    @property
    def d(self) -> int:
        return int(self.X.shape[0])


@dataclasses.dataclass
class Projections:
    """CSR list of sparse +-1 projections (features ascending within a row)."""

    ptr: np.ndarray        # int32 [P+1]
    feat: np.ndarray       # int32 [nnz]
    sign: np.ndarray       # int8  [nnz], values +1 / -1

    @property
    def n_proj(self) -> int:
        return int(self.ptr.shape[0] - 1)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _distinct(rng: np.random.Generator, d: int, k: int) -> np.ndarray:
    return np.sort(rng.choice(d, size=k, replace=False)).astype(np.int64)


def _flip_exact(rng: np.random.Generator, y: np.ndarray, frac: float, n_classes: int) -> None:
    """Flip exactly round(frac*n) distinct labels (binary: 1-y; multiclass: +1 mod C)."""
    n = y.shape[0]
    k = int(round(frac * n))
    if k == 0:
        return
    which = rng.choice(n, size=k, replace=False)
    if n_classes == 2:
        y[which] = 1 - y[which]
    else:
        y[which] = (y[which] + 1) % n_classes


def gaussian_features(rng: np.random.Generator, n: int, d: int) -> np.ndarray:
    X = np.empty((d, n), dtype=np.float32)
    for f in range(d):
        X[f] = rng.standard_normal(n, dtype=np.float32)
    return X


def binary_sum_labels(rng: np.random.Generator, X: np.ndarray, n_feat: int = 4,
                      flip: float = 0.05) -> np.ndarray:
    """y = [sum of n_feat distinct random features > 0], then exact flips."""
    d, n = X.shape
    S = _distinct(rng, d, min(n_feat, d))
    score = np.zeros(n, dtype=np.float64)
    for f in S:
        score += X[f].astype(np.float64)
    y = (score > 0).astype(np.uint8)
    _flip_exact(rng, y, flip, 2)
    return y


def argmax_sparse_labels(rng: np.random.Generator, X: np.ndarray, n_classes: int,
                         sparsity: int, noise_std: float) -> np.ndarray:
    """y = argmax_c (sum_{j in S_c} w_j x_j + eps_c), |S_c| = sparsity, w = +-1."""
    d, n = X.shape
    scores = np.empty((n_classes, n), dtype=np.float64)
    for c in range(n_classes):
        S = _distinct(rng, d, min(sparsity, d))
        w = rng.choice(np.array([-1.0, 1.0]), size=S.shape[0])
        acc = np.zeros(n, dtype=np.float64)
        for f, s in zip(S, w):
            acc += s * X[f].astype(np.float64)
        acc += noise_std * rng.standard_normal(n)
        scores[c] = acc
    return np.argmax(scores, axis=0).astype(np.uint8)


def random_projections(rng: np.random.Generator, P: int, d: int, lam: float,
                       cap: int) -> Projections:
    """P projections with nnz = min(cap, d, 1 + Poisson(lam)) distinct features and +-1 signs.

    Used where the projections are an *argument* of the call (single split
    searches).  Trees sample their own projections inside the library.
    """
    nnz = np.minimum(np.minimum(1 + rng.poisson(lam, size=P), cap), d).astype(np.int64)
    ptr = np.zeros(P + 1, dtype=np.int32)
    ptr[1:] = np.cumsum(nnz)
    feat = np.empty(int(ptr[-1]), dtype=np.int32)
    sign = np.empty(int(ptr[-1]), dtype=np.int8)
    for p in range(P):
        feat[ptr[p]:ptr[p + 1]] = _distinct(rng, d, int(nnz[p]))
        sign[ptr[p]:ptr[p + 1]] = rng.choice(np.array([-1, 1], dtype=np.int8), size=int(nnz[p]))
    return Projections(ptr=ptr, feat=feat, sign=sign)


# ----------------------------------------------------------------------------
# The five workloads (sizes overridable)
# ----------------------------------------------------------------------------

def tree_small(n: int = 8192, d: int = 32, seed: int = DATA_SEED_BASE + 0) -> Dataset:
    rng = _rng(seed)
    X = gaussian_features(rng, n, d)
    y = binary_sum_labels(rng, X, 4, 0.05)
    return Dataset(X, y, 2, "tree_small")


def root_4m(n: int = 4 * 1024 * 1024, d: int = 64, seed: int = DATA_SEED_BASE + 1) -> Dataset:
    rng = _rng(seed)
    X = gaussian_features(rng, n, d)
    y = argmax_sparse_labels(rng, X, 3, 4, 0.5)
    return Dataset(X, y, 3, "root_4m")


def frontier_1m(n: int = 1024 * 1024, d: int = 128, seed: int = DATA_SEED_BASE + 2) -> Dataset:
    rng = _rng(seed)
    X = gaussian_features(rng, n, d)
    y = binary_sum_labels(rng, X, 4, 0.05)
    return Dataset(X, y, 2, "frontier_1m")


def forest_2m(n: int = 2 * 1024 * 1024, d: int = 256, seed: int = DATA_SEED_BASE + 3) -> Dataset:
    rng = _rng(seed)
    X = np.empty((d, n), dtype=np.float32)
    for f in range(d):
        X[f] = np.exp(rng.standard_normal(n)).astype(np.float32)
    S = _distinct(rng, d, min(8, d))
    s = rng.choice(np.array([-1.0, 1.0]), size=S.shape[0])
    score = np.zeros(n, dtype=np.float64)
    for f, w in zip(S, s):
        score += w * X[f].astype(np.float64)
    y = (score > np.median(score)).astype(np.uint8)
    _flip_exact(rng, y, 0.10, 2)
    return Dataset(X, y, 2, "forest_2m")


def _wide_block(X: np.ndarray, f0: int, f1: int, ss: np.random.SeedSequence) -> None:
    rng = np.random.default_rng(ss)
    n = X.shape[1]
    nz = rng.random((f1 - f0, n), dtype=np.float32) < np.float32(0.1)
    k = int(nz.sum())
    # zero-truncated Poisson(3) by rejection of zeros
    vals = rng.poisson(3.0, size=k)
    while True:
        zero = vals == 0
        if not zero.any():
            break
        vals[zero] = rng.poisson(3.0, size=int(zero.sum()))
    sub = X[f0:f1]
    sub[nz] = vals.astype(np.float32)


def wide_counts(n: int = 500_000, d: int = 4096, seed: int = DATA_SEED_BASE + 4) -> Dataset:
    """Blocks of 64 features each draw from their own child stream of the
    seed, so the blocks can be filled by a thread pool in any order."""
    from concurrent.futures import ThreadPoolExecutor
    X = np.zeros((d, n), dtype=np.float32)
    blk = 64
    starts = list(range(0, d, blk))
    children = np.random.SeedSequence(seed).spawn(len(starts) + 1)
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(lambda a: _wide_block(X, a[0], min(d, a[0] + blk), a[1]), zip(starts, children[:-1])))
    y = argmax_sparse_labels(np.random.default_rng(children[-1]), X, 5, 16, 0.5)
    return Dataset(X, y, 5, "wide_counts")


def _trunk_block(X: np.ndarray, f0: int, f1: int, sgn: np.ndarray, ss: np.random.SeedSequence) -> None:
    rng = np.random.default_rng(ss)
    n = X.shape[1]
    for f in range(f0, f1):
        mu = np.float32(1.0 / np.sqrt(f + 1.0))
        X[f] = rng.standard_normal(n, dtype=np.float32) + sgn * mu


def trunk(n: int = 1_000_000, p: int = 1024, seed: int = DATA_SEED_BASE + 5) -> Dataset:
    """Trunk: exactly balanced classes in a seeded random order; class 0 drawn
    from N(+mu, I), class 1 from N(-mu, I), mu_j = 1/sqrt(j) for j = 1..p.
    64-feature blocks draw from child streams of the seed (thread pool)."""
    from concurrent.futures import ThreadPoolExecutor
    root = np.random.SeedSequence(seed)
    children = root.spawn((p + 63) // 64 + 1)
    y = np.zeros(n, dtype=np.uint8)
    y[n // 2:] = 1
    np.random.default_rng(children[-1]).shuffle(y)
    sgn = np.where(y == 0, np.float32(1.0), np.float32(-1.0)).astype(np.float32)
    X = np.empty((p, n), dtype=np.float32)
    starts = list(range(0, p, 64))
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        list(ex.map(lambda a: _trunk_block(X, a[0], min(p, a[0] + 64), sgn, a[1]), zip(starts, children[:-1])))
    return Dataset(X, y, 2, "trunk")


def trunk_streamed(n: int, p: int, fill_block, seed: int = DATA_SEED_BASE + 5, workers: int = 4):
    """The Trunk dataset of trunk(n, p, seed), value for value, handed over in
    64-feature blocks instead of one host array (for sizes whose matrix does
    not fit in host memory): fill_block(f0, block) receives rows f0..f0+63 as
    a float32 [rows, n] array, at most `workers` blocks alive at a time.
    Returns the labels."""
    from concurrent.futures import ThreadPoolExecutor
    root = np.random.SeedSequence(seed)
    children = root.spawn((p + 63) // 64 + 1)
    y = np.zeros(n, dtype=np.uint8)
    y[n // 2:] = 1
    np.random.default_rng(children[-1]).shuffle(y)
    sgn = np.where(y == 0, np.float32(1.0), np.float32(-1.0)).astype(np.float32)

    def one(a):
        f0, ss = a
        f1 = min(p, f0 + 64)
        blk = np.empty((f1 - f0, n), dtype=np.float32)
        rng = np.random.default_rng(ss)
        for f in range(f0, f1):
            mu = np.float32(1.0 / np.sqrt(f + 1.0))
            blk[f - f0] = rng.standard_normal(n, dtype=np.float32) + sgn * mu
        return f0, blk

    starts = list(range(0, p, 64))
    with ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        for i in range(0, len(starts), workers):
            for f0, blk in ex.map(one, list(zip(starts, children[:-1]))[i:i + workers]):
                fill_block(f0, blk)
    return y


def lognormal_node_sizes(rng: np.random.Generator, m: int, n: int,
                         mu: float = 5.0, sigma: float = 2.0) -> np.ndarray:
    """m node sizes ~ lognormal(mu, sigma) rescaled to sum to n (each >= 1)."""
    raw = rng.lognormal(mu, sigma, size=m)
    s = np.maximum(1, np.round(raw * n / raw.sum())).astype(np.int64)
    s[int(np.argmax(s))] += n - int(s.sum())
    assert s.min() >= 1 and int(s.sum()) == n
    return s


def frontier_nodes(n: int, m: int, seed: int = PROJ_SEED_BASE + 2,
                   mu: float = 5.0, sigma: float = 2.0):
    """Index lists of m frontier nodes: consecutive chunks of a permutation, each sorted.

    Returns (idx int32 [n], node_off int64 [m+1]).
    """
    rng = _rng(seed)
    sizes = lognormal_node_sizes(rng, m, n, mu, sigma)
    perm = rng.permutation(n).astype(np.int32)
    off = np.zeros(m + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    idx = np.empty(n, dtype=np.int32)
    for j in range(m):
        idx[off[j]:off[j + 1]] = np.sort(perm[off[j]:off[j + 1]])
    return idx, off


def bootstrap_indices(n: int, tree_id: int, seed: int = PROJ_SEED_BASE + 3,
                      n_draws: Optional[int] = None) -> np.ndarray:
    """n draws with replacement for one tree, sorted ascending (multiplicity kept)."""
    rng = _rng(seed * 1_000_003 + tree_id)
    k = n if n_draws is None else n_draws
    return np.sort(rng.integers(0, n, size=k)).astype(np.int32)


def all_indices(n: int) -> np.ndarray:
    return np.arange(n, dtype=np.int32)


# Tree / split parameters of each workload.
WORKLOAD_PARAMS = {
    "tree_small": dict(n_proj=32, lam=1.5, cap=8, n_bins=256, sort_below=1024),
    "root_4m": dict(n_proj=256, lam=1.5, cap=8, n_bins=256, sort_below=0, hist_only=1),
    "frontier_1m": dict(n_proj=64, lam=1.5, cap=8, n_bins=256, sort_below=1024, n_nodes=4096),
    "forest_2m": dict(n_proj=128, lam=1.5, cap=8, n_bins=256, sort_below=1024, n_trees=128),
    "wide_counts": dict(n_proj=128, lam=3.0, cap=16, n_bins=256, sort_below=1024),
    # P = 1.5 sqrt(p) projections of about 2 non-zeros each (3 sqrt(p) non-zeros
    # in all, the paper's Section 3 density) for p = 1024
    "trunk": dict(n_proj=48, lam=1.0, cap=8, n_bins=256, sort_below=1024),
}
