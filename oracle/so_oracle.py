"""ctypes wrapper over the plain-C oracle (oracle/so_oracle.c).

Test infrastructure only.  Every function mirrors one step of the method as
the paper states it (Section 3 steps 1-3, Section 3.1 switch by node size,
Section 3.3 the two GPU kernels' outputs, Appendix A Floyd sampling); the
arithmetic lives in the C file, which documents each reading.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_sm64_next.restype = C.c_uint64
        L.orc_sm64_next.argtypes = [C.POINTER(C.c_uint64)]
        L.orc_sm64.restype = C.c_uint64
        L.orc_sm64.argtypes = [C.c_uint64]
        L.orc_root_key.restype = C.c_uint64
        L.orc_root_key.argtypes = [C.c_uint64, C.c_int32]
        L.orc_child_key.restype = C.c_uint64
        L.orc_child_key.argtypes = [C.c_uint64, C.c_int]
        L.orc_poisson_cdf.restype = None
        L.orc_poisson_cdf.argtypes = [C.c_double, C.c_int, C.c_void_p]
        L.orc_sample_node.restype = C.c_int
        L.orc_sample_node.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_double, C.c_int,
                                      C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_project.restype = None
        L.orc_project.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                  C.c_void_p, C.c_int, C.c_void_p]
        L.orc_gini_gain.restype = C.c_double
        L.orc_gini_gain.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_int64]
        L.orc_boundaries.restype = None
        L.orc_boundaries.argtypes = [C.c_float, C.c_float, C.c_int, C.c_void_p]
        L.orc_rw_boundaries.restype = None
        L.orc_rw_boundaries.argtypes = [C.c_uint64, C.c_int, C.c_float, C.c_float, C.c_int, C.c_void_p]
        L.orc_split_search_rule.restype = C.c_int
        L.orc_split_search_rule.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_void_p,
                                            C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                            C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p]
        L.orc_ln.restype = C.c_double
        L.orc_ln.argtypes = [C.c_double]
        L.orc_xlnx.restype = C.c_double
        L.orc_xlnx.argtypes = [C.c_int64]
        L.orc_entropy_gain.restype = C.c_double
        L.orc_entropy_gain.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int64, C.c_int64]
        L.orc_bin.restype = C.c_int
        L.orc_bin.argtypes = [C.c_void_p, C.c_int, C.c_float]
        L.orc_midpoint.restype = C.c_float
        L.orc_midpoint.argtypes = [C.c_float, C.c_float]
        L.orc_split_search.restype = C.c_int
        L.orc_split_search.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_void_p,
                                       C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_partition.restype = C.c_int64
        L.orc_partition.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                                    C.c_void_p, C.c_int, C.c_float]
        L.orc_train_tree.restype = C.c_int
        L.orc_train_tree.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int,
                                     C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_int, C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_int32,
                                     C.c_int32, C.c_void_p]
        L.orc_train_tree_mt.restype = C.c_int
        L.orc_train_tree_mt.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int,
                                        C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int,
                                        C.c_int, C.c_int, C.c_double, C.c_int, C.c_uint64, C.c_int32,
                                        C.c_int32, C.c_int, C.c_int64, C.c_void_p]
        L.orc_tree_free.restype = None
        L.orc_tree_free.argtypes = [C.c_void_p]
        L.orc_split_search_mt.restype = C.c_int
        L.orc_split_search_mt.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int, C.c_void_p,
                                          C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                          C.c_int, C.c_void_p, C.c_void_p]
        L.orc_predict_tree.restype = None
        L.orc_predict_tree.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                       C.c_int64, C.c_void_p]
        _lib = L
    return _lib


class OrcSplit(C.Structure):
    _fields_ = [("valid", C.c_int32), ("proj", C.c_int32), ("path", C.c_int32),
                ("cand", C.c_int32), ("threshold", C.c_float), ("gain", C.c_double),
                ("n_left", C.c_int64), ("n_right", C.c_int64)]


class OrcTree(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_classes", C.c_int32), ("cap", C.c_int32),
                ("left", C.POINTER(C.c_int32)), ("right", C.POINTER(C.c_int32)),
                ("depth", C.POINTER(C.c_int32)), ("leaf_class", C.POINTER(C.c_int32)),
                ("proj_nnz", C.POINTER(C.c_int32)), ("feat", C.POINTER(C.c_int32)),
                ("cand", C.POINTER(C.c_int32)), ("sign", C.POINTER(C.c_int8)),
                ("path", C.POINTER(C.c_int8)), ("threshold", C.POINTER(C.c_float)),
                ("n_samples", C.POINTER(C.c_int64)), ("class_counts", C.POINTER(C.c_int64)),
                ("gain", C.POINTER(C.c_double))]


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- random streams

def sm64_next(state: int):
    s = C.c_uint64(state)
    r = lib().orc_sm64_next(C.byref(s))
    return int(r), int(s.value)


def sm64(x: int) -> int:
    return int(lib().orc_sm64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def root_key(seed: int, tree_id: int) -> int:
    return int(lib().orc_root_key(C.c_uint64(seed), tree_id))


def child_key(key: int, side: int) -> int:
    return int(lib().orc_child_key(C.c_uint64(key), side))


def poisson_cdf(lam: float, cap: int) -> np.ndarray:
    out = np.zeros(max(cap - 1, 1), dtype=np.float64)
    lib().orc_poisson_cdf(lam, cap, _p(out))
    return out[:cap - 1]


def sample_node(key: int, P: int, d: int, lam: float, cap: int):
    """Returns (nnz int32[P], feat int32[P,cap], sign int8[P,cap]) for one node."""
    nnz = np.zeros(P, dtype=np.int32)
    feat = np.zeros((P, cap), dtype=np.int32)
    sign = np.zeros((P, cap), dtype=np.int8)
    rc = lib().orc_sample_node(C.c_uint64(key), P, d, lam, cap, _p(nnz), _p(feat), _p(sign))
    if rc:
        raise ValueError("orc_sample_node: bad arguments")
    return nnz, feat, sign


def slots_to_csr(nnz, feat, sign):
    P = nnz.shape[0]
    ptr = np.zeros(P + 1, dtype=np.int32)
    ptr[1:] = np.cumsum(nnz)
    f = np.concatenate([feat[p, :nnz[p]] for p in range(P)]).astype(np.int32) if P else np.zeros(0, np.int32)
    s = np.concatenate([sign[p, :nnz[p]] for p in range(P)]).astype(np.int8) if P else np.zeros(0, np.int8)
    return ptr, f, s


# ---------------------------------------------------------------- split search

def project(X: np.ndarray, idx: np.ndarray, feat: np.ndarray, sign: np.ndarray) -> np.ndarray:
    X = _c(X, np.float32)
    idx = _c(idx, np.int32)
    feat = _c(feat, np.int32)
    sign = _c(sign, np.int8)
    out = np.empty(idx.shape[0], dtype=np.float32)
    lib().orc_project(_p(X), X.shape[1], _p(idx), idx.shape[0], _p(feat), _p(sign),
                      feat.shape[0], _p(out))
    return out


def gini_gain(L, N, n: int, nL: int) -> float:
    L = _c(L, np.int64)
    N = _c(N, np.int64)
    return float(lib().orc_gini_gain(_p(L), _p(N), L.shape[0], n, nL))


def ln(x: float) -> float:
    """The entropy criterion's natural log (atanh series)."""
    return float(lib().orc_ln(float(x)))


def xlnx(x: int) -> float:
    return float(lib().orc_xlnx(int(x)))


def entropy_gain(L, N, n: int, nL: int) -> float:
    L = _c(L, np.int64)
    N = _c(N, np.int64)
    return float(lib().orc_entropy_gain(_p(L), _p(N), L.shape[0], n, nL))


def boundaries(mn: float, mx: float, B: int) -> np.ndarray:
    t = np.empty(B - 1, dtype=np.float32)
    lib().orc_boundaries(C.c_float(mn), C.c_float(mx), B, _p(t))
    return t


def rw_boundaries(key: int, p: int, mn: float, mx: float, B: int) -> np.ndarray:
    """Random-width boundaries t_1..t_{B-1} of projection p at the node with key `key`."""
    t = np.empty(B - 1, dtype=np.float32)
    lib().orc_rw_boundaries(C.c_uint64(key & 0xFFFFFFFFFFFFFFFF), p, C.c_float(mn), C.c_float(mx), B, _p(t))
    return t


def bin_of(t: np.ndarray, v: float) -> int:
    t = _c(t, np.float32)
    return int(lib().orc_bin(_p(t), t.shape[0], C.c_float(v)))


def midpoint(a: float, b: float) -> float:
    return float(np.float32(lib().orc_midpoint(C.c_float(a), C.c_float(b))))


@dataclasses.dataclass
class SplitResult:
    valid: int
    proj: int
    path: int
    cand: int
    threshold: np.float32
    gain: float
    n_left: int
    n_right: int
    left_counts: np.ndarray
    minmax: Optional[np.ndarray] = None     # float32 [P, 2]
    hist: Optional[np.ndarray] = None       # int32 [P, B, C]
    gains: Optional[np.ndarray] = None      # float64 [P, B-1]
    bounds: Optional[np.ndarray] = None     # float32 [P, B-1] boundaries t_1..t_{B-1}


def split_search(X: np.ndarray, y: np.ndarray, n_classes: int, idx: np.ndarray,
                 ptr: np.ndarray, feat: np.ndarray, sign: np.ndarray, n_bins: int = 256,
                 sort_below: int = 1024, hist_only: bool = False,
                 want_debug: bool = False, bin_rule: int = 0, bin_key: int = 0,
                 criterion: int = 0) -> SplitResult:
    """bin_rule 0: equal-width boundaries; 1: random-width boundaries drawn
    from the node key bin_key.  criterion 0: Gini decrease; 1: information gain."""
    X = _c(X, np.float32)
    y = _c(y, np.uint8)
    idx = _c(idx, np.int32)
    ptr = _c(ptr, np.int32)
    feat = _c(feat, np.int32)
    sign = _c(sign, np.int8)
    P = ptr.shape[0] - 1
    out = OrcSplit()
    lc = np.zeros(n_classes, dtype=np.int64)
    mm = hist = gains = bounds = None
    if want_debug:
        mm = np.zeros((P, 2), dtype=np.float32)
        hist = np.zeros((P, n_bins, n_classes), dtype=np.int32)
        gains = np.full((P, n_bins - 1), -1.0, dtype=np.float64)
        bounds = np.zeros((P, n_bins - 1), dtype=np.float32)
    opt = lambda a: _p(a) if a is not None else None  # noqa: E731
    rc = lib().orc_split_search_rule(
        _p(X), X.shape[1], _p(y), n_classes, _p(idx), idx.shape[0], P, _p(ptr), _p(feat),
        _p(sign), n_bins, sort_below, int(bool(hist_only)), int(bin_rule),
        C.c_uint64(bin_key & 0xFFFFFFFFFFFFFFFF), 0, int(criterion), C.byref(out), _p(lc), opt(mm),
        opt(hist), opt(gains), opt(bounds))
    if rc:
        raise ValueError("orc_split_search_rule failed")
    return SplitResult(out.valid, out.proj, out.path, out.cand, np.float32(out.threshold),
                       out.gain, out.n_left, out.n_right, lc, mm, hist, gains, bounds)


def split_search_mt(X: np.ndarray, y: np.ndarray, n_classes: int, idx: np.ndarray,
                    ptr: np.ndarray, feat: np.ndarray, sign: np.ndarray, n_bins: int = 256,
                    sort_below: int = 1024, hist_only: bool = False, n_threads: int = 1,
                    bin_rule: int = 0, bin_key: int = 0, criterion: int = 0) -> SplitResult:
    """split_search with the projections divided over n_threads host threads
    (same result; no debug outputs)."""
    X = _c(X, np.float32)
    y = _c(y, np.uint8)
    idx = _c(idx, np.int32)
    ptr = _c(ptr, np.int32)
    feat = _c(feat, np.int32)
    sign = _c(sign, np.int8)
    P = ptr.shape[0] - 1
    out = OrcSplit()
    lc = np.zeros(n_classes, dtype=np.int64)
    rc = lib().orc_split_search_mt(_p(X), X.shape[1], _p(y), n_classes, _p(idx), idx.shape[0], P, _p(ptr),
                                   _p(feat), _p(sign), n_bins, sort_below, int(bool(hist_only)),
                                   int(bin_rule), C.c_uint64(bin_key & 0xFFFFFFFFFFFFFFFF), int(criterion),
                                   n_threads, C.byref(out), _p(lc))
    if rc:
        raise ValueError("orc_split_search_mt failed")
    return SplitResult(out.valid, out.proj, out.path, out.cand, np.float32(out.threshold),
                       out.gain, out.n_left, out.n_right, lc)


def partition(X: np.ndarray, idx: np.ndarray, feat, sign, threshold: float):
    """Stable partition; returns (new idx, n_left)."""
    X = _c(X, np.float32)
    out = _c(idx, np.int32).copy()
    feat = _c(feat, np.int32)
    sign = _c(sign, np.int8)
    nl = lib().orc_partition(_p(X), X.shape[1], _p(out), out.shape[0], _p(feat), _p(sign),
                             feat.shape[0], C.c_float(threshold))
    if nl < 0:
        raise MemoryError
    return out, int(nl)


# ---------------------------------------------------------------- trees

@dataclasses.dataclass
class Tree:
    n_nodes: int
    left: np.ndarray
    right: np.ndarray
    depth: np.ndarray
    leaf_class: np.ndarray
    proj_nnz: np.ndarray
    feat: np.ndarray        # [n_nodes, cap]
    sign: np.ndarray        # [n_nodes, cap]
    cand: np.ndarray
    path: np.ndarray
    threshold: np.ndarray
    n_samples: np.ndarray
    class_counts: np.ndarray  # [n_nodes, C]
    gain: np.ndarray

    FIELDS = ("left", "right", "depth", "leaf_class", "proj_nnz", "feat", "sign", "cand",
              "path", "threshold", "n_samples", "class_counts", "gain")


def train_tree(X: np.ndarray, y: np.ndarray, n_classes: int, root_idx: np.ndarray, *,
               n_proj: int, lam: float, cap: int, n_bins: int = 256, sort_below: int = 1024,
               hist_only: bool = False, seed: int = 0, tree_id: int = 0,
               max_depth: int = -1, bin_rule: int = 0, criterion: int = 0,
               n_threads: Optional[int] = None, big_node: int = 65536) -> Tree:
    """n_threads None: orc_train_tree; an int: orc_train_tree_mt on that many
    host threads (each level's nodes searched in parallel, nodes of at least
    big_node samples with their projections divided over the threads; the
    same tree)."""
    X = _c(X, np.float32)
    y = _c(y, np.uint8)
    root_idx = _c(root_idx, np.int32)
    t = OrcTree()
    args = (_p(X), X.shape[1], X.shape[0], _p(y), n_classes, _p(root_idx),
            root_idx.shape[0], n_bins, sort_below, int(bool(hist_only)),
            int(bin_rule), int(criterion), n_proj, lam, cap, C.c_uint64(seed), tree_id,
            max_depth)
    if n_threads is None:
        rc = lib().orc_train_tree(*args, C.byref(t))
    else:
        rc = lib().orc_train_tree_mt(*args, int(n_threads), int(big_node), C.byref(t))
    if rc:
        raise RuntimeError("orc_train_tree failed")
    try:
        m = int(t.n_nodes)

        def arr(ptr, count, dtype):
            return np.ctypeslib.as_array(ptr, shape=(count,)).astype(dtype, copy=True)

        tree = Tree(
            n_nodes=m,
            left=arr(t.left, m, np.int32), right=arr(t.right, m, np.int32),
            depth=arr(t.depth, m, np.int32), leaf_class=arr(t.leaf_class, m, np.int32),
            proj_nnz=arr(t.proj_nnz, m, np.int32),
            feat=arr(t.feat, m * cap, np.int32).reshape(m, cap),
            sign=arr(t.sign, m * cap, np.int8).reshape(m, cap),
            cand=arr(t.cand, m, np.int32), path=arr(t.path, m, np.int8),
            threshold=arr(t.threshold, m, np.float32),
            n_samples=arr(t.n_samples, m, np.int64),
            class_counts=arr(t.class_counts, m * n_classes, np.int64).reshape(m, n_classes),
            gain=arr(t.gain, m, np.float64))
    finally:
        lib().orc_tree_free(C.byref(t))
    return tree


def predict_tree(tree: Tree, X: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Leaf class of each row (plain traversal, v < threshold goes left)."""
    X = _c(X, np.float32)
    out = np.empty(rows.shape[0], dtype=np.int32)
    for r_i, r in enumerate(rows):
        node = 0
        while tree.left[node] >= 0:
            k = tree.proj_nnz[node]
            acc = np.float32(0.0)
            for q in range(k):
                x = X[tree.feat[node, q], r]
                acc = np.float32(acc + (x if tree.sign[node, q] == 1 else -x))
            node = tree.left[node] if acc < tree.threshold[node] else tree.right[node]
        out[r_i] = tree.leaf_class[node]
    return out


def predict_tree_c(tree: Tree, X: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Leaf class of each row through the C traversal (orc_predict_tree)."""
    X = _c(X, np.float32)
    rows = _c(rows, np.int32)
    keep = {f: np.ascontiguousarray(getattr(tree, f)) for f in Tree.FIELDS}
    t = OrcTree()
    t.n_nodes = tree.n_nodes
    t.n_classes = keep["class_counts"].shape[1] if keep["class_counts"].ndim == 2 else 1
    t.cap = keep["feat"].shape[1]
    for f, ct in (("left", C.c_int32), ("right", C.c_int32), ("depth", C.c_int32), ("leaf_class", C.c_int32),
                  ("proj_nnz", C.c_int32), ("feat", C.c_int32), ("cand", C.c_int32), ("sign", C.c_int8),
                  ("path", C.c_int8), ("threshold", C.c_float), ("n_samples", C.c_int64),
                  ("class_counts", C.c_int64), ("gain", C.c_double)):
        setattr(t, f, keep[f].ctypes.data_as(C.POINTER(ct)))
    out = np.empty(rows.shape[0], dtype=np.int32)
    lib().orc_predict_tree(C.byref(t), _p(X), X.shape[1], _p(rows), rows.shape[0], _p(out))
    return out


def predict_forest(trees, X: np.ndarray, rows: np.ndarray, n_classes: int):
    """Majority vote of the trees' leaf classes; ties go to the lowest class.
    Returns (pred int32 [n], votes int32 [n, n_classes])."""
    votes = np.zeros((rows.shape[0], n_classes), dtype=np.int32)
    for t in trees:
        cls = predict_tree_c(t, X, rows)
        np.add.at(votes, (np.arange(rows.shape[0]), cls), 1)
    return np.argmax(votes, axis=1).astype(np.int32), votes
