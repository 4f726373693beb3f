"""Thin Python binding of the C ABI in include/soforest.h.

Argument marshalling only: every step of the split search runs in the CUDA
library (lib/libsoforest.so).  Device memory and streams come from PyTorch.
There is no fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsoforest.so")

SO_OK, SO_EINVAL, SO_ENOMEM, SO_ECUDA, SO_ETIMEOUT, SO_EINTERNAL = range(6)


class SoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"soforest status {status}: {msg}")
        self.status = status


# ---------------------------------------------------------------- C structs
class so_dataset(C.Structure):
    _fields_ = [("X", C.c_void_p), ("n", C.c_int64), ("d", C.c_int32), ("ld", C.c_int64),
                ("y", C.c_void_p), ("n_classes", C.c_int32), ("Xr", C.c_void_p)]


class so_projs(C.Structure):
    _fields_ = [("n_proj", C.c_int32), ("ptr", C.c_void_p), ("feat", C.c_void_p), ("sign", C.c_void_p),
                ("max_nnz", C.c_int32)]


SO_BINS_EQUAL_WIDTH = 0
SO_BINS_RANDOM_WIDTH = 1
SO_CRIT_GINI = 0
SO_CRIT_ENTROPY = 1


class so_split_params(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("sort_below", C.c_int32), ("hist_only", C.c_int32),
                ("rescore_rel_eps", C.c_float), ("bin_rule", C.c_int32), ("criterion", C.c_int32),
                ("bin_keys", C.c_void_p), ("proj_per_cta", C.c_int32), ("chunk", C.c_int32)]


class so_split(C.Structure):
    _fields_ = [("valid", C.c_int32), ("proj", C.c_int32), ("path", C.c_int32), ("cand", C.c_int32),
                ("threshold", C.c_float), ("gain", C.c_double), ("n_left", C.c_int64),
                ("n_right", C.c_int64)]


class so_tree_params(C.Structure):
    _fields_ = [("n_bins", C.c_int32), ("sort_below", C.c_int32), ("hist_only", C.c_int32),
                ("rescore_rel_eps", C.c_float), ("n_proj", C.c_int32), ("lambda_", C.c_double),
                ("nnz_cap", C.c_int32), ("seed", C.c_uint64), ("tree_id", C.c_int32),
                ("max_depth", C.c_int32), ("bin_rule", C.c_int32), ("criterion", C.c_int32),
                ("proj_per_cta", C.c_int32), ("chunk", C.c_int32)]


class so_tree(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_classes", C.c_int32), ("cap", C.c_int32),
                ("left", C.POINTER(C.c_int32)), ("right", C.POINTER(C.c_int32)),
                ("depth", C.POINTER(C.c_int32)), ("leaf_class", C.POINTER(C.c_int32)),
                ("proj_nnz", C.POINTER(C.c_int32)), ("feat", C.POINTER(C.c_int32)),
                ("cand", C.POINTER(C.c_int32)), ("sign", C.POINTER(C.c_int8)),
                ("path", C.POINTER(C.c_int8)), ("threshold", C.POINTER(C.c_float)),
                ("n_samples", C.POINTER(C.c_int64)), ("class_counts", C.POINTER(C.c_int64)),
                ("gain", C.POINTER(C.c_double))]


class so_forest(C.Structure):
    _fields_ = [("n_trees", C.c_int32), ("n_classes", C.c_int32), ("cap", C.c_int32),
                ("tree_off", C.c_void_p), ("left", C.c_void_p), ("right", C.c_void_p),
                ("leaf_class", C.c_void_p), ("proj_nnz", C.c_void_p), ("feat", C.c_void_p),
                ("sign", C.c_void_p), ("threshold", C.c_void_p)]


class so_profile_entry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


# numpy view of an so_split array (48 bytes per record)
SPLIT_DTYPE = np.dtype([("valid", "<i4"), ("proj", "<i4"), ("path", "<i4"), ("cand", "<i4"),
                        ("threshold", "<f4"), ("_pad", "<i4"), ("gain", "<f8"),
                        ("n_left", "<i8"), ("n_right", "<i8")])
assert SPLIT_DTYPE.itemsize == C.sizeof(so_split) == 48

_V, _P, _I32, _I64, _U64, _F, _D, _SZ = (C.c_void_p, C.POINTER, C.c_int32, C.c_int64, C.c_uint64,
                                         C.c_float, C.c_double, C.c_size_t)

_SIGS = {
    "so_split_search": (_I32, [C.POINTER(so_dataset), _V, _I64, C.POINTER(so_projs),
                               C.POINTER(so_split_params), C.POINTER(so_split), _V, _V, _SZ, _V]),
    "so_split_search_batch": (_I32, [C.POINTER(so_dataset), _V, _I64, _V, _I32, C.POINTER(so_projs),
                                     C.POINTER(so_split_params), _V, _V, _V, _SZ, _V]),
    "so_split_search_noalloc": (_I32, [C.POINTER(so_dataset), _V, _I64, C.POINTER(so_projs),
                                       C.POINTER(so_split_params), C.POINTER(so_split), _V, _V]),
    "so_split_search_ws_bytes": (_SZ, [_I32, _I64, _I32, _I32, C.POINTER(so_split_params)]),
    "so_partition": (_I32, [C.POINTER(so_dataset), _V, _I64, _V, _V, _I32, _F, C.POINTER(C.c_int64), _V]),
    "so_partition_batch": (_I32, [C.POINTER(so_dataset), _V, _V, _I64, _V, _I32, C.POINTER(so_projs),
                                  _V, _V]),
    "so_sample_projections": (_I32, [_I32, _V, _I32, _I32, _D, _I32, _V, _V, _V, _V]),
    "so_histograms": (_I32, [C.POINTER(so_dataset), _V, _I64, _V, _I32, C.POINTER(so_projs),
                             C.POINTER(so_split_params), _V, _V, _V, _V, _V]),
    "so_train_tree": (_I32, [C.POINTER(so_dataset), _V, _I64, C.POINTER(so_tree_params),
                             C.POINTER(so_tree), _V]),
    "so_tree_free": (None, [C.POINTER(so_tree)]),
    "so_autotune": (_I32, [C.POINTER(so_dataset), _I32, _D, _I32, C.POINTER(so_split_params), _V, _V, _V, _V]),
    "so_predict": (_I32, [_V, _I64, _I32, _I64, C.POINTER(so_forest), _V, _V, _V]),
    "so_row_major": (_I32, [_V, _I64, _I32, _I64, _V, _V]),
    "so_last_error": (C.c_char_p, []),
    "so_shutdown": (None, []),
    "so_version": (C.c_char_p, []),
    "so_profile_enable": (None, [_I32]),
    "so_profile_read": (_I32, [C.POINTER(so_profile_entry), _I32]),
    "so_launch_count": (_I64, []),
}

_lib = None


def lib():
    """Loads libsoforest.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2603_00326_b300.build)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != SO_OK:
        raise SoError(status, lib().so_last_error().decode())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


# ---------------------------------------------------------------- wrappers
@dataclasses.dataclass
class DeviceDataset:
    """X: cuda float32 [d, n] (row f holds feature f), y: cuda uint8 [n].
    Xr: optional cuda float32 [n, d], the same values row-major (see
    with_row_major); used to read scattered samples' feature rows."""
    X: "object"
    y: "object"
    n_classes: int
    Xr: "object" = None

    def c(self) -> so_dataset:
        X = self.X
        assert X.is_cuda and X.dtype.__str__() == "torch.float32" and X.dim() == 2
        assert X.stride(1) == 1
        xr = 0
        if self.Xr is not None:
            assert self.Xr.is_cuda and tuple(self.Xr.shape) == (X.shape[1], X.shape[0]) and self.Xr.is_contiguous()
            xr = self.Xr.data_ptr()
        return so_dataset(X.data_ptr(), X.shape[1], X.shape[0], X.stride(0), self.y.data_ptr(),
                          self.n_classes, xr)

    def with_row_major(self, stream=None) -> "DeviceDataset":
        """The same dataset with a row-major copy of X on the device (so_row_major)."""
        import torch
        X = self.X
        Xr = torch.empty((X.shape[1], X.shape[0]), dtype=torch.float32, device=X.device)
        _check(lib().so_row_major(X.data_ptr(), X.shape[1], X.shape[0], X.stride(0), Xr.data_ptr(),
                                  _stream(stream)))
        return DeviceDataset(self.X, self.y, self.n_classes, Xr)


@dataclasses.dataclass
class DeviceProjs:
    """CSR projection rows on the device: ptr int32 [rows+1], feat int32, sign int8.
    max_nnz: upper bound of the row lengths (0 = unknown)."""
    n_proj: int
    ptr: "object"
    feat: "object"
    sign: "object"
    max_nnz: int = 0

    def c(self) -> so_projs:
        return so_projs(self.n_proj, self.ptr.data_ptr(), self.feat.data_ptr(), self.sign.data_ptr(),
                        self.max_nnz)


def split_params(n_bins=256, sort_below=1024, hist_only=False, rescore_rel_eps=0.0, bin_rule=0,
                 bin_keys=None, criterion=0, proj_per_cta=0, chunk=0) -> so_split_params:
    """bin_rule SO_BINS_RANDOM_WIDTH needs bin_keys: a device int64 tensor [m]
    holding the nodes' uint64 keys (kept alive by the returned struct).
    criterion SO_CRIT_GINI or SO_CRIT_ENTROPY.  proj_per_cta, chunk: the
    histogram work decomposition (0: defaults; so_autotune picks them)."""
    p = so_split_params(n_bins, sort_below, 1 if hist_only else 0, rescore_rel_eps, bin_rule, criterion,
                        _ptr(bin_keys), proj_per_cta, chunk)
    p._keys = bin_keys
    return p


def so_version() -> str:
    return lib().so_version().decode()


def so_last_error() -> str:
    return lib().so_last_error().decode()


def so_shutdown():
    lib().so_shutdown()


def so_launch_count() -> int:
    return int(lib().so_launch_count())


def so_profile_enable(on: bool):
    lib().so_profile_enable(1 if on else 0)


def so_profile_read() -> dict:
    arr = (so_profile_entry * 64)()
    k = lib().so_profile_read(arr, 64)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(k)}


def so_split_search(ds: DeviceDataset, idx, projs: DeviceProjs, params: so_split_params,
                    workspace=None, stream=None):
    """One node.  Returns (so_split, left_counts numpy int64[C])."""
    out = so_split()
    lc = np.zeros(8, dtype=np.int64)
    d = ds.c()
    p = projs.c()
    n = 0 if idx is None else int(idx.numel())
    _check(lib().so_split_search(C.byref(d), _ptr(idx), n, C.byref(p), C.byref(params), C.byref(out),
                                 lc.ctypes.data_as(C.c_void_p), _ptr(workspace),
                                 0 if workspace is None else workspace.numel() * workspace.element_size(),
                                 _stream(stream)))
    return out, lc[:ds.n_classes].copy()


def so_split_search_noalloc(ds: DeviceDataset, idx, projs: DeviceProjs, params: so_split_params, stream=None):
    """One node with the library's static scratch (no device allocation).
    Returns (so_split, left_counts numpy int64[C])."""
    out = so_split()
    lc = np.zeros(8, dtype=np.int64)
    d = ds.c()
    p = projs.c()
    n = 0 if idx is None else int(idx.numel())
    _check(lib().so_split_search_noalloc(C.byref(d), _ptr(idx), n, C.byref(p), C.byref(params), C.byref(out),
                                         lc.ctypes.data_as(C.c_void_p), _stream(stream)))
    return out, lc[:ds.n_classes].copy()


def so_split_search_ws_bytes(m, n_total, n_proj, n_classes, params) -> int:
    return int(lib().so_split_search_ws_bytes(m, n_total, n_proj, n_classes, C.byref(params)))


def so_split_search_batch(ds: DeviceDataset, idx, node_off, projs: DeviceProjs, params: so_split_params,
                          out=None, left_counts=None, workspace=None, stream=None):
    """m nodes (node_off: cuda int64 [m+1]).  Returns (out uint8 tensor [m*48], left_counts int64 [m*C])."""
    import torch
    m = int(node_off.numel()) - 1
    dev = idx.device
    if out is None:
        out = torch.empty(m * SPLIT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    if left_counts is None:
        left_counts = torch.empty(m * ds.n_classes, dtype=torch.int64, device=dev)
    d = ds.c()
    p = projs.c()
    _check(lib().so_split_search_batch(
        C.byref(d), _ptr(idx), int(idx.numel()), _ptr(node_off), m, C.byref(p), C.byref(params),
        _ptr(out), _ptr(left_counts), _ptr(workspace),
        0 if workspace is None else workspace.numel() * workspace.element_size(), _stream(stream)))
    return out, left_counts


def splits_to_numpy(out) -> np.ndarray:
    return out.cpu().numpy().view(SPLIT_DTYPE)


def so_partition(ds: DeviceDataset, idx, feat, sign, threshold: float, stream=None) -> int:
    d = ds.c()
    nl = C.c_int64(0)
    _check(lib().so_partition(C.byref(d), _ptr(idx), int(idx.numel()), _ptr(feat), _ptr(sign),
                              int(feat.numel()), C.c_float(threshold), C.byref(nl), _stream(stream)))
    return int(nl.value)


def so_partition_batch(ds: DeviceDataset, idx_in, idx_out, node_off, projs: DeviceProjs, splits,
                       stream=None):
    d = ds.c()
    p = projs.c()
    _check(lib().so_partition_batch(C.byref(d), _ptr(idx_in), _ptr(idx_out), int(idx_in.numel()),
                                    _ptr(node_off), int(node_off.numel()) - 1, C.byref(p), _ptr(splits),
                                    _stream(stream)))


def so_sample_projections(keys, n_proj: int, d: int, lam: float, cap: int, stream=None):
    """keys: cuda int64 [m] (bit patterns of uint64 keys).  Returns (nnz, feat, sign) slot tensors."""
    import torch
    m = int(keys.numel())
    nnz = torch.empty(m * n_proj, dtype=torch.int32, device=keys.device)
    feat = torch.zeros(m * n_proj * cap, dtype=torch.int32, device=keys.device)
    sign = torch.zeros(m * n_proj * cap, dtype=torch.int8, device=keys.device)
    _check(lib().so_sample_projections(m, _ptr(keys), n_proj, d, lam, cap, _ptr(nnz), _ptr(feat),
                                       _ptr(sign), _stream(stream)))
    return nnz, feat, sign


def so_histograms(ds: DeviceDataset, idx, node_off, projs: DeviceProjs, n_bins: int, want_gains=False,
                  stream=None, bin_rule=0, bin_keys=None, want_bounds=False):
    """Histogram stage of m nodes.  Returns (minmax [m,P,2], hist [m,P,B,C],
    gains [m,P,B-1] or None); with want_bounds also the boundaries [m,P,B-1]."""
    import torch
    m = int(node_off.numel()) - 1
    P, Cc = projs.n_proj, ds.n_classes
    dev = idx.device
    mm = torch.zeros((m, P, 2), dtype=torch.float32, device=dev)
    hist = torch.zeros((m, P, n_bins, Cc), dtype=torch.int32, device=dev)
    gains = torch.zeros((m, P, n_bins - 1), dtype=torch.float32, device=dev) if want_gains else None
    bounds = torch.zeros((m, P, n_bins - 1), dtype=torch.float32, device=dev) if want_bounds else None
    d = ds.c()
    p = projs.c()
    prm = split_params(n_bins, bin_rule=bin_rule, bin_keys=bin_keys)
    _check(lib().so_histograms(C.byref(d), _ptr(idx), int(idx.numel()), _ptr(node_off), m, C.byref(p),
                               C.byref(prm), _ptr(mm), _ptr(hist), _ptr(gains), _ptr(bounds), _stream(stream)))
    if want_bounds:
        return mm, hist, gains, bounds
    return mm, hist, gains


@dataclasses.dataclass
class Tree:
    n_nodes: int
    left: np.ndarray
    right: np.ndarray
    depth: np.ndarray
    leaf_class: np.ndarray
    proj_nnz: np.ndarray
    feat: np.ndarray
    sign: np.ndarray
    cand: np.ndarray
    path: np.ndarray
    threshold: np.ndarray
    n_samples: np.ndarray
    class_counts: np.ndarray
    gain: np.ndarray

    FIELDS = ("left", "right", "depth", "leaf_class", "proj_nnz", "feat", "sign", "cand",
              "path", "threshold", "n_samples", "class_counts", "gain")


def tree_params(n_proj, lam, cap, n_bins=256, sort_below=1024, hist_only=False, seed=0, tree_id=0,
                max_depth=-1, rescore_rel_eps=0.0, bin_rule=0, criterion=0, proj_per_cta=0,
                chunk=0) -> so_tree_params:
    return so_tree_params(n_bins, sort_below, 1 if hist_only else 0, rescore_rel_eps, n_proj, lam, cap,
                          seed & 0xFFFFFFFFFFFFFFFF, tree_id, max_depth, bin_rule, criterion, proj_per_cta,
                          chunk)


def so_train_tree(ds: DeviceDataset, root_idx, params: so_tree_params, stream=None) -> Tree:
    d = ds.c()
    t = so_tree()
    _check(lib().so_train_tree(C.byref(d), _ptr(root_idx), int(root_idx.numel()), C.byref(params),
                               C.byref(t), _stream(stream)))
    try:
        m, cap, Cc = int(t.n_nodes), int(t.cap), int(t.n_classes)

        def arr(ptr, count, dtype):
            return np.ctypeslib.as_array(ptr, shape=(count,)).astype(dtype, copy=True)

        return Tree(
            n_nodes=m, left=arr(t.left, m, np.int32), right=arr(t.right, m, np.int32),
            depth=arr(t.depth, m, np.int32), leaf_class=arr(t.leaf_class, m, np.int32),
            proj_nnz=arr(t.proj_nnz, m, np.int32),
            feat=arr(t.feat, m * cap, np.int32).reshape(m, cap),
            sign=arr(t.sign, m * cap, np.int8).reshape(m, cap),
            cand=arr(t.cand, m, np.int32), path=arr(t.path, m, np.int8),
            threshold=arr(t.threshold, m, np.float32), n_samples=arr(t.n_samples, m, np.int64),
            class_counts=arr(t.class_counts, m * Cc, np.int64).reshape(m, Cc),
            gain=arr(t.gain, m, np.float64))
    finally:
        lib().so_tree_free(C.byref(t))


@dataclasses.dataclass
class DeviceForest:
    """Trees' node arrays concatenated on the device (see so_forest)."""
    n_trees: int
    n_classes: int
    cap: int
    arrays: dict

    def c(self) -> so_forest:
        a = self.arrays
        return so_forest(self.n_trees, self.n_classes, self.cap, a["tree_off"].data_ptr(), a["left"].data_ptr(),
                         a["right"].data_ptr(), a["leaf_class"].data_ptr(), a["proj_nnz"].data_ptr(),
                         a["feat"].data_ptr(), a["sign"].data_ptr(), a["threshold"].data_ptr())


def upload_forest(trees: List[Tree], n_classes: int, device="cuda") -> DeviceForest:
    """Concatenates host trees (so_train_tree results) into a DeviceForest."""
    import torch
    cap = max(int(t.feat.shape[1]) for t in trees) if trees else 1
    sizes = [int(t.n_nodes) for t in trees]
    off = np.zeros(len(trees) + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)

    def cat(field, dtype, width=None):
        parts = []
        for t in trees:
            a = getattr(t, field)
            if width is not None:
                b = np.zeros((a.shape[0], width), dtype=dtype)
                b[:, :a.shape[1]] = a
                a = b
            parts.append(np.ascontiguousarray(a, dtype=dtype).reshape(-1))
        return np.concatenate(parts) if parts else np.zeros(1, dtype=dtype)

    host = {"tree_off": off, "left": cat("left", np.int32), "right": cat("right", np.int32),
            "leaf_class": cat("leaf_class", np.int32), "proj_nnz": cat("proj_nnz", np.int32),
            "feat": cat("feat", np.int32, cap), "sign": cat("sign", np.int8, cap),
            "threshold": cat("threshold", np.float32)}
    dev = {k: torch.from_numpy(v).to(device) for k, v in host.items()}
    return DeviceForest(len(trees), n_classes, cap, dev)


def so_predict(X, forest: DeviceForest, want_votes: bool = False, stream=None):
    """Majority-vote prediction of every column of X (cuda float32 [d, n]).
    Returns (pred int32 [n], votes int32 [n, C] or None) as cuda tensors."""
    import torch
    assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
    n, d = X.shape[1], X.shape[0]
    pred = torch.empty(n, dtype=torch.int32, device=X.device)
    votes = torch.empty((n, forest.n_classes), dtype=torch.int32, device=X.device) if want_votes else None
    f = forest.c()
    _check(lib().so_predict(X.data_ptr(), n, d, X.stride(0), C.byref(f), votes.data_ptr() if votes is not None else None,
                            pred.data_ptr(), _stream(stream)))
    return pred, votes


# the tuner's procedure: cached choices of an older procedure are not reused
AUTOTUNE_VERSION = 2


def _autotune_key(ds, n_proj, lam, cap, params, gpu: str) -> str:
    return (f"v{AUTOTUNE_VERSION}|{gpu}|n={ds.X.shape[1]}|d={ds.X.shape[0]}|C={ds.n_classes}|P={n_proj}|lam={lam}|cap={cap}"
            f"|B={params.n_bins}|rule={params.bin_rule}|crit={params.criterion}|rowmajor={int(ds.Xr is not None)}")


def autotune_cached(ds: DeviceDataset, n_proj: int, lam: float, cap: int, params: so_split_params,
                    cache_path=None, stream=None):
    """so_autotune with its choices (crossover T, projections per CTA, samples
    per item) cached as JSON per GPU model and workload shape; a later call
    with the same key reuses them without timing.  Returns (params, cached)."""
    import json
    import os
    import torch
    path = cache_path or os.path.join(os.path.expanduser("~"), ".cache", "soforest", "autotune.json")
    dev = ds.X.device
    gpu = torch.cuda.get_device_name(dev) if dev.type == "cuda" else str(dev)
    key = _autotune_key(ds, n_proj, lam, cap, params, gpu)
    try:
        with open(path) as fh:
            table = json.load(fh)
    except (OSError, ValueError):
        table = {}
    hit = table.get(key)
    if hit is not None:
        params.sort_below, params.proj_per_cta, params.chunk = hit["sort_below"], hit["proj_per_cta"], hit["chunk"]
        return params, True
    params, _, _ = so_autotune(ds, n_proj, lam, cap, params, stream)
    table[key] = {"sort_below": int(params.sort_below), "proj_per_cta": int(params.proj_per_cta),
                  "chunk": int(params.chunk)}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return params, False


def so_autotune(ds: DeviceDataset, n_proj: int, lam: float, cap: int, params: so_split_params, stream=None):
    """Crossover microbenchmark; sets params.sort_below.  Returns (params, sizes, times_ms[n,2])."""
    d = ds.c()
    sizes = np.zeros(16, dtype=np.int32)
    times = np.zeros(32, dtype=np.float32)
    k = C.c_int32(0)
    _check(lib().so_autotune(C.byref(d), n_proj, lam, cap, C.byref(params), sizes.ctypes.data_as(C.c_void_p),
                             times.ctypes.data_as(C.c_void_p), C.byref(k), _stream(stream)))
    n = int(k.value)
    return params, sizes[:n].copy(), times[:2 * n].reshape(n, 2).copy()
