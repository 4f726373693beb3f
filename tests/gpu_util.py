"""Helpers for the GPU parity tests: upload seeded inputs, run the oracle on
the same inputs, and compare results field by field."""
import numpy as np

import oracle as O


def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


def upload_dataset(X, y, C):
    torch = torch_cuda()
    from paper_2603_00326_b300 import soforest as S
    Xt = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
    yt = torch.from_numpy(np.ascontiguousarray(y, dtype=np.uint8)).cuda()
    return S.DeviceDataset(Xt, yt, C)


def upload_projs(ptr, feat, sign, P, max_nnz=None):
    """max_nnz=None: the true longest row (selects the narrowest kernel variant);
    0: unknown (widest variant)."""
    torch = torch_cuda()
    from paper_2603_00326_b300 import soforest as S
    if max_nnz is None:
        max_nnz = int(np.diff(np.asarray(ptr)).max()) if len(ptr) > 1 else 0
    return S.DeviceProjs(P, torch.from_numpy(np.ascontiguousarray(ptr, np.int32)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(feat, np.int32)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(sign, np.int8)).cuda(), max_nnz)


def i32(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()


def i64(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, np.int64)).cuda()


def concat_projs(proj_list):
    """List of per-node (ptr, feat, sign) CSR -> one node-major CSR."""
    ptrs, feats, signs = [np.zeros(1, np.int32)], [], []
    base = 0
    for (ptr, feat, sign) in proj_list:
        ptrs.append(ptr[1:] + base)
        feats.append(feat)
        signs.append(sign)
        base += int(ptr[-1])
    return (np.concatenate(ptrs).astype(np.int32), np.concatenate(feats).astype(np.int32),
            np.concatenate(signs).astype(np.int8))


def f32bits(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def f64bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def assert_split_equal(gpu, orc, ctx=""):
    """gpu: record with fields (numpy structured row or ctypes so_split); orc: oracle SplitResult."""
    g = {k: (gpu[k] if not hasattr(gpu, "_fields_") else getattr(gpu, k))
         for k in ("valid", "proj", "path", "cand", "threshold", "gain", "n_left", "n_right")}
    assert int(g["valid"]) == orc.valid, (ctx, g, orc)
    assert int(g["path"]) == orc.path, (ctx, g, orc)
    if orc.valid:
        assert int(g["proj"]) == orc.proj, (ctx, g, orc)
        assert int(g["cand"]) == orc.cand, (ctx, g, orc)
        assert f32bits(g["threshold"]) == f32bits(orc.threshold), (ctx, g, orc)
        assert f64bits(g["gain"]) == f64bits(orc.gain), (ctx, g, orc)
        assert int(g["n_left"]) == orc.n_left and int(g["n_right"]) == orc.n_right, (ctx, g, orc)
    else:
        assert int(g["proj"]) == -1 and int(g["cand"]) == -1, (ctx, g, orc)


def oracle_node_projs(ptr, feat, sign, P, j):
    """CSR rows of node j out of a node-major CSR."""
    rows = ptr[j * P:(j + 1) * P + 1]
    base = int(rows[0])
    return (rows - base).astype(np.int32), feat[base:int(rows[-1])], sign[base:int(rows[-1])]


def assert_tree_equal(gt, ot, ctx=""):
    """Every field of two trees bit for bit; names the first differing node."""
    assert gt.n_nodes == ot.n_nodes, (ctx, gt.n_nodes, ot.n_nodes)
    for f in O.Tree.FIELDS:
        a, b = np.asarray(getattr(gt, f)), np.asarray(getattr(ot, f))
        assert a.shape == b.shape, (ctx, f)
        bad = np.flatnonzero((a.view(np.uint8).reshape(a.shape[0], -1) !=
                              b.view(np.uint8).reshape(b.shape[0], -1)).any(axis=1))
        assert bad.size == 0, (ctx, f, "first differing node", int(bad[0]) if bad.size else None)


def oracle_tree_all_cores(X, y, C, root, **kw):
    """The oracle's tree grown on every host core (orc_train_tree_mt)."""
    import os
    return O.train_tree(X, y, C, root, n_threads=os.cpu_count() or 1, **kw)
