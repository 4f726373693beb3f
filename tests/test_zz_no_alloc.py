"""so_split_search_noalloc -- the single-node split search for callers that
cannot allocate device memory (a framework's memory pool owns the device,
a fixed memory budget, or a loop that must not pay for cudaMalloc's implicit
synchronisation).  Its scratch is a static device array inside the library.

Checked through the C ABI against so_split_search (which uses a workspace) on
the same inputs, two calls in a row with different nodes, so leftovers of the
first call in the shared static scratch cannot change the second result.
Collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2603_00326_b300 import datagen as G

pytestmark = pytest.mark.gpu


def _node_inputs(seed, n_data, d, C_, n_node, P):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((d, n_data)).astype(np.float32)
    y = rng.integers(0, C_, n_data).astype(np.uint8)
    idx = rng.integers(0, n_data, n_node).astype(np.int32)
    pr = G.random_projections(rng, P, d, 1.5, 8)
    return X, y, idx, pr


def _to_device(torch, X, y, idx, pr, C_):
    from paper_2603_00326_b300 import soforest as S
    ds = S.DeviceDataset(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), C_)
    pj = S.DeviceProjs(pr.n_proj, torch.from_numpy(pr.ptr).cuda(), torch.from_numpy(pr.feat).cuda(),
                       torch.from_numpy(pr.sign).cuda(), int(np.diff(pr.ptr).max()))
    return ds, pj, torch.from_numpy(idx).cuda()


def _same(a, b):
    for f in ("valid", "proj", "path", "cand", "n_left", "n_right"):
        assert getattr(a, f) == getattr(b, f), f
    assert np.float32(a.threshold).tobytes() == np.float32(b.threshold).tobytes()
    assert np.float64(a.gain).tobytes() == np.float64(b.gain).tobytes()


def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    from paper_2603_00326_b300 import build, soforest as S
    build.build()
    cases = [
        # (seed, n_data, d, C, n_node, P, params): a histogram-path node, then an exact-path node
        (11, 200000, 32, 3, 150000, 64, S.split_params(256, 0, True)),
        (12, 50000, 16, 5, 900, 32, S.split_params(256, 1024, False)),
    ]
    for seed, n_data, d, C_, n_node, P, prm in cases:
        X, y, idx, pr = _node_inputs(seed, n_data, d, C_, n_node, P)
        ds, pj, it = _to_device(torch, X, y, idx, pr, C_)
        ref, ref_lc = S.so_split_search(ds, it, pj, prm)
        got, got_lc = S.so_split_search_noalloc(ds, it, pj, prm)
        assert ref.valid == 1
        _same(got, ref)
        np.testing.assert_array_equal(got_lc, ref_lc)


def test_noalloc_rejects_nodes_beyond_the_static_scratch():
    import torch
    from paper_2603_00326_b300 import soforest as S
    X, y, idx, pr = _node_inputs(13, 5000, 16, 8, 4000, 1024)
    ds, pj, it = _to_device(torch, X, y, idx, pr, 8)
    with pytest.raises(S.SoError) as ei:
        S.so_split_search_noalloc(ds, it, pj, S.split_params(256, 0, True))
    assert ei.value.status == S.SO_EINVAL
    assert "static" in str(ei.value)
