"""so_split_search_noalloc -- the single-node split search for callers that
cannot allocate device memory (a framework's memory pool owns the device,
a fixed memory budget, or a loop that must not pay for cudaMalloc's implicit
synchronisation).  Its scratch is a static device array inside the library.

Checked through the C ABI against the oracle's split search and against
so_split_search (which uses a workspace) on the same inputs, several calls in
a row with different nodes, so leftovers of one call in the shared static
scratch cannot change the next result: a histogram-path node and an
exact-path node, under the Gini criterion with equal-width bins, under the
entropy criterion (its x ln x table lives in the static scratch) and with
random-width bins (their boundary tables live there too).  Collected last on
purpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import gpu_util as U

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


def _same(a, b, ctx):
    for f in ("valid", "proj", "path", "cand", "n_left", "n_right"):
        assert getattr(a, f) == getattr(b, f), (ctx, f)
    assert np.float32(a.threshold).tobytes() == np.float32(b.threshold).tobytes(), ctx
    assert np.float64(a.gain).tobytes() == np.float64(b.gain).tobytes(), ctx


# (seed, n_data, d, C, n_node, P, T, hist_only, bin_rule, criterion)
CASES = [
    (11, 200000, 32, 3, 150000, 64, 0, True, 0, 0),      # histogram path, Gini, equal width
    (12, 50000, 16, 5, 900, 32, 1024, False, 0, 0),      # exact path (one CTA sorts), Gini
    (13, 120000, 24, 4, 60000, 48, 0, True, 0, 1),       # histogram path, entropy
    (14, 40000, 12, 3, 1500, 24, 2048, False, 0, 1),     # exact path, entropy
    (15, 150000, 20, 2, 100000, 32, 0, True, 1, 0),      # histogram path, random-width bins
    (16, 90000, 28, 3, 70000, 40, 1024, False, 1, 1),    # random-width bins and entropy together
]


def test_noalloc_matches_oracle_and_workspace_entry_point():
    import torch
    from paper_2603_00326_b300 import build, soforest as S
    build.build()
    for rnd in range(2):  # every case twice, the calls back to back
        for seed, n_data, d, C_, n_node, P, T, ho, rule, crit in CASES:
            ctx = (seed, rnd)
            X, y, idx, pr = _node_inputs(seed, n_data, d, C_, n_node, P)
            ds, pj, it = _to_device(torch, X, y, idx, pr, C_)
            key = (0x9E3779B97F4A7C15 * (seed + 1)) & 0xFFFFFFFFFFFFFFFF
            keys = torch.tensor([key - (1 << 64) if key >= (1 << 63) else key], dtype=torch.int64, device="cuda")
            prm = S.split_params(256, T, ho, bin_rule=rule, bin_keys=keys if rule else None, criterion=crit)
            got, got_lc = S.so_split_search_noalloc(ds, it, pj, prm)
            r = O.split_search(X, y, C_, idx, pr.ptr, pr.feat, pr.sign, n_bins=256, sort_below=T, hist_only=ho,
                               bin_rule=rule, bin_key=key, criterion=crit)
            assert r.valid == 1, ctx
            U.assert_split_equal(got, r, ctx)
            np.testing.assert_array_equal(got_lc, r.left_counts, err_msg=str(ctx))
            ref, ref_lc = S.so_split_search(ds, it, pj, prm)
            _same(got, ref, ctx)
            np.testing.assert_array_equal(got_lc, ref_lc, err_msg=str(ctx))


def test_noalloc_rejects_nodes_beyond_the_static_scratch():
    import torch
    from paper_2603_00326_b300 import soforest as S
    X, y, idx, pr = _node_inputs(13, 5000, 16, 8, 4000, 1024)
    ds, pj, it = _to_device(torch, X, y, idx, pr, 8)
    with pytest.raises(S.SoError) as ei:
        S.so_split_search_noalloc(ds, it, pj, S.split_params(256, 0, True))
    assert ei.value.status == S.SO_EINVAL
    assert "static" in str(ei.value)
