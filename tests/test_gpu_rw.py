"""GPU parity of the random-width histogram (boundaries at random intervals,
the YDF default that the paper's Section 1 footnote names) through the C ABI,
against the CPU oracle.

Bit-exact: every boundary, histogram, chosen split (projection, candidate,
threshold bits, double gain bits, child sizes, left class counts), partition
and whole tree.  Float gains of every candidate within 1e-6 relative of the
oracle's double gain.  Covered: the staged kernels (tile path, projected-value
path of batches, wide groups), the general kernels (more than 65536
features), guided bins and the binary search of zero, tiny and
ill-conditioned ranges, one-node, allocation-free and batched calls, trees,
the autotuner, and the benchmark's root and forest workloads at full size.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

GAIN32_REL_TOL = 1e-6
RW = 1


@pytest.fixture(scope="module")
def S():
    from paper_2603_00326_b300 import build, soforest
    build.build()
    return soforest


def _keys(rng, m):
    k = rng.integers(0, 2 ** 63, m, dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1)
    if m > 1:
        k[1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    return k


def _kt(keys):
    return U.torch_cuda().from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()


def _mixed_nodes(rng, n, sizes):
    idx = np.concatenate([rng.integers(0, n, s) for s in sizes]).astype(np.int32)
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    return idx, off


def _check_hist_stage(S, X, y, C, idx, off, ptr, feat, sign, P, B, keys, max_nnz=None, gains=True):
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(ptr, feat, sign, P, max_nnz=max_nnz)
    mm, hist, g32, bnd = S.so_histograms(ds, U.i32(idx), U.i64(off), pj, B, want_gains=gains, bin_rule=RW,
                                         bin_keys=_kt(keys), want_bounds=True)
    mm, hist, bnd = mm.cpu().numpy(), hist.cpu().numpy(), bnd.cpu().numpy()
    g32 = g32.cpu().numpy() if gains else None
    worst = 0.0
    for j in range(len(off) - 1):
        s = int(off[j + 1] - off[j])
        if s == 0:
            continue
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, C, idx[off[j]:off[j + 1]], nptr, nf, ns, n_bins=B, hist_only=True,
                           want_debug=True, bin_rule=RW, bin_key=int(keys[j]))
        np.testing.assert_array_equal(U.f32bits(mm[j]), U.f32bits(r.minmax), err_msg=f"minmax node {j}")
        np.testing.assert_array_equal(U.f32bits(bnd[j]), U.f32bits(r.bounds), err_msg=f"bounds node {j}")
        np.testing.assert_array_equal(hist[j], r.hist, err_msg=f"hist node {j}")
        if gains:
            skip = r.gains < 0
            np.testing.assert_array_equal(g32[j][skip], -1.0)
            ok = (~skip) & (r.gains > 0)
            if ok.any():
                g = g32[j][ok].astype(np.float64) / (float(s) * float(s))
                worst = max(worst, float((np.abs(g - r.gains[ok]) / r.gains[ok]).max()))
    assert worst <= GAIN32_REL_TOL, worst


@pytest.mark.parametrize("B,C", [(256, 3), (7, 2), (64, 5), (256, 8)])
def test_rw_histogram_stage_parity(S, B, C):
    rng = np.random.default_rng(310 + B + C)
    n, d, P = 60000, 24, 12
    X = rng.standard_normal((d, n)).astype(np.float32)
    X[5] = 1.25  # a constant feature: a projection on it alone has min == max
    X[6] = np.round(X[6] * 2)  # ties
    X[7] = X[7] * np.float32(1e-3) + np.float32(300.0)  # narrow range at a large offset
    y = rng.integers(0, C, n).astype(np.uint8)
    sizes = [1, 2, 31, 33, 1000, 4095, 16384, 16385, 23457]  # chunk boundaries and ragged tails
    idx, off = _mixed_nodes(rng, n, sizes)
    projs = [G.random_projections(rng, P, d, 1.5, 8) for _ in sizes]
    projs = [(q.ptr, q.feat, q.sign) for q in projs]
    for j, f in ((0, 5), (3, 7)):  # node 0: the constant feature alone; node 3: the offset one
        p0, f0, s0 = projs[j]
        k0 = int(p0[1])
        projs[j] = (np.concatenate([[0, 1], p0[2:] - k0 + 1]).astype(np.int32),
                    np.concatenate([[f], f0[k0:]]).astype(np.int32), np.concatenate([[1], s0[k0:]]).astype(np.int8))
    ptr, feat, sign = U.concat_projs(projs)
    _check_hist_stage(S, X, y, C, idx, off, ptr, feat, sign, P, B, _keys(rng, len(sizes)),
                      max_nnz=None if B != 64 else 0)


def test_rw_ill_conditioned_ranges(S):
    """Ranges a few ulps wide up to 2^-20 of the value, and zero ranges: the
    boundaries round onto few floats and the bins come from binary search."""
    rng = np.random.default_rng(78)
    n, d = 5000, 7
    base = np.float32(1000.0)
    X = np.empty((d, n), np.float32)
    X[0] = base + np.float32(2.0 ** -13) * rng.integers(0, 4, n).astype(np.float32)
    X[1] = np.where(rng.random(n) < 0.5, base, np.nextafter(base, np.float32(2000)))
    X[2] = rng.standard_normal(n).astype(np.float32) * np.float32(1e-3) + np.float32(7.0)
    X[3] = rng.standard_normal(n).astype(np.float32)
    X[4] = np.float32(3.0)
    X[5] = rng.standard_normal(n).astype(np.float32) * np.float32(1e4)
    X[6] = rng.standard_normal(n).astype(np.float32) * np.float32(1e-30)
    y = rng.integers(0, 2, n).astype(np.uint8)
    ptr = np.arange(d + 1, dtype=np.int32)
    feat = np.arange(d, dtype=np.int32)
    sign = np.ones(d, np.int8)
    idx = np.arange(n, dtype=np.int32)
    off = np.array([0, n], np.int64)
    keys = _keys(rng, 1)
    _check_hist_stage(S, X, y, 2, idx, off, ptr, feat, sign, d, 256, keys)
    ds = U.upload_dataset(X, y, 2)
    pj = U.upload_projs(ptr, feat, sign, d)
    out, _ = S.so_split_search(ds, U.i32(idx), pj, S.split_params(256, 0, True, bin_rule=RW, bin_keys=_kt(keys)))
    r = O.split_search(X, y, 2, idx, ptr, feat, sign, hist_only=True, bin_rule=RW, bin_key=int(keys[0]))
    U.assert_split_equal(out, r)


@pytest.mark.parametrize("d,cap,P", [(4096, 16, 96), (600, 32, 40), (70000, 8, 8)])
def test_rw_histogram_stage_wide(S, d, cap, P):
    """Device-formed projection groups, groups wider than a tile (direct
    path), and more than 65536 features (general kernels, binary search)."""
    rng = np.random.default_rng(d + cap + 5)
    n = 3000 if d > 10000 else 20000
    X = rng.standard_normal((d, n)).astype(np.float32)
    y = rng.integers(0, 3, n).astype(np.uint8)
    sizes = [4000, 2500, 333] if n > 5000 else [2000, 999]
    idx, off = _mixed_nodes(rng, n, sizes)
    projs = [G.random_projections(rng, P, d, 8.0, cap) for _ in sizes]
    ptr, feat, sign = U.concat_projs([(p.ptr, p.feat, p.sign) for p in projs])
    _check_hist_stage(S, X, y, 3, idx, off, ptr, feat, sign, P, 256, _keys(rng, len(sizes)), gains=False)


@pytest.mark.parametrize("n,T,ho", [(30000, 0, True), (5000, 1024, False), (900, 1024, False), (2, 0, True)])
@pytest.mark.parametrize("C", [2, 5])
def test_rw_single_and_noalloc_parity(S, n, T, ho, C):
    rng = np.random.default_rng(n * 3 + C)
    n_data, d, P = 40000, 16, 24
    X = rng.standard_normal((d, n_data)).astype(np.float32)
    X[3] = np.round(X[3])
    y = rng.integers(0, C, n_data).astype(np.uint8)
    idx = rng.integers(0, n_data, n).astype(np.int32)
    pr = G.random_projections(rng, P, d, 1.5, 8)
    keys = _keys(rng, 1)
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(pr.ptr, pr.feat, pr.sign, P)
    prm = S.split_params(256, T, ho, bin_rule=RW, bin_keys=_kt(keys))
    r = O.split_search(X, y, C, idx, pr.ptr, pr.feat, pr.sign, sort_below=T, hist_only=ho, bin_rule=RW,
                       bin_key=int(keys[0]))
    out, lc = S.so_split_search(ds, U.i32(idx), pj, prm)
    U.assert_split_equal(out, r, f"n={n}")
    np.testing.assert_array_equal(lc, r.left_counts if r.valid else np.zeros(C, np.int64))
    out2, lc2 = S.so_split_search_noalloc(ds, U.i32(idx), pj, prm)
    U.assert_split_equal(out2, r, f"noalloc n={n}")
    np.testing.assert_array_equal(lc2, lc)


def test_rw_needs_keys(S):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4, 100)).astype(np.float32)
    y = rng.integers(0, 2, 100).astype(np.uint8)
    ds = U.upload_dataset(X, y, 2)
    pj = U.upload_projs(np.array([0, 1]), np.array([0]), np.array([1]), 1)
    for prm in (S.split_params(256, 0, True, bin_rule=RW), S.split_params(256, 0, True, bin_rule=2)):
        with pytest.raises(S.SoError) as ei:
            S.so_split_search(ds, U.i32(np.arange(100)), pj, prm)
        assert ei.value.status == S.SO_EINVAL


@pytest.mark.parametrize("T", [1024, 64, 0])
def test_rw_batch_frontier_and_partition(S, T):
    """A lognormal frontier in one batched call (exact and histogram nodes;
    histogram nodes read the projected values kept by the min / max pass)."""
    rng = np.random.default_rng(51 + T)
    n, d, m, P, C = 120000, 32, 400, 16, 2
    X = rng.standard_normal((d, n)).astype(np.float32)
    y = G.binary_sum_labels(rng, X, 4, 0.05)
    idx, off = G.frontier_nodes(n, m, seed=52 + T)
    projs = [G.random_projections(rng, P, d, 1.5, 8) for _ in range(m)]
    ptr, feat, sign = U.concat_projs([(p.ptr, p.feat, p.sign) for p in projs])
    keys = _keys(rng, m)
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(ptr, feat, sign, P)
    prm = S.split_params(256, T, T == 0, bin_rule=RW, bin_keys=_kt(keys))
    out, lc = S.so_split_search_batch(ds, U.i32(idx), U.i64(off), pj, prm)
    rec = S.splits_to_numpy(out)
    lc = lc.cpu().numpy().reshape(m, C)
    for j in range(m):
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, C, idx[off[j]:off[j + 1]], nptr, nf, ns, sort_below=T, hist_only=(T == 0),
                           bin_rule=RW, bin_key=int(keys[j]))
        U.assert_split_equal(rec[j], r, f"node {j} size {off[j + 1] - off[j]}")
        np.testing.assert_array_equal(lc[j], r.left_counts if r.valid else 0)
    torch = U.torch_cuda()
    idx_out = torch.empty(n, dtype=torch.int32, device="cuda")
    S.so_partition_batch(ds, U.i32(idx), idx_out, U.i64(off), pj, out)
    got = idx_out.cpu().numpy()
    for j in range(m):
        seg = idx[off[j]:off[j + 1]]
        if rec[j]["valid"]:
            p = int(rec[j]["proj"])
            nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
            exp, nl = O.partition(X, seg, nf[nptr[p]:nptr[p + 1]], ns[nptr[p]:nptr[p + 1]],
                                  float(rec[j]["threshold"]))
            assert nl == rec[j]["n_left"]
        else:
            exp = seg
        np.testing.assert_array_equal(got[off[j]:off[j + 1]], exp, err_msg=f"node {j}")


def _train_both(S, X, y, C, root, **kw):
    ds = U.upload_dataset(X, y, C)
    if kw.pop("row_major", False):
        ds = ds.with_row_major()
    tp = S.tree_params(kw["n_proj"], kw["lam"], kw["cap"], kw.get("n_bins", 256), kw.get("sort_below", 1024),
                       kw.get("hist_only", False), kw.get("seed", 0), kw.get("tree_id", 0), kw.get("max_depth", -1),
                       bin_rule=RW)
    gt = S.so_train_tree(ds, U.i32(root), tp)
    ot = O.train_tree(X, y, C, root, bin_rule=RW, **kw)
    return gt, ot


@pytest.mark.parametrize("variant", ["tree_small", "multiclass_bootstrap", "hist_only_b32", "counts_ties",
                                     "trunk_row_major"])
def test_rw_tree_parity(S, variant):
    if variant == "tree_small":
        ds = G.tree_small(n=8192, d=32, seed=93)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=32, lam=1.5, cap=8, sort_below=1024, seed=12)
    elif variant == "multiclass_bootstrap":
        ds = G.root_4m(n=6000, d=20, seed=92)
        root = G.bootstrap_indices(ds.n, 3, seed=17)
        kw = dict(n_proj=24, lam=1.5, cap=8, sort_below=300, seed=13, tree_id=2)
    elif variant == "hist_only_b32":
        ds = G.tree_small(n=3000, d=16, seed=91)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=12, lam=1.5, cap=8, n_bins=32, hist_only=True, sort_below=0, seed=14)
    elif variant == "counts_ties":
        ds = G.wide_counts(n=4000, d=256, seed=90)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=32, lam=3.0, cap=16, sort_below=256, seed=15)
    else:
        ds = G.trunk(n=6000, p=64, seed=89)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=12, lam=1.0, cap=8, sort_below=200, seed=16, row_major=True)
    gt, ot = _train_both(S, ds.X, ds.y, ds.n_classes, root, **kw)
    U.assert_tree_equal(gt, ot)
    assert np.any(gt.path == 0)


def test_rw_autotune_and_tree(S):
    ds_np = G.tree_small(n=20000, d=16, seed=56)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2)
    prm, sizes, times = S.so_autotune(ds, 16, 1.5, 8, S.split_params(256, 1024, False, bin_rule=RW))
    T = prm.sort_below
    assert 32 <= T <= 2048 and np.all(times > 0)
    gt, ot = _train_both(S, ds_np.X, ds_np.y, 2, G.all_indices(ds_np.n), n_proj=16, lam=1.5, cap=8,
                         sort_below=T, seed=4)
    U.assert_tree_equal(gt, ot)


# ---------------------------------------------------------------- full size

def test_rw_root_4m_full_size(S):
    """Root split of n=4M, d=64, 3 classes, 256 projections on the histogram
    path with random-width bins, in the launch configuration of the benchmark's
    random-width leg; the split, left counts and partition against the oracle
    (projections divided over the host's threads)."""
    import os
    torch = U.torch_cuda()
    ds_np = G.root_4m()
    p = G.WORKLOAD_PARAMS["root_4m"]
    rng = np.random.default_rng(G.PROJ_SEED_BASE + 1)
    pr = G.random_projections(rng, p["n_proj"], ds_np.d, p["lam"], p["cap"])
    key = G.PROJ_SEED_BASE + 11
    ds = U.upload_dataset(ds_np.X, ds_np.y, 3)
    pj = U.upload_projs(pr.ptr, pr.feat, pr.sign, p["n_proj"])
    idx = G.all_indices(ds_np.n)
    prm = S.split_params(256, 0, True, bin_rule=RW, bin_keys=_kt(np.array([key], np.uint64)))
    off = U.i64([0, ds_np.n])
    out, lc = S.so_split_search_batch(ds, U.i32(idx), off, pj, prm)
    rec = S.splits_to_numpy(out)[0]
    r = O.split_search_mt(ds_np.X, ds_np.y, 3, idx, pr.ptr, pr.feat, pr.sign, hist_only=True,
                          n_threads=min(32, os.cpu_count() or 1), bin_rule=RW, bin_key=key)
    U.assert_split_equal(rec, r, "root_4m random width")
    np.testing.assert_array_equal(lc.cpu().numpy(), r.left_counts)
    idx_out = torch.empty(ds_np.n, dtype=torch.int32, device="cuda")
    S.so_partition_batch(ds, U.i32(idx), idx_out, off, pj, out)
    exp, nl = O.partition(ds_np.X, idx, pr.feat[pr.ptr[r.proj]:pr.ptr[r.proj + 1]],
                          pr.sign[pr.ptr[r.proj]:pr.ptr[r.proj + 1]], float(r.threshold))
    np.testing.assert_array_equal(idx_out.cpu().numpy(), exp)


def test_rw_forest_2m_tree_full_size(S):
    """Tree 0 of the forest workload (n=2M, d=256, bootstrap, 128
    projections/node, T=1024, row-major copy) with random-width bins,
    identical to the oracle's tree field by field."""
    from paper_2603_00326_b300 import forest as F
    ds_np = G.forest_2m()
    p = G.WORKLOAD_PARAMS["forest_2m"]
    cfg = F.ForestConfig(n_trees=p["n_trees"], n_proj=p["n_proj"], lam=p["lam"], cap=p["cap"],
                         sort_below=p["sort_below"])
    root = F.root_indices(ds_np.n, 0, cfg)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2).with_row_major()
    tp = S.tree_params(p["n_proj"], p["lam"], p["cap"], p["n_bins"], p["sort_below"], False, cfg.seed, 0, -1,
                       bin_rule=RW)
    gt = S.so_train_tree(ds, U.i32(root), tp)
    del ds
    U.torch_cuda().cuda.empty_cache()
    assert set(np.unique(gt.path)) >= {0, 1}
    ot = U.oracle_tree_all_cores(ds_np.X, ds_np.y, 2, root, n_proj=p["n_proj"], lam=p["lam"], cap=p["cap"],
                                 n_bins=p["n_bins"], sort_below=p["sort_below"], seed=cfg.seed, tree_id=0,
                                 bin_rule=RW)
    U.assert_tree_equal(gt, ot, "random-width forest_2m tree 0")
