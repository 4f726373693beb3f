"""GPU parity of the entropy criterion (information gain, the criterion of the
YDF learner the paper builds on, Section 3 step 3) through the C ABI, against
the CPU oracle.

Bit-exact: chosen splits (projection, candidate, threshold bits, double gain
bits, child sizes, left class counts), partitions and whole trees, on every
path: histogram nodes (float keys, double re-score of the window), register
sorted and CTA sorted exact nodes, one-node, allocation-free and batched
calls, trees (also with random-width bins), the autotuner, and the
benchmark's root and forest workloads at full size.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

ENT = 1


@pytest.fixture(scope="module")
def S():
    from paper_2603_00326_b300 import build, soforest
    build.build()
    return soforest


def _cases():
    return [dict(n=30000, T=0, ho=True), dict(n=5000, T=1024, ho=False), dict(n=900, T=1024, ho=False),
            dict(n=20, T=1024, ho=False), dict(n=128, T=1024, ho=False), dict(n=129, T=1024, ho=False),
            dict(n=2047, T=2048, ho=False), dict(n=2, T=0, ho=True), dict(n=1, T=1024, ho=False)]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: f"n{c['n']}_T{c['T']}")
@pytest.mark.parametrize("C", [2, 5])
def test_entropy_single_and_noalloc(S, case, C):
    rng = np.random.default_rng(case["n"] * 11 + C)
    n_data, d, P = 40000, 16, 24
    X = rng.standard_normal((d, n_data)).astype(np.float32)
    X[3] = np.round(X[3])
    y = rng.integers(0, C, n_data).astype(np.uint8)
    idx = rng.integers(0, n_data, case["n"]).astype(np.int32)
    pr = G.random_projections(rng, P, d, 1.5, 8)
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(pr.ptr, pr.feat, pr.sign, P)
    prm = S.split_params(256, case["T"], case["ho"], criterion=ENT)
    r = O.split_search(X, y, C, idx, pr.ptr, pr.feat, pr.sign, sort_below=case["T"], hist_only=case["ho"],
                       criterion=ENT)
    out, lc = S.so_split_search(ds, U.i32(idx), pj, prm)
    U.assert_split_equal(out, r, str(case))
    np.testing.assert_array_equal(lc, r.left_counts if r.valid else np.zeros(C, np.int64))
    out2, lc2 = S.so_split_search_noalloc(ds, U.i32(idx), pj, prm)
    U.assert_split_equal(out2, r, "noalloc " + str(case))
    np.testing.assert_array_equal(lc2, lc)


def test_entropy_pure_constant_and_bad_criterion(S):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 5000)).astype(np.float32)
    X[2] = 7.0
    y = np.zeros(5000, np.uint8)
    y[:2500] = 1
    ds = U.upload_dataset(X, y, 2)
    ptr, feat, sign = np.array([0, 1, 2], np.int32), np.array([2, 2], np.int32), np.array([1, -1], np.int8)
    pj = U.upload_projs(ptr, feat, sign, 2)
    for n, T, ho in ((3000, 0, True), (300, 1024, False), (10, 1024, False)):
        idx = rng.integers(0, 5000, n).astype(np.int32)
        out, _ = S.so_split_search(ds, U.i32(idx), pj, S.split_params(256, T, ho, criterion=ENT))
        assert out.valid == 0
    with pytest.raises(S.SoError) as ei:
        S.so_split_search(ds, U.i32(np.arange(100)), pj, S.split_params(256, 0, True, criterion=2))
    assert ei.value.status == S.SO_EINVAL


@pytest.mark.parametrize("T", [1024, 64, 0])
def test_entropy_batch_frontier_and_partition(S, T):
    rng = np.random.default_rng(61 + T)
    n, d, m, P, C = 120000, 32, 400, 16, 3
    X = rng.standard_normal((d, n)).astype(np.float32)
    y = rng.integers(0, C, n).astype(np.uint8)
    y[X[0] + X[3] > 0.5] = 2
    idx, off = G.frontier_nodes(n, m, seed=62 + T)
    projs = [G.random_projections(rng, P, d, 1.5, 8) for _ in range(m)]
    ptr, feat, sign = U.concat_projs([(p.ptr, p.feat, p.sign) for p in projs])
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(ptr, feat, sign, P)
    prm = S.split_params(256, T, T == 0, criterion=ENT)
    out, lc = S.so_split_search_batch(ds, U.i32(idx), U.i64(off), pj, prm)
    rec = S.splits_to_numpy(out)
    lc = lc.cpu().numpy().reshape(m, C)
    for j in range(m):
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, C, idx[off[j]:off[j + 1]], nptr, nf, ns, sort_below=T, hist_only=(T == 0),
                           criterion=ENT)
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


def _train_both(S, X, y, C, root, bin_rule=0, **kw):
    ds = U.upload_dataset(X, y, C)
    tp = S.tree_params(kw["n_proj"], kw["lam"], kw["cap"], kw.get("n_bins", 256), kw.get("sort_below", 1024),
                       kw.get("hist_only", False), kw.get("seed", 0), kw.get("tree_id", 0), kw.get("max_depth", -1),
                       bin_rule=bin_rule, criterion=ENT)
    gt = S.so_train_tree(ds, U.i32(root), tp)
    ot = O.train_tree(X, y, C, root, bin_rule=bin_rule, criterion=ENT, **kw)
    return gt, ot


@pytest.mark.parametrize("variant", ["tree_small", "multiclass_bootstrap", "hist_only_b32", "counts_ties",
                                     "random_width"])
def test_entropy_tree_parity(S, variant):
    rule = 0
    if variant == "tree_small":
        ds = G.tree_small(n=8192, d=32, seed=83)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=32, lam=1.5, cap=8, sort_below=1024, seed=22)
    elif variant == "multiclass_bootstrap":
        ds = G.root_4m(n=6000, d=20, seed=82)
        root = G.bootstrap_indices(ds.n, 3, seed=27)
        kw = dict(n_proj=24, lam=1.5, cap=8, sort_below=300, seed=23, tree_id=2)
    elif variant == "hist_only_b32":
        ds = G.tree_small(n=3000, d=16, seed=81)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=12, lam=1.5, cap=8, n_bins=32, hist_only=True, sort_below=0, seed=24)
    elif variant == "counts_ties":
        ds = G.wide_counts(n=4000, d=256, seed=80)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=32, lam=3.0, cap=16, sort_below=256, seed=25)
    else:
        ds = G.tree_small(n=6000, d=16, seed=79)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=16, lam=1.5, cap=8, sort_below=400, seed=26)
        rule = 1
    gt, ot = _train_both(S, ds.X, ds.y, ds.n_classes, root, bin_rule=rule, **kw)
    U.assert_tree_equal(gt, ot)


def test_entropy_autotune_and_tree(S):
    ds_np = G.tree_small(n=20000, d=16, seed=57)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2)
    prm, sizes, times = S.so_autotune(ds, 16, 1.5, 8, S.split_params(256, 1024, False, criterion=ENT))
    T = prm.sort_below
    assert 32 <= T <= 2048 and np.all(times > 0)
    gt, ot = _train_both(S, ds_np.X, ds_np.y, 2, G.all_indices(ds_np.n), n_proj=16, lam=1.5, cap=8,
                         sort_below=T, seed=5)
    U.assert_tree_equal(gt, ot)


# ---------------------------------------------------------------- full size

def test_entropy_root_4m_full_size(S):
    """Root split of the benchmark's n=4M, d=64, 3-class node (256
    projections, histogram path) under the entropy criterion, against the
    oracle with the projections divided over the host's threads."""
    import os
    torch = U.torch_cuda()
    ds_np = G.root_4m()
    p = G.WORKLOAD_PARAMS["root_4m"]
    rng = np.random.default_rng(G.PROJ_SEED_BASE + 1)
    pr = G.random_projections(rng, p["n_proj"], ds_np.d, p["lam"], p["cap"])
    ds = U.upload_dataset(ds_np.X, ds_np.y, 3)
    pj = U.upload_projs(pr.ptr, pr.feat, pr.sign, p["n_proj"])
    idx = G.all_indices(ds_np.n)
    off = U.i64([0, ds_np.n])
    out, lc = S.so_split_search_batch(ds, U.i32(idx), off, pj, S.split_params(256, 0, True, criterion=ENT))
    rec = S.splits_to_numpy(out)[0]
    r = O.split_search_mt(ds_np.X, ds_np.y, 3, idx, pr.ptr, pr.feat, pr.sign, hist_only=True,
                          n_threads=min(32, os.cpu_count() or 1), criterion=ENT)
    U.assert_split_equal(rec, r, "root_4m entropy")
    np.testing.assert_array_equal(lc.cpu().numpy(), r.left_counts)
    idx_out = torch.empty(ds_np.n, dtype=torch.int32, device="cuda")
    S.so_partition_batch(ds, U.i32(idx), idx_out, off, pj, out)
    exp, nl = O.partition(ds_np.X, idx, pr.feat[pr.ptr[r.proj]:pr.ptr[r.proj + 1]],
                          pr.sign[pr.ptr[r.proj]:pr.ptr[r.proj + 1]], float(r.threshold))
    np.testing.assert_array_equal(idx_out.cpu().numpy(), exp)


def test_entropy_forest_2m_tree_full_size(S):
    """Tree 0 of the forest workload (n=2M, d=256, bootstrap, 128
    projections/node, T=1024, row-major copy) under the entropy criterion,
    identical to the oracle's tree field by field."""
    from paper_2603_00326_b300 import forest as F
    ds_np = G.forest_2m()
    p = G.WORKLOAD_PARAMS["forest_2m"]
    cfg = F.ForestConfig(n_trees=p["n_trees"], n_proj=p["n_proj"], lam=p["lam"], cap=p["cap"],
                         sort_below=p["sort_below"], criterion=ENT)
    root = F.root_indices(ds_np.n, 0, cfg)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2).with_row_major()
    trees, _ = F.train_forest(dataclass_one(cfg), ds)
    gt = trees[0]
    del ds
    U.torch_cuda().cuda.empty_cache()
    assert set(np.unique(gt.path)) >= {0, 1}
    ot = U.oracle_tree_all_cores(ds_np.X, ds_np.y, 2, root, n_proj=p["n_proj"], lam=p["lam"], cap=p["cap"],
                                 n_bins=p["n_bins"], sort_below=p["sort_below"], seed=cfg.seed, tree_id=0,
                                 criterion=ENT)
    U.assert_tree_equal(gt, ot, "entropy forest_2m tree 0")


def dataclass_one(cfg):
    import dataclasses
    return dataclasses.replace(cfg, n_trees=1)
