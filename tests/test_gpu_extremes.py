"""GPU parity at the edges of the parameter space: the most projections per
node (1024) with the longest rows (32 non-zeros), the most classes (8), the
fewest bins (2), a single class, a single feature and a two-sample dataset --
each against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2603_00326_b300 import build, soforest
    build.build()
    return soforest


@pytest.mark.parametrize("B,rule", [(256, 0), (2, 0), (256, 1)])
def test_max_projections_rows_and_classes(S, B, rule):
    rng = np.random.default_rng(B + rule)
    n_data, d, P, C = 40000, 64, 1024, 8
    X = rng.standard_normal((d, n_data)).astype(np.float32)
    y = rng.integers(0, C, n_data).astype(np.uint8)
    pr = G.random_projections(rng, P, d, 40.0, 32)
    assert int(np.diff(pr.ptr).max()) == 32
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(pr.ptr, pr.feat, pr.sign, P)
    for n, T, ho in ((20000, 0, True), (700, 1024, False), (100, 1024, False)):
        if rule and not ho:
            continue
        idx = rng.integers(0, n_data, n).astype(np.int32)
        key = int(rng.integers(0, 2 ** 62))
        prm = S.split_params(B, T, ho, bin_rule=rule, bin_keys=U.i64([key]) if rule else None)
        out, lc = S.so_split_search(ds, U.i32(idx), pj, prm)
        r = O.split_search(X, y, C, idx, pr.ptr, pr.feat, pr.sign, n_bins=B, sort_below=T, hist_only=ho,
                           bin_rule=rule, bin_key=key)
        U.assert_split_equal(out, r, f"n={n} B={B} rule={rule}")
        np.testing.assert_array_equal(lc, r.left_counts if r.valid else np.zeros(C, np.int64))


def test_single_class_dataset(S):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((6, 3000)).astype(np.float32)
    y = np.zeros(3000, np.uint8)
    ds = U.upload_dataset(X, y, 1)
    pr = G.random_projections(rng, 8, 6, 1.5, 8)
    pj = U.upload_projs(pr.ptr, pr.feat, pr.sign, 8)
    for n, T, ho in ((3000, 0, True), (500, 1024, False)):
        out, _ = S.so_split_search(ds, U.i32(np.arange(n)), pj, S.split_params(256, T, ho))
        assert out.valid == 0
    tp = S.tree_params(8, 1.5, 8, seed=2)
    gt = S.so_train_tree(ds, U.i32(np.arange(3000)), tp)
    assert gt.n_nodes == 1 and gt.leaf_class[0] == 0 and gt.path[0] == -1
    pred, _ = S.so_predict(ds.X, S.upload_forest([gt], 1))
    assert int(pred.max().item()) == 0


@pytest.mark.parametrize("crit", [0, 1])
def test_single_feature_tree(S, crit):
    rng = np.random.default_rng(2)
    X = np.round(rng.standard_normal((1, 4000)) * 8).astype(np.float32)  # one feature, many ties
    y = (X[0] + rng.standard_normal(4000) * 4 > 0).astype(np.uint8)
    root = G.all_indices(4000)
    ds = U.upload_dataset(X, y, 2)
    tp = S.tree_params(4, 1.5, 8, sort_below=700, seed=3, criterion=crit)
    gt = S.so_train_tree(ds, U.i32(root), tp)
    ot = O.train_tree(X, y, 2, root, n_proj=4, lam=1.5, cap=8, sort_below=700, seed=3, criterion=crit)
    U.assert_tree_equal(gt, ot)
    assert np.all(gt.proj_nnz[gt.left >= 0] == 1)


def test_two_sample_dataset(S):
    X = np.array([[0.5, -1.25], [2.0, 2.0]], np.float32)
    for y in (np.array([0, 1], np.uint8), np.array([1, 1], np.uint8)):
        ds = U.upload_dataset(X, y, 2)
        root = np.arange(2, dtype=np.int32)
        tp = S.tree_params(6, 1.5, 8, seed=4)
        gt = S.so_train_tree(ds, U.i32(root), tp)
        ot = O.train_tree(X, y, 2, root, n_proj=6, lam=1.5, cap=8, seed=4)
        U.assert_tree_equal(gt, ot)
        assert gt.n_nodes == (3 if y[0] != y[1] else 1)


def test_eight_class_tree(S):
    ds = G.root_4m(n=5000, d=24, seed=77)
    y = (ds.y.astype(np.int32) * 3 + (ds.X[0] > 0)).astype(np.uint8) % 8
    root = G.bootstrap_indices(ds.n, 5, seed=8)
    dsd = U.upload_dataset(ds.X, y, 8)
    tp = S.tree_params(16, 1.5, 8, sort_below=400, seed=6)
    gt = S.so_train_tree(dsd, U.i32(root), tp)
    ot = O.train_tree(ds.X, y, 8, root, n_proj=16, lam=1.5, cap=8, sort_below=400, seed=6)
    U.assert_tree_equal(gt, ot)
    assert len(np.unique(gt.leaf_class)) >= 6
