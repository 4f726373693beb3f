"""Forest inference on the GPU against the oracle's traversal and vote:
predictions and vote counts bit-exact on training and out-of-bag samples,
and device-side rejection of a malformed forest."""
import numpy as np
import pytest

from oracle import so_oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2603_00326_b300 import soforest
    soforest.lib()
    return soforest


@pytest.mark.parametrize("C", [2, 5])
def test_forest_predictions_match_oracle(S, C):
    from paper_2603_00326_b300 import forest as F
    torch = U.torch_cuda()
    if C == 2:
        ds_np = G.forest_2m(n=8000, d=24, seed=61)
    else:
        ds_np = G.wide_counts(n=6000, d=128, seed=62)
    ds = U.upload_dataset(ds_np.X, ds_np.y, C)
    cfg = F.ForestConfig(n_trees=5, n_proj=12, lam=1.5 if C == 2 else 3.0, cap=8 if C == 2 else 16,
                         sort_below=400)
    trees, _ = F.train_forest(cfg, ds)
    forest = S.upload_forest(trees, C)
    rows = np.arange(ds_np.n, dtype=np.int32)
    pred, votes = S.so_predict(ds.X, forest, want_votes=True)
    opred, ovotes = O.predict_forest(trees, ds_np.X, rows, C)
    np.testing.assert_array_equal(votes.cpu().numpy(), ovotes)
    np.testing.assert_array_equal(pred.cpu().numpy(), opred)
    # out-of-bag accuracy of tree 0 (samples its bootstrap never drew)
    inbag = np.zeros(ds_np.n, bool)
    inbag[F.root_indices(ds_np.n, 0, cfg)] = True
    oob = np.flatnonzero(~inbag).astype(np.int32)
    one = S.upload_forest(trees[:1], C)
    p1, _ = S.so_predict(ds.X, one)
    o1 = O.predict_tree_c(trees[0], ds_np.X, oob)
    np.testing.assert_array_equal(p1.cpu().numpy()[oob], o1)
    assert (o1 == ds_np.y[oob]).mean() > 1.0 / C


def test_malformed_forest_rejected_on_device(S):
    torch = U.torch_cuda()
    ds_np = G.tree_small(n=2000, d=8, seed=63)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2)
    tp = S.tree_params(8, 1.5, 8, 256, 300, False, 1, 0, -1)
    t = S.so_train_tree(ds, U.i32(G.all_indices(ds_np.n)), tp)
    internal = np.flatnonzero(t.left >= 0)
    assert internal.size > 0
    t.feat[internal[0], 0] = 9  # feature id >= d
    forest = S.upload_forest([t], 2)
    with pytest.raises(S.SoError) as ei:
        S.so_predict(ds.X, forest)
    assert ei.value.status == S.SO_EINTERNAL
