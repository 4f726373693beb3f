"""The threaded tree grower of the oracle grows the plain grower's tree.

orc_train_tree_mt searches the nodes of each level on several host threads
(a node's split depends only on its own samples and key, Section 2 item 2)
and takes the results in breadth-first order; it is what lets the GPU tests
compare whole full-size trees against the oracle.  Here it is pinned to the
single-threaded orc_train_tree, every field bit for bit, over thread counts,
both node schedules (nodes searched whole on one thread, and nodes with their
projections divided over the threads), bootstraps, both bin rules, both
criteria, count ties and a depth limit.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G


def _same(a, b):
    assert a.n_nodes == b.n_nodes
    for f in O.Tree.FIELDS:
        x, y = getattr(a, f), getattr(b, f)
        assert x.dtype == y.dtype and x.shape == y.shape, f
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8)), f


CASES = {
    # name: (dataset factory, classes, tree kwargs, bootstrap)
    "tree_small": (lambda: G.tree_small(n=3000, d=16, seed=21), 2,
                   dict(n_proj=16, lam=1.5, cap=8, sort_below=256, seed=3), False),
    "bootstrap_lognormal": (lambda: G.forest_2m(n=4000, d=24, seed=22), 2,
                            dict(n_proj=12, lam=1.5, cap=8, sort_below=300, seed=4, tree_id=5), True),
    "counts_five_classes": (lambda: G.wide_counts(n=2500, d=64, seed=23), 5,
                            dict(n_proj=10, lam=3.0, cap=16, sort_below=200, seed=6), False),
    "random_width_entropy": (lambda: G.tree_small(n=2500, d=12, seed=24), 2,
                             dict(n_proj=8, lam=1.5, cap=8, sort_below=128, seed=7, bin_rule=1, criterion=1),
                             True),
    "hist_only_depth4": (lambda: G.root_4m(n=5000, d=16, seed=25), 3,
                         dict(n_proj=8, lam=1.5, cap=8, hist_only=True, seed=8, max_depth=4), False),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_threaded_tree_equals_plain(name):
    make, C, kw, boot = CASES[name]
    ds = make()
    root = (G.bootstrap_indices(ds.n, kw.get("tree_id", 0), seed=9, n_draws=ds.n) if boot
            else G.all_indices(ds.n))
    plain = O.train_tree(ds.X, ds.y, C, root, **kw)
    assert plain.n_nodes > 20
    for nt, big in ((1, 1 << 40), (2, 1 << 40), (5, 1 << 40), (16, 1 << 40), (5, 0), (3, 700)):
        _same(plain, O.train_tree(ds.X, ds.y, C, root, n_threads=nt, big_node=big, **kw))


def test_threaded_tree_single_node_and_pure_root():
    """Degenerate roots: one sample, and a pure node (no search at all)."""
    ds = G.tree_small(n=64, d=4, seed=26)
    for root in (np.array([5], np.int32), np.flatnonzero(ds.y == 1).astype(np.int32)):
        a = O.train_tree(ds.X, ds.y, 2, root, n_proj=4, lam=1.5, cap=8, seed=1)
        b = O.train_tree(ds.X, ds.y, 2, root, n_proj=4, lam=1.5, cap=8, seed=1, n_threads=4, big_node=0)
        assert a.n_nodes == 1
        _same(a, b)
