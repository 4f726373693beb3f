"""The sampled-node tree checker, run on trees the oracle grows itself (CPU).

An oracle tree must pass with every node re-searched; a tree with one planted
mistake (a threshold one ulp off, a swapped projection sign, a wrong leaf
class, a wrong count, a wrong gain bit) must fail.
"""
import copy

import numpy as np
import pytest

from oracle import so_oracle as O
from paper_2603_00326_b300 import datagen as G

from tests.tree_check import route_and_sample

KW = dict(n_proj=12, lam=1.5, cap=8, n_bins=64, sort_below=200, seed=4, tree_id=2)


@pytest.fixture(scope="module")
def grown():
    ds = G.tree_small(n=1500, d=12, seed=71)
    root = G.bootstrap_indices(ds.n, 2, seed=9)
    t = O.train_tree(ds.X, ds.y, 2, root, **KW)
    assert t.n_nodes > 30 and set(np.unique(t.path)) >= {-1, 0, 1}
    return ds, root, t


def test_oracle_tree_passes_with_every_node_searched(grown):
    ds, root, t = grown
    n = route_and_sample(t, ds.X, ds.y, 2, root, check_ids=range(t.n_nodes), **KW)
    assert n == int(np.count_nonzero(t.path >= 0))


def _internal(t, k=0):
    return int(np.flatnonzero(t.left >= 0)[k])


@pytest.mark.parametrize("plant", ["threshold_ulp", "sign", "leaf_class", "count", "gain_bit", "cand"])
def test_planted_mistake_fails(grown, plant):
    ds, root, t = grown
    bad = copy.deepcopy(t)
    v = _internal(t, 3)
    if plant == "threshold_ulp":
        bad.threshold[v] = np.nextafter(bad.threshold[v], np.float32(np.inf), dtype=np.float32)
    elif plant == "sign":
        bad.sign[v, 0] = -bad.sign[v, 0]
    elif plant == "leaf_class":
        leaf = int(np.flatnonzero(t.left < 0)[0])
        bad.leaf_class[leaf] = 1 - bad.leaf_class[leaf]
    elif plant == "count":
        bad.class_counts[v, 0] += 1
    elif plant == "gain_bit":
        bad.gain[v] = np.nextafter(bad.gain[v], 2.0)
    else:
        bad.cand[v] += 1
    with pytest.raises(AssertionError):
        route_and_sample(bad, ds.X, ds.y, 2, root, check_ids=range(t.n_nodes), **KW)
