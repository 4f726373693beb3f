"""GPU parity of the exact path's CTA-sorted nodes at every padded size.

The CTA sort pads a node of n_v samples to NP = max(256, next power of two)
positions and skips every comparator that reaches beyond n_v, so the sizes
around each power of two (and 2047, the largest exact node) are the edge
cases.  Nodes above 256 samples take the segmented radix sort instead (8-bit
digits of the value key, digits constant over the node skipped), so sizes
around 256 switch between the two.  Nodes of those sizes, with duplicated
samples and few-valued features (ties), a pure node and a constant node, run
in one batched search on the column layout and on the row-major copy, under
both criteria; integer counts (whose keys share their low digits, so the
radix sort skips those passes) run the same sizes.  Every node's split is
checked bit for bit against the oracle (Section 3.1).
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

SIZES = [129, 130, 200, 255, 256, 257, 383, 511, 512, 513, 700, 1023, 1024, 1025, 1536, 2047]
T = 2048


@pytest.fixture(scope="module")
def S():
    from paper_2603_00326_b300 import build, soforest
    build.build()
    return soforest


def _nodes(rng, y, n_data):
    """Index lists: every size twice (sampled with repeats), a pure node and
    a node of one repeated sample."""
    lists = [rng.integers(0, n_data, s) for s in SIZES + SIZES[::-1]]
    lists.append(rng.choice(np.flatnonzero(y == 1), 513))
    lists.append(np.full(1024, int(rng.integers(0, n_data))))
    return lists


@pytest.mark.parametrize("row_major", [False, True], ids=["columns", "rows"])
@pytest.mark.parametrize("crit", [0, 1], ids=["gini", "entropy"])
def test_cta_sort_every_padded_size(S, row_major, crit):
    rng = np.random.default_rng(31 + 2 * crit + int(row_major))
    n_data, d, P, C = 30000, 24, 12, 3
    X = rng.standard_normal((d, n_data)).astype(np.float32)
    X[::3] = np.round(X[::3] * 2)  # a third of the features take few distinct values
    y = rng.integers(0, C, n_data).astype(np.uint8)
    lists = _nodes(rng, y, n_data)
    m = len(lists)
    idx = np.concatenate(lists).astype(np.int32)
    off = np.zeros(m + 1, np.int64)
    off[1:] = np.cumsum([len(a) for a in lists])
    projs = [G.random_projections(rng, P, d, 1.5, 8) for _ in range(m)]
    ptr, feat, sign = U.concat_projs([(p.ptr, p.feat, p.sign) for p in projs])
    ds = U.upload_dataset(X, y, C)
    if row_major:
        ds = ds.with_row_major()
    pj = U.upload_projs(ptr, feat, sign, P)
    out, lc = S.so_split_search_batch(ds, U.i32(idx), U.i64(off), pj, S.split_params(256, T, False, criterion=crit))
    rec = S.splits_to_numpy(out)
    lc = lc.cpu().numpy().reshape(m, C)
    n_valid = 0
    for j in range(m):
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, C, idx[off[j]:off[j + 1]], nptr, nf, ns, sort_below=T, criterion=crit)
        assert r.path == 1
        U.assert_split_equal(rec[j], r, f"node {j} size {off[j + 1] - off[j]}")
        np.testing.assert_array_equal(lc[j], r.left_counts if r.valid else 0)
        n_valid += int(r.valid)
    assert n_valid == m - 2 and not rec[m - 2]["valid"] and not rec[m - 1]["valid"]


@pytest.mark.parametrize("crit", [0, 1], ids=["gini", "entropy"])
def test_cta_radix_on_integer_counts(S, crit):
    """Count features (0..~12): every projected value is a small integer, so
    the low 16 bits of each order-preserving key are equal across the node and
    the radix sort runs only its upper passes."""
    rng = np.random.default_rng(77 + crit)
    n_data, d, P, C = 30000, 16, 12, 4
    X = rng.poisson(3.0, (d, n_data)).astype(np.float32)
    y = rng.integers(0, C, n_data).astype(np.uint8)
    lists = [rng.integers(0, n_data, s) for s in SIZES]
    m = len(lists)
    idx = np.concatenate(lists).astype(np.int32)
    off = np.zeros(m + 1, np.int64)
    off[1:] = np.cumsum([len(a) for a in lists])
    projs = [G.random_projections(rng, P, d, 1.5, 8) for _ in range(m)]
    ptr, feat, sign = U.concat_projs([(p.ptr, p.feat, p.sign) for p in projs])
    ds = U.upload_dataset(X, y, C).with_row_major()
    pj = U.upload_projs(ptr, feat, sign, P)
    out, lc = S.so_split_search_batch(ds, U.i32(idx), U.i64(off), pj, S.split_params(256, T, False, criterion=crit))
    rec = S.splits_to_numpy(out)
    lc = lc.cpu().numpy().reshape(m, C)
    for j in range(m):
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, C, idx[off[j]:off[j + 1]], nptr, nf, ns, sort_below=T, criterion=crit)
        assert r.path == 1 and r.valid
        U.assert_split_equal(rec[j], r, f"node {j} size {off[j + 1] - off[j]}")
        np.testing.assert_array_equal(lc[j], r.left_counts)
