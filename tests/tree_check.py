"""Oracle checks of a GPU tree too large for the oracle to grow whole.

`route_and_sample` walks the GPU tree in BFS order and re-derives every node
from the root sample list with the oracle alone:

* each internal node's samples are split with the oracle's projection
  arithmetic (Section 3's sparse sum in ascending feature order, left iff
  v < threshold) using the GPU tree's stored projection and threshold, so the
  sample count, class counts and depth of every node, and the majority class
  of every leaf, are checked for the whole tree;
* node keys follow the tree order (root key from seed and tree id, child key
  from the parent key and the side), so for a chosen set of nodes the oracle
  re-samples the node's projections and re-runs the whole split search on the
  node's samples; the GPU's recorded split (winning projection, candidate,
  path, threshold bits, FP64 gain bits, left count) must be the oracle's, and
  a searched leaf must be one where the oracle finds no valid split.

Together this pins the tree: a node that is not re-searched still has its
samples, counts and children checked, and every re-searched node is compared
bit for bit.
"""
import numpy as np

from oracle import so_oracle as O


def _f32(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def _f64(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def choose_nodes(gt, n_internal=12, n_leaves=6, seed=0):
    """Node ids to re-search: the root, the first and the deepest internal
    node of each eighth of the depth range, random internal nodes, and random
    searched leaves."""
    rng = np.random.default_rng(seed)
    internal = np.flatnonzero(gt.left >= 0)
    searched_leaves = np.flatnonzero((gt.left < 0) & (gt.path >= 0))
    ids = {0}
    if internal.size:
        dmax = int(gt.depth[internal].max())
        for k in range(8):
            d = (k * dmax) // 7 if dmax else 0
            at = internal[gt.depth[internal] == d]
            if at.size:
                ids.add(int(at[0]))
                ids.add(int(at[-1]))
        ids.update(int(v) for v in rng.choice(internal, size=min(n_internal, internal.size), replace=False))
    if searched_leaves.size:
        ids.update(int(v) for v in rng.choice(searched_leaves, size=min(n_leaves, searched_leaves.size),
                                             replace=False))
    return sorted(ids)


def route_and_sample(gt, X, y, C, root, *, n_proj, lam, cap, n_bins=256, sort_below=1024, hist_only=False,
                     seed=0, tree_id=0, max_depth=-1, check_ids=None, bin_rule=0, criterion=0):
    """Checks the GPU tree `gt` against the oracle; returns the number of
    nodes re-searched."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.uint8)
    d = X.shape[0]
    n_nodes = int(gt.n_nodes)
    check = set(check_ids if check_ids is not None else choose_nodes(gt))
    samples = {0: np.ascontiguousarray(root, dtype=np.int32)}
    keys = {0: O.root_key(seed, tree_id)}
    next_id = 1
    searched = 0
    for v in range(n_nodes):
        s = samples.pop(v)
        key = keys.pop(v)
        ctx = f"node {v}"
        cnt = np.bincount(y[s], minlength=C)[:C].astype(np.int64)
        assert int(gt.n_samples[v]) == s.shape[0], ctx
        np.testing.assert_array_equal(gt.class_counts[v], cnt, err_msg=ctx)
        leaf = gt.left[v] < 0
        searchable = s.shape[0] >= 2 and np.count_nonzero(cnt) >= 2 and (max_depth < 0 or gt.depth[v] < max_depth)
        if not searchable:
            assert leaf and int(gt.path[v]) == -1, ctx
        if v in check and searchable:
            nnz, feat, sign = O.sample_node(key, n_proj, d, lam, cap)
            ptr, f, sg = O.slots_to_csr(nnz, feat, sign)
            r = O.split_search(X, y, C, s, ptr, f, sg, n_bins=n_bins, sort_below=sort_below, hist_only=hist_only,
                               bin_rule=bin_rule, bin_key=key, criterion=criterion)
            searched += 1
            assert int(gt.path[v]) == r.path, (ctx, int(gt.path[v]), r.path)
            assert (not leaf) == bool(r.valid), ctx
            if r.valid:
                k = int(nnz[r.proj])
                assert int(gt.proj_nnz[v]) == k, ctx
                np.testing.assert_array_equal(gt.feat[v, :k], feat[r.proj, :k], err_msg=ctx)
                np.testing.assert_array_equal(gt.sign[v, :k], sign[r.proj, :k], err_msg=ctx)
                assert int(gt.cand[v]) == r.cand, ctx
                assert _f32(gt.threshold[v]) == _f32(r.threshold), ctx
                assert _f64(gt.gain[v]) == _f64(r.gain), ctx
        if leaf:
            assert int(gt.leaf_class[v]) == int(np.argmax(cnt)), ctx
            continue
        assert searchable, ctx
        k = int(gt.proj_nnz[v])
        assert 1 <= k <= cap, ctx
        fv = gt.feat[v, :k]
        assert np.all(np.diff(fv) > 0) and fv[0] >= 0 and fv[-1] < d, ctx
        pv = O.project(X, s, fv, gt.sign[v, :k])
        go_left = pv < np.float32(gt.threshold[v])
        L, R = s[go_left], s[~go_left]
        assert L.shape[0] > 0 and R.shape[0] > 0, ctx
        assert gt.left[v] == next_id and gt.right[v] == next_id + 1, ctx
        assert gt.depth[next_id] == gt.depth[v] + 1 and gt.depth[next_id + 1] == gt.depth[v] + 1, ctx
        samples[next_id], samples[next_id + 1] = L, R
        keys[next_id], keys[next_id + 1] = O.child_key(key, 0), O.child_key(key, 1)
        next_id += 2
    assert next_id == n_nodes and not samples
    return searched
