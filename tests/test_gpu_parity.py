"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bit-exact: sampled projections, min/max, histograms, chosen splits
(projection, candidate, threshold bits, double gain bits, child sizes, left
class counts), partitions and whole trees.  Float gains of every histogram
candidate: within 1e-6 relative of the oracle's double gain.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_00326_b300 import datagen as G
from tests import gpu_util as U

pytestmark = pytest.mark.gpu

GAIN32_REL_TOL = 1e-6


@pytest.fixture(scope="module")
def S():
    from paper_2603_00326_b300 import build, soforest
    build.build()
    return soforest


# ---------------------------------------------------------------- sampler

@pytest.mark.parametrize("P,d,lam,cap", [(32, 64, 1.5, 8), (128, 4096, 3.0, 16), (16, 5, 1.5, 8), (8, 1, 2.0, 4)])
def test_sampler_matches_oracle(S, P, d, lam, cap):
    torch = U.torch_cuda()
    rng = np.random.default_rng(d + P)
    keys = rng.integers(0, 2 ** 63, 300, dtype=np.int64).astype(np.uint64)
    keys[0] = 0
    keys[1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    nnz, feat, sign = S.so_sample_projections(kt, P, d, lam, cap)
    nnz = nnz.cpu().numpy().reshape(-1, P)
    feat = feat.cpu().numpy().reshape(-1, P, cap)
    sign = sign.cpu().numpy().reshape(-1, P, cap)
    for j, k in enumerate(keys):
        on, of, os_ = O.sample_node(int(k), P, d, lam, cap)
        np.testing.assert_array_equal(nnz[j], on)
        for p in range(P):
            np.testing.assert_array_equal(feat[j, p, :on[p]], of[p, :on[p]])
            np.testing.assert_array_equal(sign[j, p, :on[p]], os_[p, :on[p]])


# ---------------------------------------------------------------- histogram stage

def _mixed_nodes(rng, n, sizes):
    idx = np.concatenate([rng.integers(0, n, s) for s in sizes]).astype(np.int32)
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    return idx, off


@pytest.mark.parametrize("B,C", [(256, 3), (7, 2), (64, 5)])
def test_histogram_stage_parity(S, B, C):
    rng = np.random.default_rng(10 + B)
    n, d, P = 60000, 24, 12
    X = rng.standard_normal((d, n)).astype(np.float32)
    X[5] = 1.25  # a constant feature: projections on it have min == max
    X[6] = np.round(X[6] * 2)  # ties
    y = rng.integers(0, C, n).astype(np.uint8)
    sizes = [1, 2, 31, 33, 1000, 4095, 16384, 16385, 23457]  # chunk boundaries and ragged tails
    idx, off = _mixed_nodes(rng, n, sizes)
    projs = []
    for j in range(len(sizes)):
        pr = G.random_projections(rng, P, d, 1.5, 8)
        projs.append((pr.ptr, pr.feat, pr.sign))
    # projection 0 of node 0 reads the constant feature alone (min == max)
    p0, f0, s0 = projs[0]
    k0 = int(p0[1])
    projs[0] = (np.concatenate([[0, 1], p0[2:] - k0 + 1]).astype(np.int32),
                np.concatenate([[5], f0[k0:]]).astype(np.int32), np.concatenate([[1], s0[k0:]]).astype(np.int8))
    ptr, feat, sign = U.concat_projs(projs)
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(ptr, feat, sign, P, max_nnz=None if B != 64 else 0)
    mm, hist, g32 = S.so_histograms(ds, U.i32(idx), U.i64(off), pj, B, want_gains=True)
    mm, hist, g32 = mm.cpu().numpy(), hist.cpu().numpy(), g32.cpu().numpy()
    worst = 0.0
    for j, s in enumerate(sizes):
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, C, idx[off[j]:off[j + 1]], nptr, nf, ns, n_bins=B, hist_only=True,
                           want_debug=True)
        np.testing.assert_array_equal(U.f32bits(mm[j]), U.f32bits(r.minmax), err_msg=f"minmax node {j}")
        np.testing.assert_array_equal(hist[j], r.hist, err_msg=f"hist node {j}")
        skip = r.gains < 0
        np.testing.assert_array_equal(g32[j][skip], -1.0)
        if (~skip).any():
            g = g32[j][~skip].astype(np.float64) / (float(s) * float(s))
            rel = np.abs(g - r.gains[~skip]) / np.maximum(r.gains[~skip], 1e-300)
            rel = rel[r.gains[~skip] > 0]
            if rel.size:
                worst = max(worst, float(rel.max()))
    assert worst <= GAIN32_REL_TOL, worst


@pytest.mark.parametrize("d,cap,P", [(4096, 16, 96), (600, 32, 40), (70000, 8, 8)])
def test_histogram_stage_wide(S, d, cap, P):
    """Wide data: projection groups are formed on the device under the tile's
    feature budget; groups wider than a tile take the direct path; more than
    65536 features use the general kernels."""
    rng = np.random.default_rng(d + cap)
    n = 3000 if d > 10000 else 20000
    X = rng.standard_normal((d, n)).astype(np.float32)
    y = rng.integers(0, 3, n).astype(np.uint8)
    sizes = [4000, 2500, 333] if n > 5000 else [2000, 999]
    idx, off = _mixed_nodes(rng, n, sizes)
    projs = [G.random_projections(rng, P, d, 8.0, cap) for _ in sizes]
    ptr, feat, sign = U.concat_projs([(p.ptr, p.feat, p.sign) for p in projs])
    ds = U.upload_dataset(X, y, 3)
    pj = U.upload_projs(ptr, feat, sign, P)
    mm, hist, _ = S.so_histograms(ds, U.i32(idx), U.i64(off), pj, 256)
    mm, hist = mm.cpu().numpy(), hist.cpu().numpy()
    for j in range(len(sizes)):
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, 3, idx[off[j]:off[j + 1]], nptr, nf, ns, hist_only=True, want_debug=True)
        np.testing.assert_array_equal(U.f32bits(mm[j]), U.f32bits(r.minmax), err_msg=f"minmax node {j}")
        np.testing.assert_array_equal(hist[j], r.hist, err_msg=f"hist node {j}")


def test_ill_conditioned_ranges(S):
    """Projections whose range is tiny against their magnitude (a few ulps wide
    up to 2^-20 of the value) take the exact bin rule; boundaries coincide."""
    rng = np.random.default_rng(77)
    n, d = 5000, 6
    base = np.float32(1000.0)
    X = np.empty((d, n), np.float32)
    X[0] = base + np.float32(2.0 ** -13) * rng.integers(0, 4, n).astype(np.float32)   # 4 distinct values
    X[1] = np.where(rng.random(n) < 0.5, base, np.nextafter(base, np.float32(2000)))
    X[2] = rng.standard_normal(n).astype(np.float32) * np.float32(1e-3) + np.float32(7.0)
    X[3] = rng.standard_normal(n).astype(np.float32)
    X[4] = np.float32(3.0)
    X[5] = rng.standard_normal(n).astype(np.float32) * np.float32(1e4)
    y = rng.integers(0, 2, n).astype(np.uint8)
    ptr = np.arange(d + 1, dtype=np.int32)
    feat = np.arange(d, dtype=np.int32)
    sign = np.ones(d, np.int8)
    idx = np.arange(n, dtype=np.int32)
    off = np.array([0, n], np.int64)
    ds = U.upload_dataset(X, y, 2)
    pj = U.upload_projs(ptr, feat, sign, d)
    mm, hist, _ = S.so_histograms(ds, U.i32(idx), U.i64(off), pj, 256)
    r = O.split_search(X, y, 2, idx, ptr, feat, sign, hist_only=True, want_debug=True)
    np.testing.assert_array_equal(U.f32bits(mm.cpu().numpy()[0]), U.f32bits(r.minmax))
    np.testing.assert_array_equal(hist.cpu().numpy()[0], r.hist)
    out, _ = S.so_split_search(ds, U.i32(idx), pj, S.split_params(256, 0, True))
    U.assert_split_equal(out, r)


# ---------------------------------------------------------------- single-node search

def _single_cases():
    return [
        dict(n=30000, hist_only=True, T=0),
        dict(n=5000, hist_only=False, T=1024),     # histogram by size
        dict(n=900, hist_only=False, T=1024),      # medium exact path
        dict(n=20, hist_only=False, T=1024),       # tiny exact path
        dict(n=33, hist_only=False, T=1024),
        dict(n=128, hist_only=False, T=1024),      # largest register-sorted node
        dict(n=129, hist_only=False, T=1024),      # smallest CTA-sorted node
        dict(n=257, hist_only=False, T=1024),
        dict(n=1, hist_only=False, T=1024),
        dict(n=2, hist_only=True, T=0),
        dict(n=2047, hist_only=False, T=2048),     # largest exact node
    ]


@pytest.mark.parametrize("case", _single_cases(), ids=lambda c: f"n{c['n']}_h{int(c['hist_only'])}_T{c['T']}")
@pytest.mark.parametrize("C", [2, 5])
def test_split_search_single_parity(S, case, C):
    rng = np.random.default_rng(case["n"] * 7 + C)
    n_data, d, P = 40000, 16, 24
    X = rng.standard_normal((d, n_data)).astype(np.float32)
    X[3] = np.round(X[3])
    y = rng.integers(0, C, n_data).astype(np.uint8)
    idx = rng.integers(0, n_data, case["n"]).astype(np.int32)
    pr = G.random_projections(rng, P, d, 1.5, 8)
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(pr.ptr, pr.feat, pr.sign, P, max_nnz=None if C == 2 else 0)
    prm = S.split_params(256, case["T"], case["hist_only"])
    out, lc = S.so_split_search(ds, U.i32(idx), pj, prm)
    r = O.split_search(X, y, C, idx, pr.ptr, pr.feat, pr.sign, sort_below=case["T"], hist_only=case["hist_only"])
    U.assert_split_equal(out, r, str(case))
    np.testing.assert_array_equal(lc, r.left_counts if r.valid else np.zeros(C, np.int64))


def test_pure_and_constant_nodes(S):
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
        out, _ = S.so_split_search(ds, U.i32(idx), pj, S.split_params(256, T, ho))
        r = O.split_search(X, y, 2, idx, ptr, feat, sign, sort_below=T, hist_only=ho)
        assert r.valid == 0
        U.assert_split_equal(out, r)
    # pure node
    pj2 = U.upload_projs(np.array([0, 1], np.int32), np.array([0], np.int32), np.array([1], np.int8), 1)
    idx = np.arange(2500, 5000, dtype=np.int32)
    for T, ho in ((0, True), (4096 // 2, False)):
        out, _ = S.so_split_search(ds, U.i32(idx), pj2, S.split_params(256, T, ho))
        assert out.valid == 0


def test_malformed_projection_rows_rejected(S):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((4, 100)).astype(np.float32)
    y = rng.integers(0, 2, 100).astype(np.uint8)
    ds = U.upload_dataset(X, y, 2)
    idx = U.i32(np.arange(100))
    for ptr, feat, sign in ((np.array([0, 1]), np.array([4]), np.array([1])),        # feature >= d
                            (np.array([0, 2]), np.array([2, 1]), np.array([1, 1])),  # not ascending
                            (np.array([0, 1]), np.array([1]), np.array([3]))):       # sign not +-1
        pj = U.upload_projs(ptr, feat, sign, 1)
        with pytest.raises(S.SoError) as ei:
            S.so_split_search(ds, idx, pj, S.split_params(256, 1024, False))
        assert ei.value.status == S.SO_EINVAL


# ---------------------------------------------------------------- batched frontier

def _frontier_case(n, d, m, P, seed, C=2):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((d, n)).astype(np.float32)
    y = rng.integers(0, C, n).astype(np.uint8) if C > 2 else G.binary_sum_labels(rng, X, 4, 0.05)
    idx, off = G.frontier_nodes(n, m, seed=seed + 1)
    projs = [G.random_projections(rng, P, d, 1.5, 8) for _ in range(m)]
    ptr, feat, sign = U.concat_projs([(p.ptr, p.feat, p.sign) for p in projs])
    return X, y, idx, off, ptr, feat, sign


@pytest.mark.parametrize("T", [1024, 64, 0])
def test_batch_parity_lognormal_frontier(S, T):
    n, d, m, P, C = 120000, 32, 400, 16, 2
    X, y, idx, off, ptr, feat, sign = _frontier_case(n, d, m, P, 21 + T)
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(ptr, feat, sign, P)
    prm = S.split_params(256, T, T == 0)
    out, lc = S.so_split_search_batch(ds, U.i32(idx), U.i64(off), pj, prm)
    rec = S.splits_to_numpy(out)
    lc = lc.cpu().numpy().reshape(m, C)
    for j in range(m):
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, C, idx[off[j]:off[j + 1]], nptr, nf, ns, sort_below=T, hist_only=(T == 0))
        U.assert_split_equal(rec[j], r, f"node {j} size {off[j + 1] - off[j]}")
        np.testing.assert_array_equal(lc[j], r.left_counts if r.valid else 0)
    # batched partition of the same frontier
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


def test_partition_single_parity(S):
    rng = np.random.default_rng(5)
    n, d = 70001, 8
    X = rng.standard_normal((d, n)).astype(np.float32)
    y = rng.integers(0, 2, n).astype(np.uint8)
    ds = U.upload_dataset(X, y, 2)
    idx = np.sort(rng.integers(0, n, 50000)).astype(np.int32)
    feat, sign = np.array([1, 4, 6], np.int32), np.array([1, -1, 1], np.int8)
    for thr in (0.3, -10.0, 10.0):
        t = U.i32(idx)
        nl = S.so_partition(ds, t, U.i32(feat), U.torch_cuda().from_numpy(sign).cuda(), thr)
        exp, enl = O.partition(X, idx, feat, sign, thr)
        assert nl == enl
        np.testing.assert_array_equal(t.cpu().numpy(), exp)


# ---------------------------------------------------------------- trees

def _train_both(S, X, y, C, root, **kw):
    ds = U.upload_dataset(X, y, C)
    tp = S.tree_params(kw["n_proj"], kw["lam"], kw["cap"], kw.get("n_bins", 256), kw.get("sort_below", 1024),
                       kw.get("hist_only", False), kw.get("seed", 0), kw.get("tree_id", 0),
                       kw.get("max_depth", -1))
    gt = S.so_train_tree(ds, U.i32(root), tp)
    ot = O.train_tree(X, y, C, root, n_proj=kw["n_proj"], lam=kw["lam"], cap=kw["cap"],
                      n_bins=kw.get("n_bins", 256), sort_below=kw.get("sort_below", 1024),
                      hist_only=kw.get("hist_only", False), seed=kw.get("seed", 0),
                      tree_id=kw.get("tree_id", 0), max_depth=kw.get("max_depth", -1))
    return gt, ot


def test_tree_parity_tree_small_full(S):
    """One tree grown to purity on n=8192, d=32, 32 projections/node, T=1024."""
    ds = G.tree_small()
    p = G.WORKLOAD_PARAMS["tree_small"]
    gt, ot = _train_both(S, ds.X, ds.y, 2, G.all_indices(ds.n), n_proj=p["n_proj"], lam=p["lam"], cap=p["cap"],
                         sort_below=p["sort_below"], seed=G.PROJ_SEED_BASE)
    U.assert_tree_equal(gt, ot)
    assert set(np.unique(gt.path)) >= {0, 1}


@pytest.mark.parametrize("variant", ["multiclass_bootstrap", "hist_only_b32", "max_depth", "counts_ties",
                                     "tiny_T", "trunk"])
def test_tree_parity_variants(S, variant):
    if variant == "multiclass_bootstrap":
        ds = G.root_4m(n=6000, d=20, seed=99)
        root = G.bootstrap_indices(ds.n, 3, seed=7)
        kw = dict(n_proj=24, lam=1.5, cap=8, sort_below=300, seed=11, tree_id=3)
    elif variant == "hist_only_b32":
        ds = G.tree_small(n=3000, d=16, seed=98)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=12, lam=1.5, cap=8, n_bins=32, hist_only=True, sort_below=0, seed=5)
    elif variant == "max_depth":
        ds = G.tree_small(n=5000, d=16, seed=97)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=16, lam=1.5, cap=8, sort_below=512, seed=6, max_depth=4)
    elif variant == "counts_ties":
        ds = G.wide_counts(n=4000, d=256, seed=96)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=32, lam=3.0, cap=16, sort_below=1024, seed=8)
    elif variant == "trunk":
        ds = G.trunk(n=6000, p=64, seed=94)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=12, lam=1.0, cap=8, sort_below=700, seed=10)
    else:
        ds = G.tree_small(n=4000, d=16, seed=95)
        root = G.all_indices(ds.n)
        kw = dict(n_proj=8, lam=1.5, cap=8, sort_below=40, seed=9)
    gt, ot = _train_both(S, ds.X, ds.y, ds.n_classes, root, **kw)
    U.assert_tree_equal(gt, ot)


# ---------------------------------------------------------------- full-size workloads

def test_root_4m_full_size(S):
    """Root split on n=4M, d=64, 3 classes, 256 projections, histogram path,
    in the same launch configuration the benchmark times; every output
    compared with the oracle over all 256 projections."""
    torch = U.torch_cuda()
    ds_np = G.root_4m()
    p = G.WORKLOAD_PARAMS["root_4m"]
    rng = np.random.default_rng(G.PROJ_SEED_BASE + 1)
    pr = G.random_projections(rng, p["n_proj"], ds_np.d, p["lam"], p["cap"])
    ds = U.upload_dataset(ds_np.X, ds_np.y, 3)
    pj = U.upload_projs(pr.ptr, pr.feat, pr.sign, p["n_proj"])
    idx = G.all_indices(ds_np.n)
    prm = S.split_params(256, 0, True)
    off = U.i64([0, ds_np.n])
    out, lc = S.so_split_search_batch(ds, U.i32(idx), off, pj, prm)
    rec = S.splits_to_numpy(out)[0]
    r = O.split_search(ds_np.X, ds_np.y, 3, idx, pr.ptr, pr.feat, pr.sign, hist_only=True)
    U.assert_split_equal(rec, r, "root_4m")
    np.testing.assert_array_equal(lc.cpu().numpy(), r.left_counts)
    idx_out = torch.empty(ds_np.n, dtype=torch.int32, device="cuda")
    S.so_partition_batch(ds, U.i32(idx), idx_out, off, pj, out)
    exp, nl = O.partition(ds_np.X, idx, pr.feat[pr.ptr[r.proj]:pr.ptr[r.proj + 1]],
                          pr.sign[pr.ptr[r.proj]:pr.ptr[r.proj + 1]], float(r.threshold))
    np.testing.assert_array_equal(idx_out.cpu().numpy(), exp)


def test_frontier_1m_full_size(S):
    """4096 frontier nodes with lognormal(5, 2) sizes over n=1M, d=128, 64
    projections/node, mixed exact and histogram paths in one call, with the
    row-major feature copy and the autotuned crossover T as the benchmark runs
    it (and at T = 1024); every node compared with the oracle."""
    ds_np = G.frontier_1m()
    p = G.WORKLOAD_PARAMS["frontier_1m"]
    idx, off = G.frontier_nodes(ds_np.n, p["n_nodes"])
    rng = np.random.default_rng(G.PROJ_SEED_BASE + 2)
    m, P = p["n_nodes"], p["n_proj"]
    projs = [G.random_projections(rng, P, ds_np.d, p["lam"], p["cap"]) for _ in range(m)]
    ptr, feat, sign = U.concat_projs([(q.ptr, q.feat, q.sign) for q in projs])
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2).with_row_major()
    pj = U.upload_projs(ptr, feat, sign, P)
    tuned, _, _ = S.so_autotune(ds, P, p["lam"], p["cap"], S.split_params(256, p["sort_below"], False))
    for T in sorted({int(tuned.sort_below), p["sort_below"]}):
        prm = S.split_params(256, T, False)
        out, lc = S.so_split_search_batch(ds, U.i32(idx), U.i64(off), pj, prm)
        rec = S.splits_to_numpy(out)
        for j in range(m):
            q = projs[j]
            r = O.split_search(ds_np.X, ds_np.y, 2, idx[off[j]:off[j + 1]], q.ptr, q.feat, q.sign, sort_below=T)
            U.assert_split_equal(rec[j], r, f"node {j} T {T}")


# ---------------------------------------------------------------- crossover autotune

def test_autotune_crossover_and_tree_with_tuned_T(S):
    """The start-up microbenchmark returns a crossover within the supported
    range; a tree grown with that T is still identical to the oracle's tree
    grown with the same T."""
    ds_np = G.tree_small(n=20000, d=16, seed=55)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2)
    prm, sizes, times = S.so_autotune(ds, 16, 1.5, 8, S.split_params(256, 1024, False))
    T = prm.sort_below
    assert 32 <= T <= 2048
    assert len(sizes) >= 8 and np.all(times > 0)
    root = G.all_indices(ds_np.n)
    gt, ot = _train_both(S, ds_np.X, ds_np.y, 2, root, n_proj=16, lam=1.5, cap=8, sort_below=T, seed=3)
    U.assert_tree_equal(gt, ot)


# ---------------------------------------------------------------- forest

@pytest.mark.parametrize("row_major", [False, True])
def test_forest_bootstrap_trees_match_oracle(S, row_major):
    """A small forest (lognormal heavy-tailed features, 8-sparse median-centred
    labels, 10% flips): every bootstrapped tree identical to the oracle's, with
    and without the row-major copy of the features (scattered samples' rows)."""
    from paper_2603_00326_b300 import forest as F
    ds_np = G.forest_2m(n=6000, d=32, seed=91)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2)
    if row_major:
        ds = ds.with_row_major()
        np.testing.assert_array_equal(ds.Xr.cpu().numpy(), ds_np.X.T)
    cfg = F.ForestConfig(n_trees=4, n_proj=16, lam=1.5, cap=8, sort_below=512)
    trees, _ = F.train_forest(cfg, ds)
    assert len(trees) == 4
    for t, gt in enumerate(trees):
        root = F.root_indices(ds_np.n, t, cfg)
        ot = O.train_tree(ds_np.X, ds_np.y, 2, root, n_proj=16, lam=1.5, cap=8, sort_below=512, seed=cfg.seed,
                          tree_id=t)
        U.assert_tree_equal(gt, ot)


# ---------------------------------------------------------------- work decomposition

@pytest.mark.parametrize("ppc,chunk", [(1, 512), (2, 1000), (7, 4096), (16, 2048), (32, 16384), (64, 8192)])
@pytest.mark.parametrize("rule", [0, 1])
def test_decomposition_knobs_leave_results_unchanged(S, ppc, chunk, rule):
    """Projections per CTA and samples per histogram item change only the work
    decomposition: histograms and splits stay the oracle's."""
    rng = np.random.default_rng(ppc * 31 + chunk + rule)
    n, d, P, C = 50000, 24, 40, 3
    X = rng.standard_normal((d, n)).astype(np.float32)
    y = rng.integers(0, C, n).astype(np.uint8)
    sizes = [30001, 7777, 1500]
    idx, off = _mixed_nodes(rng, n, sizes)
    projs = [G.random_projections(rng, P, d, 1.5, 8) for _ in sizes]
    ptr, feat, sign = U.concat_projs([(q.ptr, q.feat, q.sign) for q in projs])
    keys = rng.integers(0, 2 ** 62, len(sizes), dtype=np.int64)
    kt = U.i64(keys) if rule else None
    ds = U.upload_dataset(X, y, C)
    pj = U.upload_projs(ptr, feat, sign, P)
    prm = S.split_params(256, 1024, True, bin_rule=rule, bin_keys=kt, proj_per_cta=ppc, chunk=chunk)
    out, lc = S.so_split_search_batch(ds, U.i32(idx), U.i64(off), pj, prm)
    rec = S.splits_to_numpy(out)
    for j in range(len(sizes)):
        nptr, nf, ns = U.oracle_node_projs(ptr, feat, sign, P, j)
        r = O.split_search(X, y, C, idx[off[j]:off[j + 1]], nptr, nf, ns, hist_only=True, bin_rule=rule,
                           bin_key=int(keys[j]))
        U.assert_split_equal(rec[j], r, f"node {j} ppc {ppc} chunk {chunk}")
    one, _ = S.so_split_search(ds, U.i32(idx[:sizes[0]]), U.upload_projs(*U.oracle_node_projs(ptr, feat, sign, P, 0),
                                                                         P), prm)
    U.assert_split_equal(one, O.split_search(X, y, C, idx[:sizes[0]], *U.oracle_node_projs(ptr, feat, sign, P, 0),
                                             hist_only=True, bin_rule=rule, bin_key=int(keys[0])))


def test_autotuned_decomposition_and_tree(S):
    ds_np = G.tree_small(n=20000, d=16, seed=58)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2)
    prm, _, _ = S.so_autotune(ds, 16, 1.5, 8, S.split_params(256, 1024, False))
    assert prm.proj_per_cta in (16, 32, 64) and prm.chunk in (4096, 8192, 16384)
    tp = S.tree_params(16, 1.5, 8, 256, prm.sort_below, seed=3, proj_per_cta=prm.proj_per_cta, chunk=prm.chunk)
    gt = S.so_train_tree(ds, U.i32(G.all_indices(ds_np.n)), tp)
    ot = O.train_tree(ds_np.X, ds_np.y, 2, G.all_indices(ds_np.n), n_proj=16, lam=1.5, cap=8,
                      sort_below=prm.sort_below, seed=3)
    U.assert_tree_equal(gt, ot)


def test_forest_training_is_deterministic(S):
    """The same forest trained twice gives identical tree arrays (every field,
    every tree), hashed."""
    import hashlib
    from paper_2603_00326_b300 import forest as F
    ds_np = G.forest_2m(n=20000, d=32, seed=88)
    ds = U.upload_dataset(ds_np.X, ds_np.y, 2).with_row_major()
    cfg = F.ForestConfig(n_trees=3, n_proj=16, lam=1.5, cap=8, sort_below=512)

    def digest(trees):
        h = hashlib.sha256()
        for t in trees:
            for f in S.Tree.FIELDS:
                h.update(np.ascontiguousarray(getattr(t, f)).tobytes())
        return h.hexdigest()
    a, _ = F.train_forest(cfg, ds)
    b, _ = F.train_forest(cfg, ds)
    assert digest(a) == digest(b)
