"""Benchmark: root-node split search of sparse oblique forest training on B300.

Workload (the metric's configuration): single root-node split search on the
histogram path, n = 4,194,304 samples, d = 64 float32 N(0,1) features,
3 classes from sparse linear scores, 256 projections with 1+Poisson(1.5)
(cap 8) +-1 non-zeros, 256 equal-width bins.  One step = the whole hot path
for that node: min/max of every projection, histograms, Gini scan with double
re-score, selection, and the stable partition of the node's samples.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is whole-job sample-projections per second
(n * P per step, summed over ranks), inputs resident in HBM.  Under torchrun
(N > 1) every rank runs an independent replica: the split search of one node
does not shard without collectives, so N GPUs run N replicas ("replicas
only"), with a barrier and max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "projected sample-projections/s in split search"
UNIT = "sample-projections/s"
WORKLOAD = "root_4m"
FALLBACK_HBM_GBS = 6400.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_inputs(n=None):
    """The root node's inputs; n: a smaller node of the same recipe (profiling
    cases), default the benchmark's 4M samples."""
    from paper_2603_00326_b300 import datagen as G
    ds = G.root_4m() if n is None else G.root_4m(n=n)
    p = G.WORKLOAD_PARAMS[WORKLOAD]
    rng = np.random.default_rng(G.PROJ_SEED_BASE + 1)
    pr = G.random_projections(rng, p["n_proj"], ds.d, p["lam"], p["cap"])
    return ds, pr, p


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(ds, pr, n_sample_proj: int, threads: int = 1):
    """The oracle as it stands on all n samples and the first n_sample_proj
    projections (a bounded sample of the same workload), its projections
    divided over `threads` host threads."""
    import oracle as O
    from paper_2603_00326_b300 import datagen as G
    idx = G.all_indices(ds.n)
    ptr = pr.ptr[:n_sample_proj + 1]
    t0 = time.perf_counter()
    O.split_search_mt(ds.X, ds.y, ds.n_classes, idx, ptr, pr.feat, pr.sign, hist_only=True, n_threads=threads)
    O.partition(ds.X, idx, pr.feat[pr.ptr[0]:pr.ptr[1]], pr.sign[pr.ptr[0]:pr.ptr[1]], 0.0)
    dt = time.perf_counter() - t0
    return ds.n * n_sample_proj / dt, dt


def profile_summary(name):
    """The committed ncu summary profiles/<name>.json of a kernel, if it was
    taken on the kernel source this run executes (the sha256 of the source
    file it names matches); otherwise None, so that counters of an older
    kernel are never reported as this one's."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", name + ".json")) as fh:
            rec = json.load(fh)
        with open(os.path.join(ROOT, rec["source"]), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest() != rec["source_sha256"]:
                return None
        return rec
    except (OSError, ValueError, KeyError):
        return None


def roofline_block(achieved, hbm, peak_kind, alg_bytes, k_avg_ms, clk, full_size=True):
    """The histogram kernel against the measured HBM copy bandwidth, with its
    DRAM traffic and its two on-chip ceilings from the committed ncu summary
    of the same kernel source: the shared-memory pipe (one 128-byte wavefront
    per SM per clock) and instruction issue (four warp-instructions per SM per
    clock), each as the time that many wavefronts or instructions need at the
    SM clock sampled during this run, over the measured launch time."""
    out = {"bound": "hbm", "kernel": "k_hist", "achieved": achieved, "peak": hbm, "unit": "GB/s",
           "frac": (achieved / hbm) if achieved else None, "traffic": None, "peak_source": peak_kind,
           "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": k_avg_ms}
    rec = profile_summary("k_hist_staged_root_4m") if full_size else None
    if rec is None or not k_avg_ms:
        out["traffic_note"] = ("no ncu summary of this kernel source under profiles/" if full_size else
                               "the committed ncu summary describes the full-size node, not this one")
        return out
    out["traffic"] = rec["dram_bytes_per_launch"]
    mhz = (clk or {}).get("sm_mhz") or 2032.0
    sms = rec.get("sms", 148)
    per_ms = sms * mhz * 1e3  # SM-clocks per millisecond
    sram_ms = rec["shared_wavefronts_per_launch"] / per_ms
    issue_ms = rec["warp_instructions_per_launch"] / (4 * per_ms)
    out["ceilings"] = {
        "shared_pipe": {"wavefronts_per_launch": rec["shared_wavefronts_per_launch"], "floor_ms": sram_ms,
                        "frac": sram_ms / k_avg_ms},
        "issue": {"warp_instructions_per_launch": rec["warp_instructions_per_launch"], "floor_ms": issue_ms,
                  "frac": issue_ms / k_avg_ms},
        "source": rec.get("summary", "profiles/k_hist_staged_root_4m.md")}
    return out


def gain_error(S, torch, ds, ds_np, pr, idx, off, n_proj=8):
    """Largest relative error of the GPU's float Gini gains against the
    oracle's double gains, over every candidate of positive double gain, for
    the first n_proj projections of the benchmark node: the oracle's
    per-candidate gains beside the float gains the GPU's histogram stage
    exports (which lack the constant 1/n^2 factor: n^2 is a power of two here,
    so the division is exact)."""
    import oracle as O
    from paper_2603_00326_b300 import datagen as G
    ptr = np.ascontiguousarray(pr.ptr[:n_proj + 1])
    r = O.split_search(ds_np.X, ds_np.y, ds_np.n_classes, G.all_indices(ds_np.n), ptr, pr.feat, pr.sign,
                       hist_only=True, want_debug=True)
    dev = idx.device
    pj = S.DeviceProjs(n_proj, torch.from_numpy(ptr).to(dev), torch.from_numpy(pr.feat).to(dev),
                       torch.from_numpy(pr.sign).to(dev), int(np.diff(ptr).max()))
    _, _, g32 = S.so_histograms(ds, idx, off, pj, 256, want_gains=True)
    g32 = g32.cpu().numpy()[0].astype(np.float64) / (float(ds_np.n) ** 2)
    g64 = r.gains
    pos = g64 > 0
    rel = np.abs(g32[pos] - g64[pos]) / g64[pos]
    return {"max_rel": float(rel.max()), "candidates": int(pos.sum()), "projections": n_proj,
            "bound_stated": 1e-6,
            "what": "max |gain32 - gain64| / gain64 over candidates with gain64 > 0 (float Gini key of the "
                    "histogram stage against the oracle's double gain); the chosen split's gain is the double "
                    "re-score itself"}


def extra_legs(S, torch, dev, forest_trees=2, only=None, wide_trees=1, rw_tree=True, batched_only=False,
               wide_n=None, frontier_fixed=None):
    """Secondary measurements: the batched frontier against the node-at-a-time
    form on the same GPU (frontier_1m: n=1M, d=128, 4096 lognormal nodes,
    64 projections/node, crossover T autotuned), one tree grown to purity
    (tree_small), trees of the forest (forest_2m) and the wide tree."""
    from paper_2603_00326_b300 import datagen as G
    out = {}
    if only not in (None, "frontier"):
        return _later_legs(S, torch, dev, forest_trees, only, out, wide_trees, rw_tree=rw_tree, wide_n=wide_n)
    ds_np = G.frontier_1m()
    p = G.WORKLOAD_PARAMS["frontier_1m"]
    idx_np, off_np = G.frontier_nodes(ds_np.n, p["n_nodes"])
    rng = np.random.default_rng(G.PROJ_SEED_BASE + 2)
    m, P = p["n_nodes"], p["n_proj"]
    projs = [G.random_projections(rng, P, ds_np.d, p["lam"], p["cap"]) for _ in range(m)]
    ptrs = [np.zeros(1, np.int32)]
    base = 0
    for q in projs:
        ptrs.append(q.ptr[1:] + base)
        base += int(q.ptr[-1])
    ptr = np.concatenate(ptrs).astype(np.int32)
    feat = np.concatenate([q.feat for q in projs]).astype(np.int32)
    sign = np.concatenate([q.sign for q in projs]).astype(np.int8)
    dd = S.DeviceDataset(torch.from_numpy(ds_np.X).to(dev), torch.from_numpy(ds_np.y).to(dev), 2).with_row_major()
    cap = int(p["cap"])
    pj = S.DeviceProjs(P, torch.from_numpy(ptr).to(dev), torch.from_numpy(feat).to(dev),
                       torch.from_numpy(sign).to(dev), cap)
    idx = torch.from_numpy(idx_np).to(dev)
    off = torch.from_numpy(off_np).to(dev)
    # the crossover T from the start-up microbenchmark (Section 3.1), as this
    # workload specifies; both forms below use it
    if frontier_fixed:
        # profiling case: the given crossover and decomposition instead of the
        # start-up microbenchmark (whose timings a profiler distorts)
        T_, ppc_, ch_ = frontier_fixed
        prm = S.split_params(256, T_, False, proj_per_cta=ppc_, chunk=ch_)
    else:
        prm, tune_sizes, tune_ms = S.so_autotune(dd, P, p["lam"], int(p["cap"]),
                                                 S.split_params(256, p["sort_below"], False))
    ws = torch.empty(S.so_split_search_ws_bytes(m, ds_np.n, P, 2, prm), dtype=torch.uint8, device=dev)
    outb = torch.empty(m * S.SPLIT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    for _ in range(3):
        S.so_split_search_batch(dd, idx, off, pj, prm, out=outb, workspace=ws)
    torch.cuda.synchronize()
    reps = 10
    t0 = time.perf_counter()
    for _ in range(reps):
        S.so_split_search_batch(dd, idx, off, pj, prm, out=outb, workspace=ws)
    torch.cuda.synchronize()
    batched_ms = (time.perf_counter() - t0) * 1000.0 / reps
    sp = float(ds_np.n * P)
    if batched_only:
        return {"frontier_1m": {"nodes": m, ("fixed_sort_below" if frontier_fixed else "autotuned_sort_below"):
                                int(prm.sort_below), "proj_per_cta": int(prm.proj_per_cta), "chunk": int(prm.chunk),
                                "batched_ms": batched_ms,
                                "batched_sample_projections_per_s": sp / (batched_ms / 1000.0)}}
    # node-at-a-time: one synchronous call per node (the paper's offload form)
    views = []
    for j in range(m):
        a, b = int(off_np[j]), int(off_np[j + 1])
        r0, r1 = int(ptr[j * P]), int(ptr[(j + 1) * P])
        views.append((idx[a:b], S.DeviceProjs(P, pj.ptr[j * P:(j + 1) * P + 1] - r0, pj.feat[r0:r1],
                                              pj.sign[r0:r1], cap)))
    wsn = torch.empty(S.so_split_search_ws_bytes(1, int(np.diff(off_np).max()), P, 2, prm) + 4096 + 1024,
                      dtype=torch.uint8, device=dev)
    for j in range(min(m, 64)):
        S.so_split_search(dd, views[j][0], views[j][1], prm, workspace=wsn)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = []
    for j in range(m):
        plain.append(S.so_split_search(dd, views[j][0], views[j][1], prm, workspace=wsn)[0])
    plain_ms = (time.perf_counter() - t0) * 1000.0
    rec = S.splits_to_numpy(outb)
    same = all(int(rec[j]["proj"]) == plain[j].proj and int(rec[j]["cand"]) == plain[j].cand and
               float(rec[j]["gain"]) == plain[j].gain for j in range(m))
    out["frontier_1m"] = {"nodes": m, "autotuned_sort_below": int(prm.sort_below),
                          "autotuned_proj_per_cta": int(prm.proj_per_cta), "autotuned_chunk": int(prm.chunk),
                          "batched_ms": batched_ms, "plain_ms": plain_ms,
                          "speedup": plain_ms / batched_ms, "identical": bool(same),
                          "batched_sample_projections_per_s": sp / (batched_ms / 1000.0)}
    del dd, idx, off, ws, outb, views
    if only == "frontier":
        return out
    return _later_legs(S, torch, dev, forest_trees, only, out, wide_trees, rw_tree=rw_tree, wide_n=wide_n)


def _later_legs(S, torch, dev, forest_trees, only, out, wide_trees=1, trunk_trees=1, rw_tree=True, wide_n=None):
    from paper_2603_00326_b300 import datagen as G
    if only in (None, "tree"):
        # one tree to purity
        ts = G.tree_small()
        tp = G.WORKLOAD_PARAMS["tree_small"]
        dd = S.DeviceDataset(torch.from_numpy(ts.X).to(dev), torch.from_numpy(ts.y).to(dev), 2)
        root = torch.from_numpy(G.all_indices(ts.n)).to(dev)
        prm = S.tree_params(tp["n_proj"], tp["lam"], tp["cap"], 256, tp["sort_below"], seed=G.PROJ_SEED_BASE)
        S.so_train_tree(dd, root, prm)
        times = []
        for _ in range(5):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tr = S.so_train_tree(dd, root, prm)
            times.append(time.perf_counter() - t0)
        out["tree_small"] = {"train_s": min(times), "median_s": statistics.median(times), "nodes": tr.n_nodes,
                             "depth": int(tr.depth.max())}
        del dd, root
    if forest_trees > 0 and only in (None, "forest"):
        from paper_2603_00326_b300 import forest as F
        fs = G.forest_2m()
        fp = G.WORKLOAD_PARAMS["forest_2m"]
        dd = S.DeviceDataset(torch.from_numpy(fs.X).to(dev), torch.from_numpy(fs.y).to(dev), 2).with_row_major()
        cfg = F.ForestConfig(n_trees=forest_trees, n_proj=fp["n_proj"], lam=fp["lam"], cap=fp["cap"],
                             sort_below=fp["sort_below"])
        F.train_forest(F.ForestConfig(n_trees=1, n_proj=8, lam=1.5, cap=8), dd)  # warm-up
        torch.cuda.synchronize()
        trees, secs = F.train_forest(cfg, dd)
        # inference: every sample through every trained tree, and each tree's
        # out-of-bag accuracy (samples its bootstrap never drew)
        fo = S.upload_forest(trees, 2)
        S.so_predict(dd.X, fo)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.so_predict(dd.X, fo)
        torch.cuda.synchronize()
        pred_s = time.perf_counter() - t0
        oob_acc = []
        votes = torch.zeros((fs.n, 2), dtype=torch.int32, device=dev)  # out-of-bag votes per sample
        for t, tr in enumerate(trees):
            inbag = np.zeros(fs.n, bool)
            inbag[F.root_indices(fs.n, t, cfg)] = True
            p1, _ = S.so_predict(dd.X, S.upload_forest([tr], 2))
            oob = ~inbag
            oob_acc.append(float((p1.cpu().numpy()[oob] == fs.y[oob]).mean()))
            ob = torch.from_numpy(np.flatnonzero(oob)).to(dev)
            votes[ob, p1[ob].long()] += 1
        has = votes.sum(1) > 0
        ens = (votes.argmax(1).to(torch.uint8) == torch.from_numpy(fs.y).to(dev)) & has
        oob_ensemble = float(ens.sum().item() / max(int(has.sum().item()), 1))
        out["forest_2m"] = {"trees": forest_trees, "of": fp["n_trees"], "train_s": secs,
                            "s_per_tree": secs / forest_trees,
                            "projected_forest_s": secs / forest_trees * fp["n_trees"],
                            "mean_nodes": float(np.mean([t.n_nodes for t in trees])),
                            "max_depth": int(max(int(t.depth.max()) for t in trees)),
                            "predict_sample_trees_per_s": fs.n * forest_trees / pred_s,
                            "oob_accuracy_per_tree": oob_acc[:8], "oob_accuracy_mean": float(np.mean(oob_acc)),
                            "oob_ensemble_accuracy": oob_ensemble}
        if rw_tree:
            # tree 0 again with random-width bins (the YDF default of the
            # paper's Section 1 footnote): time and out-of-bag accuracy
            import dataclasses
            rcfg = dataclasses.replace(cfg, n_trees=1, bin_rule=S.SO_BINS_RANDOM_WIDTH)
            torch.cuda.synchronize()
            rtrees, rsecs = F.train_forest(rcfg, dd)
            inbag = np.zeros(fs.n, bool)
            inbag[F.root_indices(fs.n, 0, rcfg)] = True
            p1, _ = S.so_predict(dd.X, S.upload_forest(rtrees, 2))
            out["forest_2m"]["random_width_tree0"] = {
                "train_s": rsecs, "nodes": rtrees[0].n_nodes, "depth": int(rtrees[0].depth.max()),
                "oob_accuracy": float((p1.cpu().numpy()[~inbag] == fs.y[~inbag]).mean())}
            # and with the entropy criterion (information gain, YDF's)
            ecfg = dataclasses.replace(cfg, n_trees=1, criterion=S.SO_CRIT_ENTROPY)
            torch.cuda.synchronize()
            etrees, esecs = F.train_forest(ecfg, dd)
            p1, _ = S.so_predict(dd.X, S.upload_forest(etrees, 2))
            out["forest_2m"]["entropy_tree0"] = {
                "train_s": esecs, "nodes": etrees[0].n_nodes, "depth": int(etrees[0].depth.max()),
                "oob_accuracy": float((p1.cpu().numpy()[~inbag] == fs.y[~inbag]).mean())}
            del rtrees, etrees
        del dd, trees, fo
    if wide_trees > 0 and only in (None, "wide"):
        # wide count-like data: n=500k, d=4096, 90% zeros, 5 classes, grown to purity
        ws_np = G.wide_counts() if wide_n is None else G.wide_counts(n=wide_n)
        wp = G.WORKLOAD_PARAMS["wide_counts"]
        dd = S.DeviceDataset(torch.from_numpy(ws_np.X).to(dev), torch.from_numpy(ws_np.y).to(dev), 5)
        root = torch.from_numpy(G.all_indices(ws_np.n)).to(dev)
        prm = S.tree_params(wp["n_proj"], wp["lam"], wp["cap"], wp["n_bins"], wp["sort_below"],
                            seed=G.PROJ_SEED_BASE + 4)
        S.so_train_tree(dd, root, S.tree_params(8, 1.5, 8, 256, 1024, seed=1, max_depth=3))  # warm-up
        times = []
        for _ in range(wide_trees):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tr = S.so_train_tree(dd, root, prm)
            times.append(time.perf_counter() - t0)
        out["wide_counts"] = {"train_s": min(times), "trees": wide_trees, "nodes": tr.n_nodes,
                              "depth": int(tr.depth.max()), "n": ws_np.n}
        del dd, root
    if trunk_trees > 0 and only in (None, "trunk"):
        # the Trunk generator at the paper's 100k and 1M rows, p = 1024: one
        # tree to purity each (the paper's Trunk rows are 128-tree forests)
        tp_ = G.WORKLOAD_PARAMS["trunk"]
        res = {}
        for n_tr in (100_000, 1_000_000):
            tk = G.trunk(n=n_tr, p=1024)
            dd = S.DeviceDataset(torch.from_numpy(tk.X).to(dev), torch.from_numpy(tk.y).to(dev), 2).with_row_major()
            root = torch.from_numpy(G.all_indices(tk.n)).to(dev)
            prm = S.tree_params(tp_["n_proj"], tp_["lam"], tp_["cap"], tp_["n_bins"], tp_["sort_below"],
                                seed=G.PROJ_SEED_BASE + 5)
            S.so_train_tree(dd, root, S.tree_params(8, 1.0, 8, 256, 1024, seed=1, max_depth=3))  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tr = S.so_train_tree(dd, root, prm)
            res[f"trunk_{n_tr // 1000}k"] = {"train_s": time.perf_counter() - t0, "nodes": tr.n_nodes,
                                             "depth": int(tr.depth.max())}
            del dd, root, tk
        out["trunk_p1024"] = res
    if only == "trunk10m":
        out["trunk_10m_p1024"] = trunk_10m_tree(S, torch, dev)
    torch.cuda.empty_cache()
    return out


def trunk_10m_tree(S, torch, dev, n=10_000_000, p=1024):
    """One tree to purity on Trunk at the paper's largest Trunk size (Table 3:
    10M rows; p = 1024 here), 48 projections per node of 1+Poisson(1)
    non-zeros, T = 1024, with the row-major copy.  The 41 GB feature matrix
    is generated in 64-feature blocks straight into device memory."""
    from paper_2603_00326_b300 import datagen as G
    tp_ = G.WORKLOAD_PARAMS["trunk"]
    t0 = time.perf_counter()
    X = torch.empty((p, n), dtype=torch.float32, device=dev)

    def fill(f0, blk):
        X[f0:f0 + blk.shape[0]].copy_(torch.from_numpy(blk))

    y = G.trunk_streamed(n, p, fill)
    gen_s = time.perf_counter() - t0
    dd = S.DeviceDataset(X, torch.from_numpy(y).to(dev), 2).with_row_major()
    root = torch.arange(n, dtype=torch.int32, device=dev)
    prm = S.tree_params(tp_["n_proj"], tp_["lam"], tp_["cap"], tp_["n_bins"], tp_["sort_below"],
                        seed=G.PROJ_SEED_BASE + 5)
    S.so_train_tree(dd, root, S.tree_params(8, 1.0, 8, 256, 1024, seed=1, max_depth=3))  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr = S.so_train_tree(dd, root, prm)
    train_s = time.perf_counter() - t0
    del dd, root, X
    return {"train_s": train_s, "nodes": tr.n_nodes, "depth": int(tr.depth.max()), "n": n, "p": p,
            "generate_s": gen_s, "device_gb": 2 * n * p * 4 / 1e9}


def variant_step(S, torch, ds, pj, idx, off, n, P, C, n_bins, steps, key=None, criterion=0):
    """The root step (search + partition) on resident inputs with random-width
    bins (key given: the YDF default of the paper's Section 1 footnote) or
    another criterion (1: information gain, YDF's): CUDA-event time per step
    and per-stage times."""
    dev = idx.device
    if key is not None:
        keys = torch.tensor([key], dtype=torch.int64, device=dev)
        prm = S.split_params(n_bins, 0, True, bin_rule=S.SO_BINS_RANDOM_WIDTH, bin_keys=keys, criterion=criterion)
    else:
        prm = S.split_params(n_bins, 0, True, criterion=criterion)
    ws = torch.empty(S.so_split_search_ws_bytes(1, n, P, C, prm), dtype=torch.uint8, device=dev)
    out = torch.empty(S.SPLIT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    lc = torch.empty(C, dtype=torch.int64, device=dev)
    idx_out = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        S.so_split_search_batch(ds, idx, off, pj, prm, out=out, left_counts=lc, workspace=ws)
        S.so_partition_batch(ds, idx, idx_out, off, pj, out)

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    S.so_profile_enable(True)  # stage times from a second, traced pass
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    S.so_profile_enable(False)
    prof = S.so_profile_read()
    stage_ms = {k: round(v[1] / max(v[0], 1), 4) for k, v in prof.items()}
    rec = S.splits_to_numpy(out)[0]
    return {"ms_per_step": ms, "sample_projections_per_s": n * P / (ms / 1000.0), "stage_ms_per_launch": stage_ms,
            "split": {"proj": int(rec["proj"]), "cand": int(rec["cand"]), "gain": float(rec["gain"])}}


def run_leg(args):
    """One secondary leg alone (for profiling): frontier | tree | forest | wide | trunk | rw."""
    import torch
    from paper_2603_00326_b300 import soforest as S
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    S.lib()
    if args.leg == "rw":
        ds_np, pr, p = make_inputs()
        n, P, C = ds_np.n, p["n_proj"], ds_np.n_classes
        ds = S.DeviceDataset(torch.from_numpy(ds_np.X).to(dev), torch.from_numpy(ds_np.y).to(dev), C)
        pj = S.DeviceProjs(P, torch.from_numpy(pr.ptr).to(dev), torch.from_numpy(pr.feat).to(dev),
                           torch.from_numpy(pr.sign).to(dev), int(np.diff(pr.ptr).max()))
        idx = torch.arange(n, dtype=torch.int32, device=dev)
        off = torch.tensor([0, n], dtype=torch.int64, device=dev)
        res = variant_step(S, torch, ds, pj, idx, off, n, P, C, p["n_bins"], args.steps, key=rw_key())
        res.update(_rw_roofline(pr, n, res["stage_ms_per_launch"].get("k_hist")))
        ent = variant_step(S, torch, ds, pj, idx, off, n, P, C, p["n_bins"], args.steps, criterion=1)
        del ds, pj, idx
        out = {"root_4m_random_width": res, "root_4m_entropy": ent}
        if args.forest_trees > 0:
            out.update(extra_legs(S, torch, dev, 1, only="forest", rw_tree=True))
        print(json.dumps({"leg": args.leg, **out}), flush=True)
        return 0
    # the forest leg alone grows only the equal-width Gini trees (the variant
    # trees run in the default extras and in --leg rw)
    out = extra_legs(S, torch, dev, args.forest_trees if args.leg == "forest" else 0, only=args.leg,
                     wide_trees=args.wide_trees if args.leg == "wide" else 0, rw_tree=False,
                     batched_only=args.batched_only, wide_n=args.wide_n,
                     frontier_fixed=tuple(int(v) for v in args.frontier_fixed.split(",")) if args.frontier_fixed else None)
    print(json.dumps({"leg": args.leg, **out}), flush=True)
    return 0


def rw_key() -> int:
    """Node key of the root in the random-width measurements (the full-size
    parity test uses the same key)."""
    from paper_2603_00326_b300 import datagen as G
    return G.PROJ_SEED_BASE + 11


def _rw_roofline(pr, n, k_hist_ms):
    hbm, peak_kind = peaks()
    alg_bytes = np.unique(pr.feat).size * n * 4 + n * 4 + n * 1
    if not k_hist_ms:
        return {}
    ach = alg_bytes / (k_hist_ms / 1000.0) / 1e9
    return {"roofline": {"bound": "hbm", "kernel": "k_hist (random width)", "achieved": ach, "peak": hbm,
                         "unit": "GB/s", "frac": ach / hbm, "peak_source": peak_kind,
                         "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": k_hist_ms}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    ds, pr, p = make_inputs()
    cores = host_cores()
    n_sample_proj = min(p["n_proj"], 2 * cores)
    for _ in range(args.warmup):
        cpu_baseline(ds, pr, n_sample_proj, cores)
    times = []
    for _ in range(args.steps):
        _, dt = cpu_baseline(ds, pr, n_sample_proj, cores)
        times.append(dt)
    ms = 1000.0 * sum(times) / len(times)
    value = ds.n * n_sample_proj / (ms / 1000.0)
    sample = (f"oracle split search (projections divided over {cores} threads) + partition on all {ds.n} "
              f"samples, first {n_sample_proj} of {p['n_proj']} projections per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": ds.n, "d": ds.d, "n_proj": p["n_proj"], "n_bins": 256,
                   "classes": ds.n_classes, "path": "histogram"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2603_00326_b300 import soforest as S

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    S.lib()

    ds_np, pr, p = make_inputs(args.root_n)
    n, d, P, C = ds_np.n, ds_np.d, p["n_proj"], ds_np.n_classes
    Xh = torch.from_numpy(ds_np.X).pin_memory()
    yh = torch.from_numpy(ds_np.y).pin_memory()
    idx_h = torch.arange(n, dtype=torch.int32).pin_memory()
    ptr_h = torch.from_numpy(pr.ptr).pin_memory()
    feat_h = torch.from_numpy(pr.feat).pin_memory()
    sign_h = torch.from_numpy(pr.sign).pin_memory()
    X = Xh.to(dev)
    y = yh.to(dev)
    idx = idx_h.to(dev)
    ptr, feat, sign = ptr_h.to(dev), feat_h.to(dev), sign_h.to(dev)
    ds = S.DeviceDataset(X, y, C)
    pj = S.DeviceProjs(P, ptr, feat, sign, int(np.diff(pr.ptr).max()))
    off = torch.tensor([0, n], dtype=torch.int64, device=dev)
    prm = S.split_params(p["n_bins"], 0, True)
    ws = torch.empty(S.so_split_search_ws_bytes(1, n, P, C, prm), dtype=torch.uint8, device=dev)
    out = torch.empty(S.SPLIT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    lc = torch.empty(C, dtype=torch.int64, device=dev)
    idx_out = torch.empty(n, dtype=torch.int32, device=dev)
    out_h = torch.empty(S.SPLIT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    stream = torch.cuda.current_stream()

    def step(idx_t):
        S.so_split_search_batch(ds, idx_t, off, pj, prm, out=out, left_counts=lc, workspace=ws)
        S.so_partition_batch(ds, idx_t, idx_out, off, pj, out)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(max(args.warmup, 3)):
        step(idx)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    launches0 = S.so_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(idx)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = S.so_launch_count() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps
    # the same steps again with the library's per-kernel CUDA events on the
    # launching stream (kept out of the region above: the event records add
    # about 0.045 ms to a step); the stage times and the roofline's kernel
    # duration come from this pass
    S.so_profile_enable(True)
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(args.steps):
        step(idx)
    ev3.record(stream)
    torch.cuda.synchronize()
    barrier()
    S.so_profile_enable(False)
    ms_traced = ev2.elapsed_time(ev3) / args.steps
    clk = clocks.stop()
    prof = S.so_profile_read()
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n * P / (ms / 1000.0)

    # ---- end to end through the public API, host buffers, copies inside the region.  Every
    # step copies all its inputs from pinned host memory and reads its split record back.
    # Pipelined as a caller streaming batches runs it: two device input sets and a copy stream,
    # step i+1's upload overlapping step i's kernels (the serial figure is reported beside it).
    e2e_steps = 0 if args.no_e2e else max(2, min(args.steps, 10))
    h2d = (Xh.numel() * 4 + yh.numel() + idx_h.numel() * 4 + ptr_h.numel() * 4 + feat_h.numel() * 4
           + sign_h.numel())
    hosts = (Xh, yh, idx_h, ptr_h, feat_h, sign_h)
    sets = [(X, y, idx, ptr, feat, sign), tuple(torch.empty_like(t) for t in (X, y, idx, ptr, feat, sign))]
    dsets = [ds, S.DeviceDataset(sets[1][0], sets[1][1], C)]
    pjs = [pj, S.DeviceProjs(P, sets[1][3], sets[1][4], sets[1][5], int(np.diff(pr.ptr).max()))]
    outs = [out, torch.empty_like(out)]
    outs_h = [out_h, torch.empty_like(out_h).pin_memory()]
    cstream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    released = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(b):
        S.so_split_search_batch(dsets[b], sets[b][2], off, pjs[b], prm, out=outs[b], left_counts=lc, workspace=ws)
        S.so_partition_batch(dsets[b], sets[b][2], idx_out, off, pjs[b], outs[b])

    def upload(b):
        with torch.cuda.stream(cstream):
            cstream.wait_event(released[b])  # the kernels of two steps back are done with set b
            for dst, src in zip(sets[b], hosts):
                dst.copy_(src, non_blocking=True)
            copied[b].record(cstream)

    def e2e_run(pipelined):
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if pipelined:
            upload(0)
            for i in range(e2e_steps):
                b = i % 2
                if i + 1 < e2e_steps:
                    upload(1 - b)
                stream.wait_event(copied[b])
                e2e_step(b)
                released[b].record(stream)
                outs_h[b].copy_(outs[b], non_blocking=True)
            stream.synchronize()
            cstream.synchronize()
        else:
            for _ in range(e2e_steps):
                for dst, src in zip(sets[0], hosts):
                    dst.copy_(src, non_blocking=True)
                e2e_step(0)
                outs_h[0].copy_(outs[0], non_blocking=True)
                stream.synchronize()
        s_ = (time.perf_counter() - t0) / max(e2e_steps, 1) if e2e_steps else float("nan")
        if world > 1:
            t = torch.tensor([s_], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            s_ = float(t.item())
        return s_

    e2e_serial_s = e2e_run(False)
    e2e_s = e2e_run(True)
    if e2e_steps:
        out_h = outs_h[(e2e_steps - 1) % 2]
    else:
        out_h.copy_(out)  # the device-timed steps' split record
    rec = S.SPLIT_DTYPE and np.frombuffer(out_h.numpy().tobytes(), dtype=S.SPLIT_DTYPE)[0]

    # ---- roofline of the dominant kernel (histogram fill)
    hbm, peak_kind = peaks()
    used_feats = np.unique(pr.feat).size
    alg_bytes = used_feats * n * 4 + n * 4 + n * 1  # feature columns + index list + labels, one pass
    k_launches, k_ms = prof.get("k_hist", (0, 0.0))
    k_avg_ms = k_ms / max(k_launches, 1)
    achieved = alg_bytes / (k_avg_ms / 1000.0) / 1e9 if k_avg_ms > 0 else None
    stage_ms = {k: round(v[1] / max(v[0], 1), 4) for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.root_n is None else f"root node of {n} samples (profiling case)",
                   "n": n, "d": d, "n_proj": P, "n_bins": p["n_bins"], "classes": C,
                   "path": "histogram", "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs {X.numel() * 4 / 1e9:.2f} GB > 126 MB L2; no flush needed"},
        "e2e": {"value": (world * n * P / e2e_s) if e2e_steps else None, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(out_h.numel()), "steps": e2e_steps,
                "pipelined": "step i+1's host-to-device copies overlap step i's kernels (two device input sets)",
                "serial_value": (world * n * P / e2e_serial_s) if e2e_steps else None},
        "gpu_launches": int(launches),
        "roofline": roofline_block(achieved, hbm, peak_kind, alg_bytes, k_avg_ms, clk, full_size=args.root_n is None),
        "stage_ms_per_launch": stage_ms,
        "stage_timing": f"a second pass of the {args.steps} steps with per-kernel CUDA events on the launching "
                        f"stream ({ms_traced:.4f} ms per step with the events)",
        "clocks": clk,
        "split": {"proj": int(rec["proj"]), "cand": int(rec["cand"]), "gain": float(rec["gain"]),
                  "n_left": int(rec["n_left"])},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        # the same step with random-width bins, on the resident inputs
        rw = variant_step(S, torch, ds, pj, idx, off, n, P, C, p["n_bins"], args.steps, key=rw_key())
        rw.update(_rw_roofline(pr, n, rw["stage_ms_per_launch"].get("k_hist")))
        line["random_width"] = rw
        line["entropy"] = variant_step(S, torch, ds, pj, idx, off, n, P, C, p["n_bins"], args.steps, criterion=1)
        line["extras"] = extra_legs(S, torch, dev, args.forest_trees, wide_trees=args.wide_trees)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        n_cpu = min(P, 8 * cores)
        v, dt = cpu_baseline(ds_np, pr, n_cpu, cores)
        n_one = 4
        v1, dt1 = cpu_baseline(ds_np, pr, n_one, 1)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"oracle split search (projections divided over {cores} threads) + "
                                          f"partition on all {n} samples, first {n_cpu} of {P} projections "
                                          f"({dt:.1f} s)",
                                "value_1thread": v1,
                                "sample_1thread": f"the same on one thread, first {n_one} of {P} projections "
                                                  f"({dt1:.1f} s)"}
        line["gain_error"] = gain_error(S, torch, ds, ds_np, pr, idx, off)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer leg")
    ap.add_argument("--no-extras", action="store_true", help="skip the frontier, tree and forest legs")
    ap.add_argument("--leg", default=None, choices=["frontier", "tree", "forest", "wide", "trunk", "trunk10m", "rw"],
                    help="run one secondary leg alone and print its JSON")
    ap.add_argument("--forest-trees", type=int, default=2,
                    help="trees of the n=2M, d=256 forest timed in the extras (0 skips)")
    ap.add_argument("--wide-trees", type=int, default=1,
                    help="timed trees of the n=500k, d=4096 wide count-like workload (0 skips)")
    ap.add_argument("--root-n", type=int, default=None,
                    help="profiling case: the root step on a node of this many samples (same recipe); "
                         "the printed line then describes that smaller node")
    ap.add_argument("--wide-n", type=int, default=None,
                    help="profiling case: the wide tree on this many samples (same recipe)")
    ap.add_argument("--batched-only", action="store_true",
                    help="frontier leg: time the batched search only (no node-at-a-time loop)")
    ap.add_argument("--frontier-fixed", default=None, metavar="T,PPC,CHUNK",
                    help="profiling case: frontier leg with this crossover, projections per CTA and chunk "
                         "instead of the autotuner's")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.leg:
        return run_leg(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
