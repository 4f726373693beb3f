// so_api.cu -- the C ABI (include/soforest.h): argument validation, the
// internal device arena, and the host orchestration of the batched split
// search, partition, sampling and breadth-first tree growth.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <algorithm>
#include <vector>

#include "so_internal.h"

using namespace sof;

namespace {
thread_local std::string g_err;
}  // namespace

namespace sof {
so_status fail(so_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}
}  // namespace sof

namespace {

#define SO_CK(call)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) return fail(SO_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---- internal arena: one grow-only device buffer per device -----------------
struct Arena {
  std::mutex mu;
  void* ptr = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;
};
std::mutex g_arenas_mu;
std::map<int, Arena*> g_arenas;

Arena& arena_for_current() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_arenas_mu);
  Arena*& a = g_arenas[dev];
  if (!a) a = new Arena();
  return *a;
}

// Holds the arena for one call: later users on any stream wait for the work
// this call enqueued (an event recorded on release).
class ArenaLease {
 public:
  ArenaLease() = default;
  ~ArenaLease() { release(); }
  so_status acquire(size_t bytes, cudaStream_t st) {
    a_ = &arena_for_current();
    a_->mu.lock();
    st_ = st;
    if (!a_->done) {
      if (cudaEventCreateWithFlags(&a_->done, cudaEventDisableTiming) != cudaSuccess) {
        a_->done = nullptr;
        return fail(SO_ECUDA, "cudaEventCreate failed");
      }
      cudaEventRecord(a_->done, st);
    }
    if (a_->cap < bytes) {
      cudaEventSynchronize(a_->done);
      if (a_->ptr) cudaFree(a_->ptr);
      a_->ptr = nullptr;
      a_->cap = 0;
      const size_t want = bytes + bytes / 8 + (1 << 20);
      if (cudaMalloc(&a_->ptr, want) != cudaSuccess) {
        cudaGetLastError();
        a_->ptr = nullptr;
        return fail(SO_ENOMEM, "device allocation of %zu bytes failed", want);
      }
      a_->cap = want;
    }
    cudaStreamWaitEvent(st, a_->done, 0);
    held_ = true;
    return SO_OK;
  }
  void* ptr() const { return a_ ? a_->ptr : nullptr; }
  size_t cap() const { return a_ ? a_->cap : 0; }
  void release() {
    if (held_) {
      cudaEventRecord(a_->done, st_);
      a_->mu.unlock();
      held_ = false;
    }
  }

 private:
  Arena* a_ = nullptr;
  cudaStream_t st_ = nullptr;
  bool held_ = false;
};

}  // namespace

namespace sof {

so_status check_dataset(const so_dataset* ds) {
  if (!ds) return fail(SO_EINVAL, "dataset is NULL");
  if (!ds->X || !ds->y) return fail(SO_EINVAL, "dataset X or y is NULL");
  if (ds->n < 1 || ds->n > INT32_MAX) return fail(SO_EINVAL, "dataset n=%lld out of range", (long long)ds->n);
  if (ds->d < 1) return fail(SO_EINVAL, "dataset d=%d < 1", ds->d);
  if (ds->ld < ds->n) return fail(SO_EINVAL, "dataset ld=%lld < n", (long long)ds->ld);
  if (ds->n_classes < 1 || ds->n_classes > kMaxClasses)
    return fail(SO_EINVAL, "n_classes=%d outside 1..8", ds->n_classes);
  return SO_OK;
}

// keys_given: the caller supplies the random-width node keys through
// p->bin_keys (the tree trainer and the autotuner use keys of their own).
so_status check_params(const so_split_params* p, bool keys_given) {
  if (!p) return fail(SO_EINVAL, "params is NULL");
  if (p->n_bins < 2 || p->n_bins > kMaxBins) return fail(SO_EINVAL, "n_bins=%d outside 2..256", p->n_bins);
  if (p->sort_below < 0 || p->sort_below > kMaxSortBelow)
    return fail(SO_EINVAL, "sort_below=%d outside 0..%d", p->sort_below, kMaxSortBelow);
  if (p->bin_rule != SO_BINS_EQUAL_WIDTH && p->bin_rule != SO_BINS_RANDOM_WIDTH)
    return fail(SO_EINVAL, "bin_rule=%d is neither equal width (0) nor random width (1)", p->bin_rule);
  if (keys_given && p->bin_rule == SO_BINS_RANDOM_WIDTH && !p->bin_keys)
    return fail(SO_EINVAL, "random-width bins need bin_keys");
  if (p->criterion != SO_CRIT_GINI && p->criterion != SO_CRIT_ENTROPY)
    return fail(SO_EINVAL, "criterion=%d is neither Gini (0) nor entropy (1)", p->criterion);
  if (p->proj_per_cta < 0 || p->proj_per_cta > 64)
    return fail(SO_EINVAL, "proj_per_cta=%d outside 0..64", p->proj_per_cta);
  if (p->chunk != 0 && (p->chunk < 512 || p->chunk > 16384))
    return fail(SO_EINVAL, "chunk=%d is neither 0 nor in 512..16384", p->chunk);
  return SO_OK;
}

// The histogram work decomposition a caller (or so_autotune) chose.
void apply_tuning(SearchArgs& a, int32_t proj_per_cta, int32_t chunk) {
  a.tune.staged_pg = proj_per_cta;
  if (chunk > 0) a.tune.chunk = chunk;
}

so_status check_projs(const so_projs* pr) {
  if (!pr) return fail(SO_EINVAL, "projs is NULL");
  if (pr->n_proj < 1 || pr->n_proj > kMaxProj) return fail(SO_EINVAL, "n_proj=%d outside 1..1024", pr->n_proj);
  if (!pr->ptr || !pr->feat || !pr->sign) return fail(SO_EINVAL, "projection arrays are NULL");
  if (pr->max_nnz < 0 || pr->max_nnz > kMaxCap) return fail(SO_EINVAL, "max_nnz=%d outside 0..32", pr->max_nnz);
  return SO_OK;
}

// The float gain's relative error is below (C+6) 2^-24; the re-score window
// must exceed three times that: the double winner then always enters the
// re-score, and every projection holding a double tie of it keeps its float
// maximum within the window.
float effective_eps(float eps, int C) {
  const float floor_eps = 3.5f * (float)(C + 6) * 5.9604645e-8f;
  if (!(eps > 0.0f)) eps = 4e-6f;
  return eps < floor_eps ? floor_eps : eps;
}

DatasetView view_of(const so_dataset* ds) {
  DatasetView v;
  v.X = ds->X;
  v.n = ds->n;
  v.ld = ds->ld;
  v.y = ds->y;
  v.d = ds->d;
  v.C = ds->n_classes;
  v.Xr = ds->Xr;
  return v;
}

int32_t projs_max_nnz(const so_projs* pr) {
  return (pr->max_nnz >= 1 && pr->max_nnz <= kMaxCap) ? pr->max_nnz : kMaxCap;
}

ProjView csr_view(const so_projs* pr) {
  ProjView v;
  v.beg = pr->ptr;
  v.end = pr->ptr + 1;
  v.feat = pr->feat;
  v.sign = pr->sign;
  v.P = pr->n_proj;
  return v;
}

}  // namespace sof

namespace {

size_t search_bytes(int32_t m, int64_t n_total, int32_t P, int32_t C, int32_t B, int32_t T, int32_t hist_only,
                    int32_t bin_rule) {
  Carver cv;
  cv.dry = true;
  SearchScratch s;
  carve_search(cv, s, m, n_total, P, C, B, T, hist_only, bin_rule);
  return cv.used + 256;
}

// A batch of more than one node also reserves a [P][n_total] float buffer:
// its histogram-path nodes are gathered, so the min/max pass keeps their
// projected values for the histogram pass (4 bytes per sample-projection
// instead of a second gather of the feature columns).
size_t batch_vbuf_floats(int32_t m, int64_t n_total, int32_t P) {
  return m > 1 ? (size_t)P * (size_t)n_total : 0;
}

size_t batch_bytes(int32_t m, int64_t n_total, int32_t P, int32_t C, int32_t B, int32_t T, int32_t hist_only,
                   int32_t bin_rule) {
  const size_t vb = batch_vbuf_floats(m, n_total, P);
  return search_bytes(m, n_total, P, C, B, T, hist_only, bin_rule) + (vb ? vb * sizeof(float) + 256 : 0);
}

}  // namespace

namespace sof {
// Sets the thread-local message returned by so_last_error() (for entry points
// defined in other translation units).
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }
}  // namespace sof

extern "C" {

const char* so_last_error(void) { return g_err.c_str(); }

const char* so_version(void) { return "soforest-b300 0.1 (sm_103a)"; }

void so_shutdown(void) {
  noalloc_forget();
  std::lock_guard<std::mutex> lk(g_arenas_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_arenas) {
    Arena* a = kv.second;
    std::lock_guard<std::mutex> al(a->mu);
    cudaSetDevice(kv.first);
    if (a->done) {
      cudaEventSynchronize(a->done);
      cudaEventDestroy(a->done);
      a->done = nullptr;
    }
    if (a->ptr) cudaFree(a->ptr);
    a->ptr = nullptr;
    a->cap = 0;
  }
  cudaSetDevice(cur);
}

size_t so_split_search_ws_bytes(int32_t m, int64_t n_total, int32_t n_proj, int32_t n_classes,
                                const so_split_params* params) {
  if (!params || m < 0 || n_proj < 1 || n_classes < 1) return 0;
  const size_t extra = 4096 + sizeof(so_split) + 64 * (size_t)n_classes;
  return batch_bytes(m, n_total, n_proj, n_classes, params->n_bins, params->sort_below, params->hist_only,
                     params->bin_rule) + extra;
}

so_status so_split_search_batch(const so_dataset* ds, const int32_t* idx, int64_t n_total, const int64_t* node_off,
                                int32_t m, const so_projs* projs, const so_split_params* params, so_split* out_dev,
                                int64_t* left_counts_dev, void* workspace, size_t ws_bytes, void* stream) {
  return guarded([&]() -> so_status {
    so_status st;
    if ((st = check_dataset(ds)) || (st = check_params(params)) || (st = check_projs(projs))) return st;
    if (m < 0) return fail(SO_EINVAL, "m < 0");
    if (m == 0) return SO_OK;
    if (!idx || !node_off || !out_dev) return fail(SO_EINVAL, "idx, node_off or out_dev is NULL");
    if (n_total < 0 || n_total > INT32_MAX) return fail(SO_EINVAL, "n_total out of range");
    cudaStream_t cs = (cudaStream_t)stream;
    const int C = ds->n_classes, P = projs->n_proj;
    const size_t need =
        batch_bytes(m, n_total, P, C, params->n_bins, params->sort_below, params->hist_only, params->bin_rule);
    ArenaLease lease;
    char* base = (char*)workspace;
    size_t cap = ws_bytes;
    if (!workspace) {
      if ((st = lease.acquire(need, cs))) return st;
      base = (char*)lease.ptr();
      cap = lease.cap();
    } else if (ws_bytes < need) {
      return fail(SO_ENOMEM, "workspace of %zu bytes < %zu needed", ws_bytes, need);
    }
    Carver cv;
    cv.base = base;
    cv.cap = cap;
    SearchScratch s;
    carve_search(cv, s, m, n_total, P, C, params->n_bins, params->sort_below, params->hist_only, params->bin_rule);
    const size_t vbf = batch_vbuf_floats(m, n_total, P);
    float* vbuf = vbf ? cv.take<float>(vbf) : nullptr;
    if (!cv.ok()) return fail(SO_ENOMEM, "workspace too small");
    SearchArgs a;
    a.vbuf = vbuf;
    a.ds = view_of(ds);
    a.idx = idx;
    a.n_total = n_total;
    a.node_off = node_off;
    a.m = m;
    a.pv = csr_view(projs);
    a.B = params->n_bins;
    a.T = params->sort_below;
    a.hist_only = params->hist_only ? 1 : 0;
    a.eps = effective_eps(params->rescore_rel_eps, C);
    a.max_nnz = projs_max_nnz(projs);
    a.out = out_dev;
    a.left_counts = left_counts_dev;
    a.bin_rule = params->bin_rule;
    a.bin_keys = params->bin_keys;
    a.criterion = params->criterion;
    apply_tuning(a, params->proj_per_cta, params->chunk);
    SO_CK(launch_search(a, s, cs));
    return SO_OK;
  });
}

so_status so_split_search(const so_dataset* ds, const int32_t* idx, int64_t n_node, const so_projs* projs,
                          const so_split_params* params, so_split* out_host, int64_t* left_counts_host,
                          void* workspace, size_t ws_bytes, void* stream) {
  return guarded([&]() -> so_status {
    so_status st;
    if ((st = check_dataset(ds)) || (st = check_params(params)) || (st = check_projs(projs))) return st;
    if (!out_host) return fail(SO_EINVAL, "out_host is NULL");
    if (n_node < 0 || n_node > INT32_MAX) return fail(SO_EINVAL, "n_node out of range");
    if (n_node > 0 && !idx) return fail(SO_EINVAL, "idx is NULL");
    cudaStream_t cs = (cudaStream_t)stream;
    const int C = ds->n_classes, P = projs->n_proj;
    const size_t need = search_bytes(1, n_node, P, C, params->n_bins, params->sort_below, params->hist_only,
                                     params->bin_rule) +
                        4096 + sizeof(so_split) + 64 * C;
    ArenaLease lease;
    char* base = (char*)workspace;
    size_t cap = ws_bytes;
    if (!workspace) {
      if ((st = lease.acquire(need, cs))) return st;
      base = (char*)lease.ptr();
      cap = lease.cap();
    } else if (ws_bytes < need) {
      return fail(SO_ENOMEM, "workspace of %zu bytes < %zu needed", ws_bytes, need);
    }
    Carver cv;
    cv.base = base;
    cv.cap = cap;
    int64_t* off = cv.take<int64_t>(2);
    so_split* out_dev = cv.take<so_split>(1);
    int64_t* lc = cv.take<int64_t>(kMaxClasses);
    SearchScratch s;
    carve_search(cv, s, 1, n_node, P, C, params->n_bins, params->sort_below, params->hist_only, params->bin_rule);
    if (!cv.ok()) return fail(SO_ENOMEM, "workspace too small");
    SO_CK(launch_fill_off(off, n_node, cs));
    SearchArgs a;
    a.ds = view_of(ds);
    a.idx = idx;
    a.n_total = n_node;
    a.node_off = off;
    a.m = 1;
    a.pv = csr_view(projs);
    a.B = params->n_bins;
    a.T = params->sort_below;
    a.hist_only = params->hist_only ? 1 : 0;
    a.eps = effective_eps(params->rescore_rel_eps, C);
    a.max_nnz = projs_max_nnz(projs);
    a.out = out_dev;
    a.left_counts = lc;
    a.bin_rule = params->bin_rule;
    a.bin_keys = params->bin_keys;
    a.criterion = params->criterion;
    apply_tuning(a, params->proj_per_cta, params->chunk);
    SO_CK(launch_search(a, s, cs));
    int64_t lch[kMaxClasses];
    SO_CK(cudaMemcpyAsync(out_host, out_dev, sizeof(so_split), cudaMemcpyDeviceToHost, cs));
    SO_CK(cudaMemcpyAsync(lch, lc, sizeof(int64_t) * C, cudaMemcpyDeviceToHost, cs));
    SO_CK(cudaStreamSynchronize(cs));
    if (left_counts_host) memcpy(left_counts_host, lch, sizeof(int64_t) * C);
    if (out_host->path == -2) return fail(SO_EINVAL, "a projection row is malformed (length, order, range or sign)");
    return SO_OK;
  });
}

so_status so_partition(const so_dataset* ds, int32_t* idx_inout, int64_t n_node, const int32_t* feat,
                       const int8_t* sign, int32_t nnz, float threshold, int64_t* n_left_out, void* stream) {
  return guarded([&]() -> so_status {
    so_status st;
    if ((st = check_dataset(ds))) return st;
    if (n_node < 0 || n_node > INT32_MAX) return fail(SO_EINVAL, "n_node out of range");
    if (nnz < 1 || nnz > kMaxCap) return fail(SO_EINVAL, "nnz=%d outside 1..32", nnz);
    if (!feat || !sign || !n_left_out) return fail(SO_EINVAL, "NULL argument");
    if (n_node == 0) {
      *n_left_out = 0;
      return SO_OK;
    }
    if (!idx_inout) return fail(SO_EINVAL, "idx is NULL");
    cudaStream_t cs = (cudaStream_t)stream;
    Carver dry;
    dry.dry = true;
    dry.take<int32_t>(n_node);
    dry.take<uint8_t>(n_node);
    dry.take<int64_t>(part_tiles(n_node) + 1);
    dry.take<PartNode>(1);
    dry.take<int64_t>(2);
    dry.take<int64_t>(1);
    dry.take<int32_t>(1);
    ArenaLease lease;
    if ((st = lease.acquire(dry.used + 4096, cs))) return st;
    Carver cv;
    cv.base = (char*)lease.ptr();
    cv.cap = lease.cap();
    int32_t* tmp = cv.take<int32_t>(n_node);
    uint8_t* flags = cv.take<uint8_t>(n_node);
    int64_t* tiles = cv.take<int64_t>(part_tiles(n_node) + 1);
    PartNode* node = cv.take<PartNode>(1);
    int64_t* off = cv.take<int64_t>(2);
    int64_t* ones = cv.take<int64_t>(1);
    int32_t* err = cv.take<int32_t>(1);
    SO_CK(cudaMemsetAsync(err, 0, sizeof(int32_t), cs));
    SO_CK(launch_part_single(n_node, nnz, threshold, node, off, cs));
    PartArgs a;
    a.ds = view_of(ds);
    a.idx_in = idx_inout;
    a.idx_out = tmp;
    a.n = n_node;
    a.node_off = off;
    a.m = 1;
    a.nodes = node;
    a.feat = feat;
    a.sign = sign;
    a.flags = flags;
    a.tile_cnt = tiles;
    a.ones_total = ones;
    a.err = err;
    a.n_out = n_node;
    a.fix_node = node;
    SO_CK(launch_partition(a, cs));
    SO_CK(cudaMemcpyAsync(idx_inout, tmp, sizeof(int32_t) * n_node, cudaMemcpyDeviceToDevice, cs));
    int64_t nl = 0;
    int32_t e = 0;
    SO_CK(cudaMemcpyAsync(&nl, ones, sizeof(int64_t), cudaMemcpyDeviceToHost, cs));
    SO_CK(cudaMemcpyAsync(&e, err, sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
    SO_CK(cudaStreamSynchronize(cs));
    if (e) return fail(SO_EINTERNAL, "partition consistency check failed (code %d)", e);
    *n_left_out = nl;
    return SO_OK;
  });
}

so_status so_partition_batch(const so_dataset* ds, const int32_t* idx_in, int32_t* idx_out, int64_t n_total,
                             const int64_t* node_off, int32_t m, const so_projs* projs, const so_split* splits_dev,
                             void* stream) {
  return guarded([&]() -> so_status {
    so_status st;
    if ((st = check_dataset(ds)) || (st = check_projs(projs))) return st;
    if (m < 0) return fail(SO_EINVAL, "m < 0");
    if (m == 0 || n_total == 0) return SO_OK;
    if (!idx_in || !idx_out || !node_off || !splits_dev) return fail(SO_EINVAL, "NULL argument");
    if (n_total < 0 || n_total > INT32_MAX) return fail(SO_EINVAL, "n_total out of range");
    cudaStream_t cs = (cudaStream_t)stream;
    Carver dry;
    dry.dry = true;
    dry.take<PartNode>(m);
    dry.take<V4>(scan_tiles_for_host(m) + 1);
    dry.take<V4>(1);
    dry.take<uint8_t>(n_total);
    dry.take<int64_t>(part_tiles(n_total) + 1);
    dry.take<int64_t>(1);
    dry.take<int32_t>(1);
    ArenaLease lease;
    if ((st = lease.acquire(dry.used + 4096, cs))) return st;
    Carver cv;
    cv.base = (char*)lease.ptr();
    cv.cap = lease.cap();
    PartNode* nodes = cv.take<PartNode>(m);
    V4* tiles = cv.take<V4>(scan_tiles_for_host(m) + 1);
    V4* total = cv.take<V4>(1);
    uint8_t* flags = cv.take<uint8_t>(n_total);
    int64_t* tcnt = cv.take<int64_t>(part_tiles(n_total) + 1);
    int64_t* ones = cv.take<int64_t>(1);
    int32_t* err = cv.take<int32_t>(1);
    SO_CK(cudaMemsetAsync(err, 0, sizeof(int32_t), cs));
    const ProjView pv = csr_view(projs);
    SO_CK(launch_part_nodes_from_splits(node_off, m, splits_dev, pv, nodes, tiles, total, cs));
    PartArgs a;
    a.ds = view_of(ds);
    a.idx_in = idx_in;
    a.idx_out = idx_out;
    a.n = n_total;
    a.node_off = node_off;
    a.m = m;
    a.nodes = nodes;
    a.feat = projs->feat;
    a.sign = projs->sign;
    a.flags = flags;
    a.tile_cnt = tcnt;
    a.ones_total = ones;
    a.err = err;
    a.n_out = n_total;
    a.fix_node = nullptr;
    SO_CK(launch_partition(a, cs));
    return SO_OK;
  });
}

so_status so_sample_projections(int32_t m, const uint64_t* keys, int32_t n_proj, int32_t d, double lambda,
                                int32_t cap, int32_t* nnz_out, int32_t* feat_out, int8_t* sign_out, void* stream) {
  return guarded([&]() -> so_status {
    if (m < 0 || n_proj < 1 || n_proj > kMaxProj || d < 1) return fail(SO_EINVAL, "bad m, n_proj or d");
    if (cap < 1 || cap > kMaxCap) return fail(SO_EINVAL, "cap=%d outside 1..32", cap);
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(SO_EINVAL, "lambda must be finite and >= 0");
    if (m == 0) return SO_OK;
    if (!keys || !nnz_out || !feat_out || !sign_out) return fail(SO_EINVAL, "NULL argument");
    SO_CK(launch_sample(m, keys, n_proj, d, lambda, cap, nnz_out, feat_out, sign_out, nullptr, nullptr,
                        (cudaStream_t)stream));
    return SO_OK;
  });
}

so_status so_histograms(const so_dataset* ds, const int32_t* idx, int64_t n_total, const int64_t* node_off,
                        int32_t m, const so_projs* projs, const so_split_params* params, float* minmax_dev,
                        int32_t* hist_dev, float* gain32_dev, float* bounds_dev, void* stream) {
  return guarded([&]() -> so_status {
    so_status st;
    if ((st = check_dataset(ds)) || (st = check_projs(projs)) || (st = check_params(params))) return st;
    const int32_t n_bins = params->n_bins, rule = params->bin_rule;
    if (m < 0) return fail(SO_EINVAL, "m < 0");
    if (m == 0) return SO_OK;
    if (!idx || !node_off || !minmax_dev || !hist_dev) return fail(SO_EINVAL, "NULL argument");
    cudaStream_t cs = (cudaStream_t)stream;
    const int C = ds->n_classes, P = projs->n_proj;
    Carver dry;
    dry.dry = true;
    SearchScratch ds0;
    carve_search(dry, ds0, m, n_total, P, C, n_bins, 0, 1, rule);
    dry.take<float>((size_t)m * P * (n_bins - 1));
    ArenaLease lease;
    if ((st = lease.acquire(dry.used + 4096, cs))) return st;
    Carver cv;
    cv.base = (char*)lease.ptr();
    cv.cap = lease.cap();
    SearchScratch s;
    carve_search(cv, s, m, n_total, P, C, n_bins, 0, 1, rule);
    float* gtmp = cv.take<float>((size_t)m * P * (n_bins - 1));
    if (!cv.ok()) return fail(SO_ENOMEM, "arena too small");
    SearchArgs a;
    a.ds = view_of(ds);
    a.idx = idx;
    a.n_total = n_total;
    a.node_off = node_off;
    a.m = m;
    a.pv = csr_view(projs);
    a.B = n_bins;
    a.T = 0;
    a.hist_only = 1;
    a.max_nnz = projs_max_nnz(projs);
    a.minmax_out = minmax_dev;
    a.hist_out = hist_dev;
    a.gain32_out = gain32_dev;
    a.bounds_out = bounds_dev;
    a.bin_rule = rule;
    a.bin_keys = params->bin_keys;
    SO_CK(launch_hist_inspect(a, s, gain32_dev ? gtmp : nullptr, cs));
    return SO_OK;
  });
}

void so_tree_free(so_tree* t) {
  if (!t) return;
  free(t->left); free(t->right); free(t->depth); free(t->leaf_class); free(t->proj_nnz); free(t->feat);
  free(t->cand); free(t->sign); free(t->path); free(t->threshold); free(t->n_samples); free(t->class_counts);
  free(t->gain);
  memset(t, 0, sizeof(*t));
}

so_status so_train_tree(const so_dataset* ds, const int32_t* root_idx, int64_t n_root, const so_tree_params* tp,
                        so_tree* out, void* stream) {
  return guarded([&]() -> so_status {
    so_status st;
    if ((st = check_dataset(ds))) return st;
    if (!tp || !out) return fail(SO_EINVAL, "params or out is NULL");
    memset(out, 0, sizeof(*out));
    if (n_root < 1 || n_root > INT32_MAX / 2) return fail(SO_EINVAL, "n_root out of range");
    if (!root_idx) return fail(SO_EINVAL, "root_idx is NULL");
    so_split_params sp{tp->n_bins,   tp->sort_below, tp->hist_only, tp->rescore_rel_eps,
                       tp->bin_rule, tp->criterion,  nullptr,       tp->proj_per_cta,
                       tp->chunk};
    if ((st = check_params(&sp, false))) return st;
    if (tp->n_proj < 1 || tp->n_proj > kMaxProj) return fail(SO_EINVAL, "n_proj outside 1..1024");
    if (tp->nnz_cap < 1 || tp->nnz_cap > kMaxCap) return fail(SO_EINVAL, "nnz_cap outside 1..32");
    if (!(tp->lambda >= 0.0) || !std::isfinite(tp->lambda)) return fail(SO_EINVAL, "lambda must be >= 0");
    cudaStream_t cs = (cudaStream_t)stream;
    const int C = ds->n_classes, P = tp->n_proj, cap = tp->nnz_cap, B = tp->n_bins;
    const int T = tp->sort_below, HO = tp->hist_only ? 1 : 0;
    const int64_t Mcap = n_root / 2 + 2;
    const int64_t Ncap = 2 * n_root + 1;
    // batch of nodes searched at once: bounded projection slots and histograms
    // sampled slots and the exact path's per-(node, projection) results
    const size_t per_node_proj = (size_t)P * ((size_t)cap * 5 + 12 + sort_res_bytes());
    int64_t Mb = (int64_t)((size_t)512 << 20) / (int64_t)per_node_proj;
    if (HO) {
      const size_t per_hist = (size_t)P * B * C * 4 + (size_t)P * 16;
      Mb = std::min<int64_t>(Mb, (int64_t)(((size_t)1 << 30) / per_hist));
    }
    Mb = std::max<int64_t>(1, std::min<int64_t>(Mb, Mcap));

    // projected values of the histogram-path samples, kept between the two
    // histogram passes of a level (gathered nodes: 8 bytes per
    // sample-projection instead of gathering the feature columns twice)
    const bool use_vbuf = (size_t)P * (size_t)n_root * sizeof(float) <= ((size_t)16 << 30);
    auto layout = [&](Carver& cv, int32_t** idx_a, int32_t** idx_b, Frontier* fa, Frontier* fb, so_split** spl,
                      int64_t** lc, PartNode** pn, V4** tiles, V4** total, uint8_t** flags, int64_t** ptiles,
                      int64_t** ones, int32_t** snnz, int32_t** sbeg, int32_t** send, int32_t** sfeat,
                      int8_t** ssign, TreeDev* td, LevelStats** stats, SearchScratch* ss, float** vbuf) {
      *idx_a = cv.take<int32_t>(n_root);
      *idx_b = cv.take<int32_t>(n_root);
      for (Frontier* f : {fa, fb}) {
        f->off = cv.take<int64_t>(Mcap + 1);
        f->key = cv.take<uint64_t>(Mcap);
        f->id = cv.take<int32_t>(Mcap);
        f->depth = cv.take<int32_t>(Mcap);
        f->counts = cv.take<int32_t>(Mcap * C);
      }
      *spl = cv.take<so_split>(Mcap);
      *lc = cv.take<int64_t>(Mcap * C);
      *pn = cv.take<PartNode>(Mcap);
      *tiles = cv.take<V4>(scan_tiles_for_host(Mcap) + 1);
      *total = cv.take<V4>(1);
      *flags = cv.take<uint8_t>(n_root);
      *ptiles = cv.take<int64_t>(part_tiles(n_root) + 1);
      *ones = cv.take<int64_t>(1);
      *snnz = cv.take<int32_t>(Mb * P);
      *sbeg = cv.take<int32_t>(Mb * P);
      *send = cv.take<int32_t>(Mb * P);
      *sfeat = cv.take<int32_t>(Mb * P * cap);
      *ssign = cv.take<int8_t>(Mb * P * cap);
      td->left = cv.take<int32_t>(Ncap);
      td->right = cv.take<int32_t>(Ncap);
      td->depth = cv.take<int32_t>(Ncap);
      td->leaf_class = cv.take<int32_t>(Ncap);
      td->proj_nnz = cv.take<int32_t>(Ncap);
      td->cand = cv.take<int32_t>(Ncap);
      td->feat = cv.take<int32_t>(Ncap * cap);
      td->sign = cv.take<int8_t>(Ncap * cap);
      td->path = cv.take<int8_t>(Ncap);
      td->threshold = cv.take<float>(Ncap);
      td->n_samples = cv.take<int64_t>(Ncap);
      td->class_counts = cv.take<int64_t>(Ncap * C);
      td->gain = cv.take<double>(Ncap);
      td->cap = cap;
      td->C = C;
      *stats = cv.take<LevelStats>(1);
      carve_search(cv, *ss, (int32_t)Mb, n_root, P, C, B, T, HO, tp->bin_rule);
      *vbuf = use_vbuf ? cv.take<float>((size_t)P * (size_t)n_root) : nullptr;
    };
    int32_t *idx_a, *idx_b, *snnz, *sbeg, *send, *sfeat;
    int8_t* ssign;
    Frontier fa{}, fb{};
    so_split* spl;
    int64_t *lc, *ptiles, *ones;
    PartNode* pn;
    V4 *tiles, *total;
    uint8_t* flags;
    TreeDev td{};
    LevelStats* stats;
    SearchScratch ss;
    float* vbuf = nullptr;
    Carver dry;
    dry.dry = true;
    layout(dry, &idx_a, &idx_b, &fa, &fb, &spl, &lc, &pn, &tiles, &total, &flags, &ptiles, &ones, &snnz, &sbeg,
           &send, &sfeat, &ssign, &td, &stats, &ss, &vbuf);
    ArenaLease lease;
    if ((st = lease.acquire(dry.used + 4096, cs))) return st;
    Carver cv;
    cv.base = (char*)lease.ptr();
    cv.cap = lease.cap();
    layout(cv, &idx_a, &idx_b, &fa, &fb, &spl, &lc, &pn, &tiles, &total, &flags, &ptiles, &ones, &snnz, &sbeg,
           &send, &sfeat, &ssign, &td, &stats, &ss, &vbuf);
    if (!cv.ok()) return fail(SO_ENOMEM, "arena too small");

    const DatasetView dv = view_of(ds);
    const uint64_t kG = 0x9E3779B97F4A7C15ull;
    uint64_t root_key_state = tp->seed ^ ((uint64_t)(int64_t)tp->tree_id * kG);
    // root key: one splitmix64 step from the state above
    uint64_t z = (root_key_state += kG);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    const uint64_t root_key = z ^ (z >> 31);

    SO_CK(cudaMemcpyAsync(idx_a, root_idx, sizeof(int32_t) * n_root, cudaMemcpyDeviceToDevice, cs));
    SO_CK(launch_tree_root(dv, idx_a, n_root, root_key, tp->max_depth, td, fa, stats, cs));
    LevelStats hs{};
    SO_CK(cudaMemcpyAsync(&hs, stats, sizeof(LevelStats), cudaMemcpyDeviceToHost, cs));
    SO_CK(cudaStreamSynchronize(cs));
    if (hs.err & 16) return fail(SO_EINVAL, "root_idx holds a sample index outside [0, n)");
    if (hs.err & 32) return fail(SO_EINVAL, "a label is outside [0, n_classes)");
    int64_t m = hs.m_next, n_level = n_root, n_nodes = 1;
    int64_t max_nv = hs.max_next;  // the current frontier's largest node
    Frontier cur = fa, nxt = fb;
    int32_t *cidx = idx_a, *nidx = idx_b;
    const float eps = effective_eps(tp->rescore_rel_eps, C);
    // Each level's launches (sampling, split search, split records, next
    // frontier, partition, statistics copy) are captured into a CUDA graph on
    // a private stream and launched as one; the executable graph is updated
    // in place from level to level while the launch sequence keeps its shape.
    // With tracing on, the launches go to the stream directly.
    LevelStats* hsp = nullptr;
    SO_CK(cudaMallocHost(&hsp, sizeof(LevelStats)));  // graph memcpy nodes need page-locked memory
    struct LevelResources {
      LevelStats* pinned = nullptr;
      cudaStream_t stream = nullptr;
      cudaGraphExec_t exec = nullptr;
      ~LevelResources() {
        if (exec) cudaGraphExecDestroy(exec);
        if (stream) cudaStreamDestroy(stream);
        if (pinned) cudaFreeHost(pinned);
      }
    } lr;
    lr.pinned = hsp;
    bool use_graph = !profiling_on();
    if (use_graph && cudaStreamCreateWithFlags(&lr.stream, cudaStreamNonBlocking) != cudaSuccess) {
      (void)cudaGetLastError();
      lr.stream = nullptr;
      use_graph = false;
    }
    const cudaStream_t ls = use_graph ? lr.stream : cs;
    while (m > 0) {
      auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int64_t j0 = 0; j0 < m && e == cudaSuccess; j0 += Mb) {
          const int32_t mb = (int32_t)std::min<int64_t>(Mb, m - j0);
          e = launch_sample(mb, cur.key + j0, P, ds->d, tp->lambda, cap, snnz, sfeat, ssign, sbeg, send, ls);
          if (e != cudaSuccess) break;
          SearchArgs a;
          a.ds = dv;
          a.idx = cidx;
          a.n_total = n_level;
          a.node_off = cur.off + j0;
          a.m = mb;
          a.pv = ProjView{sbeg, send, sfeat, ssign, P};
          a.B = B;
          a.T = T;
          a.hist_only = HO;
          a.eps = eps;
          a.max_nnz = cap;
          a.out = spl + j0;
          a.left_counts = lc + j0 * C;
          a.vbuf = vbuf;
          a.bin_rule = tp->bin_rule;
          a.bin_keys = cur.key + j0;  // random-width boundaries from the node keys
          a.criterion = tp->criterion;
          a.rows_trusted = 1;  // sampled by k_sample this level
          a.max_nv_hint = max_nv;
          // most histogram-path nodes of a tree are gathered nodes of a few
          // thousand samples: smaller items balance the SMs better
          apply_tuning(a, tp->proj_per_cta, tp->chunk > 0 ? tp->chunk : 4096);
          e = launch_search(a, ss, ls);
          if (e == cudaSuccess)
            e = launch_tree_record_splits((int32_t)j0, mb, cur, spl, snnz, sfeat, ssign, P, cap, td, ls);
        }
        if (e == cudaSuccess)
          e = launch_tree_level((int32_t)m, cur, nxt, spl, lc, tp->max_depth, n_nodes, td, pn, tiles, total, stats,
                                ls);
        if (e != cudaSuccess) return e;
        PartArgs pa;
        pa.ds = dv;
        pa.idx_in = cidx;
        pa.idx_out = nidx;
        pa.n = n_level;
        pa.node_off = cur.off;
        pa.m = (int32_t)m;
        pa.nodes = pn;
        pa.feat = td.feat;
        pa.sign = td.sign;
        pa.flags = flags;
        pa.tile_cnt = ptiles;
        pa.ones_total = ones;
        pa.err = &stats->err;
        pa.n_out = n_root;
        pa.fix_node = nullptr;
        e = launch_partition(pa, ls);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hsp, stats, sizeof(LevelStats), cudaMemcpyDeviceToHost, ls);
        return e;
      };
      cudaError_t e;
      if (use_graph) {
        e = cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const cudaError_t e1 = enqueue();
          cudaGraph_t g = nullptr;
          const cudaError_t e2 = cudaStreamEndCapture(ls, &g);
          e = e1 != cudaSuccess ? e1 : e2;
          if (e == cudaSuccess && lr.exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(lr.exec, g, &info) != cudaSuccess) {
              (void)cudaGetLastError();
              cudaGraphExecDestroy(lr.exec);
              lr.exec = nullptr;
            }
          }
          if (e == cudaSuccess && !lr.exec) e = cudaGraphInstantiate(&lr.exec, g, 0);
          if (e == cudaSuccess) e = cudaGraphLaunch(lr.exec, ls);
          if (g) cudaGraphDestroy(g);
        }
      } else {
        e = enqueue();
      }
      SO_CK(e);
      SO_CK(cudaStreamSynchronize(ls));
      hs = *hsp;
      if (hs.err) return fail(SO_EINTERNAL, "partition consistency check failed (code %d)", hs.err);
      n_nodes += hs.new_nodes;
      if (n_nodes > Ncap) return fail(SO_EINTERNAL, "node capacity exceeded");
      m = hs.m_next;
      n_level = hs.n_next;
      max_nv = hs.max_next;
      std::swap(cur, nxt);
      std::swap(cidx, nidx);
    }
    // copy the tree out
    so_tree t{};
    t.n_nodes = n_nodes;
    t.n_classes = C;
    t.cap = cap;
    const size_t N = (size_t)n_nodes;
    t.left = (int32_t*)malloc(N * 4);
    t.right = (int32_t*)malloc(N * 4);
    t.depth = (int32_t*)malloc(N * 4);
    t.leaf_class = (int32_t*)malloc(N * 4);
    t.proj_nnz = (int32_t*)malloc(N * 4);
    t.cand = (int32_t*)malloc(N * 4);
    t.feat = (int32_t*)malloc(N * cap * 4);
    t.sign = (int8_t*)malloc(N * cap);
    t.path = (int8_t*)malloc(N);
    t.threshold = (float*)malloc(N * 4);
    t.n_samples = (int64_t*)malloc(N * 8);
    t.class_counts = (int64_t*)malloc(N * C * 8);
    t.gain = (double*)malloc(N * 8);
    if (!t.left || !t.right || !t.depth || !t.leaf_class || !t.proj_nnz || !t.cand || !t.feat || !t.sign ||
        !t.path || !t.threshold || !t.n_samples || !t.class_counts || !t.gain) {
      so_tree_free(&t);
      return fail(SO_ENOMEM, "host allocation of the tree failed");
    }
    struct Cp {
      void* dst;
      const void* src;
      size_t bytes;
    } cps[] = {{t.left, td.left, N * 4},
               {t.right, td.right, N * 4},
               {t.depth, td.depth, N * 4},
               {t.leaf_class, td.leaf_class, N * 4},
               {t.proj_nnz, td.proj_nnz, N * 4},
               {t.cand, td.cand, N * 4},
               {t.feat, td.feat, N * cap * 4},
               {t.sign, td.sign, N * cap},
               {t.path, td.path, N},
               {t.threshold, td.threshold, N * 4},
               {t.n_samples, td.n_samples, N * 8},
               {t.class_counts, td.class_counts, N * C * 8},
               {t.gain, td.gain, N * 8}};
    for (const Cp& c : cps) {
      const cudaError_t e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, cs);
      if (e != cudaSuccess) {
        so_tree_free(&t);
        return fail(SO_ECUDA, "tree copy: %s", cudaGetErrorString(e));
      }
    }
    const cudaError_t e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) {
      so_tree_free(&t);
      return fail(SO_ECUDA, "tree copy: %s", cudaGetErrorString(e));
    }
    *out = t;
    return SO_OK;
  });
}

so_status so_autotune(const so_dataset* ds, int32_t n_proj, double lambda, int32_t nnz_cap,
                      so_split_params* params, int32_t* sizes_host, float* times_ms_host, int32_t* n_sizes_out,
                      void* stream) {
  return guarded([&]() -> so_status {
    so_status st;
    if ((st = check_dataset(ds)) || (st = check_params(params, false))) return st;
    if (n_proj < 1 || n_proj > kMaxProj) return fail(SO_EINVAL, "n_proj outside 1..1024");
    if (nnz_cap < 1 || nnz_cap > kMaxCap) return fail(SO_EINVAL, "nnz_cap outside 1..32");
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return fail(SO_EINVAL, "lambda must be finite and >= 0");
    cudaStream_t cs = (cudaStream_t)stream;
    const int C = ds->n_classes, P = n_proj, cap = nnz_cap, B = params->n_bins;
    static const int kSizes[] = {32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2047};
    const int n_sizes = (int)(sizeof(kSizes) / sizeof(kSizes[0]));
    // nodes per size: enough work to time, bounded by the data
    const int64_t budget = std::min<int64_t>(ds->n, (int64_t)1 << 18);
    // histograms of every node must fit 256 MB in the histogram-only pass
    const int64_t hist_nodes_max =
        std::max<int64_t>(1, ((int64_t)256 << 20) / ((int64_t)P * B * C * 4 + 64));
    auto nodes_for = [&](int s) {
      return (int32_t)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(4096, hist_nodes_max), budget / s));
    };
    int32_t mcap = 1;
    for (int si = 0; si < n_sizes; ++si) mcap = std::max<int32_t>(mcap, nodes_for(kSizes[si]));
    const int64_t ncap = (int64_t)mcap * kSizes[n_sizes - 1] + budget;
    // projected-value buffer of the histogram path, as batched calls use it
    int64_t max_nt = 0;
    for (int si = 0; si < n_sizes; ++si) max_nt = std::max<int64_t>(max_nt, (int64_t)nodes_for(kSizes[si]) * kSizes[si]);
    auto layout = [&](Carver& cv, int32_t** idx, int64_t** off, uint64_t** keys, int32_t** snnz, int32_t** sbeg,
                      int32_t** send, int32_t** sfeat, int8_t** ssign, so_split** out, SearchScratch* ss,
                      float** vbuf) {
      *idx = cv.take<int32_t>(ncap);
      *off = cv.take<int64_t>(mcap + 1);
      *keys = cv.take<uint64_t>(mcap);
      *snnz = cv.take<int32_t>((size_t)mcap * P);
      *sbeg = cv.take<int32_t>((size_t)mcap * P);
      *send = cv.take<int32_t>((size_t)mcap * P);
      *sfeat = cv.take<int32_t>((size_t)mcap * P * cap);
      *ssign = cv.take<int8_t>((size_t)mcap * P * cap);
      *out = cv.take<so_split>(mcap);
      carve_search(cv, *ss, mcap, ncap, P, C, B, kMaxSortBelow, 1, params->bin_rule);  // histogram scratch, every node
      *vbuf = cv.take<float>((size_t)P * (size_t)max_nt);
    };
    int32_t *idx, *snnz, *sbeg, *send, *sfeat;
    int64_t* off;
    uint64_t* keys;
    int8_t* ssign;
    so_split* out;
    SearchScratch ss;
    float* vbuf = nullptr;
    Carver dry;
    dry.dry = true;
    layout(dry, &idx, &off, &keys, &snnz, &sbeg, &send, &sfeat, &ssign, &out, &ss, &vbuf);
    ArenaLease lease;
    if ((st = lease.acquire(dry.used + 4096, cs))) return st;
    Carver cv;
    cv.base = (char*)lease.ptr();
    cv.cap = lease.cap();
    layout(cv, &idx, &off, &keys, &snnz, &sbeg, &send, &sfeat, &ssign, &out, &ss, &vbuf);
    if (!cv.ok()) return fail(SO_ENOMEM, "arena too small");
    cudaEvent_t e0, e1;
    SO_CK(cudaEventCreate(&e0));
    SO_CK(cudaEventCreate(&e1));
    int best = kMaxSortBelow;
    int found = 0;
    for (int si = 0; si < n_sizes; ++si) {
      const int s = kSizes[si];
      const int32_t m = nodes_for(s);
      SO_CK(launch_bench_nodes(m, s, ds->n, 0x5EEDull + (uint64_t)si, idx, off, keys, cs));
      SO_CK(launch_sample(m, keys, P, ds->d, lambda, cap, snnz, sfeat, ssign, sbeg, send, cs));
      float tms[2] = {0.0f, 0.0f};
      for (int path = 0; path < 2; ++path) {
        SearchArgs a;
        a.ds = view_of(ds);
        a.idx = idx;
        a.n_total = (int64_t)m * s;
        a.node_off = off;
        a.m = m;
        a.pv = ProjView{sbeg, send, sfeat, ssign, P};
        a.B = B;
        a.T = path == 0 ? kMaxSortBelow : 0;
        a.hist_only = path == 1 ? 1 : 0;
        a.eps = effective_eps(params->rescore_rel_eps, C);
        a.max_nnz = cap;
        a.out = out;
        a.left_counts = nullptr;
        a.vbuf = m > 1 ? vbuf : nullptr;
        a.bin_rule = params->bin_rule;
        a.bin_keys = keys;
        a.criterion = params->criterion;
        SO_CK(launch_search(a, ss, cs));  // warm-up
        SO_CK(cudaEventRecord(e0, cs));
        const int reps = 3;
        for (int r = 0; r < reps; ++r) SO_CK(launch_search(a, ss, cs));
        SO_CK(cudaEventRecord(e1, cs));
        SO_CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        SO_CK(cudaEventElapsedTime(&ms, e0, e1));
        tms[path] = ms / reps / (float)m;  // per node
      }
      if (sizes_host) sizes_host[si] = s;
      if (times_ms_host) {
        times_ms_host[2 * si] = tms[0];
        times_ms_host[2 * si + 1] = tms[1];
      }
      if (!found && tms[1] <= tms[0]) {
        best = s;
        found = 1;
      }
    }
    // histogram work decomposition: each projections-per-CTA and chunk
    // candidate is timed on two workloads of the histogram path -- one node
    // of up to 2^20 sorted random draws (a bootstrap-like root) and a batch of
    // gathered nodes of 2048 samples (a frontier's mid-size nodes, whose
    // projected values go through the buffer) -- each the better of two
    // timings; the pair with the least sum of times relative to each
    // workload's fastest is kept
    int best_pg = 0, best_chunk = 0;
    {
      const bool rw = params->bin_rule == SO_BINS_RANDOM_WIDTH;
      const int pg_max = staged_supported(ds->d) ? hist_group_size(B, C, rw) : 0;
      struct Cfg {
        int pg, ch;
        float ms[2];
      };
      Cfg cfgs[9];
      int n_cfg = 0;
      for (int pg : {16, 32, 64}) {
        if (pg_max == 0 ? pg != 16 : pg > pg_max) continue;  // general kernels: the chunk alone
        for (int ch : {4096, 8192, 16384}) cfgs[n_cfg++] = Cfg{pg_max == 0 ? 0 : pg, ch, {0.0f, 0.0f}};
      }
      const int32_t nh = (int32_t)std::min<int64_t>(std::min<int64_t>(ds->n, (int64_t)1 << 20), ncap);
      const int32_t sb = (int32_t)std::min<int64_t>(2048, std::max<int64_t>(1, ds->n / 2));
      const int32_t mb = (int32_t)std::max<int64_t>(
          1, std::min<int64_t>(std::min<int64_t>(128, mcap), std::min<int64_t>(max_nt, ncap) / sb));
      for (int wl = 0; wl < 2; ++wl) {
        const int32_t m_w = wl == 0 ? 1 : mb;
        const int32_t s_w = wl == 0 ? nh : sb;
        SO_CK(launch_bench_nodes(m_w, s_w, ds->n, wl == 0 ? 0x5EED7ull : 0x5EED9ull, idx, off, keys, cs));
        SO_CK(launch_sample(m_w, keys, P, ds->d, lambda, cap, snnz, sfeat, ssign, sbeg, send, cs));
        for (int c = 0; c < n_cfg; ++c) {
          SearchArgs a;
          a.ds = view_of(ds);
          a.idx = idx;
          a.n_total = (int64_t)m_w * s_w;
          a.node_off = off;
          a.m = m_w;
          a.pv = ProjView{sbeg, send, sfeat, ssign, P};
          a.B = B;
          a.T = 0;
          a.hist_only = 1;
          a.eps = effective_eps(params->rescore_rel_eps, C);
          a.max_nnz = cap;
          a.out = out;
          a.vbuf = m_w > 1 ? vbuf : nullptr;
          a.bin_rule = params->bin_rule;
          a.bin_keys = keys;
          a.criterion = params->criterion;
          apply_tuning(a, cfgs[c].pg, cfgs[c].ch);
          SO_CK(launch_search(a, ss, cs));  // warm-up
          float best_t = 0.0f;
          for (int rep = 0; rep < 2; ++rep) {
            SO_CK(cudaEventRecord(e0, cs));
            for (int r = 0; r < 3; ++r) SO_CK(launch_search(a, ss, cs));
            SO_CK(cudaEventRecord(e1, cs));
            SO_CK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            SO_CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep == 0 || ms < best_t) best_t = ms;
          }
          cfgs[c].ms[wl] = best_t;
        }
      }
      float lo[2] = {0.0f, 0.0f};
      for (int wl = 0; wl < 2; ++wl)
        for (int c = 0; c < n_cfg; ++c)
          if (c == 0 || cfgs[c].ms[wl] < lo[wl]) lo[wl] = cfgs[c].ms[wl];
      float best_score = 0.0f;
      for (int c = 0; c < n_cfg; ++c) {
        const float score = cfgs[c].ms[0] / std::max(lo[0], 1e-6f) + cfgs[c].ms[1] / std::max(lo[1], 1e-6f);
        if (c == 0 || score < best_score) {
          best_score = score;
          best_pg = cfgs[c].pg;
          best_chunk = cfgs[c].ch;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_sizes_out) *n_sizes_out = n_sizes;
    params->sort_below = best;
    params->proj_per_cta = best_pg;
    params->chunk = best_chunk;
    return SO_OK;
  });
}

}  // extern "C"
