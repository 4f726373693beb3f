// so_noalloc.cu -- so_split_search_noalloc: the single-node split search with
// its device scratch in a fixed, statically allocated array, for callers that
// must not allocate device memory.
//
// The scratch is a file-scope __device__ array of kNoallocScratchBytes.  In
// host code its name only stands in for the symbol; the device address is
// obtained once per device with cudaGetSymbolAddress (on the first call made
// with that device current) and cached.  Every call on a device shares the
// array: nothing is assumed to be zero (the search kernels initialise every
// scratch word they read), and calls that overlap on the GPU race on it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "so_internal.h"

namespace sof {
void set_last_error(const char* msg);
}

namespace {

constexpr size_t kNoallocScratchBytes = size_t(8) << 20;  // 8 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {nullptr};

so_status noalloc_fail(so_status st, const char* msg) {
  sof::set_last_error(msg);
  return st;
}

}  // namespace

extern "C" so_status so_split_search_noalloc(const so_dataset* ds, const int32_t* idx, int64_t n_node,
                                             const so_projs* projs, const so_split_params* params,
                                             so_split* out_host, int64_t* left_counts_host, void* stream) {
  using namespace sof;
  char msg[256];
  if (!ds || !ds->X || !ds->y || ds->n < 1 || ds->n > INT32_MAX || ds->d < 1 || ds->ld < ds->n ||
      ds->n_classes < 1 || ds->n_classes > kMaxClasses)
    return noalloc_fail(SO_EINVAL, "so_split_search_noalloc: bad dataset");
  if (!params || params->n_bins < 2 || params->n_bins > kMaxBins || params->sort_below < 0 ||
      params->sort_below > kMaxSortBelow ||
      (params->bin_rule != SO_BINS_EQUAL_WIDTH && params->bin_rule != SO_BINS_RANDOM_WIDTH) ||
      (params->bin_rule == SO_BINS_RANDOM_WIDTH && !params->bin_keys) ||
      (params->criterion != SO_CRIT_GINI && params->criterion != SO_CRIT_ENTROPY) || params->proj_per_cta < 0 ||
      params->proj_per_cta > 64 || (params->chunk != 0 && (params->chunk < 512 || params->chunk > 16384)))
    return noalloc_fail(SO_EINVAL, "so_split_search_noalloc: bad split parameters");
  if (!projs || projs->n_proj < 1 || projs->n_proj > kMaxProj || !projs->ptr || !projs->feat || !projs->sign ||
      projs->max_nnz < 0 || projs->max_nnz > kMaxCap)
    return noalloc_fail(SO_EINVAL, "so_split_search_noalloc: bad projections");
  if (!out_host || n_node < 0 || n_node > INT32_MAX || (n_node > 0 && !idx))
    return noalloc_fail(SO_EINVAL, "so_split_search_noalloc: bad node arguments");
  const int C = ds->n_classes, P = projs->n_proj;
  cudaStream_t cs = (cudaStream_t)stream;

  // size of the scratch this node needs (a dry carve, no memory touched)
  Carver dry;
  dry.dry = true;
  dry.take<int64_t>(2);
  dry.take<so_split>(1);
  dry.take<int64_t>(kMaxClasses);
  SearchScratch s0;
  carve_search(dry, s0, 1, n_node, P, C, params->n_bins, params->sort_below, params->hist_only, params->bin_rule);
  if (dry.used > kNoallocScratchBytes) {
    snprintf(msg, sizeof(msg),
             "so_split_search_noalloc: this node needs %zu bytes of scratch, above the %zu-byte static "
             "maximum (fewer projections, bins or classes fit)",
             dry.used, kNoallocScratchBytes);
    return noalloc_fail(SO_EINVAL, msg);
  }

  // device address of the static scratch, looked up once per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(SO_ECUDA, "so_split_search_noalloc: no current CUDA device");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        snprintf(msg, sizeof(msg), "so_split_search_noalloc: cudaGetSymbolAddress failed: %s",
                 cudaGetErrorString(e));
        return noalloc_fail(SO_ECUDA, msg);
      }
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }

  Carver cv;
  cv.base = static_cast<char*>(base);
  cv.cap = kNoallocScratchBytes;
  int64_t* off = cv.take<int64_t>(2);
  so_split* out_dev = cv.take<so_split>(1);
  int64_t* lc = cv.take<int64_t>(kMaxClasses);
  SearchScratch s;
  carve_search(cv, s, 1, n_node, P, C, params->n_bins, params->sort_below, params->hist_only, params->bin_rule);
  if (!cv.ok()) return noalloc_fail(SO_EINTERNAL, "so_split_search_noalloc: scratch layout overflow");

  SearchArgs a;
  a.ds.X = ds->X;
  a.ds.n = ds->n;
  a.ds.ld = ds->ld;
  a.ds.y = ds->y;
  a.ds.d = ds->d;
  a.ds.C = C;
  a.ds.Xr = ds->Xr;
  a.idx = idx;
  a.n_total = n_node;
  a.node_off = off;
  a.m = 1;
  a.pv.beg = projs->ptr;
  a.pv.end = projs->ptr + 1;
  a.pv.feat = projs->feat;
  a.pv.sign = projs->sign;
  a.pv.P = P;
  a.B = params->n_bins;
  a.T = params->sort_below;
  a.hist_only = params->hist_only ? 1 : 0;
  {
    // same re-score window rule as the allocating entry points
    const float floor_eps = 3.5f * (float)(C + 6) * 5.9604645e-8f;
    float eps = params->rescore_rel_eps > 0.0f ? params->rescore_rel_eps : 4e-6f;
    a.eps = eps < floor_eps ? floor_eps : eps;
  }
  a.max_nnz = (projs->max_nnz >= 1) ? projs->max_nnz : kMaxCap;
  a.out = out_dev;
  a.left_counts = lc;
  a.bin_rule = params->bin_rule;
  a.bin_keys = params->bin_keys;
  a.criterion = params->criterion;
  a.tune.staged_pg = params->proj_per_cta;
  if (params->chunk > 0) a.tune.chunk = params->chunk;

  cudaError_t e = launch_fill_off(off, n_node, cs);
  if (e == cudaSuccess) e = launch_search(a, s, cs);
  int64_t lch[kMaxClasses];
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, out_dev, sizeof(so_split), cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(lch, lc, sizeof(int64_t) * C, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "so_split_search_noalloc: %s", cudaGetErrorString(e));
    return noalloc_fail(SO_ECUDA, msg);
  }
  if (left_counts_host) memcpy(left_counts_host, lch, sizeof(int64_t) * C);
  if (out_host->path == -2)
    return noalloc_fail(SO_EINVAL, "so_split_search_noalloc: a projection row is malformed");
  return SO_OK;
}
