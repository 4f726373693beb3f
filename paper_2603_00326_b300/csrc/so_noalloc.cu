// so_noalloc.cu -- so_split_search_noalloc: the single-node split search with
// its device scratch in a fixed, statically allocated array, for callers that
// must not allocate device memory.
//
// The scratch is a file-scope __device__ array of kNoallocScratchBytes.  In
// host code its name only stands in for the symbol; the device address is
// obtained once per device with cudaGetSymbolAddress (on the first call made
// with that device current) and cached until so_shutdown.  Every call on a
// device shares the array: nothing is assumed to be zero (the search kernels
// initialise every scratch word they read), and calls that overlap on the GPU
// race on it.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "so_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = size_t(8) << 20;  // 8 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {nullptr};

}  // namespace

namespace sof {
void noalloc_forget() {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  for (int i = 0; i < kMaxDevices; ++i) g_noalloc_addr[i] = nullptr;
}
}  // namespace sof

extern "C" so_status so_split_search_noalloc(const so_dataset* ds, const int32_t* idx, int64_t n_node,
                                             const so_projs* projs, const so_split_params* params,
                                             so_split* out_host, int64_t* left_counts_host, void* stream) {
  using namespace sof;
  return guarded([&]() -> so_status {
    // the same argument checks as so_split_search
    so_status st;
    if ((st = check_dataset(ds)) || (st = check_params(params)) || (st = check_projs(projs))) return st;
    if (!out_host) return fail(SO_EINVAL, "so_split_search_noalloc: out_host is NULL");
    if (n_node < 0 || n_node > INT32_MAX) return fail(SO_EINVAL, "so_split_search_noalloc: n_node out of range");
    if (n_node > 0 && !idx) return fail(SO_EINVAL, "so_split_search_noalloc: idx is NULL");
    const int C = ds->n_classes, P = projs->n_proj;
    cudaStream_t cs = (cudaStream_t)stream;

    // size of the scratch this node needs (a dry carve, no memory touched)
    Carver dry;
    dry.dry = true;
    dry.take<int64_t>(2);
    dry.take<so_split>(1);
    dry.take<int64_t>(kMaxClasses);
    SearchScratch s0;
    carve_search(dry, s0, 1, n_node, P, C, params->n_bins, params->sort_below, params->hist_only,
                 params->bin_rule);
    if (dry.used > kNoallocScratchBytes)
      return fail(SO_EINVAL,
                  "so_split_search_noalloc: this node needs %zu bytes of scratch, above the %zu-byte static "
                  "maximum (fewer projections, bins or classes fit)",
                  dry.used, kNoallocScratchBytes);

    // device address of the static scratch, looked up once per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
      return fail(SO_ECUDA, "so_split_search_noalloc: no current CUDA device");
    void* base = nullptr;
    {
      std::lock_guard<std::mutex> lk(g_noalloc_mu);
      if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
          return fail(SO_ECUDA, "so_split_search_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
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
    if (!cv.ok()) return fail(SO_EINTERNAL, "so_split_search_noalloc: scratch layout overflow");

    // the same search arguments as so_split_search
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

    cudaError_t e = launch_fill_off(off, n_node, cs);
    if (e == cudaSuccess) e = launch_search(a, s, cs);
    int64_t lch[kMaxClasses];
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, out_dev, sizeof(so_split), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lch, lc, sizeof(int64_t) * C, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return fail(SO_ECUDA, "so_split_search_noalloc: %s", cudaGetErrorString(e));
    if (left_counts_host) memcpy(left_counts_host, lch, sizeof(int64_t) * C);
    if (out_host->path == -2) return fail(SO_EINVAL, "so_split_search_noalloc: a projection row is malformed");
    return SO_OK;
  });
}
