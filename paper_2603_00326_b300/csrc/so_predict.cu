// so_predict.cu -- forest inference: every tree routes every sample from its
// root with the projection arithmetic of Section 3 step 1 (float, +0 start,
// ascending features, one rounding per term; left iff the value is below the
// node's threshold) and votes its leaf's class; the prediction is the class
// with most votes, ties to the lowest id.
//
// One thread per sample, trees in order, votes in registers.  Consecutive
// threads are consecutive samples, so a feature read by a warp whose samples
// sit at the same node is one coalesced access of the column-major matrix.
#include <climits>
#include <cstdio>

#include "so_device.cuh"
#include "so_internal.h"

namespace sof {
void set_last_error(const char* msg);

namespace {

constexpr int kPredThreads = 256;
constexpr int kMaxRoute = 1 << 20;  // nodes visited per (sample, tree) before giving up

__global__ void __launch_bounds__(kPredThreads) k_predict(const float* __restrict__ X, int64_t n, int32_t d, int64_t ld,
                                                         so_forest f, int32_t* votes, int32_t* pred,
                                                         int32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cnt[kMaxClasses];
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) cnt[c] = 0;
  for (int t = 0; t < f.n_trees; ++t) {
    const int64_t base = f.tree_off[t];
    const int64_t size = f.tree_off[t + 1] - base;
    int64_t v = 0;
    int steps = 0;
    bool ok = size > 0;
    while (ok) {
      const int64_t g = base + v;
      const int l = f.left[g];
      if (l < 0) break;
      const int r = f.right[g];
      const int k = f.proj_nnz[g];
      if (k < 1 || k > f.cap || l >= size || r < 0 || r >= size || ++steps > kMaxRoute) {
        ok = false;
        break;
      }
      float acc = 0.0f;
      for (int q = 0; q < k; ++q) {
        const int fe = f.feat[g * f.cap + q];
        if (fe < 0 || fe >= d) {
          ok = false;
          break;
        }
        const float x = __ldg(X + (int64_t)fe * ld + i);
        acc = __fadd_rn(acc, f.sign[g * f.cap + q] == 1 ? x : -x);
      }
      if (!ok) break;
      v = (acc < f.threshold[g]) ? l : r;
    }
    if (!ok) {
      atomicOr(err, 1);
      continue;
    }
    const int cls = f.leaf_class[base + v];
#pragma unroll
    for (int c = 0; c < kMaxClasses; ++c) cnt[c] += (cls == c);
  }
  int best = 0;
#pragma unroll
  for (int c = 1; c < kMaxClasses; ++c)
    if (c < f.n_classes && cnt[c] > cnt[best]) best = c;
  pred[i] = best;
  if (votes)
    for (int c = 0; c < f.n_classes; ++c) votes[i * f.n_classes + c] = cnt[c];
}

so_status pfail(so_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

}  // namespace
}  // namespace sof

extern "C" so_status so_predict(const float* X, int64_t n, int32_t d, int64_t ld, const so_forest* forest,
                                int32_t* votes, int32_t* pred, void* stream) {
  using namespace sof;
  if (!forest || !pred) return pfail(SO_EINVAL, "so_predict: forest or pred is NULL");
  if (n < 0 || d < 1 || ld < n) return pfail(SO_EINVAL, "so_predict: bad matrix shape");
  if (n > 0 && !X) return pfail(SO_EINVAL, "so_predict: X is NULL");
  const so_forest& f = *forest;
  if (f.n_trees < 0 || f.n_classes < 1 || f.n_classes > kMaxClasses || f.cap < 1 || f.cap > kMaxCap)
    return pfail(SO_EINVAL, "so_predict: bad forest header");
  if (f.n_trees > 0 && (!f.tree_off || !f.left || !f.right || !f.leaf_class || !f.proj_nnz || !f.feat || !f.sign ||
                        !f.threshold))
    return pfail(SO_EINVAL, "so_predict: a forest array is NULL");
  if (n == 0) return SO_OK;
  cudaStream_t cs = (cudaStream_t)stream;
  int32_t* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, sizeof(int32_t), cs);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), cs);
  if (e == cudaSuccess) {
    ProfScope ps_("k_predict", cs);
    k_predict<<<(unsigned)((n + kPredThreads - 1) / kPredThreads), kPredThreads, 0, cs>>>(X, n, d, ld, f, votes,
                                                                                            pred, err);
    e = cudaGetLastError();
  }
  int32_t herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, cs);
  if (err) {
    const cudaError_t e2 = cudaFreeAsync(err, cs);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) {
    char msg[192];
    snprintf(msg, sizeof(msg), "so_predict: %s", cudaGetErrorString(e));
    return pfail(SO_ECUDA, msg);
  }
  if (herr) return pfail(SO_EINTERNAL, "so_predict: a node has a bad feature, projection length or child id");
  return SO_OK;
}
