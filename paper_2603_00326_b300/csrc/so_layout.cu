// so_layout.cu -- the optional row-major copy of the feature matrix
// (so_dataset.Xr): Xr[i*d + f] = X[f*ld + i], by 32 x 32 tiles transposed in
// shared memory (coalesced reads along samples, coalesced writes along
// features).
#include <cstdio>

#include "so_internal.h"

namespace sof {
void set_last_error(const char* msg);

namespace {

__global__ void __launch_bounds__(256) k_row_major(const float* __restrict__ X, int64_t n, int32_t d, int64_t ld,
                                                  float* __restrict__ Xr) {
  __shared__ float t[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;  // samples
  const int f0 = blockIdx.y * 32;               // features
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int f = f0 + r;
    const int64_t i = i0 + tx;
    if (f < d && i < n) t[r][tx] = X[(int64_t)f * ld + i];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r;
    const int f = f0 + tx;
    if (f < d && i < n) Xr[i * d + f] = t[tx][r];
  }
}

}  // namespace
}  // namespace sof

extern "C" so_status so_row_major(const float* X, int64_t n, int32_t d, int64_t ld, float* Xr, void* stream) {
  using namespace sof;
  if (!X || !Xr || n < 1 || d < 1 || ld < n) {
    set_last_error("so_row_major: bad arguments");
    return SO_EINVAL;
  }
  if ((n + 31) / 32 > 0x7fffffffLL || (d + 31) / 32 > 65535) {
    set_last_error("so_row_major: matrix too large for one launch");
    return SO_EINVAL;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  {
    ProfScope ps_("k_row_major", cs);
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((d + 31) / 32));
    k_row_major<<<grid, 256, 0, cs>>>(X, n, d, ld, Xr);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "so_row_major: %s", cudaGetErrorString(e));
    set_last_error(msg);
    return SO_ECUDA;
  }
  return SO_OK;
}
