// so_rw.cu -- random-width histogram boundaries (the YDF default that the
// paper's Section 1 footnote names: bin boundaries at random intervals, so
// that bins follow no fixed grid).
//
// One warp per (histogram node, projection), after the min / max pass:
//  1. draws the B-1 splitmix64 outputs of the projection's boundary stream
//     and keeps their top 23 bits;
//  2. sorts them (bitonic, 256 slots in shared memory);
//  3. places t_j = min + ((2u+1) 2^-24) * (max - min), float, two roundings;
//  4. builds the guide of the histogram kernels: for the monotone cell map
//     v -> clamp(floor(fma(v, s, o)), 0, 255) with s = 256 / (max - min) and
//     o = -min * s, cell c stores lo = #{ j : cell(t_j) < c } and the count k
//     of boundaries with cell(t_j) == c (those are t_lo .. t_{lo+k-1}).  A
//     value v in cell c has every boundary of a lower cell below it and every
//     boundary of a higher cell above it, so its bin is lo plus the number of
//     the cell's k boundaries that are <= v.  Boundaries are uniform over the
//     range, so k is 0, 1 or 2 for 92% of cells.
// Projections whose range is zero or tiny against its magnitude (boundaries
// that round onto a few floats) get no guide (s = -1) and are binned by
// binary search; the bin is the same either way.
#include "so_device.cuh"
#include "so_internal.h"

namespace sof {
namespace {

constexpr int kRwWarps = 8;
constexpr float kRwCondLimit = 16384.0f;  // guide only when max(|min|, |max|) <= 2^14 (max - min)

__global__ void __launch_bounds__(kRwWarps * 32) k_rw_bounds(const V4* plan_total, const int32_t* hist_nodes,
                                                            const uint64_t* __restrict__ keys, int32_t P, int32_t B,
                                                            const uint32_t* __restrict__ mm, RwTables rw) {
  __shared__ uint32_t s_u[kRwWarps][kRwRow];
  __shared__ uint8_t s_c[kRwWarps][kRwRow];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t total = plan_total->x * (int64_t)P;
  const int nb = B - 1;
  uint32_t* u = s_u[warp];
  uint8_t* cell = s_c[warp];
  for (int64_t wi = (int64_t)blockIdx.x * kRwWarps + warp; wi < total; wi += (int64_t)gridDim.x * kRwWarps) {
    const int64_t h = wi / P;
    const int p = (int)(wi - h * P);
    const uint64_t s0 = rw_state(keys[hist_nodes[h]], p);
    for (int j = lane; j < kRwRow; j += 32) u[j] = j < nb ? (uint32_t)(sm64_at(s0, j) >> 41) : 0xFFFFFFFFu;
    __syncwarp();
    // bitonic sort, ascending; the padding (all ones) sorts last.  In each
    // step the lane holding i owns the pair (i, i ^ jj) with i < i ^ jj.
    for (int k = 2; k <= kRwRow; k <<= 1) {
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int i = lane; i < kRwRow; i += 32) {
          const int l = i ^ jj;
          if (l > i) {
            const uint32_t x = u[i], y = u[l];
            const bool asc = (i & k) == 0;
            if (asc ? (x > y) : (x < y)) {
              u[i] = y;
              u[l] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    const float mn = key2f(mm[wi * 2]), mx = key2f(mm[wi * 2 + 1]);
    const float w = __fsub_rn(mx, mn);
    float s = __fdiv_rn((float)kRwCells, w);
    float o = __fmul_rn(-mn, s);
    const float M = fmaxf(fabsf(mn), fabsf(mx));
    const bool guided = w > 0.0f && s > 0.0f && isfinite(s) && isfinite(o) && M <= kRwCondLimit * w;
    if (!guided) {
      s = -1.0f;
      o = 0.0f;
    }
    float* trow = rw.t + wi * kRwRow;
    for (int j = lane; j < kRwRow; j += 32) {
      const float t = j < nb ? rw_boundary(u[j], mn, w) : INFINITY;
      trow[j] = t;
      cell[j] = (uint8_t)((guided && j < nb) ? rw_cell(t, s, o) : kRwCells - 1);
    }
    __syncwarp();
    // cells ascend with j (sorted boundaries, monotone map): the first j
    // whose cell is >= c, and the first whose cell is > c
    uint16_t* grow = rw.g + wi * kRwRow;
    for (int c = lane; c < kRwCells; c += 32) {
      int lo = 0, hi = nb;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)cell[mid] < c) lo = mid + 1;
        else hi = mid;
      }
      int up = lo, hi2 = nb;
      while (up < hi2) {
        const int mid = (up + hi2) >> 1;
        if ((int)cell[mid] <= c) up = mid + 1;
        else hi2 = mid;
      }
      grow[c] = guided ? (uint16_t)(lo | ((up - lo) << 8)) : (uint16_t)0;
    }
    if (lane == 0) rw.so[wi] = make_float2(s, o);
    __syncwarp();  // the next iteration rewrites u and cell
  }
}

}  // namespace

cudaError_t launch_rw_bounds(const SearchArgs& a, const V4* plan_total, const int32_t* hist_nodes,
                             const uint32_t* mm, const RwTables& rw, cudaStream_t st) {
  const DeviceInfo& di = device_info();
  ProfScope ps_("k_rw_bounds", st);
  k_rw_bounds<<<di.num_sms * 4, kRwWarps * 32, 0, st>>>(plan_total, hist_nodes, a.bin_keys, a.pv.P, a.B, mm, rw);
  return cudaGetLastError();
}

}  // namespace sof
