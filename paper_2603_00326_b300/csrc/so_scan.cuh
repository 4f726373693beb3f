// so_scan.cuh -- generic three-phase exclusive scan of 4-lane int64 vectors
// (tile reduce -> scan of tile sums in one block -> tile scan + apply).
// A functor F supplies `V4 value(int64_t i)` and `void apply(int64_t i, V4 excl)`.
// Used for node-level bookkeeping (path plan, next frontier), where element
// counts are known on the host and kept modest.
#pragma once

#include "so_internal.h"

namespace sof {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 2;
constexpr int kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ V4 v4add(const V4& a, const V4& b) {
  return V4{a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w};
}
__device__ __forceinline__ V4 v4zero() { return V4{0, 0, 0, 0}; }
__device__ __forceinline__ V4 v4shfl_up(const V4& v, int o) {
  return V4{__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o),
            __shfl_up_sync(0xffffffffu, v.z, o), __shfl_up_sync(0xffffffffu, v.w, o)};
}

// Exclusive block scan of one V4 per thread (NT threads); returns the
// exclusive prefix and writes the block total into *total (all threads see it
// after return).
template <int NT = kScanThreads>
__device__ __forceinline__ V4 block_excl_scan(V4 v, V4* total) {
  __shared__ V4 warp_tot[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V4 inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V4 u = v4shfl_up(inc, o);
    if (lane >= o) inc = v4add(inc, u);
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    V4 w = (lane < NT / 32) ? warp_tot[lane] : v4zero();
    V4 wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const V4 u = v4shfl_up(wi, o);
      if (lane >= o) wi = v4add(wi, u);
    }
    if (lane < NT / 32) warp_tot[lane] = V4{wi.x - w.x, wi.y - w.y, wi.z - w.z, wi.w - w.w};
    if (lane == NT / 32 - 1) *total = wi;
  }
  __syncthreads();
  const V4 wp = warp_tot[warp];
  const V4 ex = V4{inc.x - v.x, inc.y - v.y, inc.z - v.z, inc.w - v.w};
  const V4 r = v4add(wp, ex);
  __syncthreads();
  return r;
}

template <class F>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(F f, int64_t n, V4* tiles) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  V4 acc = v4zero();
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t i = base + k;
    if (i < n) acc = v4add(acc, f.value(i));
  }
  __shared__ V4 tot;
  block_excl_scan(acc, &tot);
  if (threadIdx.x == 0) tiles[blockIdx.x] = tot;
}

// One block: exclusive scan of the tile sums in place; total to *total.
template <class Fin>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(V4* tiles, int64_t n_tiles, V4* total, Fin fin) {
  __shared__ V4 tot;
  V4 carry = v4zero();
  for (int64_t base = 0; base < n_tiles; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    const V4 v = (i < n_tiles) ? tiles[i] : v4zero();
    const V4 ex = block_excl_scan(v, &tot);
    if (i < n_tiles) tiles[i] = v4add(carry, ex);
    carry = v4add(carry, tot);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (total) *total = carry;
    fin(carry);
  }
}

template <class F>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(F f, int64_t n, const V4* tiles) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  V4 vals[kScanPer];
  V4 acc = v4zero();
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t i = base + k;
    vals[k] = (i < n) ? f.value(i) : v4zero();
    acc = v4add(acc, vals[k]);
  }
  __shared__ V4 tot;
  V4 run = v4add(tiles[blockIdx.x], block_excl_scan(acc, &tot));
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    const int64_t i = base + k;
    if (i < n) f.apply(i, run);
    run = v4add(run, vals[k]);
  }
}

// Small scans in one launch: one block of kScanSingleThreads threads, one
// element per thread (a tree level's three launches of the general form cost
// more than that).
constexpr int kScanSingleThreads = 1024;
constexpr int64_t kScanSingleMax = kScanSingleThreads;

// A scan's optional last step, given the grand total (after every apply).
struct NoFinish {
  __device__ void operator()(const V4&) const {}
};

template <class F, class Fin>
__global__ void __launch_bounds__(kScanSingleThreads) k_scan_single(F f, int64_t n, V4* total, Fin fin) {
  __shared__ V4 tot;
  const int64_t i = threadIdx.x;
  const V4 v = (i < n) ? f.value(i) : v4zero();
  const V4 ex = block_excl_scan<kScanSingleThreads>(v, &tot);
  if (i < n) f.apply(i, ex);
  if (threadIdx.x == 0) {
    if (total) *total = tot;
    fin(tot);
  }
}

// Runs the scan over n elements (n known on the host).  `tiles` needs
// ceil(n / kScanTile) entries; the grand total goes to *total (device).
// fin(total) runs once the total is known; in the three-launch form that is
// before the apply launch, so fin must not read what apply writes.
template <class F, class Fin = NoFinish>
cudaError_t run_scan(const F& f, int64_t n, V4* tiles, V4* total, cudaStream_t st,
                     const char* name = "scan", Fin fin = Fin()) {
  if (n <= kScanSingleMax) {
    ProfScope ps_(name, st, 1);
    k_scan_single<F, Fin><<<1, kScanSingleThreads, 0, st>>>(f, n, total, fin);
    return cudaGetLastError();
  }
  const int64_t n_tiles = (n + kScanTile - 1) / kScanTile;
  ProfScope ps_(name, st, n_tiles > 0 ? 3 : 1);
  if (n_tiles > 0) {
    k_scan_reduce<F><<<(unsigned)n_tiles, kScanThreads, 0, st>>>(f, n, tiles);
  }
  k_scan_tiles<Fin><<<1, kScanThreads, 0, st>>>(tiles, n_tiles, total, fin);
  if (n_tiles > 0) {
    k_scan_apply<F><<<(unsigned)n_tiles, kScanThreads, 0, st>>>(f, n, tiles);
  }
  return cudaGetLastError();
}

inline int64_t scan_tiles_for(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

}  // namespace sof
