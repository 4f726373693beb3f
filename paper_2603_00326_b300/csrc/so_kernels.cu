// so_kernels.cu -- CUDA kernels (sm_103a) of the sparse-oblique split search.
//
// One batched pass over a frontier of m nodes:
//   plan        node -> path (exact sort below T, histogram otherwise;
//               Section 3.1), histogram work items (node, sample chunk,
//               projection group)
//   k_minmax    per (node, projection): projected values (Section 3 step 1)
//               reduced to min / max
//   k_hist      per (node, projection): equal-width bins, class counts in
//               shared memory, flushed with integer atomics (Section 3 step 2;
//               the paper's first GPU kernel, Section 3.3)
//   k_gini_scan per (node, projection): prefix counts over bins, float Gini
//               gain of every boundary, the projection's best (Section 3 step 3)
//   k_hist_select per node: double re-score of the float near-ties, the
//               lexicographic best (the paper's second GPU kernel)
//   (features up to 65536: the staged-tile kernels of so_hist_staged.cu
//   take the place of k_minmax and k_hist; exact path for small nodes:
//   so_sort_warp.cu)
// plus the device sampler (Appendix A), the stable partition, and the
// breadth-first frontier bookkeeping of tree growth.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <climits>
#include <cstdio>

#include "so_device.cuh"
#include "so_internal.h"
#include "so_scan.cuh"

namespace sof {

// ============================================================================
// Device info
// ============================================================================
const DeviceInfo& device_info() {
  static thread_local DeviceInfo info;
  static thread_local int cached = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (cached != dev) {
    info.device = dev;
    int sms = 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) info.num_sms = sms;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && optin > 0)
      info.smem_optin = optin;
    cached = dev;
  }
  return info;
}

// ============================================================================
// Projection-row validation (CSR inputs) and row loading
// ============================================================================
// Rows must hold 1..32 distinct ascending features in [0, d) with +-1 signs.
// A node with a bad row is marked and skipped (path -2); kernels additionally
// clamp what they load so that a bad row can never address outside X.
__global__ void k_validate_rows(ProjView pv, int32_t m, int32_t d, int32_t max_nnz, int32_t* bad_node) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)m * pv.P) return;
  const int32_t b = pv.beg[q], e = pv.end[q];
  bool ok = (e - b >= 1) && (e - b <= max_nnz) && b >= 0;
  if (ok) {
    int prev = -1;
    for (int i = b; i < e; ++i) {
      const int f = pv.feat[i];
      const int s = pv.sign[i];
      if (f <= prev || f >= d || (s != 1 && s != -1)) { ok = false; break; }
      prev = f;
    }
  }
  if (!ok) atomicOr(&bad_node[q / pv.P], 1);
}

// Loads row q into per-warp shared arrays (lanes < k); returns k (clamped).
__device__ __forceinline__ int load_row(const ProjView& pv, int64_t q, int d, int32_t* sf, int8_t* ss,
                                        int lane) {
  const int rb = pv.beg[q];
  int k = pv.end[q] - rb;
  k = k < 0 ? 0 : (k > kMaxCap ? kMaxCap : k);
  if (lane < k) {
    int f = pv.feat[rb + lane];
    f = (f < 0 || f >= d) ? 0 : f;
    sf[lane] = f;
    ss[lane] = pv.sign[rb + lane];
  }
  __syncwarp();
  return k;
}

// ============================================================================
// Plan: path per node and histogram work items
// ============================================================================
struct PlanF {
  const int64_t* off;
  int64_t n_total;
  const int32_t* bad;
  int32_t T, hist_only, force_hist, C;
  int64_t S;
  int32_t G;
  int32_t* hist_nodes;
  int32_t* tiny_nodes;
  int32_t* med_nodes;
  int64_t* item_off;
  so_split* out;
  int64_t* left_counts;

  // kind: 0 histogram, 1 exact path, one warp in registers (<= kSortRegMax
  // samples), 2 exact path, one CTA in shared memory (up to T-1 samples), 3 skip
  // a node whose rows are malformed or whose segment leaves [0, n_total) is skipped
  __device__ bool is_bad(int64_t j) const {
    const int64_t b = off[j], e = off[j + 1];
    return (bad && bad[j]) || b < 0 || e < b || e > n_total;
  }
  __device__ int kind(int64_t j, int64_t nv) const {
    if (is_bad(j)) return 3;
    if (force_hist) return nv >= 1 ? 0 : 3;
    if (nv < 2) return 3;
    if (!hist_only && nv < T) return nv <= kSortRegMax ? 1 : 2;
    return 0;
  }
  __device__ V4 value(int64_t j) const {
    const int64_t nv = is_bad(j) ? 0 : off[j + 1] - off[j];
    const int k = kind(j, nv);
    const long long items = (k == 0) ? ((nv + S - 1) / S) * G : 0;
    return V4{k == 0, k == 1, items, k == 2};
  }
  __device__ void apply(int64_t j, V4 ex) const {
    const int64_t nv = is_bad(j) ? 0 : off[j + 1] - off[j];
    const int k = kind(j, nv);
    if (k == 0) {
      hist_nodes[ex.x] = (int32_t)j;
      item_off[ex.x] = ex.z;
    } else if (k == 1) {
      tiny_nodes[ex.y] = (int32_t)j;
    } else if (k == 2) {
      med_nodes[ex.w] = (int32_t)j;
    } else if (out) {
      so_split r;
      r.valid = 0;
      r.proj = -1;
      r.cand = -1;
      r.path = is_bad(j) ? -2 : ((!hist_only && nv < T) ? 1 : 0);
      r.threshold = 0.0f;
      r.gain = 0.0;
      r.n_left = 0;
      r.n_right = 0;
      out[j] = r;
      if (left_counts)
        for (int c = 0; c < C; ++c) left_counts[j * C + c] = 0;
    }
  }
};

// ============================================================================
// Histogram scratch initialisation (sized by the device-resident count)
// ============================================================================
__global__ void k_hist_init(const V4* plan_total, int32_t P, int32_t BC, uint32_t* mm, int32_t* hist,
                            float* max32) {
  const int64_t mh = plan_total->x;
  const int64_t n_mm = mh * P;
  const int64_t n_h = mh * P * BC;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n_mm; i += stride) {
    mm[2 * i] = 0xFFFFFFFFu;
    mm[2 * i + 1] = 0u;
    max32[i] = -1.0f;
  }
  int4* h4 = reinterpret_cast<int4*>(hist);
  const int64_t n4 = n_h / 4;
  for (int64_t i = tid; i < n4; i += stride) h4[i] = make_int4(0, 0, 0, 0);
  for (int64_t i = n4 * 4 + tid; i < n_h; i += stride) hist[i] = 0;
}

__device__ __forceinline__ int64_t find_item_node(const int64_t* item_off, int64_t m_hist, int64_t t) {
  int64_t lo = 0, hi = m_hist - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (item_off[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ============================================================================
// K1: min / max of every (histogram node, projection)
// ============================================================================
template <int PG>
__global__ void __launch_bounds__(PG * 32) k_minmax(DatasetView ds, const int32_t* __restrict__ idx,
                                                   const int64_t* __restrict__ off, ProjView pv,
                                                   const V4* plan_total, const int32_t* hist_nodes,
                                                   const int64_t* item_off, int64_t S, uint32_t* mm) {
  __shared__ int32_t s_f[PG][kMaxCap];
  __shared__ int8_t s_s[PG][kMaxCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m_hist = plan_total->x, n_items = plan_total->z;
  const int P = pv.P;
  const int G = (P + PG - 1) / PG;
  for (int64_t t = blockIdx.x; t < n_items; t += gridDim.x) {
    const int64_t h = find_item_node(item_off, m_hist, t);
    const int j = hist_nodes[h];
    const int64_t local = t - item_off[h];
    const int64_t chunk = local / G;
    const int g = (int)(local - chunk * G);
    const int p = g * PG + warp;
    if (p >= P) continue;
    const int64_t nb = off[j], ne = off[j + 1];
    const int64_t beg = nb + chunk * S;
    const int64_t end = min(ne, beg + S);
    __syncwarp();
    const int k = load_row(pv, (int64_t)j * P + p, ds.d, s_f[warp], s_s[warp], lane);
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t e = beg + lane; e < end; e += 32) {
      const float v = project_value(ds.X, ds.ld, safe_sample(idx[e], ds.n), s_f[warp], s_s[warp], k);
      mn = fminf(mn, v);
      mx = fmaxf(mx, v);
    }
    mn = warp_min(mn);
    mx = warp_max(mx);
    if (lane == 0 && end > beg) {
      atomicMin(&mm[(h * P + p) * 2], f2key(mn));
      atomicMax(&mm[(h * P + p) * 2 + 1], f2key(mx));
    }
  }
}

// ============================================================================
// K2: class-count histograms, privatised per work item in shared memory
// ============================================================================
template <int PG>
__global__ void __launch_bounds__(PG * 32) k_hist(DatasetView ds, const int32_t* __restrict__ idx,
                                                 const int64_t* __restrict__ off, ProjView pv,
                                                 const V4* plan_total, const int32_t* hist_nodes,
                                                 const int64_t* item_off, int64_t S, int B,
                                                 const uint32_t* __restrict__ mm, int32_t* hist,
                                                 const float* __restrict__ rw_t) {
  extern __shared__ int32_t s_hist[];  // [PG][B*C]
  __shared__ int32_t s_f[PG][kMaxCap];
  __shared__ int8_t s_s[PG][kMaxCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = ds.C;
  const int BC = B * C;
  const int64_t m_hist = plan_total->x, n_items = plan_total->z;
  const int P = pv.P;
  const int G = (P + PG - 1) / PG;
  for (int64_t t = blockIdx.x; t < n_items; t += gridDim.x) {
    const int64_t h = find_item_node(item_off, m_hist, t);
    const int j = hist_nodes[h];
    const int64_t local = t - item_off[h];
    const int64_t chunk = local / G;
    const int g = (int)(local - chunk * G);
    const int p = g * PG + warp;
    const int64_t nb = off[j], ne = off[j + 1];
    const int64_t beg = nb + chunk * S;
    const int64_t end = min(ne, beg + S);
    __syncthreads();  // previous item's flush has finished reading s_hist
    for (int e = threadIdx.x; e < PG * BC; e += blockDim.x) s_hist[e] = 0;
    int k = 0;
    float mn = 0.f, w = 0.f, inv_w = 0.f;
    if (p < P) {
      k = load_row(pv, (int64_t)j * P + p, ds.d, s_f[warp], s_s[warp], lane);
      mn = key2f(mm[(h * P + p) * 2]);
      const float mx = key2f(mm[(h * P + p) * 2 + 1]);
      w = bin_width(mn, mx, B);
      inv_w = __fdiv_rn((float)B, __fsub_rn(mx, mn));
    }
    __syncthreads();
    if (p < P) {
      int32_t* hp = s_hist + warp * BC;
      for (int64_t e = beg + lane; e < end; e += 32) {
        const int64_t s = safe_sample(idx[e], ds.n);
        const int yv = ds.y[s];
        const float v = project_value(ds.X, ds.ld, s, s_f[warp], s_s[warp], k);
        // random width: binary search of the projection's sorted boundaries
        const int b = rw_t ? bin_search(rw_t + (h * P + p) * kRwRow, B - 1, v) : bin_of(v, mn, w, inv_w, B);
        if (yv < C) atomicAdd(&hp[b * C + yv], 1);  // labels >= C are not counted
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < PG * BC; e += blockDim.x) {
      const int wv = e / BC;
      const int pp = g * PG + wv;
      const int32_t c = s_hist[e];
      if (pp < P && c) atomicAdd(&hist[((int64_t)h * P + pp) * BC + (e - wv * BC)], c);
    }
  }
}

// ============================================================================
// K4a: Gini scan over the bins of every (histogram node, projection)
// ============================================================================
// One warp per (node, projection).  The warp walks the bins in rounds of 32
// consecutive bins, lane l taking bin 32 r + l, so that each load of a round
// reads one contiguous run of counters; a warp scan per class and round
// gives the left counts (bins <= b) of candidate b.
struct BinWalk {
  int N[kMaxClasses];      // node class counts
  long long n;
  int carry[kMaxClasses];  // left counts before the current round
};

__device__ __forceinline__ void walk_init(const int32_t* __restrict__ H, int B, int C, int lane, BinWalk& w) {
  w.n = 0;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) {
    w.N[c] = 0;
    w.carry[c] = 0;
    if (c < C) {
      int t = 0;
      for (int b = lane; b < B; b += 32) t += H[b * C + c];
      w.N[c] = warp_sum(t);
      w.n += w.N[c];
    }
  }
}

// Left class counts L and left size of candidate b = 32 r + lane of round r
// (rounds in order; every lane of the warp calls it).
__device__ __forceinline__ long long walk_round(const int32_t* __restrict__ H, int B, int C, int lane, int r,
                                                BinWalk& w, int* L) {
  const int b = 32 * r + lane;
  long long nL = 0;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) {
    L[c] = 0;
    if (c < C) {
      const int inc = warp_incl_scan(b < B ? H[b * C + c] : 0, lane);
      L[c] = w.carry[c] + inc;
      w.carry[c] += __shfl_sync(0xffffffffu, inc, 31);
      nL += L[c];
    }
  }
  return nL;
}

// The same walk with the whole histogram of the projection loaded into
// registers first (lane l: bins 32 r + l, r < 8, classes c < CM), so its loads
// are in flight together instead of one round's at a time.  For B <= 256 and
// C <= CM; the round index must be a compile-time constant after unrolling.
template <int CM>
__device__ __forceinline__ void regs_init(const int32_t* __restrict__ H, int B, int C, int lane, int (&v)[8][CM],
                                          BinWalk& w) {
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int b = 32 * r + lane;
#pragma unroll
    for (int c = 0; c < CM; ++c) v[r][c] = (b < B && c < C) ? H[b * C + c] : 0;
  }
  w.n = 0;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) {
    w.N[c] = 0;
    w.carry[c] = 0;
  }
#pragma unroll
  for (int c = 0; c < CM; ++c) {
    int t = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r) t += v[r][c];
    w.N[c] = warp_sum(t);
    w.n += w.N[c];
  }
}

template <int CM>
__device__ __forceinline__ long long regs_round(const int (&v)[8][CM], int C, int lane, int r, BinWalk& w, int* L) {
  long long nL = 0;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) L[c] = 0;
#pragma unroll
  for (int c = 0; c < CM; ++c) {
    if (c < C) {
      const int inc = warp_incl_scan(v[r][c], lane);
      L[c] = w.carry[c] + inc;
      w.carry[c] += __shfl_sync(0xffffffffu, inc, 31);
      nL += L[c];
    }
  }
  return nL;
}

// One projection of k_gini_scan from registers; returns the lane's best key.
template <int CM>
__device__ __forceinline__ float gini_proj_regs(const int32_t* __restrict__ H, int B, int C, int lane, const Crit& cr,
                                                float* gain_row, BinWalk& w) {
  int v[8][CM];
  regs_init<CM>(H, B, C, lane, v, w);
  float best = key_none(cr);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    if (32 * r >= B) break;
    int L[kMaxClasses];
    const long long nL = regs_round<CM>(v, C, lane, r, w, L);
    const int b = 32 * r + lane;
    if (b > B - 2) continue;
    float g = key_none(cr);
    if (nL > 0 && nL < w.n) g = key32(cr, L, w.N, C, w.n, nL);
    best = fmaxf(best, g);
    if (gain_row) gain_row[b] = g;
  }
  return best;
}

// REGS: the register walk (B <= 256 and C <= 2; the host picks the
// instantiation, so each keeps its own register allocation)
template <int REGS>
__global__ void __launch_bounds__(256) k_gini_scan(const V4* plan_total, int32_t P, int32_t B, int32_t C,
                                                   const int32_t* __restrict__ hist, float* max32,
                                                   int32_t* node_counts, float* gain32_out, Crit cr) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t total = plan_total->x * P;
  const int R = (B + 31) / 32;
  for (int64_t wi = gw; wi < total; wi += nw) {
    const int64_t h = wi / P;
    const int p = (int)(wi - h * P);
    const int32_t* H = hist + wi * (int64_t)B * C;
    BinWalk w;
    float best = key_none(cr);
    float* gain_row = gain32_out ? gain32_out + wi * (B - 1) : nullptr;
    if (REGS) {
      // (measured: for three classes the register form was slower here,
      // 0.023 against 0.015 ms for one 256-projection node)
      best = gini_proj_regs<2>(H, B, C, lane, cr, gain_row, w);
    } else {
      walk_init(H, B, C, lane, w);
      for (int r = 0; r < R; ++r) {
        int L[kMaxClasses];
        const long long nL = walk_round(H, B, C, lane, r, w, L);
        const int b = 32 * r + lane;
        if (b > B - 2) continue;
        float g = key_none(cr);
        if (nL > 0 && nL < w.n) g = key32(cr, L, w.N, C, w.n, nL);
        best = fmaxf(best, g);
        if (gain_row) gain_row[b] = g;
      }
    }
    best = warp_max(best);
    if (lane == 0) max32[wi] = best;
    if (p == 0) {
#pragma unroll
      for (int c = 0; c < kMaxClasses; ++c)
        if (c < C && lane == c) node_counts[h * C + c] = w.N[c];
    }
  }
}

// ============================================================================
// K4b: per histogram node, double re-score of float near-ties and selection

// The candidates of projection p whose float key reaches thr, re-scored in
// double into the lane's lexicographic best.  An empty bin b repeats
// candidate b-1's partition (same double gain bits, lower index), so it can
// never be the lexicographic argmax and is skipped.
__device__ __forceinline__ void select_visit(const Crit& cr, const int* L, const BinWalk& w, int C, long long nL,
                                             long long prev, int b, int B, float thr, int p, Cand& best) {
  if (b > B - 2) return;
  const bool repeat = b > 0 && nL == prev;
  if (!repeat && nL > 0 && nL < w.n) {
    const float g = key32(cr, L, w.N, C, w.n, nL);
    if (g >= thr) {
      const Cand c{gain64c(cr, L, w.N, C, w.n, nL), p, b};
      if (better(c, best)) best = c;
    }
  }
}

__device__ __forceinline__ void select_proj(const int32_t* __restrict__ H, int B, int C, int lane, const Crit& cr,
                                            float thr, int p, Cand& best) {
  BinWalk w;
  walk_init(H, B, C, lane, w);
  long long before = 0;  // left size of bin 32 r - 1
  for (int r = 0; r * 32 < B; ++r) {
    int L[kMaxClasses];
    const long long nL = walk_round(H, B, C, lane, r, w, L);
    long long prev = __shfl_up_sync(0xffffffffu, nL, 1);
    if (lane == 0) prev = before;
    before = __shfl_sync(0xffffffffu, nL, 31);
    select_visit(cr, L, w, C, nL, prev, 32 * r + lane, B, thr, p, best);
  }
}

template <int CM>
__device__ __forceinline__ void select_proj_regs(const int32_t* __restrict__ H, int B, int C, int lane,
                                                 const Crit& cr, float thr, int p, Cand& best) {
  BinWalk w;
  int v[8][CM];
  regs_init<CM>(H, B, C, lane, v, w);
  long long before = 0;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    if (32 * r >= B) break;
    int L[kMaxClasses];
    const long long nL = regs_round<CM>(v, C, lane, r, w, L);
    long long prev = __shfl_up_sync(0xffffffffu, nL, 1);
    if (lane == 0) prev = before;
    before = __shfl_sync(0xffffffffu, nL, 31);
    select_visit(cr, L, w, C, nL, prev, 32 * r + lane, B, thr, p, best);
  }
}
// ============================================================================
__global__ void __launch_bounds__(256) k_hist_select(const V4* plan_total, const int32_t* hist_nodes,
                                                     const int64_t* off, int32_t P, int32_t B, int32_t C,
                                                     const int32_t* __restrict__ hist,
                                                     const float* __restrict__ max32,
                                                     const uint32_t* __restrict__ mm,
                                                     const float* __restrict__ rw_t, Crit cr,
                                                     so_split* out, int64_t* left_counts) {
  __shared__ float s_red[8];
  __shared__ Cand s_best[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t m_hist = plan_total->x;
  for (int64_t h = blockIdx.x; h < m_hist; h += gridDim.x) {
    const int j = hist_nodes[h];
    const int64_t n = off[j + 1] - off[j];
    float m = key_none(cr);
    for (int p = threadIdx.x; p < P; p += blockDim.x) m = fmaxf(m, max32[h * P + p]);
    m = warp_max(m);
    if (lane == 0) s_red[warp] = m;
    __syncthreads();
    float M = s_red[0];
    for (int w = 1; w < 8; ++w) M = fmaxf(M, s_red[w]);
    __syncthreads();
    if (!key_any(cr, M)) {
      if (threadIdx.x == 0) {
        so_split r;
        r.valid = 0; r.proj = -1; r.path = 0; r.cand = -1; r.threshold = 0.0f; r.gain = 0.0;
        r.n_left = 0; r.n_right = 0;
        out[j] = r;
        if (left_counts)
          for (int c = 0; c < C; ++c) left_counts[(int64_t)j * C + c] = 0;
      }
      continue;
    }
    const float thr = key_thr(cr, M, n, C);
    Cand best{-1.0, INT_MAX, INT_MAX};
    // warp w reads the float maxima of projections 256 i + w + 8 lane at
    // once and walks those within the window (the lexicographic best does
    // not depend on the order)
    for (int base = 0; base < P; base += 8 * 32) {
      const int pp = base + warp + 8 * lane;
      unsigned hits = __ballot_sync(0xffffffffu, pp < P && max32[h * P + pp] >= thr);
      while (hits) {
        const int p = base + warp + 8 * (__ffs(hits) - 1);
        hits &= hits - 1u;
        const int32_t* H = hist + (h * P + p) * (int64_t)B * C;
        if (B <= 256 && C <= 2)
          select_proj_regs<2>(H, B, C, lane, cr, thr, p, best);
        else if (B <= 256 && C <= 4)
          select_proj_regs<4>(H, B, C, lane, cr, thr, p, best);
        else
          select_proj(H, B, C, lane, cr, thr, p, best);
      }
    }
    best = warp_best(best);
    if (lane == 0) s_best[warp] = best;
    __syncthreads();
    if (warp == 0) {
      // every lane of warp 0 takes the node's best; the left class counts of
      // the chosen candidate are summed over its bins 32 at a time
      Cand f = s_best[0];
      for (int w = 1; w < 8; ++w)
        if (better(s_best[w], f)) f = s_best[w];
      if (!(f.g > 0.0)) {
        // no re-scored candidate with a positive double gain (information
        // gain can round to zero or below for a split that carries almost none)
        if (lane == 0) {
          so_split r;
          r.valid = 0; r.proj = -1; r.path = 0; r.cand = -1; r.threshold = 0.0f; r.gain = 0.0;
          r.n_left = 0; r.n_right = 0;
          out[j] = r;
          if (left_counts)
            for (int c = 0; c < C; ++c) left_counts[(int64_t)j * C + c] = 0;
        }
      } else {
        if (f.proj == INT_MAX) f.proj = 0, f.cand = 0;  // cannot happen: the float maximum is always re-scored
        const int32_t* H = hist + (h * P + f.proj) * (int64_t)B * C;
        long long Lc[kMaxClasses];
#pragma unroll
        for (int c = 0; c < kMaxClasses; ++c) Lc[c] = 0;
        for (int b = lane; b <= f.cand; b += 32)
#pragma unroll
          for (int c = 0; c < kMaxClasses; ++c)
            if (c < C) Lc[c] += H[b * C + c];
        long long nL = 0;
#pragma unroll
        for (int c = 0; c < kMaxClasses; ++c) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) Lc[c] += __shfl_xor_sync(0xffffffffu, Lc[c], o);
          nL += c < C ? Lc[c] : 0;
        }
        if (lane == 0) {
          const float mn = key2f(mm[(h * P + f.proj) * 2]);
          const float mx = key2f(mm[(h * P + f.proj) * 2 + 1]);
          const float w = bin_width(mn, mx, B);
          so_split r;
          r.valid = 1;
          r.proj = f.proj;
          r.path = 0;
          r.cand = f.cand;
          // candidate b's threshold is boundary t_{b+1}
          r.threshold = rw_t ? rw_t[(h * P + f.proj) * kRwRow + f.cand] : boundary(mn, w, f.cand + 1);
          r.gain = f.g;
          r.n_left = nL;
          r.n_right = n - nL;
          out[j] = r;
          if (left_counts)
            for (int c = 0; c < C; ++c) left_counts[(int64_t)j * C + c] = Lc[c];
        }
      }
    }
    __syncthreads();
  }
}

// x ln x for x < kXlnxTab, the exact path's table of the entropy criterion
// (each entry the value xlnx64 computes, so table and direct values agree).
__global__ void k_xlnx_table(double* tab) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < kXlnxTab) tab[x] = xlnx64(x);
}

// Copies inspection outputs of the histogram stage (slot h -> node j).
__global__ void k_hist_export(const V4* plan_total, const int32_t* hist_nodes, int32_t P, int32_t BC,
                              int32_t B, const uint32_t* mm, const int32_t* hist, const float* gain_tmp,
                              const float* rw_t, float* minmax_out, int32_t* hist_out, float* gain32_out,
                              float* bounds_out) {
  const int64_t mh = plan_total->x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < mh * P; i += stride) {
    const int64_t h = i / P, p = i - h * P;
    const int64_t j = hist_nodes[h];
    minmax_out[(j * P + p) * 2] = key2f(mm[i * 2]);
    minmax_out[(j * P + p) * 2 + 1] = key2f(mm[i * 2 + 1]);
  }
  for (int64_t i = tid; i < mh * P * BC; i += stride) {
    const int64_t hp = i / BC, r = i - hp * BC;
    const int64_t h = hp / P, p = hp - h * P;
    hist_out[((int64_t)hist_nodes[h] * P + p) * BC + r] = hist[i];
  }
  if (gain32_out && gain_tmp) {
    for (int64_t i = tid; i < mh * P * (B - 1); i += stride) {
      const int64_t hp = i / (B - 1), r = i - hp * (B - 1);
      const int64_t h = hp / P, p = hp - h * P;
      gain32_out[((int64_t)hist_nodes[h] * P + p) * (B - 1) + r] = gain_tmp[i];
    }
  }
  if (bounds_out) {
    for (int64_t i = tid; i < mh * P * (B - 1); i += stride) {
      const int64_t hp = i / (B - 1), r = i - hp * (B - 1);
      const int64_t h = hp / P, p = hp - h * P;
      float t;
      if (rw_t) {
        t = rw_t[hp * kRwRow + r];
      } else {
        const float mn = key2f(mm[hp * 2]), mx = key2f(mm[hp * 2 + 1]);
        t = boundary(mn, bin_width(mn, mx, B), (int)r + 1);
      }
      bounds_out[((int64_t)hist_nodes[h] * P + p) * (B - 1) + r] = t;
    }
  }
}

// ============================================================================
// Search driver
// ============================================================================
void carve_search(Carver& cv, SearchScratch& s, int32_t m, int64_t n_total, int32_t P, int32_t C,
                  int32_t B, int32_t T, int32_t hist_only, int32_t bin_rule) {
  int64_t mh = m;
  if (!hist_only) {
    const int64_t tt = T > 2 ? T : 2;
    mh = std::min<int64_t>(m, n_total / tt + 1);
  }
  if (mh < 1) mh = 1;
  s.m_hist_cap = mh;
  s.plan_total = cv.take<V4>(1);
  s.tiles = cv.take<V4>((size_t)scan_tiles_for(m) + 1);
  s.hist_nodes = cv.take<int32_t>((size_t)m + 1);
  s.sort_nodes = cv.take<int32_t>(2 * (size_t)m + 2);
  s.item_off = cv.take<int64_t>((size_t)m + 1);
  s.err = cv.take<int32_t>((size_t)m + 1);  // per-node bad-row flags
  s.sort_res = cv.take<unsigned char>((size_t)m * P * sort_res_bytes());
  s.node_cls = cv.take<int32_t>((size_t)m * kMaxClasses);
  s.sort_lists = cv.take<int64_t>(2 * (size_t)m * P + 2);
  s.sort_list_n = cv.take<int32_t>(2);
  s.mm_keys = cv.take<uint32_t>((size_t)mh * P * 2);
  s.max32 = cv.take<float>((size_t)mh * P);
  s.node_counts = cv.take<int32_t>((size_t)mh * C);
  s.hist = cv.take<int32_t>((size_t)mh * P * B * C);
  carve_staged(cv, s.staged, mh, P);
  s.xlnx = cv.take<double>(kXlnxTab);
  if (bin_rule == SO_BINS_RANDOM_WIDTH) {
    s.rw.t = cv.take<float>((size_t)mh * P * kRwRow);
    s.rw.g = cv.take<uint16_t>((size_t)mh * P * kRwRow);
    s.rw.so = cv.take<float2>((size_t)mh * P);
  } else {
    s.rw = RwTables{};
  }
}

namespace {
template <typename K>
int occupancy(K kernel, int threads, size_t smem) {
  int blocks = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, smem) != cudaSuccess || blocks < 1)
    blocks = 1;
  return blocks;
}
}  // namespace

cudaError_t launch_search(const SearchArgs& a, const SearchScratch& s, cudaStream_t st) {
  const DeviceInfo& di = device_info();
  const int P = a.pv.P, C = a.ds.C, B = a.B;
  constexpr int PG = 8;
  const int G = (P + PG - 1) / PG;
  int64_t S = a.tune.chunk > 0 ? a.tune.chunk : 16384;
  cudaError_t e;

  // validation of the projection rows
  e = cudaMemsetAsync(s.err, 0, sizeof(int32_t) * ((size_t)a.m + 1), st);
  if (e != cudaSuccess) return e;
  if (!a.rows_trusted) {
    const int64_t rows = (int64_t)a.m * P;
    if (rows > 0) k_validate_rows<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a.pv, a.m, a.ds.d, a.max_nnz, s.err);
  }
  PlanF pf;
  pf.off = a.node_off;
  pf.n_total = a.n_total;
  pf.bad = s.err;
  pf.T = a.T;
  pf.hist_only = a.hist_only;
  pf.force_hist = 0;
  pf.C = C;
  pf.S = S;
  pf.G = G;
  pf.hist_nodes = s.hist_nodes;
  pf.tiny_nodes = s.sort_nodes;
  pf.med_nodes = s.sort_nodes + a.m + 1;
  pf.item_off = s.item_off;
  pf.out = a.out;
  pf.left_counts = a.left_counts;
  e = run_scan(pf, a.m, s.tiles, s.plan_total, st, "plan_scan");
  if (e != cudaSuccess) return e;

  const int grid_fill = di.num_sms * 8;
  const Crit cr{a.criterion == SO_CRIT_ENTROPY ? 1 : 0, a.eps, a.criterion == SO_CRIT_ENTROPY ? s.xlnx : nullptr};
  if (cr.ent) {
    ProfScope ps_("k_xlnx_table", st);
    k_xlnx_table<<<kXlnxTab / 256, 256, 0, st>>>(s.xlnx);
  }
  // the histogram path (no node of the call reaches T: left out)
  const bool hist_any = a.hist_only || a.max_nv_hint < 0 || a.max_nv_hint >= a.T;
  const bool rw = a.bin_rule == SO_BINS_RANDOM_WIDTH;
  if (hist_any) {
    {
      ProfScope ps_("k_hist_init", st);
      k_hist_init<<<grid_fill, 256, 0, st>>>(s.plan_total, P, B * C, s.mm_keys, s.hist, s.max32);
    }
    if (staged_supported(a.ds.d)) {
      e = launch_staged(a, s.plan_total, s.hist_nodes, s.m_hist_cap, s.staged, s.mm_keys, s.hist, s.rw, S,
                        a.max_nnz, st);
      if (e != cudaSuccess) return e;
    } else {
      {
        static thread_local int occ_mm = 0;
        if (!occ_mm) occ_mm = occupancy(k_minmax<PG>, PG * 32, 0);
        ProfScope ps_("k_minmax", st);
        k_minmax<PG><<<di.num_sms * occ_mm, PG * 32, 0, st>>>(a.ds, a.idx, a.node_off, a.pv, s.plan_total,
                                                              s.hist_nodes, s.item_off, S, s.mm_keys);
      }
      if (rw) {
        e = launch_rw_bounds(a, s.plan_total, s.hist_nodes, s.mm_keys, s.rw, st);
        if (e != cudaSuccess) return e;
      }
      {
        const size_t smem = (size_t)PG * B * C * sizeof(int32_t);
        e = cudaFuncSetAttribute(k_hist<PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const int occ = occupancy(k_hist<PG>, PG * 32, smem);
        ProfScope ps_("k_hist", st);
        k_hist<PG><<<di.num_sms * occ, PG * 32, smem, st>>>(a.ds, a.idx, a.node_off, a.pv, s.plan_total,
                                                            s.hist_nodes, s.item_off, S, B, s.mm_keys, s.hist,
                                                            rw ? s.rw.t : nullptr);
      }
    }
    {
      ProfScope ps_("k_gini_scan", st);
      auto kg = (B <= 256 && C <= 2) ? k_gini_scan<1> : k_gini_scan<0>;
      kg<<<grid_fill, 256, 0, st>>>(s.plan_total, P, B, C, s.hist, s.max32, s.node_counts, nullptr, cr);
    }
    {
      ProfScope ps_("k_hist_select", st);
      k_hist_select<<<grid_fill, 256, 0, st>>>(s.plan_total, s.hist_nodes, a.node_off, P, B, C, s.hist, s.max32,
                                               s.mm_keys, rw ? s.rw.t : nullptr, cr, a.out, a.left_counts);
    }
  }  // hist_any
  // exact path (no node can take it when every node is on the histogram path
  // or T <= 2: nodes below 2 samples are never searched)
  if (!a.hist_only && a.T > 2) {
    e = launch_sort_warp(a, cr, s.plan_total, s.sort_nodes, s.sort_nodes + a.m + 1, s.sort_res, s.node_cls,
                         s.sort_lists, s.sort_list_n, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// Inspection variant: histogram stage with exported intermediates.
cudaError_t launch_hist_inspect(const SearchArgs& a, const SearchScratch& s, float* gain_tmp, cudaStream_t st) {
  const DeviceInfo& di = device_info();
  const int P = a.pv.P, C = a.ds.C, B = a.B;
  constexpr int PG = 8;
  const int G = (P + PG - 1) / PG;
  const int64_t S = a.tune.chunk > 0 ? a.tune.chunk : 16384;
  cudaError_t e = cudaMemsetAsync(s.err, 0, sizeof(int32_t) * ((size_t)a.m + 1), st);
  if (e != cudaSuccess) return e;
  const int64_t rows = (int64_t)a.m * P;
  if (rows > 0) k_validate_rows<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a.pv, a.m, a.ds.d, a.max_nnz, s.err);
  PlanF pf;
  pf.off = a.node_off;
  pf.n_total = a.n_total;
  pf.bad = s.err;
  pf.T = a.T;
  pf.hist_only = 1;
  pf.force_hist = 1;
  pf.C = C;
  pf.S = S;
  pf.G = G;
  pf.hist_nodes = s.hist_nodes;
  pf.tiny_nodes = s.sort_nodes;
  pf.med_nodes = s.sort_nodes + a.m + 1;
  pf.item_off = s.item_off;
  pf.out = nullptr;
  pf.left_counts = nullptr;
  e = run_scan(pf, a.m, s.tiles, s.plan_total, st, "plan_scan");
  if (e != cudaSuccess) return e;
  const int grid_fill = di.num_sms * 8;
  const bool rw = a.bin_rule == SO_BINS_RANDOM_WIDTH;
  {
    ProfScope ps_("k_hist_init", st);
    k_hist_init<<<grid_fill, 256, 0, st>>>(s.plan_total, P, B * C, s.mm_keys, s.hist, s.max32);
  }
  if (staged_supported(a.ds.d)) {
    e = launch_staged(a, s.plan_total, s.hist_nodes, s.m_hist_cap, s.staged, s.mm_keys, s.hist, s.rw, S,
                      a.max_nnz, st);
    if (e != cudaSuccess) return e;
  } else {
    {
      ProfScope ps_("k_minmax", st);
      k_minmax<PG><<<di.num_sms * 4, PG * 32, 0, st>>>(a.ds, a.idx, a.node_off, a.pv, s.plan_total, s.hist_nodes,
                                                       s.item_off, S, s.mm_keys);
    }
    if (rw) {
      e = launch_rw_bounds(a, s.plan_total, s.hist_nodes, s.mm_keys, s.rw, st);
      if (e != cudaSuccess) return e;
    }
    const size_t smem = (size_t)PG * B * C * sizeof(int32_t);
    e = cudaFuncSetAttribute(k_hist<PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    {
      ProfScope ps_("k_hist", st);
      k_hist<PG><<<di.num_sms * 2, PG * 32, smem, st>>>(a.ds, a.idx, a.node_off, a.pv, s.plan_total, s.hist_nodes,
                                                        s.item_off, S, B, s.mm_keys, s.hist, rw ? s.rw.t : nullptr);
    }
  }
  {
    ProfScope ps_("k_gini_scan", st);
    auto kg = (B <= 256 && C <= 2) ? k_gini_scan<1> : k_gini_scan<0>;
    kg<<<grid_fill, 256, 0, st>>>(s.plan_total, P, B, C, s.hist, s.max32, s.node_counts, gain_tmp,
                                           Crit{0, a.eps, nullptr});
  }
  {
    ProfScope ps_("k_hist_export", st);
    k_hist_export<<<grid_fill, 256, 0, st>>>(s.plan_total, s.hist_nodes, P, B * C, B, s.mm_keys, s.hist, gain_tmp,
                                             rw ? s.rw.t : nullptr, a.minmax_out, a.hist_out, a.gain32_out,
                                             a.bounds_out);
  }
  return cudaGetLastError();
}

// ============================================================================
// Projection sampler (Appendix A: Floyd; nnz by inverse-CDF Poisson)
// ============================================================================
struct CdfTable {
  double c[kMaxCap];
};

__global__ void k_sample(int32_t m, const uint64_t* __restrict__ keys, int32_t P, int32_t d, CdfTable cdf,
                         int32_t cap, int32_t* nnz, int32_t* feat, int8_t* sign, int32_t* beg, int32_t* end) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)m * P) return;
  const int64_t j = q / P;
  const int p = (int)(q - j * P);
  uint64_t st = sm64(keys[j] + (uint64_t)p * kProjMult);
  const uint64_t r = sm64_next(st);
  const double u = (double)(r >> 11) * 0x1.0p-53;
  int K = 0;
  while (K < cap - 1 && u >= cdf.c[K]) ++K;
  int k = 1 + K;
  if (k > d) k = d;
  int32_t f[kMaxCap];
  int mcount = 0;
  for (int jj = d - k; jj < d; ++jj) {
    const uint64_t rr = sm64_next(st);
    const int32_t t = (int32_t)__umul64hi(rr, (uint64_t)(jj + 1));
    bool seen = false;
    for (int i = 0; i < mcount; ++i) seen |= (f[i] == t);
    f[mcount++] = seen ? jj : t;
  }
  for (int a = 1; a < mcount; ++a) {
    const int32_t key = f[a];
    int b = a - 1;
    while (b >= 0 && f[b] > key) {
      f[b + 1] = f[b];
      --b;
    }
    f[b + 1] = key;
  }
  const uint64_t sb = sm64_next(st);
  const int64_t base = q * cap;
  for (int i = 0; i < mcount; ++i) {
    feat[base + i] = f[i];
    sign[base + i] = ((sb >> i) & 1ull) ? (int8_t)1 : (int8_t)-1;
  }
  nnz[q] = mcount;
  if (beg) beg[q] = (int32_t)base;
  if (end) end[q] = (int32_t)(base + mcount);
}

cudaError_t launch_sample(int32_t m, const uint64_t* keys, int32_t P, int32_t d, double lambda, int32_t cap,
                          int32_t* nnz, int32_t* feat, int8_t* sign, int32_t* beg, int32_t* end, cudaStream_t st) {
  // Poisson cumulative probabilities P(K <= k), k = 0..cap-2, by the
  // definition p_0 = e^-lambda, p_k = p_{k-1} * lambda / k (host, double).
  CdfTable t{};
  double pk = std::exp(-lambda);
  double c = pk;
  for (int k = 0; k < cap - 1; ++k) {
    if (k > 0) {
      pk = (pk * lambda) / (double)k;
      c = c + pk;
    }
    t.c[k] = c;
  }
  const int64_t n = (int64_t)m * P;
  if (n == 0) return cudaSuccess;
  {
    ProfScope ps_("k_sample", st);
    k_sample<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(m, keys, P, d, t, cap, nnz, feat, sign, beg, end);
  }
  return cudaGetLastError();
}

// ============================================================================
// Stable partition (batched over the frontier)
// ============================================================================
constexpr int kPartThreads = 256;
constexpr int kPartPer = 4;
constexpr int kPartTile = kPartThreads * kPartPer;

int64_t part_tiles(int64_t n) { return (n + kPartTile - 1) / kPartTile; }

__device__ __forceinline__ int find_seg(const int64_t* off, int m, int64_t q) {
  int lo = 0, hi = m - 1;  // largest j with off[j] <= q
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= q) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int part_flag(const PartArgs& a, const PartNode& nd, int32_t s) {
  if (nd.mode == PART_COPY) return 1;
  if (nd.mode == PART_DROP) return 0;
  const int k = nd.nnz < 0 ? 0 : (nd.nnz > kMaxCap ? kMaxCap : nd.nnz);
  float acc = 0.0f;
  for (int jj = 0; jj < k; ++jj) {
    int f = a.feat[nd.feat_off + jj];
    f = (f < 0 || f >= a.ds.d) ? 0 : f;
    const float x = __ldg(a.ds.X + (int64_t)f * a.ds.ld + s);
    acc = __fadd_rn(acc, a.sign[nd.feat_off + jj] == 1 ? x : -x);
  }
  return acc < nd.thr ? 1 : 0;
}

__global__ void __launch_bounds__(kPartThreads) k_part_flags(PartArgs a) {
  const int64_t base = (int64_t)blockIdx.x * kPartTile;
  const int64_t q0 = base + threadIdx.x;  // the thread's samples: q0 + k * kPartThreads
  int cnt = 0;
  int j = q0 < a.n ? find_seg(a.node_off, a.m, q0) : -1;
  const int64_t q_last = min(a.n - 1, q0 + (int64_t)(kPartPer - 1) * kPartThreads);
  if (j >= 0 && a.node_off[j + 1] > q_last) {
    // every sample of the thread in one node: the sample ids first, then each
    // term's values of all of them, so the loads of a stage are in flight
    // together; the terms are added in row order as part_flag does
    const PartNode nd = a.nodes[j];
    int32_t sid[kPartPer];
#pragma unroll
    for (int k = 0; k < kPartPer; ++k) {
      const int64_t q = q0 + (int64_t)k * kPartThreads;
      sid[k] = q < a.n ? (int32_t)safe_sample(a.idx_in[q], a.ds.n) : 0;
    }
    int fl[kPartPer];
    if (nd.mode == PART_COPY || nd.mode == PART_DROP) {
#pragma unroll
      for (int k = 0; k < kPartPer; ++k) fl[k] = nd.mode == PART_COPY ? 1 : 0;
    } else {
      const int kk = nd.nnz < 0 ? 0 : (nd.nnz > kMaxCap ? kMaxCap : nd.nnz);
      float acc[kPartPer];
#pragma unroll
      for (int k = 0; k < kPartPer; ++k) acc[k] = 0.0f;
      for (int jj = 0; jj < kk; ++jj) {
        int f = a.feat[nd.feat_off + jj];
        f = (f < 0 || f >= a.ds.d) ? 0 : f;
        const bool pos = a.sign[nd.feat_off + jj] == 1;
        const float* col = a.ds.X + (int64_t)f * a.ds.ld;
        float x[kPartPer];
#pragma unroll
        for (int k = 0; k < kPartPer; ++k) x[k] = __ldg(col + sid[k]);
#pragma unroll
        for (int k = 0; k < kPartPer; ++k) acc[k] = __fadd_rn(acc[k], pos ? x[k] : -x[k]);
      }
#pragma unroll
      for (int k = 0; k < kPartPer; ++k) fl[k] = acc[k] < nd.thr ? 1 : 0;
    }
#pragma unroll
    for (int k = 0; k < kPartPer; ++k) {
      const int64_t q = q0 + (int64_t)k * kPartThreads;
      if (q < a.n) {
        a.flags[q] = (uint8_t)fl[k];
        cnt += fl[k];
      }
    }
  } else if (j >= 0) {
    int64_t seg_end = -1;
    j = -1;
    PartNode nd;
    for (int k = 0; k < kPartPer; ++k) {
      const int64_t q = q0 + (int64_t)k * kPartThreads;
      if (q >= a.n) break;
      if (j < 0 || q >= seg_end) {
        j = find_seg(a.node_off, a.m, q);
        nd = a.nodes[j];
        seg_end = a.node_off[j + 1];
      }
      const int f = part_flag(a, nd, (int32_t)safe_sample(a.idx_in[q], a.ds.n));
      a.flags[q] = (uint8_t)f;
      cnt += f;
    }
  }
  cnt = warp_sum(cnt);
  __shared__ int s_c[kPartThreads / 32];
  if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < kPartThreads / 32; ++w) t += s_c[w];
    a.tile_cnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) k_part_scan(int64_t* tile_cnt, int64_t n_tiles, int64_t* total,
                                                   PartNode* fix) {
  __shared__ long long s_w[32];
  __shared__ long long s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n_tiles; base += 1024) {
    const int64_t i = base + threadIdx.x;
    const long long v = (i < n_tiles) ? tile_cnt[i] : 0;
    long long inc = warp_incl_scan(v, lane);
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const long long wv = s_w[lane];
      const long long wi = warp_incl_scan(wv, lane);
      s_w[lane] = wi - wv;
    }
    __syncthreads();
    const long long carry = s_carry;
    if (i < n_tiles) tile_cnt[i] = carry + s_w[warp] + inc - v;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = carry + s_w[warp] + inc;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (total) *total = s_carry;
    if (fix) {
      fix->ones = s_carry;
      fix->dst_zero = fix->dst_one + s_carry;
    }
  }
}

__global__ void __launch_bounds__(kPartThreads) k_part_scatter(PartArgs a) {
  const int64_t tile0 = (int64_t)blockIdx.x * kPartTile;
  const int64_t q0 = tile0 + (int64_t)threadIdx.x * kPartPer;
  int cnt = 0;
  uint8_t fl[kPartPer];
  int32_t iv[kPartPer];  // the samples' entries, loaded ahead of the scan
  if (q0 + kPartPer <= a.n && (reinterpret_cast<uintptr_t>(a.idx_in + q0) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(a.flags + q0) & 3) == 0) {
    static_assert(kPartPer == 4, "one 16-byte load of entries, one 4-byte load of flags");
    const int4 v = *reinterpret_cast<const int4*>(a.idx_in + q0);
    const uint32_t f4 = *reinterpret_cast<const uint32_t*>(a.flags + q0);
    iv[0] = v.x;
    iv[1] = v.y;
    iv[2] = v.z;
    iv[3] = v.w;
#pragma unroll
    for (int k = 0; k < kPartPer; ++k) fl[k] = (uint8_t)((f4 >> (8 * k)) & 0xFFu);
  } else {
#pragma unroll
    for (int k = 0; k < kPartPer; ++k) {
      const int64_t q = q0 + k;
      fl[k] = (q < a.n) ? a.flags[q] : 0;
      iv[k] = (q < a.n) ? a.idx_in[q] : 0;
    }
  }
#pragma unroll
  for (int k = 0; k < kPartPer; ++k) cnt += fl[k];
  // exclusive block scan of per-thread counts
  __shared__ int s_w[kPartThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int inc = warp_incl_scan(cnt, lane);
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int wv = (lane < kPartThreads / 32) ? s_w[lane] : 0;
    const int wi = warp_incl_scan(wv, lane);
    if (lane < kPartThreads / 32) s_w[lane] = wi - wv;
  }
  __syncthreads();
  long long ones_before = a.tile_cnt[blockIdx.x] + s_w[warp] + (inc - cnt);
  int j = -1;
  int64_t seg_end = -1;
  PartNode nd;
  for (int k = 0; k < kPartPer; ++k) {
    const int64_t q = q0 + k;
    if (q >= a.n) break;
    if (j < 0 || q >= seg_end) {
      j = find_seg(a.node_off, a.m, q);
      nd = a.nodes[j];
      seg_end = a.node_off[j + 1];
    }
    const int f = fl[k];
    const long long r1 = ones_before - nd.ones_prefix;
    const long long r0 = (q - nd.beg) - r1;
    const long long size = nd.end - nd.beg;
    if (f) {
      if (r1 < 0 || r1 >= nd.ones) {
        atomicOr(a.err, 1);
      } else if (nd.dst_one >= 0) {
        const int64_t dst = nd.dst_one + r1;
        if (dst < a.n_out) a.idx_out[dst] = iv[k];
        else atomicOr(a.err, 8);
      }
    } else {
      if (r0 < 0 || r0 >= size - nd.ones) {
        atomicOr(a.err, 2);
      } else if (nd.dst_zero >= 0) {
        const int64_t dst = nd.dst_zero + r0;
        if (dst < a.n_out) a.idx_out[dst] = iv[k];
        else atomicOr(a.err, 8);
      }
    }
    if (q == nd.end - 1 && r1 + f != nd.ones) atomicOr(a.err, 4);
    ones_before += f;
  }
}

cudaError_t launch_partition(const PartArgs& a, cudaStream_t st) {
  const int64_t tiles = part_tiles(a.n);
  if (tiles == 0) return cudaSuccess;
  {
    ProfScope ps_("k_part_flags", st);
    k_part_flags<<<(unsigned)tiles, kPartThreads, 0, st>>>(a);
  }
  {
    ProfScope ps_("k_part_scan", st);
    k_part_scan<<<1, 1024, 0, st>>>(a.tile_cnt, tiles, a.ones_total, a.fix_node);
  }
  {
    ProfScope ps_("k_part_scatter", st);
    k_part_scatter<<<(unsigned)tiles, kPartThreads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

// PartNodes from split records (batch API): valid -> split to the same
// offsets (left part first), invalid -> copied unchanged.
struct PartFromSplitsF {
  const int64_t* off;
  const so_split* sp;
  ProjView pv;
  PartNode* nodes;
  // a record that names no usable projection or an impossible left size is
  // treated as invalid (the segment is copied unchanged)
  __device__ bool usable(const so_split& r, long long size) const {
    return r.valid && r.proj >= 0 && r.proj < pv.P && r.n_left >= 0 && r.n_left <= size;
  }
  __device__ V4 value(int64_t j) const {
    const so_split r = sp[j];
    const long long size = off[j + 1] - off[j];
    return V4{usable(r, size) ? r.n_left : size, 0, 0, 0};
  }
  __device__ void apply(int64_t j, V4 ex) const {
    so_split r = sp[j];
    if (!usable(r, off[j + 1] - off[j])) r.valid = 0;
    PartNode nd;
    nd.beg = off[j];
    nd.end = off[j + 1];
    nd.ones_prefix = ex.x;
    nd.mode = r.valid ? PART_SPLIT : PART_COPY;
    nd.ones = r.valid ? r.n_left : (nd.end - nd.beg);
    nd.dst_one = nd.beg;
    nd.dst_zero = nd.beg + nd.ones;
    if (r.valid) {
      const int64_t q = j * pv.P + r.proj;
      nd.feat_off = pv.beg[q];
      nd.nnz = pv.end[q] - pv.beg[q];
    } else {
      nd.feat_off = 0;
      nd.nnz = 0;
    }
    nd.thr = r.threshold;
    nd.pad = 0;
    nodes[j] = nd;
  }
};

cudaError_t launch_part_nodes_from_splits(const int64_t* node_off, int32_t m, const so_split* splits,
                                          const ProjView pv, PartNode* nodes, V4* tiles, V4* total,
                                          cudaStream_t st) {
  PartFromSplitsF f{node_off, splits, pv, nodes};
  return run_scan(f, m, tiles, total, st, "part_nodes_scan");
}

__global__ void k_part_single(int64_t n, int32_t nnz, float thr, PartNode* node, int64_t* node_off) {
  PartNode nd;
  nd.beg = 0;
  nd.end = n;
  nd.ones_prefix = 0;
  nd.ones = n;  // unknown until the flags are counted; checks use k_part_single_fix
  nd.dst_one = 0;
  nd.dst_zero = 0;
  nd.feat_off = 0;
  nd.nnz = nnz;
  nd.thr = thr;
  nd.mode = PART_SPLIT;
  nd.pad = 0;
  *node = nd;
  node_off[0] = 0;
  node_off[1] = n;
}
cudaError_t launch_part_single(int64_t n, int32_t nnz, float thr, PartNode* node, int64_t* node_off,
                               cudaStream_t st) {
  {
    ProfScope ps_("k_part_single", st);
    k_part_single<<<1, 1, 0, st>>>(n, nnz, thr, node, node_off);
  }
  return cudaGetLastError();
}
__global__ void k_fill_off(int64_t* off, int64_t n) {
  off[0] = 0;
  off[1] = n;
}
// Synthetic nodes for the crossover benchmark: m nodes of s samples each,
// indices drawn by splitmix64 from [0, n) and sorted within each node by a
// per-node odd-even pass (order only affects memory locality), offsets j*s.
__global__ void k_bench_nodes(int32_t m, int32_t s, int64_t n, uint64_t seed, int32_t* idx, int64_t* off,
                              uint64_t* keys) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < (int64_t)m * s) idx[t] = (int32_t)(sm64(seed + (uint64_t)t) % (uint64_t)n);
  if (t <= m) off[t] = (int64_t)t * s;
  if (t < m) keys[t] = sm64(seed ^ (0xA5A5A5A5ull + (uint64_t)t));
}
cudaError_t launch_bench_nodes(int32_t m, int32_t s, int64_t n, uint64_t seed, int32_t* idx, int64_t* off,
                               uint64_t* keys, cudaStream_t st) {
  const int64_t tot = std::max<int64_t>((int64_t)m * s, m + 1);
  ProfScope ps_("k_bench_nodes", st);
  k_bench_nodes<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m, s, n, seed, idx, off, keys);
  return cudaGetLastError();
}

cudaError_t launch_fill_off(int64_t* off, int64_t n, cudaStream_t st) {
  {
    ProfScope ps_("k_fill_off", st);
    k_fill_off<<<1, 1, 0, st>>>(off, n);
  }
  return cudaGetLastError();
}

// ============================================================================
// Tree growth bookkeeping
// ============================================================================
__device__ __forceinline__ int majority(const int* cnt, int C) {
  int best = 0;
  for (int c = 1; c < C; ++c)
    if (cnt[c] > cnt[best]) best = c;
  return best;
}

__device__ __forceinline__ void write_node(TreeDev t, int64_t id, int depth, long long n, const int* cnt) {
  t.left[id] = -1;
  t.right[id] = -1;
  t.depth[id] = depth;
  t.leaf_class[id] = majority(cnt, t.C);
  t.proj_nnz[id] = 0;
  t.cand[id] = -1;
  t.path[id] = -1;
  t.threshold[id] = 0.0f;
  t.gain[id] = 0.0;
  t.n_samples[id] = n;
  for (int c = 0; c < t.C; ++c) t.class_counts[id * t.C + c] = cnt[c];
  for (int q = 0; q < t.cap; ++q) {
    t.feat[id * t.cap + q] = 0;
    t.sign[id * t.cap + q] = 0;
  }
}

__global__ void k_root_counts(const uint8_t* y, int64_t n_data, const int32_t* root_idx, int64_t n, int C,
                              int32_t* counts, LevelStats* stats) {
  __shared__ int s[kMaxClasses];
  if (threadIdx.x < kMaxClasses) s[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = root_idx[i];
    if ((uint32_t)r >= (uint64_t)n_data) {
      atomicOr(&stats->err, 16);  // sample index outside [0, n)
      continue;
    }
    const int yv = y[r];
    if (yv >= C) {
      atomicOr(&stats->err, 32);  // label outside [0, n_classes)
      continue;
    }
    atomicAdd(&s[yv], 1);
  }
  __syncthreads();
  if (threadIdx.x < C && s[threadIdx.x]) atomicAdd(&counts[threadIdx.x], s[threadIdx.x]);
}

__global__ void k_root_finish(int64_t n_root, uint64_t root_key, int32_t max_depth, TreeDev t, Frontier f,
                              LevelStats* stats) {
  int cnt[kMaxClasses];
  int present = 0;
  for (int c = 0; c < t.C; ++c) {
    cnt[c] = f.counts[c];
    present += cnt[c] > 0;
  }
  write_node(t, 0, 0, n_root, cnt);
  const bool active = n_root >= 2 && present >= 2 && (max_depth < 0 || 0 < max_depth);
  f.off[0] = 0;
  f.off[1] = n_root;
  f.key[0] = root_key;
  f.id[0] = 0;
  f.depth[0] = 0;
  stats->m_next = (active && stats->err == 0) ? 1 : 0;
  stats->n_next = n_root;
  stats->max_next = (int)n_root;
  stats->new_nodes = 1;
}

cudaError_t launch_tree_root(const DatasetView ds, const int32_t* root_idx, int64_t n_root, uint64_t root_key,
                             int32_t max_depth, TreeDev t, Frontier f, LevelStats* stats, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(f.counts, 0, sizeof(int32_t) * t.C, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(stats, 0, sizeof(LevelStats), st);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>((n_root + 255) / 256, (int64_t)device_info().num_sms * 4);
  {
    ProfScope ps_("k_root_counts", st);
    k_root_counts<<<grid > 0 ? grid : 1, 256, 0, st>>>(ds.y, ds.n, root_idx, n_root, t.C, f.counts, stats);
  }
  {
    ProfScope ps_("k_root_finish", st);
    k_root_finish<<<1, 1, 0, st>>>(n_root, root_key, max_depth, t, f, stats);
  }
  return cudaGetLastError();
}

__global__ void k_tree_record_splits(int32_t j0, int32_t mb, Frontier f, const so_split* splits, const int32_t* snnz,
                                     const int32_t* sfeat, const int8_t* ssign, int32_t P, int32_t cap, TreeDev t) {
  const int64_t jj = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (jj >= mb) return;
  const int64_t j = j0 + jj;
  const so_split r = splits[j];
  const int64_t id = f.id[j];
  t.path[id] = (int8_t)r.path;
  if (!r.valid) return;
  const int64_t q = jj * P + r.proj;
  const int k = snnz[q];
  t.proj_nnz[id] = k;
  for (int i = 0; i < k; ++i) {
    t.feat[id * t.cap + i] = sfeat[q * cap + i];
    t.sign[id * t.cap + i] = ssign[q * cap + i];
  }
  t.cand[id] = r.cand;
  t.threshold[id] = r.threshold;
  t.gain[id] = r.gain;
}

cudaError_t launch_tree_record_splits(int32_t j0, int32_t mb, const Frontier f, const so_split* splits,
                                      const int32_t* snnz, const int32_t* sfeat, const int8_t* ssign, int32_t P,
                                      int32_t cap, TreeDev t, cudaStream_t st) {
  if (mb <= 0) return cudaSuccess;
  {
    ProfScope ps_("k_tree_record_splits", st);
    k_tree_record_splits<<<(mb + 255) / 256, 256, 0, st>>>(j0, mb, f, splits, snnz, sfeat, ssign, P, cap, t);
  }
  return cudaGetLastError();
}

struct LevelF {
  Frontier cur, nxt;
  const so_split* sp;
  const int64_t* lc;
  int32_t max_depth;
  int64_t node_base_next;
  TreeDev t;
  PartNode* pn;
  LevelStats* stats;  // max_next: zeroed before the scan

  __device__ void children(int64_t j, bool& v, long long& nL, long long& nR, bool& aL, bool& aR, int* L,
                           int* R) const {
    const so_split r = sp[j];
    v = r.valid != 0;
    nL = v ? r.n_left : 0;
    nR = v ? r.n_right : 0;
    int pl = 0, pr = 0;
    for (int c = 0; c < t.C; ++c) {
      L[c] = v ? (int)lc[j * t.C + c] : 0;
      R[c] = v ? cur.counts[j * t.C + c] - L[c] : 0;
      pl += L[c] > 0;
      pr += R[c] > 0;
    }
    const int d = cur.depth[j] + 1;
    const bool deeper = max_depth < 0 || d < max_depth;
    aL = v && nL >= 2 && pl >= 2 && deeper;
    aR = v && nR >= 2 && pr >= 2 && deeper;
  }
  __device__ V4 value(int64_t j) const {
    bool v, aL, aR;
    long long nL, nR;
    int L[kMaxClasses], R[kMaxClasses];
    children(j, v, nL, nR, aL, aR, L, R);
    return V4{v ? 1 : 0, (aL ? 1 : 0) + (aR ? 1 : 0), (aL ? nL : 0) + (aR ? nR : 0), v ? nL : 0};
  }
  __device__ void apply(int64_t j, V4 ex) const {
    bool v, aL, aR;
    long long nL, nR;
    int L[kMaxClasses], R[kMaxClasses];
    children(j, v, nL, nR, aL, aR, L, R);
    const int64_t id = cur.id[j];
    PartNode nd;
    nd.beg = cur.off[j];
    nd.end = cur.off[j + 1];
    nd.ones_prefix = ex.w;
    nd.ones = v ? nL : 0;
    nd.mode = v ? PART_SPLIT : PART_DROP;
    nd.dst_one = aL ? ex.z : -1;
    nd.dst_zero = aR ? ex.z + (aL ? nL : 0) : -1;
    nd.feat_off = id * t.cap;
    nd.nnz = v ? t.proj_nnz[id] : 0;
    nd.thr = v ? sp[j].threshold : 0.0f;
    nd.pad = 0;
    pn[j] = nd;
    // the next frontier's largest node (an atomic only when this one is
    // larger than the maximum seen so far)
    const long long bl = aL ? nL : 0, br = aR ? nR : 0;
    const int big = (int)(bl > br ? bl : br);
    if (big > *(volatile int*)&stats->max_next) atomicMax(&stats->max_next, big);
    if (!v) return;
    const int64_t lid = node_base_next + 2 * ex.x;
    const int64_t rid = lid + 1;
    t.left[id] = (int32_t)lid;
    t.right[id] = (int32_t)rid;
    const int d = cur.depth[j] + 1;
    write_node(t, lid, d, nL, L);
    write_node(t, rid, d, nR, R);
    const uint64_t key = cur.key[j];
    int64_t a = ex.y;
    if (aL) {
      nxt.off[a] = ex.z;
      nxt.key[a] = sm64(2ull * key + 0ull);
      nxt.id[a] = (int32_t)lid;
      nxt.depth[a] = d;
      for (int c = 0; c < t.C; ++c) nxt.counts[a * t.C + c] = L[c];
      ++a;
    }
    if (aR) {
      nxt.off[a] = ex.z + (aL ? nL : 0);
      nxt.key[a] = sm64(2ull * key + 1ull);
      nxt.id[a] = (int32_t)rid;
      nxt.depth[a] = d;
      for (int c = 0; c < t.C; ++c) nxt.counts[a * t.C + c] = R[c];
    }
  }
};

// The next frontier's end offset and the level's counts, from the level
// scan's total (run by the scan's last step).
struct LevelFinish {
  Frontier nxt;
  LevelStats* stats;
  __device__ void operator()(const V4& tt) const {
    nxt.off[tt.y] = tt.z;
    stats->m_next = tt.y;
    stats->n_next = tt.z;
    stats->new_nodes = 2 * tt.x;
  }
};

cudaError_t launch_tree_level(int32_t m, const Frontier cur, Frontier nxt, const so_split* splits,
                              const int64_t* left_counts, int32_t max_depth, int64_t node_base_next, TreeDev t,
                              PartNode* pnodes, V4* tiles, V4* total, LevelStats* stats, cudaStream_t st) {
  LevelF f{cur, nxt, splits, left_counts, max_depth, node_base_next, t, pnodes, stats};
  cudaError_t e = cudaMemsetAsync(&stats->max_next, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  return run_scan(f, m, tiles, total, st, "level_scan", LevelFinish{nxt, stats});
}

}  // namespace sof
