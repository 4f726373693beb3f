// so_hist_staged.cu -- staged-tile kernels of the histogram path (sm_103a).
//
// A work item is (histogram node, sample chunk, projection group).  The
// item's projections use U distinct features; for each tile of St samples
// the CTA stages those U feature columns once in shared memory (one global
// read per (sample, feature)), then every projection of the group is
// evaluated from shared memory: one warp per projection, each lane a pair of
// consecutive samples, packed FP32x2 arithmetic.  Projection groups are
// formed on the device so that U stays within the tile budget.
//
//   k_groups       per histogram node: greedy grouping of its projections
//   k_mm_staged    per item: min / max of every projection (Section 3 step 2)
//   k_hist_staged  per item: equal-width bins and class counts in shared
//                  memory, flushed with integer atomics (Section 3 step 2)
//
// Exact bins without search loops.  With W = (max-min)/B and
// t_j = min + j*W (float), bin(v) = #{j in 1..B-1 : t_j <= v}.  Let
// e = v*inv_w + c with c = fl(fl(-min*inv_w) - 0.75) (one fused rounding) and
// q = round_half_even(e) (by adding 1.5*2^23).  When max(|min|,|max|) <= 2^18 W
// the combined rounding errors of e and of the t_j are below 1/4 bin, which
// gives bin(v) in {q, q+1}: bin(v) = q + [t_{q+1} <= v], with t_{q+1}
// computed exactly as the definition states.  q = -1 resolves to bin 0
// (t_0 = min <= v); q+1 = B lands in a spare bin merged into bin B-1 on flush.
// Projections outside that condition take the exact estimate-and-correct rule.
#include <climits>

#include "so_device.cuh"
#include "so_internal.h"
#include "so_scan.cuh"

namespace sof {

constexpr int kStThreads = 512;          // threads of the staged kernels (16 warps)
constexpr int kStWarps = kStThreads / 32;
constexpr int kStEpt = 32;               // staged elements per thread per tile (registers), histograms
constexpr int kMmEpt = 16;               // the same for min / max (smaller tile: two CTAs per SM)
constexpr int kStUMax = kStThreads * kStEpt / 64;  // rows of a histogram tile at St = 64 -> 256
constexpr int kMmUMax = kStThreads * kMmEpt / 64;  // rows of a min / max tile at St = 64 -> 128
constexpr int kStMaxWords = 2048;        // feature bitmap words (d <= 65536)
constexpr int kMmPPW = 16;               // min/max: projections per warp
constexpr int kMmGroup = kStWarps * kMmPPW;  // 256 projections per min/max group
constexpr float kMagic = 12582912.0f;    // 1.5 * 2^23
constexpr float kCondLimit = 262144.0f;  // 2^18

// ---- packed FP32x2 (sm_100+ PTX) ------------------------------------------
// Pairs are formed and split with mov.b64 so they stay register pairs.
// fadd2 results are only used where a later fusion could not change them.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

// ---- staged plan ------------------------------------------------------------
struct StagedPlan {
  const V4* plan_total;     // x = m_hist
  const int32_t* hist_nodes;
  const int64_t* node_off;
  const int32_t* ng;        // [m_hist_cap] groups per node
  const int32_t* gstart;    // [m_hist_cap][P+1] first projection of each group
  const int64_t* item_off;  // [m_hist_cap] first item of each node
  const V4* item_total;     // lane: items of this kernel
  int lane;                 // 0: min/max items (x), 1: histogram items (y)
  int64_t S;                // samples per chunk
};

__device__ __forceinline__ int64_t items_total(const StagedPlan& sp) {
  const V4 t = *sp.item_total;
  return sp.lane == 0 ? t.x : t.y;
}

struct ItemPos {
  int64_t h;
  int j;
  int64_t beg, end;
  int p0, np;
};

__device__ __forceinline__ ItemPos decode_item(const StagedPlan& sp, int64_t t, int P) {
  ItemPos r;
  const int64_t m_hist = sp.plan_total->x;
  int64_t lo = 0, hi = m_hist - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (sp.item_off[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  r.h = lo;
  r.j = sp.hist_nodes[lo];
  const int ng = sp.ng[lo];
  const int64_t local = t - sp.item_off[lo];
  const int64_t chunk = local / ng;
  const int g = (int)(local - chunk * ng);
  const int32_t* gs = sp.gstart + lo * (int64_t)(P + 1);
  r.p0 = gs[g];
  r.np = gs[g + 1] - gs[g];
  const int64_t nb = sp.node_off[r.j], ne = sp.node_off[r.j + 1];
  r.beg = nb + chunk * sp.S;
  r.end = min(ne, r.beg + sp.S);
  return r;
}

// ---- feature bitmap -> tile rows --------------------------------------------
// Marks the features of projections [p0, p0+np) of node j, assigns rows in
// ascending feature order and returns U.  The caller syncs before use.
__device__ __forceinline__ int build_rows(const ProjView& pv, int64_t qbase, int np, int d, uint32_t* s_bits,
                                          int* s_wpre, int* s_rowfeat, int* s_misc) {
  const int nw = (d + 31) >> 5;
  for (int w = threadIdx.x; w < nw; w += kStThreads) s_bits[w] = 0u;
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += kStThreads) {
    const int rb = pv.beg[qbase + p];
    int k = pv.end[qbase + p] - rb;
    k = k < 0 ? 0 : (k > kMaxCap ? kMaxCap : k);
    for (int jj = 0; jj < k; ++jj) {
      int f = pv.feat[rb + jj];
      f = (f < 0 || f >= d) ? 0 : f;
      atomicOr(&s_bits[f >> 5], 1u << (f & 31));
    }
  }
  __syncthreads();
  // exclusive prefix of popcounts over the words: each thread a run of words
  const int per = (nw + kStThreads - 1) / kStThreads;
  const int w0 = threadIdx.x * per;
  int own = 0;
  for (int w = w0; w < min(nw, w0 + per); ++w) own += __popc(s_bits[w]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int inc = warp_incl_scan(own, lane);
  if (lane == 31) s_misc[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int v = lane < kStWarps ? s_misc[lane] : 0;
    const int vi = warp_incl_scan(v, lane);
    if (lane < kStWarps) s_misc[lane] = vi - v;
    if (lane == kStWarps - 1) s_misc[kStWarps] = vi;
  }
  __syncthreads();
  int run = s_misc[warp] + inc - own;
  for (int w = w0; w < min(nw, w0 + per); ++w) {
    s_wpre[w] = run;
    run += __popc(s_bits[w]);
  }
  const int U = s_misc[kStWarps];
  __syncthreads();
  if (U <= kStUMax) {
    for (int w = threadIdx.x; w < nw; w += kStThreads) {
      unsigned bits = s_bits[w];
      int r = s_wpre[w];
      while (bits) {
        const int b = __ffs(bits) - 1;
        s_rowfeat[r++] = w * 32 + b;
        bits &= bits - 1u;
      }
    }
  }
  return U;
}

__device__ __forceinline__ int row_of(int f, const uint32_t* s_bits, const int* s_wpre) {
  return s_wpre[f >> 5] + __popc(s_bits[f >> 5] & ((1u << (f & 31)) - 1u));
}

// Projection descriptors of the group in shared memory: k, row of each
// non-zero (ascending feature order), sign as a float multiplier.
template <int KMAX>
__device__ __forceinline__ void build_desc(const ProjView& pv, int64_t qbase, int np, int d, const uint32_t* s_bits,
                                           const int* s_wpre, int* s_dk, int16_t* s_drow, float* s_dsg) {
  for (int e = threadIdx.x; e < np * KMAX; e += kStThreads) {
    const int p = e / KMAX, jj = e - (e / KMAX) * KMAX;
    const int rb = pv.beg[qbase + p];
    int k = pv.end[qbase + p] - rb;
    k = k < 0 ? 0 : (k > KMAX ? KMAX : k);
    if (jj == 0) s_dk[p] = k;
    if (jj < k) {
      int f = pv.feat[rb + jj];
      f = (f < 0 || f >= d) ? 0 : f;
      s_drow[p * KMAX + jj] = (int16_t)row_of(f, s_bits, s_wpre);
      s_dsg[p * KMAX + jj] = pv.sign[rb + jj] == 1 ? 1.0f : -1.0f;
    }
  }
}

// ---- tile staging through registers (prefetch of the next tile) -------------
// Scalar form: thread owns tile column i = tid % St and rows tid/St + k*(NT/St),
// one gather per element.  Vector form (a full tile of consecutive, 16-byte
// aligned samples): thread owns float4 column tid % (St/4).  Threads tid < St
// also fetch the label of tile position tid.
template <int EPT>
struct TileLoader {
  float pre[EPT];
  int ylab;  // label of position tid (tid < St), -1 for padding
  __device__ __forceinline__ void load(const DatasetView& ds, const int32_t* __restrict__ idx, int64_t tbeg,
                                       int64_t tend, int St, int U, const int* s_rowfeat, bool vec) {
    if (vec) {
      const int nq = St >> 2;
      const int q = threadIdx.x & (nq - 1);
      const int r0 = threadIdx.x / nq;
      const int rstep = kStThreads / nq;
      const int64_t sid0 = idx[tbeg];
#pragma unroll
      for (int k = 0; k < EPT / 4; ++k) {
        const int r = r0 + k * rstep;
        if (r < U) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(ds.X + (int64_t)s_rowfeat[r] * ds.ld + sid0) + q);
          pre[4 * k] = v.x;
          pre[4 * k + 1] = v.y;
          pre[4 * k + 2] = v.z;
          pre[4 * k + 3] = v.w;
        }
      }
      if (threadIdx.x < St) ylab = ds.y[sid0 + threadIdx.x];
    } else {
      const int i = threadIdx.x % St;
      const int r0 = threadIdx.x / St;
      const int rstep = kStThreads / St;
      const int64_t pos = tbeg + i;
      const bool valid = pos < tend;
      // padding positions repeat the tile's first sample (min / max unchanged)
      const int64_t sid = safe_sample(idx[valid ? pos : tbeg], ds.n);
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int r = r0 + k * rstep;
        if (r < U) pre[k] = __ldg(ds.X + (int64_t)s_rowfeat[r] * ds.ld + sid);
      }
      if (threadIdx.x < St) ylab = valid ? (int)ds.y[sid] : -1;
    }
  }
  __device__ __forceinline__ void store(float* s_tile, int St, int U, bool vec) const {
    if (vec) {
      const int nq = St >> 2;
      const int q = threadIdx.x & (nq - 1);
      const int r0 = threadIdx.x / nq;
      const int rstep = kStThreads / nq;
#pragma unroll
      for (int k = 0; k < EPT / 4; ++k) {
        const int r = r0 + k * rstep;
        if (r < U)
          reinterpret_cast<float4*>(s_tile + r * St)[q] =
              make_float4(pre[4 * k], pre[4 * k + 1], pre[4 * k + 2], pre[4 * k + 3]);
      }
    } else {
      const int i = threadIdx.x % St;
      const int r0 = threadIdx.x / St;
      const int rstep = kStThreads / St;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int r = r0 + k * rstep;
        if (r < U) s_tile[r * St + i] = pre[k];
      }
    }
  }
};

// Whether the item's samples are one run of consecutive indices that the
// vector form may read directly (all threads call; one barrier).
__device__ __forceinline__ bool item_contiguous(const DatasetView& ds, const int32_t* __restrict__ idx, int64_t beg,
                                                int64_t end) {
  const int64_t first = idx[beg];
  bool ok = first >= 0 && first + (end - beg) <= ds.n && (first & 3) == 0 && (ds.ld & 3) == 0 &&
            ((reinterpret_cast<uintptr_t>(ds.X) & 15) == 0);
  for (int64_t e = beg + threadIdx.x; ok && e < end; e += kStThreads) ok = (idx[e] == first + (e - beg));
  return __syncthreads_and(ok) != 0;
}

template <int EPT>
__device__ __forceinline__ int choose_st(int U) {
  // U * St <= kStThreads * EPT, St in {64, 128, 256}
  if (U * 256 <= kStThreads * EPT) return 256;
  if (U * 128 <= kStThreads * EPT) return 128;
  return 64;
}

// ---- k_groups: greedy projection groups per histogram node -------------------
// One warp per node.  A group is closed before a projection that would push
// its distinct features above umax or its size above pmax.
__global__ void __launch_bounds__(128) k_groups(const V4* plan_total, const int32_t* hist_nodes, ProjView pv, int d,
                                                int umax1, int pmax1, int umax2, int pmax2, int32_t* ng1,
                                                int32_t* gs1, int32_t* ng2, int32_t* gs2) {
  extern __shared__ uint32_t s_grp[];  // per warp: bitmap [nw] + set-word list [kStUMax]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (d + 31) >> 5;
  uint32_t* bits = s_grp + warp * (nw + kStUMax);
  uint32_t* setw = bits + nw;
  for (int w = lane; w < nw; w += 32) bits[w] = 0u;
  __syncwarp();
  const int64_t m_hist = plan_total->x;
  const int P = pv.P;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t h = gw; h < m_hist; h += nwarps) {
    const int64_t j = hist_nodes[h];
    for (int pass = 0; pass < 2; ++pass) {
      const int umax = pass == 0 ? umax1 : umax2;
      const int pmax = pass == 0 ? pmax1 : pmax2;
      int32_t* gs = (pass == 0 ? gs1 : gs2) + h * (int64_t)(P + 1);
      if (d <= umax) {
        // every group fits the tile whatever its features: fixed chunks of pmax
        const int ng = (P + pmax - 1) / pmax;
        for (int g = lane; g <= ng; g += 32) gs[g] = min(g * pmax, P);
        if (lane == 0) (pass == 0 ? ng1 : ng2)[h] = ng;
        continue;
      }
      int U = 0, cnt = 0, nset = 0, g = 0;
      if (lane == 0) gs[0] = 0;
      for (int p = 0; p < P; ++p) {
        const int64_t q = j * P + p;
        const int rb = pv.beg[q];
        int k = pv.end[q] - rb;
        k = k < 0 ? 0 : (k > kMaxCap ? kMaxCap : k);
        int f = 0;
        if (lane < k) {
          f = pv.feat[rb + lane];
          f = (f < 0 || f >= d) ? 0 : f;
        }
        bool fresh = lane < k && !(bits[f >> 5] & (1u << (f & 31)));
        int add = __popc(__ballot_sync(0xffffffffu, fresh));
        if (cnt > 0 && (U + add > umax || cnt + 1 > pmax)) {
          for (int s = lane; s < nset; s += 32) bits[setw[s]] = 0u;
          __syncwarp();
          U = 0;
          cnt = 0;
          nset = 0;
          ++g;
          if (lane == 0) gs[g] = p;
          fresh = lane < k;
          add = __popc(__ballot_sync(0xffffffffu, fresh));
        }
        // set the bits; record words that become non-zero
        bool newword = false;
        if (fresh) {
          const uint32_t old = atomicOr(&bits[f >> 5], 1u << (f & 31));
          newword = (old == 0u);
        }
        // a word may be set by two lanes of the same projection; only the
        // lane that saw it empty records it
        const unsigned nb = __ballot_sync(0xffffffffu, newword);
        if (newword) setw[nset + __popc(nb & ((1u << lane) - 1u))] = (uint32_t)(f >> 5);
        nset += __popc(nb);
        U += add;
        ++cnt;
        __syncwarp();
      }
      for (int s = lane; s < nset; s += 32) bits[setw[s]] = 0u;
      __syncwarp();
      if (lane == 0) {
        gs[g + 1] = P;
        (pass == 0 ? ng1 : ng2)[h] = g + 1;
      }
    }
  }
}

// Item counts per histogram node (scan over node slots; slots >= m_hist are 0).
struct ItemScanF {
  const V4* plan_total;
  const int32_t* hist_nodes;
  const int64_t* off;
  const int32_t* ng1;
  const int32_t* ng2;
  int64_t S;
  int64_t* item_off1;
  int64_t* item_off2;
  __device__ V4 value(int64_t h) const {
    if (h >= plan_total->x) return V4{0, 0, 0, 0};
    const int j = hist_nodes[h];
    const int64_t nv = off[j + 1] - off[j];
    const int64_t ch = (nv + S - 1) / S;
    return V4{ch * ng1[h], ch * ng2[h], 0, 0};
  }
  __device__ void apply(int64_t h, V4 ex) const {
    if (h >= plan_total->x) return;
    item_off1[h] = ex.x;
    item_off2[h] = ex.y;
  }
};

// ---- k_mm_staged: min / max -------------------------------------------------
// Per (projection, tile): the warp of the projection evaluates every sample
// pair of the tile with the projection's rows and signs in registers (the
// loop is specialised on the projection's non-zero count K); per-lane running
// minima and maxima live in shared memory until the item ends.
template <int K, int NPS>
__device__ __forceinline__ void mm_tile(const float* __restrict__ s_tile, const int16_t* drow, const float* dsg,
                                        int St, int lane, float& mn, float& mx) {
  int roff[K];
  float2 sg[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    roff[j] = drow[j] * St + 2 * lane;
    sg[j] = make_float2(dsg[j], dsg[j]);
  }
  // NPS > 0: the St/64 pair-steps are unrolled (St = 64 * NPS); NPS = 0: rolled
  const int nps = NPS > 0 ? NPS : (St >> 6);
#pragma unroll
  for (int q = 0; q < (NPS > 0 ? NPS : 1); ++q) {
    for (int r = 0; r < (NPS > 0 ? 1 : nps); ++r) {
      const int ps = 64 * (NPS > 0 ? q : r);
      float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < K; ++j) acc = ffma2(sg[j], *reinterpret_cast<const float2*>(s_tile + roff[j] + ps), acc);
      mn = fminf(mn, fminf(acc.x, acc.y));
      mx = fmaxf(mx, fmaxf(acc.x, acc.y));
    }
  }
}

// Dispatch on (non-zero count, pair-steps per tile); counts above 16 use the
// rolled form.
template <int KMAX>
__device__ __forceinline__ void mm_tile_k(int k, const float* s_tile, const int16_t* drow, const float* dsg, int St,
                                          int lane, float& mn, float& mx) {
  const int nps = St >> 6;
  const int key = k * 8 + (nps == 4 ? 2 : nps == 2 ? 1 : 0);
  switch (key) {
#define SOF_MM_CASE(N)                                                                                        \
  case N * 8 + 0:                                                                                             \
    if (N <= KMAX) mm_tile<(N <= KMAX ? N : 1), 1>(s_tile, drow, dsg, St, lane, mn, mx);                      \
    return;                                                                                                   \
  case N * 8 + 1:                                                                                             \
    if (N <= KMAX) mm_tile<(N <= KMAX ? N : 1), 2>(s_tile, drow, dsg, St, lane, mn, mx);                      \
    return;                                                                                                   \
  case N * 8 + 2:                                                                                             \
    if (N <= KMAX) mm_tile<(N <= KMAX ? N : 1), 4>(s_tile, drow, dsg, St, lane, mn, mx);                      \
    return;
    SOF_MM_CASE(1) SOF_MM_CASE(2) SOF_MM_CASE(3) SOF_MM_CASE(4) SOF_MM_CASE(5) SOF_MM_CASE(6) SOF_MM_CASE(7)
    SOF_MM_CASE(8) SOF_MM_CASE(9) SOF_MM_CASE(10) SOF_MM_CASE(11) SOF_MM_CASE(12) SOF_MM_CASE(13)
    SOF_MM_CASE(14) SOF_MM_CASE(15) SOF_MM_CASE(16)
#undef SOF_MM_CASE
    default:
      break;
  }
  switch (k) {
#define SOF_MM_ROLLED(N) \
  case N:                \
    if (N <= KMAX) mm_tile<(N <= KMAX ? N : 1), 0>(s_tile, drow, dsg, St, lane, mn, mx); \
    break;
    SOF_MM_ROLLED(17) SOF_MM_ROLLED(18) SOF_MM_ROLLED(19) SOF_MM_ROLLED(20) SOF_MM_ROLLED(21) SOF_MM_ROLLED(22)
    SOF_MM_ROLLED(23) SOF_MM_ROLLED(24) SOF_MM_ROLLED(25) SOF_MM_ROLLED(26) SOF_MM_ROLLED(27) SOF_MM_ROLLED(28)
    SOF_MM_ROLLED(29) SOF_MM_ROLLED(30) SOF_MM_ROLLED(31) SOF_MM_ROLLED(32)
#undef SOF_MM_ROLLED
    default:
      break;
  }
}

template <int KMAX>
__global__ void __launch_bounds__(kStThreads, (KMAX <= 8 ? 2 : 1)) k_mm_staged(DatasetView ds, const int32_t* __restrict__ idx,
                                                            ProjView pv, StagedPlan sp, uint32_t* mm) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  const int nw = (ds.d + 31) >> 5;
  float* s_tile = reinterpret_cast<float*>(s_raw);                       // [kStThreads*kMmEpt]
  float* s_pmin = s_tile + kStThreads * kMmEpt;                          // [kMmGroup*32]
  float* s_pmax = s_pmin + kMmGroup * 32;                                // [kMmGroup*32]
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(s_pmax + kMmGroup * 32);  // [nw]
  int* s_wpre = reinterpret_cast<int*>(s_bits + nw);                     // [nw]
  int* s_rowfeat = s_wpre + nw;                                          // [kStUMax]
  int* s_dk = s_rowfeat + kStUMax;                                       // [kMmGroup]
  float* s_dsg = reinterpret_cast<float*>(s_dk + kMmGroup);              // [kMmGroup*KMAX]
  int16_t* s_drow = reinterpret_cast<int16_t*>(s_dsg + kMmGroup * KMAX); // [kMmGroup*KMAX]
  __shared__ int s_misc[kStWarps + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = pv.P;
  const int64_t n_items = items_total(sp);
  for (int64_t t = blockIdx.x; t < n_items; t += gridDim.x) {
    const ItemPos it = decode_item(sp, t, P);
    const int64_t qbase = (int64_t)it.j * P + it.p0;
    __syncthreads();  // previous item done with shared memory
    const int U = build_rows(pv, qbase, it.np, ds.d, s_bits, s_wpre, s_rowfeat, s_misc);
    build_desc<KMAX>(pv, qbase, it.np, ds.d, s_bits, s_wpre, s_dk, s_drow, s_dsg);
    for (int e = threadIdx.x; e < it.np * 32; e += kStThreads) {
      s_pmin[e] = INFINITY;
      s_pmax[e] = -INFINITY;
    }
    const bool contig = item_contiguous(ds, idx, it.beg, it.end);  // includes a barrier
    if (U <= kMmUMax) {
      const int St = choose_st<kMmEpt>(U);
      const int64_t len = it.end - it.beg;
      const int64_t ntile = (len + St - 1) / St;
      TileLoader<kMmEpt> ld;
      bool vec = contig && len >= St;
      ld.load(ds, idx, it.beg, it.end, St, U, s_rowfeat, vec);
      for (int64_t tt = 0; tt < ntile; ++tt) {
        __syncthreads();
        ld.store(s_tile, St, U, vec);
        __syncthreads();
        if (tt + 1 < ntile) {
          const int64_t nb = it.beg + (tt + 1) * St;
          vec = contig && (it.end - nb) >= St;
          ld.load(ds, idx, nb, min(it.end, nb + St), St, U, s_rowfeat, vec);
        }
        for (int pl = warp; pl < it.np; pl += kStWarps) {
          float mn = s_pmin[pl * 32 + lane], mx = s_pmax[pl * 32 + lane];
          mm_tile_k<KMAX>(s_dk[pl], s_tile, s_drow + pl * KMAX, s_dsg + pl * KMAX, St, lane, mn, mx);
          s_pmin[pl * 32 + lane] = mn;
          s_pmax[pl * 32 + lane] = mx;
        }
      }
    } else {
      // direct path for wide groups: each warp gathers its projections' features
      for (int pl = warp; pl < it.np; pl += kStWarps) {
        const int64_t q = qbase + pl;
        const int rb = pv.beg[q];
        int k = pv.end[q] - rb;
        k = k < 0 ? 0 : (k > kMaxCap ? kMaxCap : k);
        float mn = INFINITY, mx = -INFINITY;
        for (int64_t e = it.beg + lane; e < it.end; e += 32) {
          const int64_t s = safe_sample(idx[e], ds.n);
          float acc = 0.0f;
          for (int jj = 0; jj < k; ++jj) {
            int f = pv.feat[rb + jj];
            f = (f < 0 || f >= ds.d) ? 0 : f;
            const float x = __ldg(ds.X + (int64_t)f * ds.ld + s);
            acc = __fadd_rn(acc, pv.sign[rb + jj] == 1 ? x : -x);
          }
          mn = fminf(mn, acc);
          mx = fmaxf(mx, acc);
        }
        s_pmin[pl * 32 + lane] = mn;
        s_pmax[pl * 32 + lane] = mx;
      }
    }
    __syncthreads();
    for (int pl = warp; pl < it.np; pl += kStWarps) {
      const float a = warp_min(s_pmin[pl * 32 + lane]), b = warp_max(s_pmax[pl * 32 + lane]);
      if (lane == 0) {
        atomicMin(&mm[(it.h * P + it.p0 + pl) * 2], f2key(a));
        atomicMax(&mm[(it.h * P + it.p0 + pl) * 2 + 1], f2key(b));
      }
    }
  }
}

// ---- k_hist_staged: class-count histograms -----------------------------------
// Histogram layout in shared memory: [pl][B+1][C] int32, one spare bin per
// projection, then a trash word.  Addresses are byte offsets clamped (as
// unsigned) to the trash word, which absorbs padding positions (label offset
// very negative), labels outside [0, C) and non-finite projected values.
struct BinParams {
  float mn, W, inv_w, c;
  unsigned hb;  // byte base of the projection's histogram minus magic*C*4 (mod 2^32)
  int fast;
};

template <int K, int NPS>
__device__ __forceinline__ void hist_tile(const float* __restrict__ s_tile, const int* __restrict__ s_y4,
                                          const int16_t* drow, const float* dsg, int St, int lane, const BinParams& bp,
                                          unsigned C4, unsigned limit, char* s_histb) {
  int roff[K];
  float2 sg[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    roff[j] = drow[j] * St + 2 * lane;
    sg[j] = make_float2(dsg[j], dsg[j]);
  }
  const float2 inv2 = make_float2(bp.inv_w, bp.inv_w);
  const float2 c2 = make_float2(bp.c, bp.c);
  const float2 m2 = make_float2(kMagic, kMagic);
  const float2 m1 = make_float2(1.0f - kMagic, 1.0f - kMagic);
  const int nps = NPS > 0 ? NPS : (St >> 6);
#pragma unroll
  for (int q = 0; q < (NPS > 0 ? NPS : 1); ++q) {
    for (int r = 0; r < (NPS > 0 ? 1 : nps); ++r) {
      const int ps = 64 * (NPS > 0 ? q : r);
      float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int j = 0; j < K; ++j) acc = ffma2(sg[j], *reinterpret_cast<const float2*>(s_tile + roff[j] + ps), acc);
      const int2 y4 = *reinterpret_cast<const int2*>(s_y4 + ps + 2 * lane);
      const float2 e = ffma2(acc, inv2, c2);
      const float2 tq = fadd2(e, m2);
      const float2 q1 = fadd2(tq, m1);
      // t_{q+1} = min + (q+1)*W with two roundings (scalar: not fused)
      const float tbx = __fadd_rn(bp.mn, __fmul_rn(q1.x, bp.W));
      const float tby = __fadd_rn(bp.mn, __fmul_rn(q1.y, bp.W));
      unsigned ax = __float_as_uint(tq.x) * C4 + (bp.hb + (unsigned)y4.x);
      unsigned ay = __float_as_uint(tq.y) * C4 + (bp.hb + (unsigned)y4.y);
      if (tbx <= acc.x) ax += C4;
      if (tby <= acc.y) ay += C4;
      ax = min(ax, limit);
      ay = min(ay, limit);
      atomicAdd(reinterpret_cast<int*>(s_histb + ax), 1);
      atomicAdd(reinterpret_cast<int*>(s_histb + ay), 1);
    }
  }
}

template <int KMAX>
__device__ __forceinline__ void hist_tile_k(int k, const float* s_tile, const int* s_y4, const int16_t* drow,
                                            const float* dsg, int St, int lane, const BinParams& bp, unsigned C4,
                                            unsigned limit, char* s_histb) {
  const int nps = St >> 6;
  const int key = k * 8 + (nps == 4 ? 2 : nps == 2 ? 1 : 0);
  switch (key) {
#define SOF_H_CASE(N)                                                                                               \
  case N * 8 + 0:                                                                                                   \
    if (N <= KMAX) hist_tile<(N <= KMAX ? N : 1), 1>(s_tile, s_y4, drow, dsg, St, lane, bp, C4, limit, s_histb);    \
    return;                                                                                                         \
  case N * 8 + 1:                                                                                                   \
    if (N <= KMAX) hist_tile<(N <= KMAX ? N : 1), 2>(s_tile, s_y4, drow, dsg, St, lane, bp, C4, limit, s_histb);    \
    return;                                                                                                         \
  case N * 8 + 2:                                                                                                   \
    if (N <= KMAX) hist_tile<(N <= KMAX ? N : 1), 4>(s_tile, s_y4, drow, dsg, St, lane, bp, C4, limit, s_histb);    \
    return;
    SOF_H_CASE(1) SOF_H_CASE(2) SOF_H_CASE(3) SOF_H_CASE(4) SOF_H_CASE(5) SOF_H_CASE(6) SOF_H_CASE(7)
    SOF_H_CASE(8) SOF_H_CASE(9) SOF_H_CASE(10) SOF_H_CASE(11) SOF_H_CASE(12) SOF_H_CASE(13) SOF_H_CASE(14)
    SOF_H_CASE(15) SOF_H_CASE(16)
#undef SOF_H_CASE
    default:
      break;
  }
  switch (k) {
#define SOF_H_ROLLED(N) \
  case N:               \
    if (N <= KMAX) hist_tile<(N <= KMAX ? N : 1), 0>(s_tile, s_y4, drow, dsg, St, lane, bp, C4, limit, s_histb); \
    break;
    SOF_H_ROLLED(17) SOF_H_ROLLED(18) SOF_H_ROLLED(19) SOF_H_ROLLED(20) SOF_H_ROLLED(21) SOF_H_ROLLED(22)
    SOF_H_ROLLED(23) SOF_H_ROLLED(24) SOF_H_ROLLED(25) SOF_H_ROLLED(26) SOF_H_ROLLED(27) SOF_H_ROLLED(28)
    SOF_H_ROLLED(29) SOF_H_ROLLED(30) SOF_H_ROLLED(31) SOF_H_ROLLED(32)
#undef SOF_H_ROLLED
    default:
      break;
  }
}

// exact estimate-and-correct rule for projections outside the fast condition
__device__ __forceinline__ void hist_tile_slow(int k, const float* __restrict__ s_tile, const int* __restrict__ s_y4,
                                               const int16_t* drow, const float* dsg, int St, int lane,
                                               const BinParams& bp, int B, int C, int hbase, int32_t* s_hist) {
  for (int i = lane; i < St; i += 32) {
    float acc = 0.0f;
    for (int j = 0; j < k; ++j) acc = __fmaf_rn(dsg[j], s_tile[drow[j] * St + i], acc);
    const int y4 = s_y4[i];
    if (y4 >= 0) atomicAdd(&s_hist[hbase + bin_of(acc, bp.mn, bp.W, bp.inv_w, B) * C + (y4 >> 2)], 1);
  }
}

template <int KMAX>
__global__ void __launch_bounds__(kStThreads, 1) k_hist_staged(DatasetView ds, const int32_t* __restrict__ idx,
                                                              ProjView pv, StagedPlan sp, int B, int PG,
                                                              const uint32_t* __restrict__ mm, int32_t* hist) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  const int nw = (ds.d + 31) >> 5;
  const int C = ds.C;
  const int HS = (B + 1) * C;  // words per projection histogram
  const int hist_words = ((PG * HS + 1) + 3) & ~3;
  // every region starts on a 16-byte boundary (s_y4 is read as int2)
  float* s_tile = reinterpret_cast<float*>(s_raw);                        // [kStThreads*kStEpt]
  int* s_y4 = reinterpret_cast<int*>(s_tile + kStThreads * kStEpt);       // [256] label byte offset
  int32_t* s_hist = s_y4 + 256;                                           // [PG*HS + 1 (trash)]
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(s_hist + hist_words);    // [nw]
  int* s_wpre = reinterpret_cast<int*>(s_bits + nw);                      // [nw]
  int* s_rowfeat = s_wpre + nw;                                           // [kStUMax]
  int* s_dk = s_rowfeat + kStUMax;                                        // [32]
  float* s_dsg = reinterpret_cast<float*>(s_dk + 32);                     // [32*KMAX]
  int16_t* s_drow = reinterpret_cast<int16_t*>(s_dsg + 32 * KMAX);        // [32*KMAX]
  __shared__ int s_misc[kStWarps + 1];
  __shared__ BinParams s_bp[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = pv.P;
  const unsigned C4 = (unsigned)C * 4u;
  const unsigned limit = (unsigned)(PG * HS) * 4u;  // byte offset of the trash word
  const unsigned magic_bits = __float_as_uint(kMagic);
  char* s_histb = reinterpret_cast<char*>(s_hist);
  const int64_t n_items = items_total(sp);
  for (int64_t t = blockIdx.x; t < n_items; t += gridDim.x) {
    const ItemPos it = decode_item(sp, t, P);
    const int64_t qbase = (int64_t)it.j * P + it.p0;
    __syncthreads();  // previous item's flush finished
    {
      int4* h4 = reinterpret_cast<int4*>(s_hist);
      for (int e = threadIdx.x; e < hist_words / 4; e += kStThreads) h4[e] = make_int4(0, 0, 0, 0);
    }
    const int U = build_rows(pv, qbase, it.np, ds.d, s_bits, s_wpre, s_rowfeat, s_misc);
    build_desc<KMAX>(pv, qbase, it.np, ds.d, s_bits, s_wpre, s_dk, s_drow, s_dsg);
    if (threadIdx.x < it.np) {
      const int pl = threadIdx.x;
      const float mn = key2f(mm[(it.h * P + it.p0 + pl) * 2]);
      const float mx = key2f(mm[(it.h * P + it.p0 + pl) * 2 + 1]);
      BinParams bp;
      bp.mn = mn;
      bp.W = bin_width(mn, mx, B);
      bp.inv_w = __frcp_rn(bp.W);
      bp.c = __fsub_rn(__fmul_rn(-mn, bp.inv_w), 0.75f);
      const float M = fmaxf(fabsf(mn), fabsf(mx));
      bp.fast = (bp.W > 0.0f && isfinite(bp.inv_w) && isfinite(bp.c) && M <= kCondLimit * bp.W) ? 1 : 0;
      bp.hb = (unsigned)(pl * HS * 4) - magic_bits * C4;
      s_bp[pl] = bp;
    }
    const bool contig = item_contiguous(ds, idx, it.beg, it.end);  // includes a barrier
    const int64_t len = it.end - it.beg;
    if (U <= kStUMax) {
      const int St = choose_st<kStEpt>(U);
      const int64_t ntile = (len + St - 1) / St;
      TileLoader<kStEpt> ld;
      bool vec = contig && len >= St;
      ld.load(ds, idx, it.beg, it.end, St, U, s_rowfeat, vec);
      for (int64_t tt = 0; tt < ntile; ++tt) {
        __syncthreads();
        ld.store(s_tile, St, U, vec);
        if (threadIdx.x < St) {
          // labels outside [0, C) and padding: a very negative offset that the
          // unsigned clamp sends to the trash word
          s_y4[threadIdx.x] = (ld.ylab >= 0 && ld.ylab < C) ? ld.ylab * 4 : (INT_MIN / 2);
        }
        __syncthreads();
        if (tt + 1 < ntile) {
          const int64_t nb = it.beg + (tt + 1) * St;
          vec = contig && (it.end - nb) >= St;
          ld.load(ds, idx, nb, min(it.end, nb + St), St, U, s_rowfeat, vec);
        }
        for (int pl = warp; pl < it.np; pl += kStWarps) {
          const BinParams bp = s_bp[pl];
          if (bp.fast)
            hist_tile_k<KMAX>(s_dk[pl], s_tile, s_y4, s_drow + pl * KMAX, s_dsg + pl * KMAX, St, lane, bp, C4, limit,
                              s_histb);
          else
            hist_tile_slow(s_dk[pl], s_tile, s_y4, s_drow + pl * KMAX, s_dsg + pl * KMAX, St, lane, bp, B, C, pl * HS,
                           s_hist);
        }
      }
    } else {
      // direct path for wide groups (rare): one warp per projection, gathers
      for (int pl = warp; pl < it.np; pl += kStWarps) {
        const int64_t q = qbase + pl;
        const int rb = pv.beg[q];
        int k = pv.end[q] - rb;
        k = k < 0 ? 0 : (k > kMaxCap ? kMaxCap : k);
        const BinParams bp = s_bp[pl];
        for (int64_t e = it.beg + lane; e < it.end; e += 32) {
          const int64_t s = safe_sample(idx[e], ds.n);
          float acc = 0.0f;
          for (int jj = 0; jj < k; ++jj) {
            int f = pv.feat[rb + jj];
            f = (f < 0 || f >= ds.d) ? 0 : f;
            const float x = __ldg(ds.X + (int64_t)f * ds.ld + s);
            acc = __fadd_rn(acc, pv.sign[rb + jj] == 1 ? x : -x);
          }
          const int yv = ds.y[s];
          if (yv < C) atomicAdd(&s_hist[pl * HS + bin_of(acc, bp.mn, bp.W, bp.inv_w, B) * C + yv], 1);
        }
      }
    }
    __syncthreads();
    // flush: the spare bin B folds into bin B-1
    const int BC = B * C;
    for (int pl = warp; pl < it.np; pl += kStWarps) {
      int32_t* g = hist + (it.h * P + it.p0 + pl) * (int64_t)BC;
      const int32_t* h = s_hist + pl * HS;
      for (int r = lane; r < BC; r += 32) {
        int v = h[r];
        if (r >= BC - C) v += h[r + C];
        if (v) atomicAdd(&g[r], v);
      }
    }
  }
}

// ---- host side ----------------------------------------------------------------
int hist_group_size(int B, int C) {
  // histogram shared memory <= 100 KB: PG * (B + 1) * C * 4
  int pg = 32;
  while (pg > 1 && (size_t)pg * (B + 1) * C * 4 > 100 * 1024) pg >>= 1;
  return pg;
}

size_t mm_smem_bytes(int d, int kmax) {
  const int nw = (d + 31) >> 5;
  return (size_t)kStThreads * kMmEpt * 4 + (size_t)kMmGroup * 32 * 8 + (size_t)nw * 8 + kStUMax * 4 +
         kMmGroup * 4 + (size_t)kMmGroup * kmax * 6 + 64;
}
size_t hist_smem_bytes(int d, int kmax, int B, int C, int PG) {
  const int nw = (d + 31) >> 5;
  const size_t hist_words = ((size_t)PG * (B + 1) * C + 1 + 3) & ~(size_t)3;
  return (size_t)kStThreads * kStEpt * 4 + 256 * 4 + hist_words * 4 + (size_t)nw * 8 + kStUMax * 4 + 32 * 4 +
         (size_t)32 * kmax * 6 + 64;
}

bool staged_supported(int d) { return d <= kStMaxWords * 32; }

void carve_staged(Carver& cv, StagedScratch& s, int64_t m_hist_cap, int P) {
  s.ng1 = cv.take<int32_t>(m_hist_cap);
  s.gs1 = cv.take<int32_t>(m_hist_cap * (P + 1));
  s.ng2 = cv.take<int32_t>(m_hist_cap);
  s.gs2 = cv.take<int32_t>(m_hist_cap * (P + 1));
  s.item_off1 = cv.take<int64_t>(m_hist_cap + 1);
  s.item_off2 = cv.take<int64_t>(m_hist_cap + 1);
  s.item_total = cv.take<V4>(1);
  s.tiles = cv.take<V4>(scan_tiles_for(m_hist_cap) + 1);
}

template <int KMAX>
cudaError_t launch_staged_k(const SearchArgs& a, const V4* plan_total, const int32_t* hist_nodes, int64_t m_hist_cap,
                            const StagedScratch& ss, uint32_t* mm, int32_t* hist, int64_t S, cudaStream_t st) {
  const DeviceInfo& di = device_info();
  const int P = a.pv.P, C = a.ds.C, B = a.B, d = a.ds.d;
  const int PG = hist_group_size(B, C);
  cudaError_t e;
  {
    const size_t smem = (size_t)4 * (((d + 31) >> 5) + kStUMax) * 4;
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_groups, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    ProfScope ps_("k_groups", st);
    k_groups<<<di.num_sms * 2, 128, smem, st>>>(plan_total, hist_nodes, a.pv, d, kMmUMax, kMmGroup, kStUMax, PG,
                                                ss.ng1, ss.gs1, ss.ng2, ss.gs2);
  }
  ItemScanF isf{plan_total, hist_nodes, a.node_off, ss.ng1, ss.ng2, S, ss.item_off1, ss.item_off2};
  e = run_scan(isf, m_hist_cap, ss.tiles, ss.item_total, st, "item_scan");
  if (e != cudaSuccess) return e;
  StagedPlan sp1{plan_total, hist_nodes, a.node_off, ss.ng1, ss.gs1, ss.item_off1, ss.item_total, 0, S};
  StagedPlan sp2{plan_total, hist_nodes, a.node_off, ss.ng2, ss.gs2, ss.item_off2, ss.item_total, 1, S};
  {
    const size_t smem = mm_smem_bytes(d, KMAX);
    e = cudaFuncSetAttribute(k_mm_staged<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mm_staged<KMAX>, kStThreads, smem);
    if (occ < 1) occ = 1;
    ProfScope ps_("k_minmax", st);
    k_mm_staged<KMAX><<<di.num_sms * occ, kStThreads, smem, st>>>(a.ds, a.idx, a.pv, sp1, mm);
  }
  {
    const size_t smem = hist_smem_bytes(d, KMAX, B, C, PG);
    e = cudaFuncSetAttribute(k_hist_staged<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope ps_("k_hist", st);
    k_hist_staged<KMAX><<<di.num_sms, kStThreads, smem, st>>>(a.ds, a.idx, a.pv, sp2, B, PG, mm, hist);
  }
  return cudaGetLastError();
}

cudaError_t launch_staged(const SearchArgs& a, const V4* plan_total, const int32_t* hist_nodes, int64_t m_hist_cap,
                          const StagedScratch& ss, uint32_t* mm, int32_t* hist, int64_t S, int kmax,
                          cudaStream_t st) {
  if (kmax <= 8) return launch_staged_k<8>(a, plan_total, hist_nodes, m_hist_cap, ss, mm, hist, S, st);
  if (kmax <= 16) return launch_staged_k<16>(a, plan_total, hist_nodes, m_hist_cap, ss, mm, hist, S, st);
  return launch_staged_k<32>(a, plan_total, hist_nodes, m_hist_cap, ss, mm, hist, S, st);
}

}  // namespace sof
