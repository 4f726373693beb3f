// so_sort_warp.cu -- exact path (Section 3.1: small nodes are split exactly by
// sorting).
//
// Pass 1, per (node, projection): gather the node's projected values and sort
// the (order-preserving key, label) pairs -- one warp in registers for nodes
// of up to kSortRegMax samples (bitonic network, lane-major layout
// e = lane*EPL + r), one CTA in shared memory for larger exact-path nodes
// (a bitonic network up to kScBitonicMax samples, a segmented radix sort of
// the value keys above) -- form class prefix counts with a packed scan, evaluate the float key of the
// criterion at every boundary between distinct values and keep the
// projection's float maximum M_p.  k_sort_node_thr then sets each node's
// window below M = max_p M_p, and a second pass redoes only the projections
// with M_p inside it (the only ones the selection reads; the double re-score
// is the costly part on this GPU), re-scoring in double every candidate
// within the window below its own M_p (Gini: M_p(1-eps); information gain:
// an absolute bound of the key's error) and storing the projection's
// lexicographic best (double gain, lowest position).
// Pass 2 (k_sortw_select): one warp per node takes M = max_p M_p and the
// lexicographic best (gain, projection, position) over the projections whose
// M_p lies in the same window below M.  The double winner of the node is
// always in its projection's re-score set (M >= M_p), and every projection
// holding a double tie of it has M_p inside the window, because the window
// exceeds twice the key's error (Gini: eps above three times its relative
// error; information gain: three times its absolute bound), so the result
// equals the double argmax.
#include <climits>

#include "so_device.cuh"
#include "so_internal.h"

namespace sof {

namespace {

struct PackedCnt {
  unsigned long long lo, hi;  // 16-bit class counters: classes 0-3 in lo, 4-7 in hi
};
__device__ __forceinline__ void pc_add(PackedCnt& a, int y) {
  if (y < 4) a.lo += 1ull << (16 * y);
  else if (y < kMaxClasses) a.hi += 1ull << (16 * (y - 4));
}
__device__ __forceinline__ int pc_get(const PackedCnt& a, int c) {
  return (int)(((c < 4) ? (a.lo >> (16 * c)) : (a.hi >> (16 * (c - 4)))) & 0xFFFFull);
}

template <int EPL>
__device__ __forceinline__ void cmpswap(unsigned long long (&k)[EPL], int r, int rp, bool up) {
  const unsigned long long a = k[r], b = k[rp];
  const bool sw = (a > b) == up;
  k[r] = sw ? b : a;
  k[rp] = sw ? a : b;
}

// Bitonic sort of 32*EPL keys, element e = lane*EPL + r, ascending.
template <int EPL>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&k)[EPL], int lane) {
  constexpr int NP = 32 * EPL;
#pragma unroll
  for (int size = 2; size <= NP; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride < EPL) {
#pragma unroll
        for (int r = 0; r < EPL; ++r) {
          const int rp = r ^ stride;
          if (rp > r) {
            const int e = lane * EPL + r;
            cmpswap<EPL>(k, r, rp, (e & size) == 0);
          }
        }
      } else {
        const int ls = stride / EPL;
        const bool lower = (lane & ls) == 0;
#pragma unroll
        for (int r = 0; r < EPL; ++r) {
          const unsigned long long o = __shfl_xor_sync(0xffffffffu, k[r], ls);
          const int e = lane * EPL + r;
          const bool up = (e & size) == 0;
          const unsigned long long mn = k[r] < o ? k[r] : o;
          const unsigned long long mx = k[r] < o ? o : k[r];
          k[r] = (lower == up) ? mn : mx;
        }
      }
    }
  }
}

struct SortNodeCtx {
  int64_t beg;
  int nv;
  int N[kMaxClasses];
};

// Loads, projects and sorts one projection of one node; returns the lane's
// keys in k[] (padding keys are all-ones and sort last).  RM: gather from the
// row-major copy ds.Xr (the node's projections then share its samples' rows
// through L2) instead of one sector per (sample, feature) of the columns.
template <int EPL, int RM>
__device__ __forceinline__ void load_sort(const DatasetView& ds, const int32_t* __restrict__ idx, const ProjView& pv,
                                          int64_t q, const SortNodeCtx& nc, int lane, unsigned long long (&k)[EPL]) {
  const int rb = pv.beg[q];
  int kk = pv.end[q] - rb;
  kk = kk < 0 ? 0 : (kk > kMaxCap ? kMaxCap : kk);
  int fl = 0, sl = 1;
  if (lane < kk) {
    fl = pv.feat[rb + lane];
    fl = (fl < 0 || fl >= ds.d) ? 0 : fl;
    sl = pv.sign[rb + lane];
  }
  int32_t sid[EPL];
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    const int e = lane * EPL + r;
    sid[r] = e < nc.nv ? (int32_t)safe_sample(idx[nc.beg + e], ds.n) : -1;
  }
  float v[EPL];
#pragma unroll
  for (int r = 0; r < EPL; ++r) v[r] = 0.0f;
  // four terms' gathers in flight at a time, added in order
  for (int j0 = 0; j0 < kk; j0 += 4) {
    float x[4][EPL];
    int sg[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int jj = j0 + u < kk ? j0 + u : j0;
      const int f = __shfl_sync(0xffffffffu, fl, jj);
      sg[u] = __shfl_sync(0xffffffffu, sl, jj);
      const float* col = RM ? ds.Xr + f : ds.X + (int64_t)f * ds.ld;
#pragma unroll
      for (int r = 0; r < EPL; ++r)
        x[u][r] = (j0 + u < kk && sid[r] >= 0) ? __ldg(col + (RM ? (int64_t)sid[r] * ds.d : (int64_t)sid[r])) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (j0 + u < kk) {
#pragma unroll
        for (int r = 0; r < EPL; ++r)
          if (sid[r] >= 0) v[r] = __fadd_rn(v[r], sg[u] == 1 ? x[u][r] : -x[u][r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    if (sid[r] >= 0) {
      const int yv = ds.y[sid[r]];
      k[r] = ((unsigned long long)f2key(v[r]) << 32) | (unsigned long long)(unsigned)yv;
    } else {
      k[r] = ~0ull;
    }
  }
  warp_bitonic<EPL>(k, lane);
}

// Walks the sorted keys; calls visit(e, run, g32, a, b) for every candidate e
// (a boundary between distinct values a < b), run = packed class counts of
// positions 0..e.
template <int EPL, class Visit>
__device__ __forceinline__ void scan_candidates(const unsigned long long (&k)[EPL], const SortNodeCtx& nc, int C,
                                                const Crit& cr, int lane, Visit visit) {
  PackedCnt own{0, 0};
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    const int e = lane * EPL + r;
    if (e < nc.nv) pc_add(own, (int)(k[r] & 0xFFull));
  }
  unsigned long long ilo = own.lo, ihi = own.hi;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long ul = __shfl_up_sync(0xffffffffu, ilo, o);
    const unsigned long long uh = __shfl_up_sync(0xffffffffu, ihi, o);
    if (lane >= o) {
      ilo += ul;
      ihi += uh;
    }
  }
  PackedCnt run{ilo - own.lo, ihi - own.hi};
  // the key right after this lane's last element: the next lane's first
  const unsigned next_first = (unsigned)(__shfl_down_sync(0xffffffffu, k[0], 1) >> 32);
#pragma unroll
  for (int r = 0; r < EPL; ++r) {
    const int e = lane * EPL + r;
    if (e < nc.nv) pc_add(run, (int)(k[r] & 0xFFull));
    if (e < nc.nv - 1) {
      const unsigned a = (unsigned)(k[r] >> 32);
      const unsigned b = (r + 1 < EPL) ? (unsigned)(k[(r + 1) < EPL ? r + 1 : r] >> 32) : next_first;
      if (a != b) {
        int L[kMaxClasses];
#pragma unroll
        for (int c = 0; c < kMaxClasses; ++c) L[c] = pc_get(run, c);
        visit(e, run, key32s(cr, L, nc.N, C, nc.nv, e + 1), a, b);
      }
    }
  }
}

// Node context from its offsets and the class counts computed once per node.
__device__ __forceinline__ void node_ctx_j(const int64_t* off, int j, const int32_t* __restrict__ node_cls,
                                           SortNodeCtx& nc) {
  nc.beg = off[j];
  nc.nv = (int)(off[j + 1] - nc.beg);
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) nc.N[c] = node_cls[(int64_t)j * kMaxClasses + c];
}
__device__ __forceinline__ void node_ctx(const int64_t* off, const int32_t* nodes, int64_t s,
                                         const int32_t* __restrict__ node_cls, SortNodeCtx& nc, int& j) {
  j = nodes[s];
  nc.beg = off[j];
  nc.nv = (int)(off[j + 1] - nc.beg);
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) nc.N[c] = node_cls[(int64_t)j * kMaxClasses + c];
}

// Per-(node, projection) result of pass 1.
struct SortRes {
  double g64;             // best double gain of the projection (-1: none)
  float m32;              // float maximum of the projection (-1: no candidate)
  int cand;               // sorted position of the best candidate
  unsigned ka, kb;        // keys of the values around the boundary
  unsigned long long llo, lhi;  // packed left class counts
};

struct Best {
  Cand c;
  unsigned ka, kb;
  PackedCnt L;  // class counts of the left side
};

__device__ __forceinline__ void best_reduce(Best& lb) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Best other;
    other.c.g = __shfl_xor_sync(0xffffffffu, lb.c.g, o);
    other.c.proj = __shfl_xor_sync(0xffffffffu, lb.c.proj, o);
    other.c.cand = __shfl_xor_sync(0xffffffffu, lb.c.cand, o);
    other.ka = __shfl_xor_sync(0xffffffffu, lb.ka, o);
    other.kb = __shfl_xor_sync(0xffffffffu, lb.kb, o);
    other.L.lo = __shfl_xor_sync(0xffffffffu, lb.L.lo, o);
    other.L.hi = __shfl_xor_sync(0xffffffffu, lb.L.hi, o);
    if (better(other.c, lb.c)) lb = other;
  }
}

// Both sweeps of pass 1 over an already sorted projection, through a
// candidate walker walk(visit); writes the projection's SortRes.
template <class Walk>
__device__ __forceinline__ void score_projection(const SortNodeCtx& nc, int C, const Crit& cr, int lane, Walk walk,
                                                 bool rescore, SortRes* out) {
  float m = key_none(cr);
  walk([&](int, const PackedCnt&, float g, unsigned, unsigned) { m = fmaxf(m, g); });
  m = warp_max(m);
  Best lb;
  lb.c = Cand{-1.0, INT_MAX, INT_MAX};
  lb.ka = lb.kb = 0u;
  lb.L = PackedCnt{0, 0};
  if (rescore && key_any(cr, m)) {
    const float thr = key_thr(cr, m, nc.nv, C);
    walk([&](int e, const PackedCnt& run, float g, unsigned a, unsigned b) {
      if (g >= thr) {
        int L[kMaxClasses];
#pragma unroll
        for (int cc = 0; cc < kMaxClasses; ++cc) L[cc] = pc_get(run, cc);
        const Cand c{gain64s(cr, L, nc.N, C, nc.nv, e + 1), 0, e};
        if (better(c, lb.c)) {
          lb.c = c;
          lb.ka = a;
          lb.kb = b;
          lb.L = run;
        }
      }
    });
    best_reduce(lb);
  }
  if (lane == 0) {
    SortRes r;
    r.m32 = m;
    r.g64 = lb.c.g;
    r.cand = lb.c.cand;
    r.ka = lb.ka;
    r.kb = lb.kb;
    r.llo = lb.L.lo;
    r.lhi = lb.L.hi;
    *out = r;
  }
}

template <int EPL, int RM>
__device__ __forceinline__ void proj_pass1_reg(const DatasetView& ds, const int32_t* idx, const ProjView& pv, int64_t q,
                                               const SortNodeCtx& nc, int lane, const Crit& cr, bool rescore,
                                               SortRes* out) {
  unsigned long long k[EPL];
  load_sort<EPL, RM>(ds, idx, pv, q, nc, lane, k);
  score_projection(nc, ds.C, cr, lane, [&](auto visit) { scan_candidates<EPL>(k, nc, ds.C, cr, lane, visit); },
                   rescore, out);
}

__device__ __forceinline__ int epl_of(int nv) { return nv <= 32 ? 1 : nv <= 64 ? 2 : 4; }

}  // namespace

// Pass 1, register form: one warp per (node of <= kSortRegMax samples,
// projection).  ENT fixes the criterion at compile time, so the Gini form
// carries none of the information gain's code.  With node_thr null the pass
// keeps only each projection's float maximum; with node_thr it redoes, with
// the double re-score, only the projections whose maximum reaches their
// node's window (listed by k_sort_node_thr) -- the only ones the selection
// reads.
template <int ENT, int RM>
__global__ void __launch_bounds__(256, 4) k_sortw_scan(DatasetView ds, const int32_t* __restrict__ idx,
                                                       const int64_t* __restrict__ off, ProjView pv,
                                                       const V4* plan_total, const int32_t* nodes,
                                                       const int32_t* __restrict__ node_cls, Crit cr_in,
                                                       SortRes* res, const int64_t* __restrict__ list,
                                                       const int32_t* __restrict__ list_n) {
  Crit cr = cr_in;
  cr.ent = ENT;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int P = pv.P;
  const bool rescore = list != nullptr;
  const int64_t total = rescore ? (int64_t)*list_n : plan_total->y * P;
  for (int64_t t = gw; t < total; t += nw) {
    SortNodeCtx nc;
    int j, p;
    if (rescore) {
      const int64_t q = list[t];
      j = (int)(q / P);
      p = (int)(q - (int64_t)j * P);
      node_ctx_j(off, j, node_cls, nc);
    } else {
      const int64_t s = t / P;
      p = (int)(t - s * P);
      node_ctx(off, nodes, s, node_cls, nc, j);
    }
    const int64_t q = (int64_t)j * P + p;
    SortRes* out = res + q;
    switch (epl_of(nc.nv)) {
      case 1: proj_pass1_reg<1, RM>(ds, idx, pv, q, nc, lane, cr, rescore, out); break;
      case 2: proj_pass1_reg<2, RM>(ds, idx, pv, q, nc, lane, cr, rescore, out); break;
      default: proj_pass1_reg<4, RM>(ds, idx, pv, q, nc, lane, cr, rescore, out); break;
    }
  }
}

// Pass 1, CTA form: one CTA of kScThreads per (node of kSortRegMax+1 .. T-1
// samples, projection).  The node's projected values are gathered by the
// whole CTA (each thread up to NP/kScThreads samples, the projection's terms
// four at a time), sorted in shared memory (nodes of up to kScBitonicMax
// samples as (key, label) pairs by a bitonic network, larger ones by value
// key with a segmented radix sort, sc_radix), and scanned in per-thread
// chunks of consecutive sorted positions with a block-wide exclusive scan of
// the packed class counters.
constexpr int kScThreads = 128;
constexpr int kScWarps = kScThreads / 32;
// CTA-sorted nodes of up to this many samples take the bitonic network, larger
// ones the radix passes (measured: the network is faster for 129..256
// samples, the radix passes from about 500 up)
constexpr int kScBitonicMax = 256;

struct ScShared {
  int feat[kMaxCap];
  int sign[kMaxCap];
  unsigned long long wlo[kScWarps], whi[kScWarps];
  float wmax[kScWarps];
  Best wbest[kScWarps];
  unsigned kor[kScWarps], kand[kScWarps];  // radix: bits set in some / every key of the node
  int wtot[kScWarps];                      // radix: warp totals of the digit-count scan
};

// Shared-memory slot of sorted position p: bits 0-3 are XORed with bits 4-7,
// so that a warp reading each thread's run of E = 2..16 consecutive positions
// touches 16 distinct 8-byte bank pairs per half-warp, while every aligned run
// of 16 positions stays a permutation of its own 16 slots (the sort's access
// pattern keeps its bank spread).
__device__ __forceinline__ int sc_slot(int p) { return p ^ ((p >> 4) & 15); }

// Writes the node's nv (key, label) pairs to positions 0..nv-1 (the sort
// never reads positions >= nv; see sc_bitonic).
// RM: read the row-major copy ds.Xr (the node's projections then share its
// samples' rows through L2) instead of one sector per (sample, feature) of
// the columns.
// The thread's OR and AND of its keys' value bits go to kor / kand.
template <int RM, class Put>
__device__ __forceinline__ void sc_gather(const DatasetView& ds, const int32_t* __restrict__ idx, const SortNodeCtx& nc,
                                          int kk, const ScShared& sh, Put put, unsigned& kor, unsigned& kand) {
  constexpr int kPer = 4;  // samples per thread per round, loads of 4 terms in flight per sample
  for (int e0 = threadIdx.x; e0 < nc.nv; e0 += kScThreads * kPer) {
    int64_t sid[kPer];
    float v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = e0 + u * kScThreads;
      sid[u] = e < nc.nv ? safe_sample(idx[nc.beg + e], ds.n) : -1;
      v[u] = 0.0f;
    }
    for (int j0 = 0; j0 < kk; j0 += 4) {
      float x[4][kPer];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int64_t f = sh.feat[j0 + jj < kk ? j0 + jj : j0];
        const float* col = RM ? ds.Xr + f : ds.X + f * ds.ld;
#pragma unroll
        for (int u = 0; u < kPer; ++u)
          x[jj][u] = (j0 + jj < kk && sid[u] >= 0) ? __ldg(col + (RM ? sid[u] * ds.d : sid[u])) : 0.0f;
      }
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        if (j0 + jj < kk) {
          const bool pos = sh.sign[j0 + jj] == 1;
#pragma unroll
          for (int u = 0; u < kPer; ++u) v[u] = __fadd_rn(v[u], pos ? x[jj][u] : -x[jj][u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = e0 + u * kScThreads;
      if (sid[u] >= 0) {
        const unsigned kv = f2key(v[u]);
        kor |= kv;
        kand &= kv;
        put(e, kv, (unsigned)ds.y[sid[u]]);
      }
    }
  }
}

// Ascending bitonic network over NP = 2^k positions of which the first nv
// hold keys: each merge of blocks of `size` first compares offset o of a
// block with its mirror size-1-o, then half-cleans with strides size/4 .. 1,
// every comparator putting the smaller key at the lower position.  Positions
// >= nv act as keys above every real key (a real key's label byte keeps it
// below all-ones), so no comparator ever moves a real key there: a
// comparator whose upper position is >= nv is a no-op and is skipped, and
// those positions are never written (nor read: registers stand in all-ones).
// Comparators within an aligned run of kScRun positions run in registers, one
// thread per run (the whole network for sizes up to kScRun, then strides
// kScRun/2 .. 1 of every larger merge); the other strides are shared-memory
// stages with a barrier each.
constexpr int kScRun = 8;

template <bool kWhole>
__device__ __forceinline__ void sc_runs(unsigned long long* keys, int NP, int nv) {
  for (int b = threadIdx.x; b < NP / kScRun; b += kScThreads) {
    const int base = b * kScRun;
    if (base >= nv) break;
    unsigned long long r[kScRun];
#pragma unroll
    for (int u = 0; u < kScRun; ++u) r[u] = base + u < nv ? keys[sc_slot(base + u)] : ~0ull;
#pragma unroll
    for (int size = kWhole ? 2 : 2 * kScRun; size <= (kWhole ? kScRun : 2 * kScRun); size <<= 1) {
      const int half = size >> 1;
#pragma unroll
      for (int stride = half < kScRun ? half : kScRun / 2; stride > 0; stride >>= 1) {
#pragma unroll
        for (int u = 0; u < kScRun; ++u) {
          const int o = u & (stride - 1);
          if ((u & stride) == 0) {
            // mirror comparator (first stage of a merge that fits the run) or half-cleaner
            const int w = (kWhole && stride == half) ? (u | (size - 1)) - o : u + stride;
            const unsigned long long a = r[u], c = r[w];
            r[u] = a < c ? a : c;
            r[w] = a < c ? c : a;
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kScRun; ++u)
      if (base + u < nv) keys[sc_slot(base + u)] = r[u];
  }
}

__device__ __forceinline__ void sc_bitonic(unsigned long long* keys, int NP, int nv) {
  sc_runs<true>(keys, NP, nv);
  __syncthreads();
  for (int size = 2 * kScRun; size <= NP; size <<= 1) {
    const int half = size >> 1;
    for (int stride = half; stride >= kScRun; stride >>= 1) {
      for (int i = threadIdx.x; i < NP / 2; i += kScThreads) {
        const int o = i & (stride - 1);
        const int lo = ((i & ~(stride - 1)) << 1) | o;
        const int hi = stride == half ? lo + size - 1 - 2 * o : lo + stride;
        if (hi >= nv) continue;
        const int sl = sc_slot(lo), sh = sc_slot(hi);
        const unsigned long long a = keys[sl], b = keys[sh];
        if (a > b) {
          keys[sl] = b;
          keys[sh] = a;
        }
      }
      __syncthreads();
    }
    sc_runs<false>(keys, NP, nv);
    __syncthreads();
  }
}

// Segmented radix sort of one node's pairs by the 32-bit value key (least
// significant digit first, 8-bit digits; a digit that is the same in every key
// of the node, bits diff = OR ^ AND of the keys, is skipped).  Value keys and
// labels sit in separate arrays with two buffers each (buffer b at offset
// b * np_max, position i at slot sc_slot(i)); each pass moves positions
// 0..nv-1 stably to the other buffer.  Warp w owns the segment
// [w * seg, (w + 1) * seg) of positions: it counts its digits with
// shared-memory reductions; the digit-major, warp-minor exclusive scan of the
// counts gives every (digit, warp) its first output position; the warp then
// walks its segment in order, 32 positions at a time, lanes holding the same
// digit finding each other with a match and their leader taking the group's
// positions from the running offset.  Counts and offsets are 16-bit halves of
// [kScWarps][128] words (digit dg: word dg >> 1, half dg & 1; both stay below
// 2048); cnt holds two such arrays, a pass counting in cnt[par] (zero on
// entry) and clearing cnt[par ^ 1] for the next.  Returns the buffer holding
// the sorted pairs.
__device__ __forceinline__ int sc_radix(unsigned* k32, uint8_t* l8, int np_max, int nv, unsigned diff,
                                             unsigned* cnt, int& par, ScShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = ((((nv + kScWarps - 1) / kScWarps) + 31) >> 5) << 5;
  const int p0 = warp * seg, p1 = min(nv, p0 + seg);
  const unsigned lt = (1u << lane) - 1u;
  int cur = 0;
  for (int sh8 = 0; sh8 < 32; sh8 += 8) {
    if (((diff >> sh8) & 255u) == 0u) continue;
    unsigned* c = cnt + par * (kScWarps * 128);
    unsigned* cn = cnt + (par ^ 1) * (kScWarps * 128);
    unsigned* wc = c + warp * 128;
    const unsigned* ka = k32 + cur * np_max;
    const uint8_t* la = l8 + cur * np_max;
    unsigned* kb = k32 + (cur ^ 1) * np_max;
    uint8_t* lb = l8 + (cur ^ 1) * np_max;
    for (int p = p0 + lane; p < p1; p += 32) {
      const unsigned dg = (ka[sc_slot(p)] >> sh8) & 255u;
      atomicAdd(&wc[dg >> 1], 1u << (16 * (dg & 1u)));
    }
    __syncthreads();
    // exclusive scan in (digit, warp) order: thread t takes digits 2t, 2t+1 (word t)
    unsigned v[kScWarps];
    int tot = 0;
#pragma unroll
    for (int w = 0; w < kScWarps; ++w) {
      v[w] = c[w * 128 + threadIdx.x];
      tot += (int)(v[w] & 0xFFFFu) + (int)(v[w] >> 16);
    }
    const int inc = warp_incl_scan(tot, lane);
    if (lane == 31) sh.wtot[warp] = inc;
    __syncthreads();
    int run = inc - tot;
    for (int w = 0; w < warp; ++w) run += sh.wtot[w];
    unsigned o[kScWarps];
#pragma unroll
    for (int w = 0; w < kScWarps; ++w) {
      o[w] = (unsigned)run;
      run += (int)(v[w] & 0xFFFFu);
    }
#pragma unroll
    for (int w = 0; w < kScWarps; ++w) {
      o[w] |= (unsigned)run << 16;
      run += (int)(v[w] >> 16);
    }
#pragma unroll
    for (int w = 0; w < kScWarps; ++w) c[w * 128 + threadIdx.x] = o[w];
    __syncthreads();
    for (int pb = p0; pb < p1; pb += 32) {
      const int p = pb + lane;
      const bool valid = p < p1;
      const int sp = sc_slot(valid ? p : p0);
      const unsigned kv = ka[sp];
      const unsigned dg = valid ? (kv >> sh8) & 255u : 256u + lane;
      const unsigned peers = __match_any_sync(0xffffffffu, dg);
      const int leader = __ffs(peers) - 1;
      const unsigned hs = 16u * (dg & 1u);
      unsigned pos = 0u;
      if (valid && lane == leader) pos = (atomicAdd(&wc[dg >> 1], (unsigned)__popc(peers) << hs) >> hs) & 0xFFFFu;
      pos = __shfl_sync(0xffffffffu, pos, leader);
      if (valid) {
        const int dp = sc_slot((int)pos + __popc(peers & lt));
        kb[dp] = kv;
        lb[dp] = la[sp];
      }
      __syncwarp();
    }
    for (int i = threadIdx.x; i < kScWarps * 128; i += kScThreads) cn[i] = 0u;
    __syncthreads();
    cur ^= 1;
    par ^= 1;
  }
  return cur;
}

// Walks this thread's chunk [i0, i0+E) of sorted positions; calls
// visit(i, run, g32, a, b) for each candidate (boundary between distinct
// values), run = packed class counts of positions 0..i.
template <class Get, class Visit>
__device__ __forceinline__ void sc_walk(Get key_at, const SortNodeCtx& nc, int C, const Crit& cr,
                                        int i0, int E, PackedCnt run, Visit visit) {
  unsigned long long x = i0 < nc.nv - 1 ? key_at(i0) : 0ull;
  for (int e = 0; e < E; ++e) {
    const int i = i0 + e;
    if (i >= nc.nv - 1) break;
    const unsigned long long nx = key_at(i + 1);
    pc_add(run, (int)(x & 0xFFull));
    const unsigned a = (unsigned)(x >> 32), b = (unsigned)(nx >> 32);
    x = nx;
    if (a != b) {
      int L[kMaxClasses];
#pragma unroll
      for (int c = 0; c < kMaxClasses; ++c) L[c] = pc_get(run, c);
      visit(i, run, key32s(cr, L, nc.N, C, nc.nv, i + 1), a, b);
    }
  }
}

// One pass per (node, projection) with the double re-score inline (the
// sort, not the re-score, dominates a CTA-sorted node).  Eight CTAs per SM:
// 64 registers a thread (the row-major form would otherwise take 72).
template <int ENT, int RM>
__global__ void __launch_bounds__(kScThreads, 8) k_sortc_scan(DatasetView ds, const int32_t* __restrict__ idx,
                                                             const int64_t* __restrict__ off, ProjView pv,
                                                             const V4* plan_total, const int32_t* nodes,
                                                             const int32_t* __restrict__ node_cls, Crit cr_in,
                                                             SortRes* res, int np_max) {
  Crit cr = cr_in;
  cr.ent = ENT;
  // bitonic: pairs [NP]; radix: value keys [2][np_max], then labels [2][np_max]
  extern __shared__ unsigned long long s_keys[];
  __shared__ ScShared sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // radix digit counts: two arrays of [kScWarps][128] words
  __shared__ unsigned s_rcnt[2 * kScWarps * 128];
  int rpar = 0;
  for (int i = threadIdx.x; i < kScWarps * 128; i += kScThreads) s_rcnt[i] = 0u;
  const int P = pv.P;
  const int64_t total = plan_total->w * P;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    SortNodeCtx nc;
    int j;
    const int64_t s = t / P;
    const int p = (int)(t - s * P);
    node_ctx(off, nodes, s, node_cls, nc, j);
    const int64_t q = (int64_t)j * P + p;
    int NP = 2 * kScThreads;
    while (NP < nc.nv) NP <<= 1;
    const int rb = pv.beg[q];
    int kk = pv.end[q] - rb;
    kk = kk < 0 ? 0 : (kk > kMaxCap ? kMaxCap : kk);
    __syncthreads();  // previous (node, projection) done with shared memory
    if (threadIdx.x < kk) {
      int f = pv.feat[rb + threadIdx.x];
      sh.feat[threadIdx.x] = (f < 0 || f >= ds.d) ? 0 : f;
      sh.sign[threadIdx.x] = pv.sign[rb + threadIdx.x];
    }
    __syncthreads();
    // nodes of up to kScBitonicMax samples: (key, label) pairs sorted by the
    // bitonic network; larger nodes: value keys and labels in separate
    // arrays, sorted by the radix passes
    const bool rdx = nc.nv > kScBitonicMax;
    unsigned* s_k32 = reinterpret_cast<unsigned*>(s_keys);             // [2][np_max] value keys
    uint8_t* s_l8 = reinterpret_cast<uint8_t*>(s_k32 + 2 * np_max);  // [2][np_max] labels
    unsigned kor = 0u, kand = ~0u;
    sc_gather<RM>(ds, idx, nc, kk, sh, [&](int e, unsigned kv, unsigned yv) {
      if (rdx) {
        s_k32[sc_slot(e)] = kv;
        s_l8[sc_slot(e)] = (uint8_t)yv;
      } else {
        s_keys[sc_slot(e)] = ((unsigned long long)kv << 32) | (unsigned long long)yv;
      }
    }, kor, kand);
    int fin = 0;
    if (rdx) {
      kor = __reduce_or_sync(0xffffffffu, kor);
      kand = __reduce_and_sync(0xffffffffu, kand);
      if (lane == 0) {
        sh.kor[warp] = kor;
        sh.kand[warp] = kand;
      }
      __syncthreads();
      for (int w = 0; w < kScWarps; ++w) {
        kor |= sh.kor[w];
        kand &= sh.kand[w];
      }
      fin = sc_radix(s_k32, s_l8, np_max, nc.nv, kor ^ kand, s_rcnt, rpar, sh);
    } else {
      __syncthreads();
      sc_bitonic(s_keys, NP, nc.nv);
    }
    const unsigned* kf = s_k32 + fin * np_max;
    const uint8_t* lf = s_l8 + fin * np_max;
    auto key_at = [&](int i) -> unsigned long long {
      const int sl = sc_slot(i);
      return rdx ? ((unsigned long long)kf[sl] << 32) | (unsigned long long)lf[sl] : s_keys[sl];
    };
    // this thread's chunk of consecutive sorted positions and its left counts
    const int E = NP / kScThreads;
    const int i0 = threadIdx.x * E;
    PackedCnt own{0, 0};
    for (int e = 0; e < E; ++e)
      if (i0 + e < nc.nv) pc_add(own, (int)(key_at(i0 + e) & 0xFFull));
    unsigned long long ilo = own.lo, ihi = own.hi;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long ul = __shfl_up_sync(0xffffffffu, ilo, o);
      const unsigned long long uh = __shfl_up_sync(0xffffffffu, ihi, o);
      if (lane >= o) {
        ilo += ul;
        ihi += uh;
      }
    }
    if (lane == 31) {
      sh.wlo[warp] = ilo;
      sh.whi[warp] = ihi;
    }
    __syncthreads();
    PackedCnt run{ilo - own.lo, ihi - own.hi};
    for (int w = 0; w < warp; ++w) {
      run.lo += sh.wlo[w];
      run.hi += sh.whi[w];
    }
    // float maximum of the projection
    float m = key_none(cr);
    sc_walk(key_at, nc, ds.C, cr, i0, E, run,
            [&](int, const PackedCnt&, float g, unsigned, unsigned) { m = fmaxf(m, g); });
    m = warp_max(m);
    if (lane == 0) sh.wmax[warp] = m;
    __syncthreads();
    m = sh.wmax[0];
    for (int w = 1; w < kScWarps; ++w) m = fmaxf(m, sh.wmax[w]);
    // double re-score of the candidates within m(1-eps); lexicographic best
    Best lb;
    lb.c = Cand{-1.0, INT_MAX, INT_MAX};
    lb.ka = lb.kb = 0u;
    lb.L = PackedCnt{0, 0};
    if (key_any(cr, m)) {
      const float thr = key_thr(cr, m, nc.nv, ds.C);
      sc_walk(key_at, nc, ds.C, cr, i0, E, run, [&](int i, const PackedCnt& r, float g, unsigned a, unsigned b) {
        if (g >= thr) {
          int L[kMaxClasses];
#pragma unroll
          for (int cc = 0; cc < kMaxClasses; ++cc) L[cc] = pc_get(r, cc);
          const Cand c{gain64s(cr, L, nc.N, ds.C, nc.nv, i + 1), 0, i};
          if (better(c, lb.c)) {
            lb.c = c;
            lb.ka = a;
            lb.kb = b;
            lb.L = r;
          }
        }
      });
    }
    best_reduce(lb);
    if (lane == 0) sh.wbest[warp] = lb;
    __syncthreads();
    if (threadIdx.x == 0) {
      Best b = sh.wbest[0];
      for (int w = 1; w < kScWarps; ++w)
        if (better(sh.wbest[w].c, b.c)) b = sh.wbest[w];
      SortRes r;
      r.m32 = m;
      r.g64 = b.c.g;
      r.cand = b.c.cand;
      r.ka = b.ka;
      r.kb = b.kb;
      r.llo = b.L.lo;
      r.lhi = b.L.hi;
      res[q] = r;
    }
  }
}

// Class counts of every exact-path node (one warp per node).
__global__ void __launch_bounds__(256) k_sortw_counts(DatasetView ds, const int32_t* __restrict__ idx,
                                                      const int64_t* __restrict__ off, const V4* plan_total,
                                                      const int32_t* tiny, const int32_t* med, int32_t* node_cls) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t m_tiny = plan_total->y, m_all = plan_total->y + plan_total->w;
  for (int64_t s = gw; s < m_all; s += nw) {
    const int j = s < m_tiny ? tiny[s] : med[s - m_tiny];
    const int64_t beg = off[j];
    const int nv = (int)(off[j + 1] - beg);
    int cnt[kMaxClasses];
#pragma unroll
    for (int c = 0; c < kMaxClasses; ++c) cnt[c] = 0;
    for (int e = lane; e < nv; e += 32) {
      const int yv = ds.y[safe_sample(idx[beg + e], ds.n)];
#pragma unroll
      for (int c = 0; c < kMaxClasses; ++c) cnt[c] += (yv == c);
    }
#pragma unroll
    for (int c = 0; c < kMaxClasses; ++c) {
      const int v = warp_sum(cnt[c]);
      if (lane == c) node_cls[(int64_t)j * kMaxClasses + c] = v;
    }
  }
}

// Pass 2: one warp per exact-path node (both forms).
__global__ void __launch_bounds__(256) k_sortw_select(const int64_t* __restrict__ off, int32_t P, int32_t C,
                                                      const V4* plan_total, const int32_t* tiny, const int32_t* med,
                                                      const SortRes* __restrict__ res, Crit cr, so_split* out,
                                                      int64_t* left_counts) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t m_tiny = plan_total->y, m_all = plan_total->y + plan_total->w;
  for (int64_t s = gw; s < m_all; s += nw) {
    const int j = s < m_tiny ? tiny[s] : med[s - m_tiny];
    const int nv = (int)(off[j + 1] - off[j]);
    const SortRes* rj = res + (int64_t)j * P;
    float M = key_none(cr);
    for (int p = lane; p < P; p += 32) M = fmaxf(M, rj[p].m32);
    M = warp_max(M);
    Cand best{-1.0, INT_MAX, INT_MAX};
    if (key_any(cr, M)) {
      const float thr = key_thr(cr, M, nv, C);
      for (int p = lane; p < P; p += 32) {
        const SortRes r = rj[p];
        if (r.m32 >= thr && r.g64 > 0.0) {
          const Cand c{r.g64, p, r.cand};
          if (better(c, best)) best = c;
        }
      }
      best = warp_best(best);
    }
    if (lane == 0) {
      so_split rec;
      rec.path = 1;
      if (best.proj == INT_MAX) {
        rec.valid = 0; rec.proj = -1; rec.cand = -1; rec.threshold = 0.0f; rec.gain = 0.0;
        rec.n_left = 0; rec.n_right = 0;
        out[j] = rec;
        if (left_counts)
          for (int c = 0; c < C; ++c) left_counts[(int64_t)j * C + c] = 0;
      } else {
        const SortRes r = rj[best.proj];
        rec.valid = 1;
        rec.proj = best.proj;
        rec.cand = r.cand;
        rec.threshold = midpoint(key2f(r.ka), key2f(r.kb));
        rec.gain = r.g64;
        rec.n_left = r.cand + 1;
        rec.n_right = nv - (r.cand + 1);
        out[j] = rec;
        if (left_counts) {
          const PackedCnt L{r.llo, r.lhi};
          for (int c = 0; c < C; ++c) left_counts[(int64_t)j * C + c] = pc_get(L, c);
        }
      }
    }
  }
}

// Between the two passes: each exact-path node's re-score window from its
// projections' float maxima (+inf when no candidate can win).
// Lists the (node, projection) pairs whose float maximum reaches the node's
// window (list 0: register-sorted nodes, list 1: CTA-sorted nodes); the order
// of a list does not matter, each entry writes its own result.
__global__ void __launch_bounds__(256) k_sort_node_thr(const int64_t* __restrict__ off, int32_t P, int32_t C,
                                                       const V4* plan_total, const int32_t* tiny, const int32_t* med,
                                                       const SortRes* __restrict__ res, Crit cr, int64_t* lists,
                                                       int64_t list_cap, int32_t* list_n, int list_med) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t m_tiny = plan_total->y, m_all = plan_total->y + plan_total->w;
  for (int64_t s = gw; s < m_all; s += nw) {
    const int j = s < m_tiny ? tiny[s] : med[s - m_tiny];
    const int which = s < m_tiny ? 0 : 1;
    if (which == 1 && !list_med) continue;
    const int nv = (int)(off[j + 1] - off[j]);
    const SortRes* rj = res + (int64_t)j * P;
    float M = key_none(cr);
    for (int p = lane; p < P; p += 32) M = fmaxf(M, rj[p].m32);
    M = warp_max(M);
    if (!key_any(cr, M)) continue;
    const float thr = key_thr(cr, M, nv, C);
    for (int p0 = 0; p0 < P; p0 += 32) {
      const int p = p0 + lane;
      const bool in = p < P && rj[p].m32 >= thr;
      const unsigned bal = __ballot_sync(0xffffffffu, in);
      int base = 0;
      if (lane == 0 && bal) base = atomicAdd(&list_n[which], __popc(bal));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (in) {
        const int pos = base + __popc(bal & ((1u << lane) - 1u));
        if (pos < list_cap) lists[which * list_cap + pos] = (int64_t)j * P + p;
      }
    }
  }
}

cudaError_t launch_sort_warp(const SearchArgs& a, const Crit& cr, const V4* plan_total, const int32_t* tiny,
                             const int32_t* med, void* res_raw, int32_t* node_cls, int64_t* lists,
                             int32_t* list_n, cudaStream_t st) {
  const DeviceInfo& di = device_info();
  SortRes* res = static_cast<SortRes*>(res_raw);
  const int64_t list_cap = (int64_t)a.m * a.pv.P;
  cudaError_t e = cudaMemsetAsync(list_n, 0, 2 * sizeof(int32_t), st);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps_("k_sortw_counts", st);
    k_sortw_counts<<<di.num_sms * 8, 256, 0, st>>>(a.ds, a.idx, a.node_off, plan_total, tiny, med, node_cls);
  }
  const bool cta = !a.hist_only && a.T > kSortRegMax + 1;
  int NPmax = 2 * kScThreads;
  while (NPmax < a.T - 1) NPmax <<= 1;
  // the larger of the bitonic network's pairs (8 bytes a position) and the
  // radix passes' two buffers of value keys and labels (10 bytes a position)
  const size_t smem = (size_t)NPmax * (NPmax > kScBitonicMax ? 10 : 8);
  auto kw = cr.ent ? (a.ds.Xr ? k_sortw_scan<1, 1> : k_sortw_scan<1, 0>)
                   : (a.ds.Xr ? k_sortw_scan<0, 1> : k_sortw_scan<0, 0>);
  auto kc = cr.ent ? (a.ds.Xr ? k_sortc_scan<1, 1> : k_sortc_scan<1, 0>)
                   : (a.ds.Xr ? k_sortc_scan<0, 1> : k_sortc_scan<0, 0>);
  // every projection's float maximum; then each node's window; then the
  // double re-score of the projections inside their node's window only
  for (int pass = 0; pass < 2; ++pass) {
    const int64_t* lw = pass == 0 ? nullptr : lists;
    {
      ProfScope ps_("k_sortw_scan", st);
      kw<<<di.num_sms * 8, 256, 0, st>>>(a.ds, a.idx, a.node_off, a.pv, plan_total, tiny, node_cls, cr, res, lw,
                                         list_n);
    }
    if (cta && pass == 0) {  // CTA-sorted nodes: one pass, re-score inline
      ProfScope ps_("k_sortc_scan", st);
      kc<<<di.num_sms * 16, kScThreads, smem, st>>>(a.ds, a.idx, a.node_off, a.pv, plan_total, med, node_cls, cr,
                                                    res, NPmax);
    }
    if (pass == 0) {
      ProfScope ps_("k_sort_node_thr", st);
      k_sort_node_thr<<<di.num_sms * 4, 256, 0, st>>>(a.node_off, a.pv.P, a.ds.C, plan_total, tiny, med, res, cr,
                                                      lists, list_cap, list_n, 0);
    }
  }
  {
    ProfScope ps_("k_sortw_select", st);
    k_sortw_select<<<di.num_sms * 8, 256, 0, st>>>(a.node_off, a.pv.P, a.ds.C, plan_total, tiny, med, res, cr,
                                                   a.out, a.left_counts);
  }
  return cudaGetLastError();
}

size_t sort_res_bytes() { return sizeof(SortRes); }

}  // namespace sof
