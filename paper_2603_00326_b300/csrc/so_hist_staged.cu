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
//   k_hist_staged  per item: bins (equal-width, or random-width from the
//                  boundary tables of so_rw.cu) and class counts in shared
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

constexpr int kStThreads = 1024;         // threads of the staged kernels (32 warps, one CTA per SM)
constexpr int kStWarps = kStThreads / 32;
constexpr int kTileF = 8192;             // floats per tile buffer (32 KB); two buffers
constexpr int kStUMax = kTileF / 64;     // rows of a tile at St = 64 -> 128
constexpr int kMmUMax = kTileF / 68;     // 120: every min/max group also fits the padded row-major tile
constexpr int kStMaxWords = 2048;        // feature bitmap words (d <= 65536)
constexpr int kMmPPW = 8;                // min/max: projections per warp
constexpr int kMmBuf = 3;                // min/max: tile buffers (kMmBuf - 1 tiles in flight)
constexpr int kMmGroup = kStWarps * kMmPPW;  // 256 projections per min/max group
constexpr int kHistPGMax = 64;           // histogram projections per item (two per warp)
constexpr int kHistPPW = kHistPGMax / kStWarps;  // histogram projections per warp
constexpr int kMaxItem = 16384;          // samples per item (label bytes kept in shared memory)
constexpr float kMagic = 12582912.0f;    // 1.5 * 2^23
constexpr float kCondLimit = 262144.0f;  // 2^18

// ---- asynchronous global -> shared copies (sm_80+ cp.async) ------------------
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---- shared-memory accesses by 32-bit shared address --------------------------
// The inner loops address shared memory with 32-bit offsets in the shared
// window directly (no generic-pointer arithmetic).
__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ float4 lds_f4(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds_f2(unsigned a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ uint4 lds_u4(unsigned a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];\n" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ unsigned lds_u32(unsigned a) {
  unsigned v;
  asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ unsigned lds_u16(unsigned a) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];\n" : "=h"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_f32(unsigned a) { return __uint_as_float(lds_u32(a)); }
__device__ __forceinline__ void reds_add(unsigned a, unsigned v) {
  asm volatile("red.shared.add.u32 [%0], %1;\n" ::"r"(a), "r"(v) : "memory");
}

// Random-width bin #{j < nb : t_j <= v} over a projection's sorted boundaries
// at shared address tb.  GUIDED: v's cell holds lo (boundaries of lower
// cells, all below v) and k (boundaries in the cell, t_lo .. t_{lo+k-1}); the
// bin is lo plus those of the k that are <= v.  The first two are compared
// without a branch (the second read may pass the row end when k < 2: it
// stays inside the table area of shared memory and is masked); cells with
// more than two boundaries (8% of cells) finish in a loop bounded by k.
// Otherwise a binary search bounded by nb.
template <bool GUIDED>
__device__ __forceinline__ int rw_bin_smem(float v, float s, float o, unsigned tb, unsigned gb, int nb) {
  if (GUIDED) {
    const unsigned g = lds_u16(gb + 2u * (unsigned)rw_cell(v, s, o));
    const unsigned lo = g & 0xffu, k = g >> 8;
    const unsigned ta = tb + 4u * lo;
    int b = (int)lo + ((k > 0u && lds_f32(ta) <= v) ? 1 : 0) + ((k > 1u && lds_f32(ta + 4u) <= v) ? 1 : 0);
    for (unsigned i = 2; i < k; ++i) b += lds_f32(ta + 4u * i) <= v ? 1 : 0;
    return b;
  }
  int lo = 0, hi = nb;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (lds_f32(tb + 4u * (unsigned)mid) <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Three-input minimum / maximum (sm_100+ PTX): the value of two chained
// two-input fminf / fmaxf, one instruction.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;\n" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;\n" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

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
  unsigned long long* ctr;  // next item to take (zeroed before the launch)
};


// Items are taken from a counter, so a CTA that drew short items takes more
// (items differ a lot in size: chunks of large nodes and whole small ones).
// Every item's output is order-independent (atomic min / max and histogram
// flushes, projected values at fixed positions).  The caller's barrier
// comes first: every thread has read the previous item number.
__device__ __forceinline__ int64_t next_item(const StagedPlan& sp, int64_t* s_item) {
  __syncthreads();
  if (threadIdx.x == 0) *s_item = (int64_t)atomicAdd(sp.ctr, 1ull);
  __syncthreads();
  return *s_item;
}

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

// The item's node h = the last node whose first item is <= t, by a 32-way
// search: each step the warp probes 32 evenly spaced first-item offsets at
// once (item_off is nondecreasing, so the probes at or below t form a prefix
// of the lanes), cutting the range 32-fold per dependent load.
__device__ __forceinline__ ItemPos decode_item(const StagedPlan& sp, int64_t t, int P) {
  ItemPos r;
  const int64_t m_hist = sp.plan_total->x;
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = m_hist - 1;  // item_off[lo] <= t; h in [lo, hi]
  while (lo < hi) {
    const int64_t step = (hi - lo + 31) >> 5;
    const int64_t pos = lo + (int64_t)(lane + 1) * step;
    const bool ok = pos <= hi && sp.item_off[pos] <= t;
    const int c = __popc(__ballot_sync(0xffffffffu, ok));
    hi = min(hi, lo + (int64_t)(c + 1) * step - 1);
    lo += (int64_t)c * step;
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

// Projection descriptors of the group in shared memory: k, and per non-zero
// (ascending feature order) a packed word with the tile byte offset
// row * St * 4 in the low 16 bits (U * St <= 8192 floats) and the sign in
// bit 31.
template <int KMAX>
__device__ __forceinline__ void build_desc(const ProjView& pv, int64_t qbase, int np, int d, int St,
                                           const uint32_t* s_bits, const int* s_wpre, int* s_dk, uint32_t* s_dpk) {
  for (int e = threadIdx.x; e < np * KMAX; e += kStThreads) {
    const int p = e / KMAX, jj = e - (e / KMAX) * KMAX;
    const int rb = pv.beg[qbase + p];
    int k = pv.end[qbase + p] - rb;
    k = k < 0 ? 0 : (k > KMAX ? KMAX : k);
    if (jj == 0) s_dk[p] = k;
    if (jj < k) {
      int f = pv.feat[rb + jj];
      f = (f < 0 || f >= d) ? 0 : f;
      s_dpk[p * KMAX + jj] = (uint32_t)(row_of(f, s_bits, s_wpre) * St * 4) | (pv.sign[rb + jj] == 1 ? 0u : 0x80000000u);
    }
  }
}

// ---- tile staging with asynchronous copies ------------------------------------
// A tile is U rows (the item's features, ascending) by St samples, row-major
// in shared memory.  Vector form (a full tile of consecutive samples, 16-byte
// aligned): 16-byte copies along each row.  Gather form: thread owns column
// i = tid % St and rows tid/St + k*(NT/St), one 4-byte copy per element;
// columns past the item's end repeat its first sample (min / max unchanged;
// their labels are marked invalid).  Nothing passes through registers.
// (Tensor-map gathers of four feature rows (cp.async.bulk.tensor gather4)
// were measured in place of the 16-byte copies: 1.91 against 1.49 ms for the
// histogram kernel on the 4M-sample root, 0.85 against 0.67 ms for the
// min / max kernel.)

// Per-thread copy plan of an item's tiles.  Every tile of an item has the same
// rows and width and only its first sample moves, so the thread's source and
// destination offsets are fixed once per item.  Vector form: the thread's (at
// most two, U * St / 4 <= 2 * kStThreads) 16-byte chunks.  Gather form: the
// thread's tile column and rows tid/St + k*(NT/St); the element offsets of the
// rows (feature * ld) sit in shared memory.
struct Stager {
  const float* src0;
  const float* src1;
  int dst0, dst1;
  int col;
  bool vec;
  // row-major gather form: the thread copies row r of every 1024/Ur-th
  // sample column from the row-major copy (feature frow, -1: no row)
  bool rowmaj;
  int Ur, r, frow, Sp;
};

__device__ __forceinline__ Stager stager_init(const DatasetView& ds, const int32_t* __restrict__ idx,
                                              const ItemPos& it, int St, int U, const int* s_rowfeat, bool contig,
                                              bool rowmaj = false, int Sp = 0) {
  Stager sg;
  sg.vec = contig;
  sg.col = threadIdx.x & (St - 1);
  sg.src0 = sg.src1 = nullptr;
  sg.dst0 = sg.dst1 = 0;
  sg.rowmaj = rowmaj;
  sg.Sp = rowmaj ? Sp : St;
  sg.Ur = 1;
  sg.r = 0;
  sg.frow = -1;
  if (rowmaj) {
    while (sg.Ur < U) sg.Ur <<= 1;
    sg.r = threadIdx.x & (sg.Ur - 1);
    sg.frow = sg.r < U ? s_rowfeat[sg.r] : -1;
  } else if (contig) {
    const int lq = __ffs(St) - 3;  // log2(St / 4)
    const int total = U << lq;
    const int64_t sid0 = idx[it.beg];
    const int e0 = threadIdx.x, e1 = threadIdx.x + kStThreads;
    if (e0 < total) {
      const int r = e0 >> lq, q = e0 & ((1 << lq) - 1);
      sg.src0 = ds.X + (int64_t)s_rowfeat[r] * ds.ld + sid0 + 4 * q;
      sg.dst0 = r * St + 4 * q;
    }
    if (e1 < total) {
      const int r = e1 >> lq, q = e1 & ((1 << lq) - 1);
      sg.src1 = ds.X + (int64_t)s_rowfeat[r] * ds.ld + sid0 + 4 * q;
      sg.dst1 = r * St + 4 * q;
    }
  }
  return sg;
}

// Issues the copies of tile t into buf.  A full tile of an aligned run of
// consecutive samples takes the vector form; the row-major form reads each
// sample's features from its row of the row-major copy (consecutive threads,
// consecutive features of one sample), into rows of stride Sp = St + 4 so
// that those threads' shared-memory writes spread over the banks; any other
// tile gathers one value per (sample, feature) from the column-major matrix.
// Columns past the item's end repeat its first sample.
__device__ __forceinline__ void stager_issue(const Stager& sg, const DatasetView& ds, const int32_t* __restrict__ idx,
                                             const ItemPos& it, int t, int St, int U, const int64_t* s_rowoff,
                                             float* buf) {
  const int64_t nb = it.beg + (int64_t)t * St;
  if (sg.rowmaj) {
    const int spp = kStThreads / sg.Ur;  // sample columns per pass
    for (int i = threadIdx.x / sg.Ur; i < St; i += spp) {
      const int64_t pos = nb + i;
      const int64_t sid = safe_sample(idx[pos < it.end ? pos : nb], ds.n);
      if (sg.frow >= 0) cp_async4(buf + sg.r * sg.Sp + i, ds.Xr + sid * ds.d + sg.frow);
    }
  } else if (sg.vec && it.end - nb >= St) {
    const int64_t o = (int64_t)t * St;
    if (sg.src0) cp_async16(buf + sg.dst0, sg.src0 + o);
    if (sg.src1) cp_async16(buf + sg.dst1, sg.src1 + o);
  } else {
    const int64_t pos = nb + sg.col;
    const int64_t sid = safe_sample(idx[pos < it.end ? pos : nb], ds.n);
    const float* xs = ds.X + sid;
    const int rstep = kStThreads / St;
    for (int r = threadIdx.x / St; r < U; r += rstep) cp_async4(buf + r * St + sg.col, xs + s_rowoff[r]);
  }
}

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

__device__ __forceinline__ int choose_st(int U) {
  // U * St <= kTileF, St in {64, 128, 256}
  if (U * 256 <= kTileF) return 256;
  if (U * 128 <= kTileF) return 128;
  return 64;
}

// Tile width of the row-major form, whose rows have stride St + 4:
// U * (St + 4) <= kTileF (U <= kRowMajUMax).
constexpr int kRowMajUMax = kMmUMax;  // 120 rows at St = 64
__device__ __forceinline__ int choose_st_pad(int U) {
  if (U * 260 <= kTileF) return 256;
  if (U * 132 <= kTileF) return 128;
  return 64;
}

// ---- k_groups: greedy projection groups per histogram node -------------------
// One warp per (node, grouping).  A group is closed before a projection that would push
// its distinct features above umax or its size above pmax.
__global__ void __launch_bounds__(128) k_groups(const V4* plan_total, const int32_t* hist_nodes, ProjView pv, int d,
                                                int umax1, int pmax1, int umax2, int pmax2, int32_t* ng1,
                                                int32_t* gs1, int32_t* ng2, int32_t* gs2) {
  // per warp: bitmap [nw], set-word list [kStUMax], and the features of 32
  // projection rows [32][32] (lane l holds feature l of each row)
  extern __shared__ uint32_t s_grp[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (d + 31) >> 5;
  uint32_t* bits = s_grp + warp * (nw + kStUMax + 32 * 33);
  uint32_t* setw = bits + nw;
  int* rowf = reinterpret_cast<int*>(setw + kStUMax);  // [32][33]: padded against bank conflicts
  for (int w = lane; w < nw; w += 32) bits[w] = 0u;
  __syncwarp();
  const int64_t m_hist = plan_total->x;
  const int P = pv.P;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // one warp per (node, pass): a node's two groupings run side by side
  for (int64_t t = gw; t < 2 * m_hist; t += nwarps) {
    const int64_t h = t >> 1;
    const int pass = (int)(t & 1);
    const int64_t j = hist_nodes[h];
    {
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
      int k_l = 0;  // lane l: length of row p0 + l
      // d <= 1024: the group's feature bitmap in registers, lane l holding
      // features 32l .. 32l+31 (a bit test is one shuffle, no atomics)
      const bool regmap = d <= 1024;
      uint32_t word = 0u;
      for (int p = 0; p < P; ++p) {
        if ((p & 31) == 0) {
          // rows p .. p+31 at once: their bounds in one load, then all their
          // features with the loads in flight together
          int rb_l = 0;
          k_l = 0;
          if (p + lane < P) {
            const int64_t q = j * P + p + lane;
            rb_l = pv.beg[q];
            const int kk = pv.end[q] - rb_l;
            k_l = kk < 0 ? 0 : (kk > kMaxCap ? kMaxCap : kk);
          }
          __syncwarp();  // the previous rows' features are no longer read
#pragma unroll 8
          for (int pp = 0; pp < 32; ++pp) {
            const int rb = __shfl_sync(0xffffffffu, rb_l, pp);
            const int kk = __shfl_sync(0xffffffffu, k_l, pp);
            int f = 0;
            if (lane < kk) {
              f = pv.feat[rb + lane];
              f = (f < 0 || f >= d) ? 0 : f;
            }
            rowf[pp * 33 + lane] = f;
          }
          __syncwarp();
        }
        const int k = __shfl_sync(0xffffffffu, k_l, p & 31);
        const int f = rowf[(p & 31) * 33 + lane];
        if (regmap) {
          const uint32_t ow = __shfl_sync(0xffffffffu, word, (f >> 5) & 31);
          bool fresh = lane < k && !((ow >> (f & 31)) & 1u);
          int add = __popc(__ballot_sync(0xffffffffu, fresh));
          if (cnt > 0 && (U + add > umax || cnt + 1 > pmax)) {
            word = 0u;
            U = 0;
            cnt = 0;
            ++g;
            if (lane == 0) gs[g] = p;
            add = __popc(__ballot_sync(0xffffffffu, lane < k));
          }
          for (int jj = 0; jj < k; ++jj) {  // each feature of the row to its owner lane
            const int fj = __shfl_sync(0xffffffffu, f, jj);
            if ((fj >> 5) == lane) word |= 1u << (fj & 31);
          }
          U += add;
          ++cnt;
          continue;
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
  int64_t S1, S2;  // samples per item of the min / max and the histogram kernels
  int64_t* item_off1;
  int64_t* item_off2;
  __device__ V4 value(int64_t h) const {
    if (h >= plan_total->x) return V4{0, 0, 0, 0};
    const int j = hist_nodes[h];
    const int64_t nv = off[j + 1] - off[j];
    return V4{(nv + S1 - 1) / S1 * ng1[h], (nv + S2 - 1) / S2 * ng2[h], 0, 0};
  }
  __device__ void apply(int64_t h, V4 ex) const {
    if (h >= plan_total->x) return;
    item_off1[h] = ex.x;
    item_off2[h] = ex.y;
  }
};

// Static assignment of an item's projections to warps, balanced by non-zero
// count: projections ranked by k (descending, counting sort) are dealt to the
// warps in snake order (0..31, 31..0, ...).  s_assign[w * nslot + s] is the
// s-th projection of warp w, or -1; s_slot (if given) is the inverse map,
// projection -> w * nslot + s.  Needs s_dk complete; the caller syncs before
// reading s_assign or s_slot.
__device__ __forceinline__ int assign_snake(int np, const int* s_dk, int* s_kcnt, int* s_assign,
                                            int* s_slot = nullptr) {
  const int nslot = (np + kStWarps - 1) / kStWarps;
  for (int e = threadIdx.x; e < kMaxCap + 1; e += kStThreads) s_kcnt[e] = 0;
  for (int e = threadIdx.x; e < nslot * kStWarps; e += kStThreads) s_assign[e] = -1;
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += kStThreads) atomicAdd(&s_kcnt[s_dk[p]], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = kMaxCap; k >= 0; --k) {
      const int c = s_kcnt[k];
      s_kcnt[k] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += kStThreads) {
    const int r = atomicAdd(&s_kcnt[s_dk[p]], 1);
    const int round = r / kStWarps, j = r - round * kStWarps;
    const int w = (round & 1) ? (kStWarps - 1 - j) : j;
    s_assign[w * nslot + round] = p;
    if (s_slot) s_slot[p] = w * nslot + round;
  }
  return nslot;
}

// ---- k_mm_staged: min / max -------------------------------------------------
// Projection descriptors are packed words: the tile offset (row * St) of a
// non-zero in the low 16 bits and its sign in bit 31.  The loop over a
// projection's non-zeros is not specialised: each term is one broadcast
// descriptor load, then NPS packed FP32x2 fused multiply-adds (one per sample
// pair-step of the tile), so a warp's work per tile needs no dispatch.
// fma(+-1, x, acc) rounds exactly like acc + (+-x).
__device__ __forceinline__ float desc_sign(uint32_t w) { return __uint_as_float((w & 0x80000000u) | 0x3f800000u); }

// Lane layout of a tile of St samples: NQ steps of 32*V consecutive samples,
// V consecutive samples per lane in each step (vector loads of V floats):
// sample(q, v) = 32*V*q + V*lane + v.  St = 64 -> (V, NQ) = (2, 1),
// St = 128 -> (4, 1), St = 256 -> (4, 2).
template <int V, int NQ>
__device__ __forceinline__ void project_term(unsigned base, uint32_t w, float (&acc)[V * NQ]) {
  const float s = desc_sign(w);
  const unsigned row = base + (w & 0xffffu);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (V == 4) {
      const float4 x = lds_f4(row + 512 * q);
      acc[4 * q] = __fmaf_rn(s, x.x, acc[4 * q]);
      acc[4 * q + 1] = __fmaf_rn(s, x.y, acc[4 * q + 1]);
      acc[4 * q + 2] = __fmaf_rn(s, x.z, acc[4 * q + 2]);
      acc[4 * q + 3] = __fmaf_rn(s, x.w, acc[4 * q + 3]);
    } else {
      const float2 x = lds_f2(row + 256 * q);
      acc[2 * q] = __fmaf_rn(s, x.x, acc[2 * q]);
      acc[2 * q + 1] = __fmaf_rn(s, x.y, acc[2 * q + 1]);
    }
  }
}

// The projection's terms in order: descriptor words four at a time (16-byte
// loads; rows are padded to a multiple of 8 words), a warp-uniform exit after
// each term.  tile and dpk are shared addresses of the tile buffer and of the
// projection's descriptor row.
template <int V, int NQ>
__device__ __forceinline__ void project_tile(unsigned tile, unsigned dpk, int k, int lane, float (&acc)[V * NQ]) {
  const unsigned base = tile + 4u * V * lane;
#pragma unroll
  for (int i = 0; i < V * NQ; ++i) acc[i] = 0.0f;
  for (int j0 = 0; j0 < k; j0 += 4) {
    const uint4 w = lds_u4(dpk + 4u * j0);
    project_term<V, NQ>(base, w.x, acc);
    if (j0 + 1 >= k) break;
    project_term<V, NQ>(base, w.y, acc);
    if (j0 + 2 >= k) break;
    project_term<V, NQ>(base, w.z, acc);
    if (j0 + 3 >= k) break;
    project_term<V, NQ>(base, w.w, acc);
  }
}

// Packed form of project_tile: sample pairs in FP32x2 registers (fma(+-1, x,
// acc) per lane of the pair, the same single rounding).
template <int V, int NQ>
__device__ __forceinline__ void project_tile2(unsigned tile, unsigned dpk, int k, int lane,
                                              float2 (&acc)[V * NQ / 2]) {
  const unsigned base = tile + 4u * V * lane;
#pragma unroll
  for (int i = 0; i < V * NQ / 2; ++i) acc[i] = make_float2(0.0f, 0.0f);
  auto term = [&](uint32_t w) {
    const float s = desc_sign(w);
    const float2 s2 = make_float2(s, s);
    const unsigned row = base + (w & 0xffffu);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (V == 4) {
        const float4 x = lds_f4(row + 512 * q);
        acc[2 * q] = ffma2(s2, make_float2(x.x, x.y), acc[2 * q]);
        acc[2 * q + 1] = ffma2(s2, make_float2(x.z, x.w), acc[2 * q + 1]);
      } else {
        acc[q] = ffma2(s2, lds_f2(row + 256 * q), acc[q]);
      }
    }
  };
  for (int j0 = 0; j0 < k; j0 += 4) {
    const uint4 w = lds_u4(dpk + 4u * j0);
    term(w.x);
    if (j0 + 1 >= k) break;
    term(w.y);
    if (j0 + 2 >= k) break;
    term(w.z);
    if (j0 + 3 >= k) break;
    term(w.w);
  }
}

// Straight-line form of project_tile2 for rows of at most 8 terms (row stride
// 8 words): one warp-uniform dispatch on k picks a fully unrolled body that
// reads the row's descriptor words in 16-byte broadcasts (one for k <= 4), so
// no loop control runs per term.  The terms are added in row order, as
// project_tile2 adds them.  (Unrolling only k <= 4 and looping over longer
// rows was measured slower: 0.77 against 0.68 ms for the min / max pass of
// the 4M-sample root.)
template <int V, int NQ, int K>
__device__ __forceinline__ void proj_fixed(unsigned base, unsigned dpk, float2 (&acc)[V * NQ / 2]) {
#pragma unroll
  for (int i = 0; i < V * NQ / 2; ++i) acc[i] = make_float2(0.0f, 0.0f);
  uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
  if (K > 0) a = lds_u4(dpk);
  if (K > 4) b = lds_u4(dpk + 16u);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const uint32_t w = j == 0 ? a.x : j == 1 ? a.y : j == 2 ? a.z : j == 3 ? a.w
                     : j == 4 ? b.x : j == 5 ? b.y : j == 6 ? b.z : b.w;
    const float s = desc_sign(w);
    const float2 s2 = make_float2(s, s);
    const unsigned row = base + (w & 0xffffu);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (V == 4) {
        const float4 x = lds_f4(row + 512 * q);
        acc[2 * q] = ffma2(s2, make_float2(x.x, x.y), acc[2 * q]);
        acc[2 * q + 1] = ffma2(s2, make_float2(x.z, x.w), acc[2 * q + 1]);
      } else {
        acc[q] = ffma2(s2, lds_f2(row + 256 * q), acc[q]);
      }
    }
  }
}

template <int V, int NQ>
__device__ __forceinline__ void proj_lean8(unsigned tile, unsigned dpk, int k, int lane, float2 (&acc)[V * NQ / 2]) {
  const unsigned base = tile + 4u * V * lane;
  switch (k) {
    case 1: proj_fixed<V, NQ, 1>(base, dpk, acc); break;
    case 2: proj_fixed<V, NQ, 2>(base, dpk, acc); break;
    case 3: proj_fixed<V, NQ, 3>(base, dpk, acc); break;
    case 4: proj_fixed<V, NQ, 4>(base, dpk, acc); break;
    case 5: proj_fixed<V, NQ, 5>(base, dpk, acc); break;
    case 6: proj_fixed<V, NQ, 6>(base, dpk, acc); break;
    case 7: proj_fixed<V, NQ, 7>(base, dpk, acc); break;
    case 8: proj_fixed<V, NQ, 8>(base, dpk, acc); break;
    default: proj_fixed<V, NQ, 0>(base, dpk, acc); break;  // an empty row projects to +0
  }
}

// The projection of a tile: the straight-line form when rows hold at most 8
// terms, else the loop.
template <int V, int NQ, int KMAX>
__device__ __forceinline__ void proj_any(unsigned tile, unsigned dpk, int k, int lane, float2 (&acc)[V * NQ / 2]) {
  if (KMAX <= 8)
    proj_lean8<V, NQ>(tile, dpk, k, lane, acc);
  else
    project_tile2<V, NQ>(tile, dpk, k, lane, acc);
}

// Label byte offsets (class * 4) of the lane's samples, in project_tile's
// order, from the item's label bytes (0xFF marks padding and labels outside
// [0, C); those get a very negative offset that the address clamp sends to
// the trash word).
__device__ __forceinline__ int label_off8(unsigned b) { return b != 0xFFu ? (int)(b * 4u) : (INT_MIN / 2); }

template <int V, int NQ>
__device__ __forceinline__ void tile_labels(unsigned lab, int lane, int (&yo)[V * NQ]) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (V == 4) {
      const unsigned w = lds_u32(lab + 128 * q + 4 * lane);
#pragma unroll
      for (int v = 0; v < 4; ++v) yo[4 * q + v] = label_off8((w >> (8 * v)) & 0xffu);
    } else {
      const unsigned w = lds_u16(lab + 64 * q + 2 * lane);
      yo[2 * q] = label_off8(w & 0xffu);
      yo[2 * q + 1] = label_off8(w >> 8);
    }
  }
}

// The item's tile loop, one instantiation per tile width St = 32 * V * NQ
// (the same for every warp of the CTA).  kMmBuf tile buffers: tiles tt+1 ..
// tt+kMmBuf-1 are in flight while tile tt is evaluated, one barrier per tile
// (four and five buffers measured no faster than three, on contiguous and on
// gathered items).  Warp w evaluates its assigned projections, keeping each
// lane's running minima and maxima in registers, then reduces them over its
// lanes into the node's keys (no shared-memory staging of the minima: the
// 64 KB it took left the L1 cache less room, 0.680 -> 0.646 ms at the root).
template <int V, int NQ, int KMAX>
__device__ __forceinline__ void mm_item(const DatasetView& ds, const int32_t* __restrict__ idx, const ItemPos& it,
                                        int U, bool contig, bool rowmaj, int Sp, float* s_tile, const int* s_rowfeat,
                                        const int64_t* s_rowoff, const int* s_assign, int nslot, const int* s_dk,
                                        const uint32_t* s_dpk, uint32_t* mm, int P, int lane, int warp, float* vbuf,
                                        int64_t n_total) {
  constexpr int St = 32 * V * NQ;
  const int ntile = (int)((it.end - it.beg + St - 1) / St);
  const int* my = s_assign + warp * nslot;
  // the lane's running minima and maxima of the warp's projections (at most
  // kMmPPW) stay in registers over the item's tiles, and so do the slots'
  // projections and row lengths (pl | k << 16, -1: empty slot)
  float mns[kMmPPW], mxs[kMmPPW];
  int pks[kMmPPW];
#pragma unroll
  for (int sl = 0; sl < kMmPPW; ++sl) {
    mns[sl] = INFINITY;
    mxs[sl] = -INFINITY;
    const int pl = sl < nslot ? my[sl] : -1;
    pks[sl] = pl < 0 ? -1 : (pl | (s_dk[pl] << 16));
  }
  const Stager sg = stager_init(ds, idx, it, St, U, s_rowfeat, contig, rowmaj, Sp);
  // tiles 0 .. kMmBuf-2 in flight before the first is evaluated
#pragma unroll
  for (int b = 0; b < kMmBuf - 1; ++b) {
    if (b < ntile) stager_issue(sg, ds, idx, it, b, St, U, s_rowoff, s_tile + b * kTileF);
    cp_async_commit();
  }
  int bc = 0, bi = kMmBuf - 1;  // buffer of tile tt, buffer of tile tt + kMmBuf - 1
  for (int tt = 0; tt < ntile; ++tt) {
    cp_async_wait_n<kMmBuf - 2>();
    __syncthreads();  // tile tt visible; every warp done with tile tt-1
    if (tt + kMmBuf - 1 < ntile) stager_issue(sg, ds, idx, it, tt + kMmBuf - 1, St, U, s_rowoff, s_tile + bi * kTileF);
    cp_async_commit();
    const unsigned tile = su32(s_tile) + 4u * kTileF * bc;
    bc = bc == kMmBuf - 1 ? 0 : bc + 1;
    bi = bi == kMmBuf - 1 ? 0 : bi + 1;
#pragma unroll
    for (int sl = 0; sl < kMmPPW; ++sl) {
      if (pks[sl] < 0) break;
      const int pl = pks[sl] & 0xffff;
      float2 acc[V * NQ / 2];
      proj_any<V, NQ, KMAX>(tile, su32(s_dpk) + 4u * pl * KMAX, pks[sl] >> 16, lane, acc);
#pragma unroll
      for (int i = 0; i < V * NQ / 2; ++i) {
        mns[sl] = fmin3(mns[sl], acc[i].x, acc[i].y);
        mxs[sl] = fmax3(mxs[sl], acc[i].x, acc[i].y);
      }
      if (vbuf) {
        // keep the values for the histogram pass (positions of this node only)
        const int64_t t0 = it.beg + (int64_t)tt * St;
        float* vp = vbuf + (int64_t)(it.p0 + pl) * n_total + t0;
        const int64_t rem = it.end - t0;
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int u = 0; u < V; ++u) {
            const int e = 32 * V * q + V * lane + u;
            const float2 a2 = acc[(V * q + u) >> 1];
            if (e < rem) vp[e] = (u & 1) ? a2.y : a2.x;
          }
      }
    }
  }
  // the warp's projections: minimum and maximum over its lanes, into the
  // node's order-preserving keys
#pragma unroll
  for (int sl = 0; sl < kMmPPW; ++sl) {
    if (pks[sl] < 0) break;
    const int pl = pks[sl] & 0xffff;
    const float a = warp_min(mns[sl]), b = warp_max(mxs[sl]);
    if (lane == 0) {
      atomicMin(&mm[(it.h * P + it.p0 + pl) * 2], f2key(a));
      atomicMax(&mm[(it.h * P + it.p0 + pl) * 2 + 1], f2key(b));
    }
  }
}

template <int KMAX>
__global__ void __launch_bounds__(kStThreads, 1) k_mm_staged(DatasetView ds, const int32_t* __restrict__ idx,
                                                            ProjView pv, StagedPlan sp, uint32_t* mm, float* vbuf,
                                                            int64_t n_total) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  const int nw = (ds.d + 31) >> 5;
  float* s_tile = reinterpret_cast<float*>(s_raw);  // [kMmBuf][kTileF]
  uint32_t* s_dpk = reinterpret_cast<uint32_t*>(s_tile + kMmBuf * kTileF);  // [kMmGroup*KMAX]
  int* s_dk = reinterpret_cast<int*>(s_dpk + kMmGroup * KMAX);             // [kMmGroup]
  int* s_assign = s_dk + kMmGroup;                                         // [kMmGroup]
  int* s_rowfeat = s_assign + kMmGroup;                                    // [kStUMax]
  int64_t* s_rowoff = reinterpret_cast<int64_t*>(s_rowfeat + kStUMax);     // [kStUMax]
  // the feature bitmap is only used while an item is set up, before tile
  // kMmBuf-1 is copied: it shares the last tile buffer
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(s_tile + (kMmBuf - 1) * kTileF);  // [nw]
  int* s_wpre = reinterpret_cast<int*>(s_bits + nw);                       // [nw]
  __shared__ int s_misc[kStWarps + 1];
  __shared__ int s_kcnt[kMaxCap + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = pv.P;
  const int64_t n_items = items_total(sp);
  __shared__ int64_t s_item;
  for (int64_t t = next_item(sp, &s_item); t < n_items; t = next_item(sp, &s_item)) {
    const ItemPos it = decode_item(sp, t, P);
    const int64_t qbase = (int64_t)it.j * P + it.p0;
    __syncthreads();  // previous item done with shared memory
    const bool contig = item_contiguous(ds, idx, it.beg, it.end);  // includes a barrier
    const int U = build_rows(pv, qbase, it.np, ds.d, s_bits, s_wpre, s_rowfeat, s_misc);
    // scattered samples whose rows are short enough: read the feature rows
    // from the row-major copy (a row of d <= 8 U floats costs fewer DRAM
    // sectors than U separate gathers)
    bool rowmaj = false;
    if (ds.Xr && !contig && U <= kRowMajUMax && ds.d <= 8 * U) {
      const int64_t span = (int64_t)idx[it.end - 1] - (int64_t)idx[it.beg];
      rowmaj = span < 0 || span > 4 * (it.end - it.beg);
    }
    const int St = rowmaj ? choose_st_pad(U) : choose_st(U);
    const int Sp = rowmaj ? St + 4 : St;  // row stride of the tile in shared memory
    build_desc<KMAX>(pv, qbase, it.np, ds.d, Sp, s_bits, s_wpre, s_dk, s_dpk);
    __syncthreads();  // s_dk and s_rowfeat complete
    for (int r = threadIdx.x; r < U && r < kStUMax; r += kStThreads) s_rowoff[r] = (int64_t)s_rowfeat[r] * ds.ld;
    const int nslot = assign_snake(it.np, s_dk, s_kcnt, s_assign);
    __syncthreads();  // assignment and row offsets visible
    if (U <= kMmUMax) {
      if (St == 256)
        mm_item<4, 2, KMAX>(ds, idx, it, U, contig, rowmaj, Sp, s_tile, s_rowfeat, s_rowoff, s_assign, nslot, s_dk,
                            s_dpk, mm, P, lane, warp, vbuf, n_total);
      else if (St == 128)
        mm_item<4, 1, KMAX>(ds, idx, it, U, contig, rowmaj, Sp, s_tile, s_rowfeat, s_rowoff, s_assign, nslot, s_dk,
                            s_dpk, mm, P, lane, warp, vbuf, n_total);
      else
        mm_item<2, 1, KMAX>(ds, idx, it, U, contig, rowmaj, Sp, s_tile, s_rowfeat, s_rowoff, s_assign, nslot, s_dk,
                            s_dpk, mm, P, lane, warp, vbuf, n_total);
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
          if (vbuf) vbuf[(int64_t)(it.p0 + pl) * n_total + e] = acc;
        }
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0) {
          atomicMin(&mm[(it.h * P + it.p0 + pl) * 2], f2key(mn));
          atomicMax(&mm[(it.h * P + it.p0 + pl) * 2 + 1], f2key(mx));
        }
      }
    }
  }
}

// ---- k_hist_staged: class-count histograms -----------------------------------
// 16-bit counters in shared memory, two counter slots per 32-bit word: slots
// (2i, 2i+1) share a [B+1][C] array of words (one spare bin), slot 2i in the
// low half, 2i+1 in the high half; then a trash word.  A projection's slot is
// its place in the warp assignment (warp w's s-th projection takes slot
// w * nslot + s), so when a warp holds two projections they share one word
// array and one base address.  A warp's atomic add touches one half only, so
// lanes of one instruction collide only on the same (bin, class).  An item
// holds at most 65535 samples, so no counter overflows.  Addresses are byte
// offsets clamped (as unsigned) to the trash word, which absorbs padding
// positions (label offset very negative), labels outside [0, C) and
// non-finite projected values.
// Counter word arrays of a group of PG projections: more than 32 projections
// take two slots per warp (slots up to 63), at most 32 one slot per warp.
__host__ __device__ __forceinline__ int hist_pairs(int PG) { return PG > kStWarps ? kStWarps : (PG + 1) >> 1; }

struct BinParams {
  float mn, W, inv_w, c;
  unsigned hb;   // byte base of the projection pair's words minus magic*C*4 (mod 2^32)
  unsigned inc;  // 1 or 1 << 16
  int fast;
};


// Label offsets of the tile (one int per sample, decoded once per tile), in
// project_tile's order.
template <int V, int NQ>
__device__ __forceinline__ void tile_offsets(unsigned yo_tile, int lane, int (&yo)[V * NQ]) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if (V == 4) {
      const uint4 y = lds_u4(yo_tile + 4u * (128 * q + 4 * lane));
      yo[4 * q] = (int)y.x;
      yo[4 * q + 1] = (int)y.y;
      yo[4 * q + 2] = (int)y.z;
      yo[4 * q + 3] = (int)y.w;
    } else {
      const float2 y = lds_f2(yo_tile + 4u * (64 * q + 2 * lane));
      yo[2 * q] = __float_as_int(y.x);
      yo[2 * q + 1] = __float_as_int(y.y);
    }
  }
}

template <int V, int NQ>
__device__ __forceinline__ void hist_tile_fast(unsigned tile, unsigned yo_tile, unsigned dpk, int k, int lane,
                                               const BinParams& bp, unsigned C4, unsigned limit) {
  float2 acc[V * NQ / 2];
  int yo[V * NQ];
  project_tile2<V, NQ>(tile, dpk, k, lane, acc);
  tile_offsets<V, NQ>(yo_tile, lane, yo);
  const float2 inv2 = make_float2(bp.inv_w, bp.inv_w);
  const float2 c2 = make_float2(bp.c, bp.c);
  const float2 m2 = make_float2(kMagic, kMagic);
  const float2 m1 = make_float2(1.0f - kMagic, 1.0f - kMagic);
#pragma unroll
  for (int i = 0; i < V * NQ / 2; ++i) {
    // q = round(v / W + c') by the 1.5 * 2^23 shift (packed: one fused
    // multiply-add, then additions that cannot fuse with it); the exact
    // boundary t_{q+1} = min + (q+1) * W with two roundings (scalar, so the
    // multiply and the add stay separate) decides between q and q+1
    const float2 e = ffma2(acc[i], inv2, c2);
    const float2 tq = fadd2(e, m2);
    const float2 q1 = fadd2(tq, m1);
    const float tbx = __fadd_rn(bp.mn, __fmul_rn(q1.x, bp.W));
    const float tby = __fadd_rn(bp.mn, __fmul_rn(q1.y, bp.W));
    unsigned ax = __float_as_uint(tq.x) * C4 + (bp.hb + (unsigned)yo[2 * i]);
    unsigned ay = __float_as_uint(tq.y) * C4 + (bp.hb + (unsigned)yo[2 * i + 1]);
    if (tbx <= acc[i].x) ax += C4;
    if (tby <= acc[i].y) ay += C4;
    reds_add(min(ax, limit), bp.inc);
    reds_add(min(ay, limit), bp.inc);
  }
}

// hist_tile_fast for the NS (1 or 2) projections a warp holds, sharing the
// tile's label offsets and their counter base (a warp's two projections take
// the two halves of one word array), with the straight-line projection for
// rows of at most 8 terms.
template <int V, int NQ, int KMAX, int NS>
__device__ __forceinline__ void hist_tile_warp(unsigned tile, unsigned yo_tile, unsigned dpk0, unsigned dpk1, int k0,
                                               int k1, int lane, const BinParams& b0, const BinParams& b1,
                                               unsigned C4, unsigned limit) {
  unsigned hy[V * NQ];
  {
    int yo[V * NQ];
    tile_offsets<V, NQ>(yo_tile, lane, yo);
#pragma unroll
    for (int i = 0; i < V * NQ; ++i) hy[i] = b0.hb + (unsigned)yo[i];
  }
  const float2 m2 = make_float2(kMagic, kMagic);
  const float2 m1 = make_float2(1.0f - kMagic, 1.0f - kMagic);
#pragma unroll
  for (int sp = 0; sp < NS; ++sp) {
    const BinParams& bp = sp ? b1 : b0;
    float2 acc[V * NQ / 2];
    proj_any<V, NQ, KMAX>(tile, sp ? dpk1 : dpk0, sp ? k1 : k0, lane, acc);
    const float2 inv2 = make_float2(bp.inv_w, bp.inv_w);
    const float2 c2 = make_float2(bp.c, bp.c);
#pragma unroll
    for (int i = 0; i < V * NQ / 2; ++i) {
      // the bin rule of hist_tile_fast
      const float2 e = ffma2(acc[i], inv2, c2);
      const float2 tq = fadd2(e, m2);
      const float2 q1 = fadd2(tq, m1);
      const float tbx = __fadd_rn(bp.mn, __fmul_rn(q1.x, bp.W));
      const float tby = __fadd_rn(bp.mn, __fmul_rn(q1.y, bp.W));
      unsigned ax = __float_as_uint(tq.x) * C4 + hy[2 * i];
      unsigned ay = __float_as_uint(tq.y) * C4 + hy[2 * i + 1];
      if (tbx <= acc[i].x) ax += C4;
      if (tby <= acc[i].y) ay += C4;
      reds_add(min(ax, limit), bp.inc);
      reds_add(min(ay, limit), bp.inc);
    }
  }
}

// exact estimate-and-correct rule for projections outside the fast condition
template <int V, int NQ>
__device__ __forceinline__ void hist_tile_slow(unsigned tile, unsigned yo_tile, unsigned dpk, int k, int lane,
                                               const BinParams& bp, int B, int C, int wbase, uint32_t* s_hist) {
  float acc[V * NQ];
  int yo[V * NQ];
  project_tile<V, NQ>(tile, dpk, k, lane, acc);
  tile_offsets<V, NQ>(yo_tile, lane, yo);
#pragma unroll
  for (int i = 0; i < V * NQ; ++i)
    if (yo[i] >= 0) atomicAdd(&s_hist[wbase + bin_of(acc[i], bp.mn, bp.W, bp.inv_w, B) * C + (yo[i] >> 2)], bp.inc);
}

// Random-width bins of a tile: the packed projection of hist_tile_fast, then
// per sample the bin from the projection's boundary tables in shared memory
// (bp.mn, bp.W hold the cell map's s and o; bp.hb the pair's counter base).
template <int V, int NQ, bool GUIDED>
__device__ __forceinline__ void hist_tile_rw(unsigned tile, unsigned yo_tile, unsigned dpk, int k, int lane,
                                             const BinParams& bp, unsigned tb, unsigned gb, int nb, unsigned C4,
                                             unsigned limit) {
  float2 acc[V * NQ / 2];
  int yo[V * NQ];
  project_tile2<V, NQ>(tile, dpk, k, lane, acc);
  tile_offsets<V, NQ>(yo_tile, lane, yo);
#pragma unroll
  for (int i = 0; i < V * NQ / 2; ++i) {
    const unsigned bx = (unsigned)rw_bin_smem<GUIDED>(acc[i].x, bp.mn, bp.W, tb, gb, nb);
    const unsigned by = (unsigned)rw_bin_smem<GUIDED>(acc[i].y, bp.mn, bp.W, tb, gb, nb);
    reds_add(min(bx * C4 + (bp.hb + (unsigned)yo[2 * i]), limit), bp.inc);
    reds_add(min(by * C4 + (bp.hb + (unsigned)yo[2 * i + 1]), limit), bp.inc);
  }
}

// The item's tile loop for tile width St = 32 * V * NQ.  Three tile buffers,
// one barrier per tile; labels go through a register one tile ahead.  Warp w
// evaluates its assigned projections (at most kHistPPW) with their bin
// parameters in registers.
template <int V, int NQ, bool RW, int KMAX>
__device__ __forceinline__ void hist_item(const DatasetView& ds, const int32_t* __restrict__ idx, const ItemPos& it,
                                          int U, bool contig, float* s_tile, const uint8_t* s_lab, int* s_yo,
                                          const int* s_rowfeat,
                                          const int64_t* s_rowoff, const int* s_assign, int nslot, const int* s_dk, const uint32_t* s_dpk,
                                          int kmax, const float4* s_bpf, const int4* s_bpi, int B, int HS,
                                          unsigned C4, unsigned limit, uint32_t* s_hist, unsigned rwt, unsigned rwg,
                                          int lane, int warp) {
  constexpr int St = 32 * V * NQ;
  const int C = ds.C;
  const int ntile = (int)((it.end - it.beg + St - 1) / St);
  int pls[kHistPPW], ks[kHistPPW];
  BinParams bps[kHistPPW];
#pragma unroll
  for (int sl = 0; sl < kHistPPW; ++sl) {
    pls[sl] = sl < nslot ? s_assign[warp * nslot + sl] : -1;
    const int pl = pls[sl] >= 0 ? pls[sl] : 0;
    ks[sl] = pls[sl] >= 0 ? s_dk[pl] : 0;
    const float4 bf = s_bpf[pl];
    const int4 bi = s_bpi[pl];
    // absolute shared address base: the unsigned wrap of the clamp is kept
    // (a valid address stays below the shared window's end, a rejected one
    // stays far above it)
    bps[sl] = BinParams{bf.x, bf.y, bf.z, bf.w, su32(s_hist) + (unsigned)bi.x, (unsigned)bi.y, bi.z};
  }
  const unsigned limit_abs = su32(s_hist) + limit;
  // every projection of the warp on the fast equal-width rule: one pass per
  // tile over both (shared label offsets and counter base)
  const int nps = (pls[0] >= 0 ? 1 : 0) + (kHistPPW > 1 && pls[kHistPPW - 1] >= 0 ? 1 : 0);
  const bool warp_fast = !RW && (pls[0] < 0 || bps[0].fast) && (kHistPPW < 2 || pls[kHistPPW - 1] < 0 ||
                                                                   bps[kHistPPW - 1].fast);
  const Stager sg = stager_init(ds, idx, it, St, U, s_rowfeat, contig);
  // label byte offsets of tile t into s_yo[t % 3], written with tile t's copies
  auto tile_yo = [&](int t, int b) {
    if ((int)threadIdx.x < St) s_yo[b * 256 + threadIdx.x] = label_off8(s_lab[t * St + threadIdx.x]);
  };
  if (ntile > 0) {
    stager_issue(sg, ds, idx, it, 0, St, U, s_rowoff, s_tile);
    tile_yo(0, 0);
  }
  cp_async_commit();
  if (ntile > 1) {
    stager_issue(sg, ds, idx, it, 1, St, U, s_rowoff, s_tile + kTileF);
    tile_yo(1, 1);
  }
  cp_async_commit();
  int bc = 0, bn = 1, bi = 2;  // buffers of tiles tt, tt + 1, tt + 2
  for (int tt = 0; tt < ntile; ++tt) {
    cp_async_wait1();
    __syncthreads();  // tile tt visible; every warp done with tile tt-1
    if (tt + 2 < ntile) {
      stager_issue(sg, ds, idx, it, tt + 2, St, U, s_rowoff, s_tile + bi * kTileF);
      tile_yo(tt + 2, bi);
    }
    cp_async_commit();
    const unsigned tile = su32(s_tile) + 4u * kTileF * bc;
    const unsigned lab = su32(s_yo) + 4u * 256 * bc;
    bc = bn;
    bn = bi;
    bi = bi == 2 ? 0 : bi + 1;
    if (warp_fast) {
      const unsigned d0 = su32(s_dpk) + 4u * (pls[0] >= 0 ? pls[0] : 0) * kmax;
      const unsigned d1 = su32(s_dpk) + 4u * (pls[kHistPPW - 1] >= 0 ? pls[kHistPPW - 1] : 0) * kmax;
      if (nps == 2)
        hist_tile_warp<V, NQ, KMAX, 2>(tile, lab, d0, d1, ks[0], ks[kHistPPW - 1], lane, bps[0], bps[kHistPPW - 1],
                                       C4, limit_abs);
      else if (nps == 1)
        hist_tile_warp<V, NQ, KMAX, 1>(tile, lab, d0, d1, ks[0], ks[0], lane, bps[0], bps[0], C4, limit_abs);
    } else {
#pragma unroll
      for (int sl = 0; sl < kHistPPW; ++sl) {
        if (pls[sl] >= 0) {
          const unsigned dpk = su32(s_dpk) + 4u * pls[sl] * kmax;
          if (RW) {
            const unsigned tb = rwt + 4u * kRwRow * pls[sl], gb = rwg + 2u * kRwRow * pls[sl];
            if (bps[sl].fast)
              hist_tile_rw<V, NQ, true>(tile, lab, dpk, ks[sl], lane, bps[sl], tb, gb, B - 1, C4, limit_abs);
            else
              hist_tile_rw<V, NQ, false>(tile, lab, dpk, ks[sl], lane, bps[sl], tb, gb, B - 1, C4, limit_abs);
          } else if (bps[sl].fast) {
            hist_tile_fast<V, NQ>(tile, lab, dpk, ks[sl], lane, bps[sl], C4, limit_abs);
          } else {
            hist_tile_slow<V, NQ>(tile, lab, dpk, ks[sl], lane, bps[sl], B, C, ((warp * nslot + sl) >> 1) * HS,
                                  s_hist);
          }
        }
      }
    }
  }
}

// The item's histograms from projected values kept by the min / max pass (the
// node's samples are gathered, so reading 4 bytes per sample-projection beats
// gathering the feature columns again).  No tiles and no barriers: each warp
// streams its assigned projections over the item, four samples per lane and
// four steps in flight.
template <bool RW>
__device__ __forceinline__ void hist_item_buf(const float* __restrict__ vbuf, int64_t n_total, const ItemPos& it,
                                              unsigned lab_base, const int* s_assign, int nslot,
                                              const float4* s_bpf, const int4* s_bpi, int B, int C, int HS,
                                              unsigned C4, unsigned limit_abs, uint32_t* s_hist, unsigned rwt,
                                              unsigned rwg, int lane, int warp) {
  const int len = (int)(it.end - it.beg);
  for (int sl = 0; sl < nslot; ++sl) {
    const int pl = s_assign[warp * nslot + sl];
    if (pl < 0) break;
    const float4 bf = s_bpf[pl];
    const int4 bi = s_bpi[pl];
    const BinParams bp{bf.x, bf.y, bf.z, bf.w, su32(s_hist) + (unsigned)bi.x, (unsigned)bi.y, bi.z};
    const float* vp = vbuf + (int64_t)(it.p0 + pl) * n_total + it.beg;
    for (int e0 = 0; e0 < len; e0 += 512) {
      float v[16];
      int yo[16];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int e = e0 + 128 * u + 4 * lane + w;
          v[4 * u + w] = e < len ? __ldg(vp + e) : __int_as_float(0x7fc00000);
        }
        const unsigned lw = lds_u32(lab_base + (unsigned)(e0 + 128 * u + 4 * lane));
#pragma unroll
        for (int w = 0; w < 4; ++w) yo[4 * u + w] = label_off8((lw >> (8 * w)) & 0xffu);
      }
      if (RW) {
        const unsigned tb = rwt + 4u * kRwRow * pl, gb = rwg + 2u * kRwRow * pl;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const unsigned b = (unsigned)(bp.fast ? rw_bin_smem<true>(v[i], bp.mn, bp.W, tb, gb, B - 1)
                                                : rw_bin_smem<false>(v[i], bp.mn, bp.W, tb, gb, B - 1));
          reds_add(min(b * C4 + (bp.hb + (unsigned)yo[i]), limit_abs), bp.inc);
        }
      } else if (bp.fast) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float tq = __fadd_rn(__fmaf_rn(v[i], bp.inv_w, bp.c), kMagic);
          const float q1 = __fadd_rn(tq, 1.0f - kMagic);
          const float tb = __fadd_rn(bp.mn, __fmul_rn(q1, bp.W));
          unsigned a = __float_as_uint(tq) * C4 + (bp.hb + (unsigned)yo[i]);
          if (tb <= v[i]) a += C4;
          reds_add(min(a, limit_abs), bp.inc);
        }
      } else {
        const int wbase = ((warp * nslot + sl) >> 1) * HS;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (yo[i] >= 0) atomicAdd(&s_hist[wbase + bin_of(v[i], bp.mn, bp.W, bp.inv_w, B) * C + (yo[i] >> 2)], bp.inc);
      }
    }
  }
}

template <int KMAX, bool RW>
__global__ void __launch_bounds__(kStThreads, 1) k_hist_staged(DatasetView ds, const int32_t* __restrict__ idx,
                                                              ProjView pv, StagedPlan sp, int B, int PG,
                                                              const uint32_t* __restrict__ mm, int32_t* hist,
                                                              const float* __restrict__ vbuf, int64_t n_total,
                                                              RwTables rw) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  const int nw = (ds.d + 31) >> 5;
  const int C = ds.C;
  const int HS = (B + 1) * C;  // words per counter pair
  const int npair = hist_pairs(PG);
  const int hist_words = (npair * HS + 1 + 3) & ~3;
  // every region starts on a 16-byte boundary
  float* s_tile = reinterpret_cast<float*>(s_raw);  // [3][kTileF]
  uint8_t* s_lab = reinterpret_cast<uint8_t*>(s_tile + 3 * kTileF);          // [kMaxItem + 512] item labels
  int* s_yo = reinterpret_cast<int*>(s_lab + kMaxItem + 512);                // [3][256] tile label offsets
  uint32_t* s_hist = reinterpret_cast<uint32_t*>(s_yo + 3 * 256);            // [hist_words]
  float* s_rwt = reinterpret_cast<float*>(s_hist + hist_words);              // RW: [PG][kRwRow] boundaries
  uint16_t* s_rwg = reinterpret_cast<uint16_t*>(s_rwt + (RW ? PG * kRwRow : 0));  // RW: [PG][kRwRow] guide
  uint32_t* s_dpk = reinterpret_cast<uint32_t*>(s_rwg + (RW ? PG * kRwRow : 0));   // [kHistPGMax*KMAX]
  int* s_dk = reinterpret_cast<int*>(s_dpk + kHistPGMax * KMAX);             // [kHistPGMax]
  int* s_assign = s_dk + kHistPGMax;                                         // [kHistPGMax]
  int* s_rowfeat = s_assign + kHistPGMax;                                    // [kStUMax]
  int64_t* s_rowoff = reinterpret_cast<int64_t*>(s_rowfeat + kStUMax);       // [kStUMax]
  // the feature bitmap is only used while an item is set up, before tile 2
  // is copied: it shares the third tile buffer
  uint32_t* s_bits = reinterpret_cast<uint32_t*>(s_tile + 2 * kTileF);       // [nw]
  int* s_wpre = reinterpret_cast<int*>(s_bits + nw);                         // [nw]
  __shared__ float4 s_bpf[kHistPGMax];  // min, W, 1/W, c
  __shared__ int4 s_bpi[kHistPGMax];    // hb, inc, fast
  __shared__ int s_slot[kHistPGMax];    // counter slot of each projection
  __shared__ int s_misc[kStWarps + 1];
  __shared__ int s_kcnt[kMaxCap + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = pv.P;
  const unsigned C4 = (unsigned)C * 4u;
  const unsigned limit = (unsigned)(npair * HS) * 4u;  // byte offset of the trash word
  const unsigned magic_bits = __float_as_uint(kMagic);
  const int64_t n_items = items_total(sp);
  __shared__ int64_t s_item;
  for (int64_t t = next_item(sp, &s_item); t < n_items; t = next_item(sp, &s_item)) {
    const ItemPos it = decode_item(sp, t, P);
    const int64_t qbase = (int64_t)it.j * P + it.p0;
    __syncthreads();  // previous item's flush finished
    {
      int4* h4 = reinterpret_cast<int4*>(s_hist);
      for (int e = threadIdx.x; e < hist_words / 4; e += kStThreads) h4[e] = make_int4(0, 0, 0, 0);
    }
    int U = 0, St = 64;
    if (!vbuf) {
      U = build_rows(pv, qbase, it.np, ds.d, s_bits, s_wpre, s_rowfeat, s_misc);
      St = choose_st(U);
      build_desc<KMAX>(pv, qbase, it.np, ds.d, St, s_bits, s_wpre, s_dk, s_dpk);
    } else if (threadIdx.x < it.np) {
      s_dk[threadIdx.x] = 1;  // every projection costs the same when its values are read back
    }
    if (RW) {
      // the group's boundary rows and guides, 16 bytes per copy
      const int64_t row0 = (it.h * P + it.p0) * (int64_t)kRwRow;
      const int4* gt = reinterpret_cast<const int4*>(rw.t + row0);
      const int4* gg = reinterpret_cast<const int4*>(rw.g + row0);
      int4* st4 = reinterpret_cast<int4*>(s_rwt);
      int4* sg4 = reinterpret_cast<int4*>(s_rwg);
      for (int e = threadIdx.x; e < it.np * (kRwRow / 4); e += kStThreads) st4[e] = gt[e];
      for (int e = threadIdx.x; e < it.np * (kRwRow / 8); e += kStThreads) sg4[e] = gg[e];
      if (threadIdx.x < it.np) {
        const int pl = threadIdx.x;
        const float2 so = rw.so[it.h * P + it.p0 + pl];
        s_bpf[pl] = make_float4(so.x, so.y, 0.0f, 0.0f);
        s_bpi[pl] = make_int4(0, 0, so.x >= 0.0f ? 1 : 0, 0);  // counter base and increment: below
      }
    } else if (threadIdx.x < it.np) {
      const int pl = threadIdx.x;
      const float mn = key2f(mm[(it.h * P + it.p0 + pl) * 2]);
      const float mx = key2f(mm[(it.h * P + it.p0 + pl) * 2 + 1]);
      const float W = bin_width(mn, mx, B);
      const float inv_w = __frcp_rn(W);
      const float c = __fsub_rn(__fmul_rn(-mn, inv_w), 0.75f);
      const float M = fmaxf(fabsf(mn), fabsf(mx));
      const int fast = (W > 0.0f && isfinite(inv_w) && isfinite(c) && M <= kCondLimit * W) ? 1 : 0;
      s_bpf[pl] = make_float4(mn, W, inv_w, c);
      s_bpi[pl] = make_int4(0, 0, fast, 0);  // counter base and increment: below
    }
    __syncthreads();  // s_dk and s_rowfeat complete
    for (int r = threadIdx.x; r < U && r < kStUMax; r += kStThreads) s_rowoff[r] = (int64_t)s_rowfeat[r] * ds.ld;
    const int nslot = assign_snake(it.np, s_dk, s_kcnt, s_assign, s_slot);
    __syncthreads();  // s_slot complete
    if (threadIdx.x < it.np) {
      // the projection's counters: word array of its slot pair, its half;
      // the fast equal-width rule adds the bin estimate's rounding shift
      // (magic * C4) to the base, so it is taken off here
      const int pl = threadIdx.x, sl = s_slot[pl];
      const unsigned base = (unsigned)((sl >> 1) * HS * 4);
      s_bpi[pl].x = (int)((RW || !s_bpi[pl].z) ? base : base - magic_bits * C4);
      s_bpi[pl].y = (int)(1u << (16 * (sl & 1)));
    }
    const bool contig = vbuf ? false : item_contiguous(ds, idx, it.beg, it.end);  // includes a barrier
    if (vbuf || U <= kStUMax) {
      // the item's labels as bytes (0xFF: padding or outside [0, C)); read
      // after the first tile barrier
      const int len = (int)(it.end - it.beg);
      for (int e = threadIdx.x; e < len + 512; e += kStThreads) {
        unsigned b = 0xFFu;
        if (e < len) {
          const unsigned y = ds.y[safe_sample(idx[it.beg + e], ds.n)];
          b = y < (unsigned)C ? y : 0xFFu;
        }
        s_lab[e] = (uint8_t)b;
      }
      const unsigned rwt = su32(s_rwt), rwg = su32(s_rwg);
      if (vbuf) {
        __syncthreads();  // labels and warp assignment visible
        hist_item_buf<RW>(vbuf, n_total, it, su32(s_lab), s_assign, nslot, s_bpf, s_bpi, B, C, HS, C4,
                          su32(s_hist) + limit, s_hist, rwt, rwg, lane, warp);
      } else if (St == 256)
        hist_item<4, 2, RW, KMAX>(ds, idx, it, U, contig, s_tile, s_lab, s_yo, s_rowfeat, s_rowoff, s_assign, nslot, s_dk, s_dpk, KMAX,
                            s_bpf, s_bpi, B, HS, C4, limit, s_hist, rwt, rwg, lane, warp);
      else if (St == 128)
        hist_item<4, 1, RW, KMAX>(ds, idx, it, U, contig, s_tile, s_lab, s_yo, s_rowfeat, s_rowoff, s_assign, nslot, s_dk, s_dpk, KMAX,
                            s_bpf, s_bpi, B, HS, C4, limit, s_hist, rwt, rwg, lane, warp);
      else
        hist_item<2, 1, RW, KMAX>(ds, idx, it, U, contig, s_tile, s_lab, s_yo, s_rowfeat, s_rowoff, s_assign, nslot, s_dk, s_dpk, KMAX,
                            s_bpf, s_bpi, B, HS, C4, limit, s_hist, rwt, rwg, lane, warp);
    } else {
      // direct path for wide groups (rare): one warp per projection, gathers
      for (int pl = warp; pl < it.np; pl += kStWarps) {
        const int64_t q = qbase + pl;
        const int rb = pv.beg[q];
        int k = pv.end[q] - rb;
        k = k < 0 ? 0 : (k > kMaxCap ? kMaxCap : k);
        const float4 bf = s_bpf[pl];
        const int slot = s_slot[pl];
        const unsigned inc = 1u << (16 * (slot & 1));
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
          int b;
          if (RW) {
            const unsigned tb = su32(s_rwt) + 4u * kRwRow * pl, gb = su32(s_rwg) + 2u * kRwRow * pl;
            b = bf.x >= 0.0f ? rw_bin_smem<true>(acc, bf.x, bf.y, tb, gb, B - 1)
                             : rw_bin_smem<false>(acc, bf.x, bf.y, tb, gb, B - 1);
          } else {
            b = bin_of(acc, bf.x, bf.y, bf.z, B);
          }
          if (yv < C) atomicAdd(&s_hist[(slot >> 1) * HS + b * C + yv], inc);
        }
      }
    }
    __syncthreads();
    // flush: the spare bin B folds into bin B-1
    const int BC = B * C;
    for (int pl = warp; pl < it.np; pl += kStWarps) {
      int32_t* g = hist + (it.h * P + it.p0 + pl) * (int64_t)BC;
      const int slot = s_slot[pl];
      const uint32_t* h = s_hist + (slot >> 1) * HS;
      const int sh = 16 * (slot & 1);
      for (int r = lane; r < BC; r += 32) {
        int v = (int)((h[r] >> sh) & 0xffffu);
        if (r >= BC - C) v += (int)((h[r + C] >> sh) & 0xffffu);
        if (v) atomicAdd(&g[r], v);
      }
    }
  }
}

// ---- host side ----------------------------------------------------------------
int hist_group_size(int B, int C, bool rw) {
  // 16-bit counters, two projections per word, plus the random-width tables
  // (boundaries and guide of each projection), in about 100 KB of shared
  // memory (a first estimate: the launch shrinks the group until the CTA's
  // whole shared memory fits the device limit).
  // Rounded down to a multiple of the 32 warps when at least 32: a group of,
  // say, 36 gives 4 warps two projections while 28 wait at every barrier.
  const int pair_bytes = (B + 1) * C * 4 + (rw ? 2 * kRwRow * 6 : 0);
  int pg = 2 * ((100 * 1024) / pair_bytes);
  if (pg >= kHistPGMax) return kHistPGMax;
  if (pg >= kStWarps) return kStWarps;
  return pg < 1 ? 1 : pg;
}

// The feature bitmap (2 * ceil(d/32) words <= 16 KB) lives in the third tile
// buffer, so d does not change the size.
static_assert(kStMaxWords * 8 <= kTileF * 4, "bitmap must fit a tile buffer");
size_t mm_smem_bytes(int /*d*/, int kmax) {
  return (size_t)kMmBuf * kTileF * 4 + (size_t)kMmGroup * kmax * 4 + kMmGroup * 8 + kStUMax * 12;
}
size_t hist_smem_bytes(int /*d*/, int kmax, int B, int C, int PG, bool rw) {
  const int npair = hist_pairs(PG);
  const size_t hist_words = ((size_t)npair * (B + 1) * C + 1 + 3) & ~(size_t)3;
  const size_t rw_bytes = rw ? (size_t)PG * kRwRow * 6 : 0;
  return (size_t)3 * kTileF * 4 + kMaxItem + 512 + 3 * 256 * 4 + hist_words * 4 + rw_bytes +
         (size_t)kHistPGMax * kmax * 4 + kHistPGMax * 8 + kStUMax * 12;
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
  s.item_ctr = cv.take<unsigned long long>(2);
}

template <int KMAX>
cudaError_t launch_staged_k(const SearchArgs& a, const V4* plan_total, const int32_t* hist_nodes, int64_t m_hist_cap,
                            const StagedScratch& ss, uint32_t* mm, int32_t* hist, const RwTables& rw, int64_t S,
                            cudaStream_t st) {
  const DeviceInfo& di = device_info();
  const int C = a.ds.C, B = a.B, d = a.ds.d;
  const bool RW = a.bin_rule == SO_BINS_RANDOM_WIDTH;
  auto kern = RW ? k_hist_staged<KMAX, true> : k_hist_staged<KMAX, false>;
  int PG = hist_group_size(B, C, RW);
  if (a.tune.staged_pg > 0 && a.tune.staged_pg < PG) PG = a.tune.staged_pg;
  {
    // the group's counters, tables and the fixed regions (which grow with
    // the row width KMAX) must fit one CTA's shared memory with the
    // kernel's static shared memory
    static thread_local size_t static_bytes[2] = {0, 0};
    static thread_local bool have[2] = {false, false};
    if (!have[RW]) {
      cudaFuncAttributes fa{};
      if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return cudaGetLastError();
      static_bytes[RW] = fa.sharedSizeBytes;
      have[RW] = true;
    }
    while (PG > 1 && hist_smem_bytes(d, KMAX, B, C, PG, RW) + static_bytes[RW] > (size_t)di.smem_optin)
      PG = PG > kStWarps ? kStWarps : PG - 1;
  }
  // histogram items: at most kMaxItem samples (label bytes in shared memory,
  // 16-bit counters); min / max items a quarter of that, so that a single
  // large node still spreads over every SM
  const int64_t S2 = S > kMaxItem ? kMaxItem : S;
  const int64_t S1 = S2 / 4 > 1024 ? S2 / 4 : (S2 < 1024 ? S2 : 1024);
  cudaError_t e;
  {
    const size_t smem = (size_t)4 * (((d + 31) >> 5) + kStUMax + 32 * 33) * 4;
    if (smem > 48 * 1024) {
      e = cudaFuncSetAttribute(k_groups, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    ProfScope ps_("k_groups", st);
    k_groups<<<di.num_sms * 2, 128, smem, st>>>(plan_total, hist_nodes, a.pv, d, kMmUMax, kMmGroup, kStUMax, PG,
                                                ss.ng1, ss.gs1, ss.ng2, ss.gs2);
  }
  ItemScanF isf{plan_total, hist_nodes, a.node_off, ss.ng1, ss.ng2, S1, S2, ss.item_off1, ss.item_off2};
  e = run_scan(isf, m_hist_cap, ss.tiles, ss.item_total, st, "item_scan");
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ss.item_ctr, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  StagedPlan sp1{plan_total, hist_nodes, a.node_off, ss.ng1, ss.gs1, ss.item_off1, ss.item_total, 0, S1,
                 ss.item_ctr};
  StagedPlan sp2{plan_total, hist_nodes, a.node_off, ss.ng2, ss.gs2, ss.item_off2, ss.item_total, 1, S2,
                 ss.item_ctr + 1};
  {
    const size_t smem = mm_smem_bytes(d, KMAX);
    e = cudaFuncSetAttribute(k_mm_staged<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope ps_("k_minmax", st);
    k_mm_staged<KMAX><<<di.num_sms, kStThreads, smem, st>>>(a.ds, a.idx, a.pv, sp1, mm, a.vbuf, a.n_total);
  }
  if (RW) {
    e = launch_rw_bounds(a, plan_total, hist_nodes, mm, rw, st);
    if (e != cudaSuccess) return e;
  }
  {
    const size_t smem = hist_smem_bytes(d, KMAX, B, C, PG, RW);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope ps_("k_hist", st);
    kern<<<di.num_sms, kStThreads, smem, st>>>(a.ds, a.idx, a.pv, sp2, B, PG, mm, hist, a.vbuf, a.n_total, rw);
  }
  return cudaGetLastError();
}

cudaError_t launch_staged(const SearchArgs& a, const V4* plan_total, const int32_t* hist_nodes, int64_t m_hist_cap,
                          const StagedScratch& ss, uint32_t* mm, int32_t* hist, const RwTables& rw, int64_t S,
                          int kmax, cudaStream_t st) {
  if (kmax <= 8) return launch_staged_k<8>(a, plan_total, hist_nodes, m_hist_cap, ss, mm, hist, rw, S, st);
  if (kmax <= 16) return launch_staged_k<16>(a, plan_total, hist_nodes, m_hist_cap, ss, mm, hist, rw, S, st);
  return launch_staged_k<32>(a, plan_total, hist_nodes, m_hist_cap, ss, mm, hist, rw, S, st);
}

}  // namespace sof
