// so_device.cuh -- device-side building blocks shared by the split-search
// kernels: ordered float keys, the projected value, the equal-width bin rule,
// the float and double Gini gains, splitmix64, and warp reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "so_internal.h"

namespace sof {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;       // splitmix64 increment
constexpr uint64_t kProjMult = 0xD2B74407B1CE6E93ull;    // separates projection streams
constexpr uint64_t kBinTag = 0x6A09E667F3BCC908ull;      // frac(sqrt 2): tags the boundary streams

// Order-preserving map float -> uint32 (total order of finite floats, -0 < +0).
__device__ __forceinline__ uint32_t f2key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  return __uint_as_float(u);
}

// Projected value of sample s (Section 3 step 1: a sparse vector sum of the
// selected columns).  Fixed order: +0, then the features in ascending order,
// each added (sign +1) or subtracted as a negated addend, round-to-nearest,
// never fused.  Starting from +0 makes a -0 result impossible.
__device__ __forceinline__ float project_value(const float* __restrict__ X, int64_t ld, int64_t s,
                                               const int32_t* f, const int8_t* sg, int k) {
  float acc = 0.0f;
  for (int j = 0; j < k; ++j) {
    const float x = __ldg(X + (int64_t)f[j] * ld + s);
    acc = __fadd_rn(acc, sg[j] == 1 ? x : -x);
  }
  return acc;
}

// Sample indices outside [0, n) are read as sample 0 (memory safety only;
// the documented contract is 0 <= idx < n).
__device__ __forceinline__ int64_t safe_sample(int32_t s, int64_t n) {
  return ((uint32_t)s < (uint64_t)n) ? (int64_t)s : 0;
}

// Equal-width bins (Section 3.2 with 256 bins): w = (max-min)/B, boundary
// t_j = min + j*w (float, round-to-nearest), bin(v) = #{ j in 1..B-1 : t_j <= v }.
__device__ __forceinline__ float bin_width(float mn, float mx, int B) {
  return __fdiv_rn(__fsub_rn(mx, mn), (float)B);
}
__device__ __forceinline__ float boundary(float mn, float w, int j) {
  return __fadd_rn(mn, __fmul_rn((float)j, w));
}
// The arithmetic estimate floor((v-min)/w) lands within one bin of the exact
// upper-bound count for well-spread ranges; the two loops correct it against
// the stored-boundary definition exactly (they run more than once only when
// the range is a few ulps wide and boundaries coincide).
__device__ __forceinline__ int bin_of(float v, float mn, float w, float inv_w, int B) {
  if (w == 0.0f) return B - 1;  // every boundary equals min <= v
  const float q = floorf(__fmul_rn(__fsub_rn(v, mn), inv_w));
  int b = (q >= 0.0f) ? ((q < (float)(B - 1)) ? (int)q : (B - 1)) : 0;
  while (b > 0 && v < boundary(mn, w, b)) --b;
  while (b < B - 1 && boundary(mn, w, b + 1) <= v) ++b;
  return b;
}

// Gini decrease of a candidate with left class counts L (node counts N):
// sum_c D_c^2 / (n^2 nL nR), D_c = n L_c - N_c nL exact in int64.
// Float version: a comparison key only (the n^2 factor is dropped); its
// relative error is at most (C+6) 2^-24 to first order.
__device__ __forceinline__ float gain32(const int* L, const int* N, int C, int64_t n, int64_t nL) {
  float num = 0.0f;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) {
    if (c < C) {
      const long long D = n * (long long)L[c] - (long long)N[c] * nL;
      const float fd = __ll2float_rn(D);
      num = __fadd_rn(num, __fmul_rn(fd, fd));
    }
  }
  const float den = __fmul_rn(__ll2float_rn(nL), __ll2float_rn(n - nL));
  return __fdiv_rn(num, den);
}

// Double version: the exact expression of the definition, one IEEE operation
// at a time: num = sum_c D_c*D_c (class order), g = num/(nL*nR), g = g/(n*n).
__device__ __forceinline__ double gain64(const int* L, const int* N, int C, int64_t n, int64_t nL) {
  double num = 0.0;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) {
    if (c < C) {
      const long long D = n * (long long)L[c] - (long long)N[c] * nL;
      const double dd = __ll2double_rn(D);
      num = __dadd_rn(num, __dmul_rn(dd, dd));
    }
  }
  const double g = __ddiv_rn(num, __dmul_rn(__ll2double_rn(nL), __ll2double_rn(n - nL)));
  return __ddiv_rn(g, __dmul_rn(__ll2double_rn(n), __ll2double_rn(n)));
}

// Exact-path threshold between consecutive distinct values a < b.
__device__ __forceinline__ float midpoint(float a, float b) {
  float t = __fadd_rn(a, __fmul_rn(0.5f, __fsub_rn(b, a)));
  if (!(a < t) || !(t <= b)) t = b;
  return t;
}

// splitmix64 (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t sm64_next(uint64_t& s) {
  uint64_t z = (s += kGamma);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sm64(uint64_t x) {
  uint64_t s = x;
  return sm64_next(s);
}
// Output j (0-based) of the generator whose state is s0: the state after j+1
// increments, mixed.
__device__ __forceinline__ uint64_t sm64_at(uint64_t s0, int j) {
  uint64_t s = s0 + (uint64_t)j * kGamma;
  return sm64_next(s);
}

// ---- random-width boundaries (the YDF default of the paper's Section 1
// footnote): projection p of the node with key K draws B-1 splitmix64 outputs
// from state sm64((K ^ kBinTag) + p*kProjMult); the top 23 bits u of each,
// sorted, give t = min + ((2u+1) 2^-24) * (max - min), float, two roundings.
__device__ __forceinline__ uint64_t rw_state(uint64_t key, int p) {
  return sm64((key ^ kBinTag) + (uint64_t)p * kProjMult);
}
__device__ __forceinline__ float rw_boundary(uint32_t u, float mn, float w) {
  const float f = __fmul_rn(__uint2float_rn(2u * u + 1u), 0x1p-24f);  // exact: 2u+1 < 2^24
  return __fadd_rn(mn, __fmul_rn(f, w));
}
// Guide cell of v: every step (one fused multiply-add, round down to an
// unsigned integer -- negative values and NaN saturate to 0 --, clamp above)
// is monotone non-decreasing in v, so cell(t) < cell(v) implies t < v and
// cell(t) > cell(v) implies t > v.
__device__ __forceinline__ int rw_cell(float v, float s, float o) {
  return (int)min(__float2uint_rd(__fmaf_rn(v, s, o)), (unsigned)(kRwCells - 1));
}
// Upper-bound count #{j < nb : t[j] <= v} by binary search (any rule).
__device__ __forceinline__ int bin_search(const float* __restrict__ t, int nb, float v) {
  int lo = 0, hi = nb;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(t + mid) <= v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---- warp helpers ---------------------------------------------------------
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

// ---- information gain (entropy criterion, the YDF learner's, Section 3 step 3)
// Definition in double, fixed order: t = f(n) - sum_c f(N_c) + sum_c f(L_c)
// - f(nL) + sum_c f(R_c) - f(nR), IG = t / n, f(x) = x ln x; IG = 0 when
// every D_c = n L_c - N_c nL is 0.  ln by a stated method so that any IEEE
// machine gets the same bits: x = 2^e m, m in [sqrt(1/2), sqrt(2)) from the
// bit pattern, s = (m-1)/(m+1), ln m = 2 s P(s^2) with the atanh series
// P(z) = sum_{k<12} z^k/(2k+1) by Horner, ln x = e ln2 + ln m.
constexpr double kLn2 = 0x1.62e42fefa39efp-1;       // ln 2 rounded to double
constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;  // sqrt(1/2) rounded to double
constexpr int kXlnxTab = 2048;                      // table of x ln x, x < 2048 (exact-path counts)

__device__ __forceinline__ double ln_series(double x) {
  // 1/(2k+1) rounded to double, k = 0..11
  constexpr double kC[12] = {0x1p+0,
                             0x1.5555555555555p-2,
                             0x1.999999999999ap-3,
                             0x1.2492492492492p-3,
                             0x1.c71c71c71c71cp-4,
                             0x1.745d1745d1746p-4,
                             0x1.3b13b13b13b14p-4,
                             0x1.1111111111111p-4,
                             0x1.e1e1e1e1e1e1ep-5,
                             0x1.af286bca1af28p-5,
                             0x1.8618618618618p-5,
                             0x1.642c8590b2164p-5};
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7ffull) - 1022;
  double m = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull));
  if (m < kSqrtHalf) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double s = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double z = __dmul_rn(s, s);
  double P = kC[11];
#pragma unroll
  for (int k = 10; k >= 0; --k) P = __dadd_rn(__dmul_rn(P, z), kC[k]);
  return __dadd_rn(__dmul_rn((double)e, kLn2), __dmul_rn(__dmul_rn(2.0, s), P));
}
__device__ __forceinline__ double xlnx64(long long x) {
  return x < 2 ? 0.0 : __dmul_rn(__ll2double_rn(x), ln_series(__ll2double_rn(x)));
}
__device__ __forceinline__ double xlnx_t(long long x, const double* tab) {
  return (tab && x < kXlnxTab) ? tab[x] : xlnx64(x);
}
__device__ __forceinline__ bool informative(const int* L, const int* N, int C, int64_t n, int64_t nL) {
  bool any = false;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) any |= (n * (long long)L[c] - (long long)N[c] * nL) != 0;
  return any;
}
__device__ __forceinline__ double ent_gain64(const int* L, const int* N, int C, int64_t n, int64_t nL,
                                             const double* tab) {
  if (!informative(L, N, C, n, nL)) return 0.0;
  double t = xlnx_t(n, tab);
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) t = __dsub_rn(t, xlnx_t(N[c], tab));
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) t = __dadd_rn(t, xlnx_t(L[c], tab));
  t = __dsub_rn(t, xlnx_t(nL, tab));
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) t = __dadd_rn(t, xlnx_t((long long)N[c] - L[c], tab));
  t = __dsub_rn(t, xlnx_t(n - nL, tab));
  return __ddiv_rn(t, __ll2double_rn(n));
}
// Float comparison key of the information gain: n IG / ln 2 without the node
// constant, sum_c (L_c lg L_c + R_c lg R_c) - nL lg nL - nR lg nR (lg = log2
// by the fast intrinsic: 2^-22 absolute error on [0.5, 2], 2 ulp elsewhere).
// Candidates without information are -inf.
__device__ __forceinline__ float xlg2x(long long x) {
  const float xf = __ll2float_rn(x);
  return x < 2 ? 0.0f : __fmul_rn(xf, __log2f(xf));
}
__device__ __forceinline__ float ent_key32(const int* L, const int* N, int C, int64_t n, int64_t nL) {
  if (!informative(L, N, C, n, nL)) return -INFINITY;
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) s = __fadd_rn(__fadd_rn(s, xlg2x(L[c])), xlg2x((long long)N[c] - L[c]));
  return __fsub_rn(__fsub_rn(s, xlg2x(nL)), xlg2x(n - nL));
}
// The same key for exact-path nodes (n < 2048, so every product n L_c fits
// 32 bits and every count converts to float exactly): the same bits with
// 32-bit arithmetic.
__device__ __forceinline__ float xlg2x_i(int x) {
  const float xf = __int2float_rn(x);
  return x < 2 ? 0.0f : __fmul_rn(xf, __log2f(xf));
}
__device__ __forceinline__ float ent_key32_small(const int* L, const int* N, int C, int n, int nL) {
  bool any = false;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) any |= n * L[c] != N[c] * nL;
  if (!any) return -INFINITY;
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) s = __fadd_rn(__fadd_rn(s, xlg2x_i(L[c])), xlg2x_i(N[c] - L[c]));
  return __fsub_rn(__fsub_rn(s, xlg2x_i(nL)), xlg2x_i(n - nL));
}

// Re-score window of the key at a node of n samples: every candidate's key
// is within E of its double gain (same units), with m = 2C+2 terms of size at
// most F = n log2 n (all terms sum to at most 2F), per-term error 2^-21
// relative plus 2^-20 absolute, float summation m 2^-24 relative:
// E <= F (2C+10) 2^-23 + (2C+2) 2^-20.  The double winner (and every double
// tie of it) lies within 2E of the float maximum; the window is 3E.
__device__ __forceinline__ float ent_window(int64_t n, int C) {
  const float nf = __ll2float_rn(n);
  const float F = __fmul_rn(__fmul_rn(nf, __log2f(nf) + 0.01f), 1.01f) + 2.0f;
  return 3.0f * (F * (float)(2 * C + 10) * 0x1p-23f + (float)(2 * C + 2) * 0x1p-20f);
}

// The split criterion as the kernels use it (Crit, so_internal.h): a float
// key for every candidate, the re-score window around the float maximum, the
// double gain.
__device__ __forceinline__ float key32(const Crit& cr, const int* L, const int* N, int C, int64_t n, int64_t nL) {
  return cr.ent ? ent_key32(L, N, C, n, nL) : gain32(L, N, C, n, nL);
}
// exact-path nodes (fewer than 2048 samples): every count is in the table
// of x ln x, so the double gain needs no logarithm (the same bits)
__device__ __forceinline__ double ent_gain64_small(const int* L, const int* N, int C, int n, int nL,
                                                   const double* __restrict__ tab) {
  bool any = false;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) any |= n * L[c] != N[c] * nL;
  if (!any) return 0.0;
  double t = tab[n];
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) t = __dsub_rn(t, tab[N[c]]);
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) t = __dadd_rn(t, tab[L[c]]);
  t = __dsub_rn(t, tab[nL]);
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c)
    if (c < C) t = __dadd_rn(t, tab[N[c] - L[c]]);
  t = __dsub_rn(t, tab[n - nL]);
  return __ddiv_rn(t, __int2double_rn(n));
}
// Gini key and gain of exact-path nodes: |D_c| < n^2 < 2^22 fits 32 bits and
// converts exactly, so these are gain32 / gain64 bit for bit
__device__ __forceinline__ float gain32_small(const int* L, const int* N, int C, int n, int nL) {
  float num = 0.0f;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) {
    if (c < C) {
      const float fd = __int2float_rn(n * L[c] - N[c] * nL);
      num = __fadd_rn(num, __fmul_rn(fd, fd));
    }
  }
  return __fdiv_rn(num, __fmul_rn(__int2float_rn(nL), __int2float_rn(n - nL)));
}
__device__ __forceinline__ double gain64_small(const int* L, const int* N, int C, int n, int nL) {
  double num = 0.0;
#pragma unroll
  for (int c = 0; c < kMaxClasses; ++c) {
    if (c < C) {
      const double dd = __int2double_rn(n * L[c] - N[c] * nL);
      num = __dadd_rn(num, __dmul_rn(dd, dd));
    }
  }
  const double g = __ddiv_rn(num, __dmul_rn(__int2double_rn(nL), __int2double_rn(n - nL)));
  return __ddiv_rn(g, __dmul_rn(__int2double_rn(n), __int2double_rn(n)));
}
__device__ __forceinline__ float key32s(const Crit& cr, const int* L, const int* N, int C, int n, int nL) {
  return cr.ent ? ent_key32_small(L, N, C, n, nL) : gain32_small(L, N, C, n, nL);
}
__device__ __forceinline__ double gain64s(const Crit& cr, const int* L, const int* N, int C, int n, int nL) {
  return cr.ent ? ent_gain64_small(L, N, C, n, nL, cr.tab) : gain64_small(L, N, C, n, nL);
}
__device__ __forceinline__ double gain64c(const Crit& cr, const int* L, const int* N, int C, int64_t n,
                                          int64_t nL) {
  return cr.ent ? ent_gain64(L, N, C, n, nL, cr.tab) : gain64(L, N, C, n, nL);
}
// key of "no candidate"; whether a float maximum has a candidate that can win
__device__ __forceinline__ float key_none(const Crit& cr) { return cr.ent ? -INFINITY : -1.0f; }
__device__ __forceinline__ bool key_any(const Crit& cr, float M) { return cr.ent ? M > -INFINITY : M > 0.0f; }
__device__ __forceinline__ float key_thr(const Crit& cr, float M, int64_t n, int C) {
  return cr.ent ? __fsub_rn(M, ent_window(n, C)) : __fmul_rn(M, 1.0f - cr.eps);
}

// A candidate of the double re-score, ordered by (gain desc, proj asc, cand asc).
struct Cand {
  double g;
  int proj;
  int cand;
};
__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  if (a.g != b.g) return a.g > b.g;
  if (a.proj != b.proj) return a.proj < b.proj;
  return a.cand < b.cand;
}
__device__ __forceinline__ Cand shfl_cand(const Cand& c, int src) {
  Cand r;
  r.g = __shfl_sync(0xffffffffu, c.g, src);
  r.proj = __shfl_sync(0xffffffffu, c.proj, src);
  r.cand = __shfl_sync(0xffffffffu, c.cand, src);
  return r;
}
__device__ __forceinline__ Cand warp_best(Cand c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Cand d;
    d.g = __shfl_xor_sync(0xffffffffu, c.g, o);
    d.proj = __shfl_xor_sync(0xffffffffu, c.proj, o);
    d.cand = __shfl_xor_sync(0xffffffffu, c.cand, o);
    if (better(d, c)) c = d;
  }
  return c;
}

}  // namespace sof
