/*
 * so_oracle.c -- plain, slow CPU oracle for sparse-oblique split search and
 * tree growth ("Vectorized Adaptive Histograms for Sparse Oblique Forests").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant generator with the CUDA library; the two meet only through the
 * seeded inputs of the input-generator module.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no intrinsics,
 * no -ffast-math).  On x86-64 float arithmetic is SSE, so every float and
 * double operation below is one IEEE-754 round-to-nearest operation.
 *
 * What is computed, and where the paper states it:
 *   - Per node, a sparse projection matrix is sampled and every row of it is
 *     evaluated (Section 3, "Method", the numbered steps 1-3).
 *   - Step 1, apply projection: a sparse vector sum over the node's active
 *     rows of the selected columns (Section 3 step 1; Section 3.3 kernel 1).
 *   - Step 2, histogram: bin the projected feature and count class instances
 *     per bin (Section 3 step 2; Section 3.2, equal-width 256-bin variant).
 *   - Step 3, split criterion at every bin boundary, best over projections
 *     (Section 3 step 3; Section 3.3 kernel 2).  Two criteria: Gini impurity
 *     decrease, and entropy (information gain), which the paper's YDF uses.
 *   - Small nodes use an exact split by sorting instead of a histogram, the
 *     switch being node cardinality (Section 3.1, Dynamic Histogramming).
 *   - Trees are grown to purity (Section 2, Background, item 2).
 *   - Projection sampling draws distinct features with Floyd's algorithm
 *     (Appendix A).
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   R1 projection value: acc = +0.0f, then acc = acc + (s>0 ? x : -x) over the
 *      projection's features in ascending order, float, no fused multiply-add.
 *   R2 histogram: w = (max-min)/B, t_j = min + j*w (float), bin(v) =
 *      #{ j in 1..B-1 : t_j <= v } (an upper-bound search, as YDF's binary
 *      search computes).  Candidate b (0..B-2) sends bins <= b left, which is
 *      exactly v < t_{b+1}; the threshold is t_{b+1}.
 *   R3 sort path: candidates only between distinct consecutive sorted values;
 *      threshold = a + 0.5f*(b-a) with a collapse guard to b.
 *   R4 gain = sum_c D_c^2 / (n^2 nL nR), D_c = n L_c - N_c nL (exact int64),
 *      evaluated in double by one fixed expression.  This equals the Gini
 *      decrease G(parent) - nL/n G(L) - nR/n G(R).
 *   R5 argmax: largest double gain; ties -> lowest projection, then lowest
 *      candidate.  A split is valid iff its gain is > 0.
 *   R6 partition: stable, left iff v < threshold (v recomputed by R1).
 *   R7 tree: breadth-first node order, children appended left then right.
 *      Node keys and projection streams use splitmix64 (Steele, Lea & Flood,
 *      OOPSLA 2014); nnz = min(cap, d, 1 + Poisson(lambda)) by inverse CDF.
 *   R14 random-width histogram (the YDF default the paper's Section 1 footnote
 *      names: boundaries at random intervals): for node key K and projection
 *      p, a splitmix64 generator with state sm64((K ^ BIN_TAG) + p*PROJ_MULT)
 *      draws B-1 outputs r_j; u_j = r_j >> 41 (23 bits) sorted ascending;
 *      f_j = (2 u_j + 1) * 2^-24, exact in float and inside (0, 1);
 *      t_j = min + f_j * (max - min), float, two roundings.  Bin, candidates
 *      and thresholds then follow R2 with these t_j.
 *   R15 entropy criterion: information gain in nats, IG = (f(n) - sum_c f(N_c)
 *      + sum_c f(L_c) - f(nL) + sum_c f(R_c) - f(nR)) / n with f(x) = x ln x,
 *      f(0) = f(1) = 0, summed in exactly that order in double; IG = 0 when
 *      every D_c = n L_c - N_c nL is 0 (the split carries no information).
 *      ln is evaluated by a stated method so that any IEEE machine gets the
 *      same bits: x = 2^e m with m in [sqrt(1/2), sqrt(2)) (exponent and
 *      mantissa from the bit pattern), s = (m-1)/(m+1), ln m = 2 s P(s^2)
 *      with P(z) = sum_{k=0}^{11} z^k / (2k+1) by Horner (the atanh series,
 *      Abramowitz & Stegun 4.1.27), ln x = e ln2 + ln m.  Argmax, ties and
 *      validity (best IG > 0) as R5.
 */
#include <math.h>
#include <stdint.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORC_GAMMA 0x9E3779B97F4A7C15ULL   /* splitmix64 increment (golden ratio) */
#define ORC_PROJ_MULT 0xD2B74407B1CE6E93ULL /* odd multiplier separating projection streams */
#define ORC_BIN_TAG 0x6A09E667F3BCC908ULL   /* first 64 fractional bits of sqrt(2): tags the
                                               boundary streams apart from the projection streams */
#define ORC_MAX_CLASSES 8
#define ORC_MAX_CAP 32

/* ------------------------------------------------------------------------ */
/* Random streams (input definition of the method's own random draws)        */
/* ------------------------------------------------------------------------ */

/* One splitmix64 step: advance the state by the golden-ratio increment and
 * return the mixed output (Steele, Lea & Flood 2014, "Fast splittable
 * pseudorandom number generators"). */
uint64_t orc_sm64_next(uint64_t *state)
{
    uint64_t z = (*state += ORC_GAMMA);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* splitmix64 output of a generator whose state is x. */
uint64_t orc_sm64(uint64_t x)
{
    uint64_t s = x;
    return orc_sm64_next(&s);
}

uint64_t orc_root_key(uint64_t seed, int32_t tree_id)
{
    return orc_sm64(seed ^ ((uint64_t)(int64_t)tree_id * ORC_GAMMA));
}

uint64_t orc_child_key(uint64_t key, int side)
{
    return orc_sm64(2u * key + (uint64_t)side);
}

/* Poisson(lambda) cumulative probabilities P(K <= k), k = 0..cap-2, by the
 * definition p_0 = e^-lambda, p_k = p_{k-1} * lambda / k. */
void orc_poisson_cdf(double lambda, int cap, double *cdf)
{
    double p = exp(-lambda);
    double c = p;
    for (int k = 0; k < cap - 1; k++) {
        if (k > 0) {
            p = (p * lambda) / (double)k;
            c = c + p;
        }
        cdf[k] = c;
    }
}

/* Samples projection p of a node: nnz by inverse-CDF Poisson, then nnz
 * distinct features by Floyd's algorithm (Appendix A cites Floyd), sorted
 * ascending, then one sign bit per feature.  Returns nnz. */
static int sample_one_projection(uint64_t node_key, int p, int d, const double *cdf,
                                 int cap, int32_t *feat, int8_t *sign)
{
    uint64_t st = orc_sm64(node_key + (uint64_t)p * ORC_PROJ_MULT);
    uint64_t r = orc_sm64_next(&st);
    double u = (double)(r >> 11) * 0x1.0p-53;
    int K = 0;
    while (K < cap - 1 && u >= cdf[K])
        K++;
    int k = 1 + K;
    if (k > d)
        k = d;
    /* Floyd: for j = d-k .. d-1 pick t uniform in [0, j]; take t unless
     * already chosen, in which case take j. */
    int m = 0;
    for (int j = d - k; j < d; j++) {
        uint64_t rr = orc_sm64_next(&st);
        int32_t t = (int32_t)(((unsigned __int128)rr * (unsigned __int128)(uint64_t)(j + 1)) >> 64);
        int seen = 0;
        for (int q = 0; q < m; q++)
            if (feat[q] == t)
                seen = 1;
        feat[m++] = seen ? j : t;
    }
    /* ascending order (insertion sort) */
    for (int a = 1; a < m; a++) {
        int32_t key = feat[a];
        int b = a - 1;
        while (b >= 0 && feat[b] > key) {
            feat[b + 1] = feat[b];
            b--;
        }
        feat[b + 1] = key;
    }
    uint64_t sb = orc_sm64_next(&st);
    for (int q = 0; q < m; q++)
        sign[q] = ((sb >> q) & 1u) ? (int8_t)1 : (int8_t)-1;
    return m;
}

/* All P projections of one node into fixed slots of width cap. */
int orc_sample_node(uint64_t node_key, int P, int d, double lambda, int cap,
                    int32_t *nnz_out, int32_t *feat_out, int8_t *sign_out)
{
    if (cap < 1 || cap > ORC_MAX_CAP || d < 1 || P < 0)
        return -1;
    double cdf[ORC_MAX_CAP];
    orc_poisson_cdf(lambda, cap, cdf);
    for (int p = 0; p < P; p++)
        nnz_out[p] = sample_one_projection(node_key, p, d, cdf, cap,
                                           feat_out + (int64_t)p * cap,
                                           sign_out + (int64_t)p * cap);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Split search                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t valid, proj, path, cand;
    float threshold;
    double gain;
    int64_t n_left, n_right;
} orc_split;

/* R1: the projected value of sample i. */
static float project(const float *X, int64_t ld, int64_t i, const int32_t *f,
                     const int8_t *s, int k)
{
    float acc = 0.0f;
    for (int j = 0; j < k; j++) {
        float x = X[(int64_t)f[j] * ld + i];
        acc = acc + (s[j] == 1 ? x : -x);
    }
    return acc;
}

void orc_project(const float *X, int64_t ld, const int32_t *idx, int64_t n,
                 const int32_t *feat, const int8_t *sign, int nnz, float *v_out)
{
    for (int64_t i = 0; i < n; i++)
        v_out[i] = project(X, ld, idx[i], feat, sign, nnz);
}

/* R4: Gini decrease for a candidate with left class counts L out of node
 * counts N (n = sum N, nL = sum L), one fixed double expression. */
double orc_gini_gain(const int64_t *L, const int64_t *N, int C, int64_t n, int64_t nL)
{
    double num = 0.0;
    for (int c = 0; c < C; c++) {
        int64_t D = n * L[c] - N[c] * nL;
        double dd = (double)D;
        num = num + dd * dd;
    }
    double g = num / ((double)nL * (double)(n - nL));
    return g / ((double)n * (double)n);
}

/* R15: natural log of a positive normal double by the atanh series. */
double orc_ln(double x)
{
    uint64_t b;
    memcpy(&b, &x, sizeof b);
    int e = (int)((b >> 52) & 0x7ff) - 1022;
    uint64_t mb = (b & 0x000FFFFFFFFFFFFFULL) | 0x3FE0000000000000ULL; /* m in [0.5, 1) */
    double m;
    memcpy(&m, &mb, sizeof m);
    if (m < sqrt(0.5)) {
        m = m * 2.0;
        e = e - 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double P = 1.0 / 23.0;
    for (int k = 10; k >= 0; k--)
        P = P * z + 1.0 / (double)(2 * k + 1);
    return (double)e * M_LN2 + (2.0 * s) * P;
}

/* R15: x ln x of a count. */
double orc_xlnx(int64_t x)
{
    return x < 2 ? 0.0 : (double)x * orc_ln((double)x);
}

/* R15: information gain of a candidate with left class counts L out of
 * node counts N (n = sum N, nL = sum L), one fixed double expression. */
double orc_entropy_gain(const int64_t *L, const int64_t *N, int C, int64_t n, int64_t nL)
{
    int informative = 0;
    for (int c = 0; c < C; c++)
        if (n * L[c] - N[c] * nL != 0)
            informative = 1;
    if (!informative)
        return 0.0;
    double t = orc_xlnx(n);
    for (int c = 0; c < C; c++)
        t = t - orc_xlnx(N[c]);
    for (int c = 0; c < C; c++)
        t = t + orc_xlnx(L[c]);
    t = t - orc_xlnx(nL);
    for (int c = 0; c < C; c++)
        t = t + orc_xlnx(N[c] - L[c]);
    t = t - orc_xlnx(n - nL);
    return t / (double)n;
}

static double criterion_gain(int criterion, const int64_t *L, const int64_t *N, int C, int64_t n,
                             int64_t nL)
{
    return criterion == 1 ? orc_entropy_gain(L, N, C, n, nL) : orc_gini_gain(L, N, C, n, nL);
}

/* R2: the B-1 boundaries t_1..t_{B-1} (t[j-1] holds t_j). */
void orc_boundaries(float mn, float mx, int B, float *t)
{
    float w = (mx - mn) / (float)B;
    for (int j = 1; j < B; j++)
        t[j - 1] = mn + (float)j * w;
}

/* R14: the B-1 random-width boundaries of projection p of the node with key
 * `key` (t[j-1] holds t_j, ascending). */
void orc_rw_boundaries(uint64_t key, int p, float mn, float mx, int B, float *t)
{
    uint32_t u[256];
    uint64_t st = orc_sm64((key ^ ORC_BIN_TAG) + (uint64_t)(int64_t)p * ORC_PROJ_MULT);
    for (int j = 0; j < B - 1; j++)
        u[j] = (uint32_t)(orc_sm64_next(&st) >> 41);
    for (int a = 1; a < B - 1; a++) { /* insertion sort, ascending */
        uint32_t v = u[a];
        int b = a - 1;
        while (b >= 0 && u[b] > v) {
            u[b + 1] = u[b];
            b--;
        }
        u[b + 1] = v;
    }
    float w = mx - mn;
    for (int j = 0; j < B - 1; j++) {
        float f = (float)(2u * u[j] + 1u) * 0x1p-24f;
        t[j] = mn + f * w;
    }
}

/* R2: bin = number of boundaries <= v, found by a textbook upper-bound
 * binary search over the non-decreasing array t[0..nb-1]. */
int orc_bin(const float *t, int nb, float v)
{
    int lo = 0, hi = nb; /* first index with t[idx] > v */
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if (t[mid] <= v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

typedef struct {
    float v;
    uint8_t y;
} orc_pair;

static int cmp_pair(const void *a, const void *b)
{
    const orc_pair *x = (const orc_pair *)a, *z = (const orc_pair *)b;
    if (x->v < z->v) return -1;
    if (x->v > z->v) return 1;
    return (int)x->y - (int)z->y;
}

/* R3: exact-path threshold between consecutive distinct values a < b. */
float orc_midpoint(float a, float b)
{
    float t = a + 0.5f * (b - a);
    if (!(a < t) || !(t <= b))
        t = b;
    return t;
}

/*
 * Best split of one node over P projections (CSR ptr/feat/sign).
 * Path: exact sort if !hist_only && n < sort_below, else histogram.
 * bin_rule 0: equal-width boundaries (R2); 1: random-width (R14) from the
 * node's key bin_key, projection p drawing from stream p_base + p (p_base is
 * nonzero only when a caller searches a sub-range of the node's projections).
 * criterion 0: Gini decrease (R4); 1: information gain (R15).
 * Optional outputs (may be NULL):
 *   left_counts[C]   class counts of the chosen left child
 *   mm_out[2P]       per projection (min, max)            (histogram path)
 *   hist_out[P*B*C]  per projection class-count histogram (histogram path)
 *   gains_out[P*(B-1)] per candidate double gain, -1 when skipped (hist path)
 *   best32_out[P]    unused by the oracle (kept NULL)
 * Returns 0, or -1 on a bad argument / allocation failure.
 */
int orc_split_search_rule(const float *X, int64_t ld, const uint8_t *y, int C,
                          const int32_t *idx, int64_t n, int P, const int32_t *ptr,
                          const int32_t *feat, const int8_t *sign, int B, int sort_below,
                          int hist_only, int bin_rule, uint64_t bin_key, int p_base,
                          int criterion, orc_split *out, int64_t *left_counts, float *mm_out,
                          int32_t *hist_out, double *gains_out, float *bounds_out)
{
    memset(out, 0, sizeof(*out));
    out->proj = -1;
    out->cand = -1;
    if (C < 1 || C > ORC_MAX_CLASSES || B < 2 || B > 256 || n < 0 || P < 0 ||
        bin_rule < 0 || bin_rule > 1 || criterion < 0 || criterion > 1)
        return -1;
    int64_t N[ORC_MAX_CLASSES] = {0};
    for (int64_t i = 0; i < n; i++)
        N[y[idx[i]]]++;
    int use_sort = (!hist_only && n < sort_below);
    out->path = use_sort ? 1 : 0;
    if (n == 0)
        return 0;

    float *v = (float *)malloc((size_t)n * sizeof(float));
    orc_pair *pairs = use_sort ? (orc_pair *)malloc((size_t)n * sizeof(orc_pair)) : NULL;
    int64_t *H = use_sort ? NULL : (int64_t *)malloc((size_t)B * C * sizeof(int64_t));
    float *t = (float *)malloc((size_t)B * sizeof(float));
    if (!v || (use_sort && !pairs) || (!use_sort && !H) || !t) {
        free(v); free(pairs); free(H); free(t);
        return -1;
    }

    double best = 0.0;
    int64_t bestL[ORC_MAX_CLASSES] = {0};
    for (int p = 0; p < P; p++) {
        const int32_t *f = feat + ptr[p];
        const int8_t *s = sign + ptr[p];
        int k = ptr[p + 1] - ptr[p];
        for (int64_t i = 0; i < n; i++)
            v[i] = project(X, ld, idx[i], f, s, k);

        if (use_sort) {
            for (int64_t i = 0; i < n; i++) {
                pairs[i].v = v[i];
                pairs[i].y = y[idx[i]];
            }
            qsort(pairs, (size_t)n, sizeof(orc_pair), cmp_pair);
            int64_t L[ORC_MAX_CLASSES] = {0};
            for (int64_t i = 0; i + 1 < n; i++) {
                L[pairs[i].y]++;
                if (!(pairs[i].v < pairs[i + 1].v))
                    continue;
                int64_t nL = i + 1;
                double g = criterion_gain(criterion, L, N, C, n, nL);
                if (g > best) {
                    best = g;
                    out->valid = 1;
                    out->proj = p;
                    out->cand = (int32_t)i;
                    out->threshold = orc_midpoint(pairs[i].v, pairs[i + 1].v);
                    out->gain = g;
                    out->n_left = nL;
                    out->n_right = n - nL;
                    memcpy(bestL, L, sizeof(L));
                }
            }
        } else {
            float mn = v[0], mx = v[0];
            for (int64_t i = 1; i < n; i++) {
                if (v[i] < mn) mn = v[i];
                if (v[i] > mx) mx = v[i];
            }
            if (mm_out) {
                mm_out[2 * p] = mn;
                mm_out[2 * p + 1] = mx;
            }
            if (bin_rule == 1)
                orc_rw_boundaries(bin_key, p_base + p, mn, mx, B, t);
            else
                orc_boundaries(mn, mx, B, t);
            if (bounds_out)
                memcpy(bounds_out + (int64_t)p * (B - 1), t, (size_t)(B - 1) * sizeof(float));
            memset(H, 0, (size_t)B * C * sizeof(int64_t));
            for (int64_t i = 0; i < n; i++) {
                int b = orc_bin(t, B - 1, v[i]);
                H[(int64_t)b * C + y[idx[i]]]++;
            }
            if (hist_out)
                for (int64_t q = 0; q < (int64_t)B * C; q++)
                    hist_out[(int64_t)p * B * C + q] = (int32_t)H[q];
            int64_t L[ORC_MAX_CLASSES] = {0};
            for (int b = 0; b + 1 < B; b++) {
                int64_t nL = 0;
                for (int c = 0; c < C; c++) {
                    L[c] += H[(int64_t)b * C + c];
                    nL += L[c];
                }
                double g = -1.0;
                if (nL > 0 && nL < n) {
                    g = criterion_gain(criterion, L, N, C, n, nL);
                    if (g > best) {
                        best = g;
                        out->valid = 1;
                        out->proj = p;
                        out->cand = b;
                        out->threshold = t[b]; /* t_{b+1} */
                        out->gain = g;
                        out->n_left = nL;
                        out->n_right = n - nL;
                        memcpy(bestL, L, sizeof(L));
                    }
                }
                if (gains_out)
                    gains_out[(int64_t)p * (B - 1) + b] = g;
            }
        }
    }
    if (left_counts)
        for (int c = 0; c < C; c++)
            left_counts[c] = bestL[c];
    free(v); free(pairs); free(H); free(t);
    return 0;
}

/* The search with equal-width boundaries (R2). */
int orc_split_search(const float *X, int64_t ld, const uint8_t *y, int C,
                     const int32_t *idx, int64_t n, int P, const int32_t *ptr,
                     const int32_t *feat, const int8_t *sign, int B, int sort_below,
                     int hist_only, orc_split *out, int64_t *left_counts,
                     float *mm_out, int32_t *hist_out, double *gains_out)
{
    return orc_split_search_rule(X, ld, y, C, idx, n, P, ptr, feat, sign, B, sort_below,
                                 hist_only, 0, 0, 0, 0, out, left_counts, mm_out, hist_out,
                                 gains_out, NULL);
}

/* R6: stable partition of idx[0..n) by v < thr; returns the left count. */
int64_t orc_partition(const float *X, int64_t ld, int32_t *idx, int64_t n,
                      const int32_t *feat, const int8_t *sign, int nnz, float thr)
{
    int32_t *tmp = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!tmp)
        return -1;
    int64_t nl = 0;
    for (int64_t i = 0; i < n; i++)
        if (project(X, ld, idx[i], feat, sign, nnz) < thr)
            tmp[nl++] = idx[i];
    int64_t r = nl;
    for (int64_t i = 0; i < n; i++)
        if (!(project(X, ld, idx[i], feat, sign, nnz) < thr))
            tmp[r++] = idx[i];
    memcpy(idx, tmp, (size_t)n * sizeof(int32_t));
    free(tmp);
    return nl;
}

/* ------------------------------------------------------------------------ */
/* Tree to purity, breadth first (R7)                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n_nodes;
    int32_t n_classes, cap;
    int32_t *left, *right, *depth, *leaf_class, *proj_nnz, *feat, *cand;
    int8_t *sign, *path;
    float *threshold;
    int64_t *n_samples, *class_counts;
    double *gain;
} orc_tree;

void orc_tree_free(orc_tree *t)
{
    free(t->left); free(t->right); free(t->depth); free(t->leaf_class);
    free(t->proj_nnz); free(t->feat); free(t->cand); free(t->sign); free(t->path);
    free(t->threshold); free(t->n_samples); free(t->class_counts); free(t->gain);
    memset(t, 0, sizeof(*t));
}

typedef struct {
    int64_t off, cnt;
    uint64_t key;
    int32_t depth;
} orc_pending;

static int tree_reserve(orc_tree *t, int64_t cap_nodes, int C, int cap)
{
#define GROW(ptr, type, per)                                                   \
    do {                                                                       \
        void *q = realloc(t->ptr, (size_t)cap_nodes * (per) * sizeof(type));   \
        if (!q)                                                                \
            return -1;                                                         \
        t->ptr = (type *)q;                                                    \
    } while (0)
    GROW(left, int32_t, 1); GROW(right, int32_t, 1); GROW(depth, int32_t, 1);
    GROW(leaf_class, int32_t, 1); GROW(proj_nnz, int32_t, 1); GROW(feat, int32_t, cap);
    GROW(cand, int32_t, 1); GROW(sign, int8_t, cap); GROW(path, int8_t, 1);
    GROW(threshold, float, 1); GROW(n_samples, int64_t, 1); GROW(class_counts, int64_t, C);
    GROW(gain, double, 1);
#undef GROW
    return 0;
}

/*
 * Grows one tree from the root sample list (which may hold repeats, e.g. a
 * bootstrap).  A node is a leaf when it has < 2 samples, is pure, reached
 * max_depth (>= 0), or has no split of positive gain.  Leaf class = majority,
 * ties to the lowest class id.  Returns 0 or -1.
 */
int orc_train_tree(const float *X, int64_t ld, int32_t d, const uint8_t *y, int C,
                   const int32_t *root_idx, int64_t n_root, int B, int sort_below,
                   int hist_only, int bin_rule, int criterion, int P, double lambda, int cap,
                   uint64_t seed, int32_t tree_id, int32_t max_depth, orc_tree *out)
{
    memset(out, 0, sizeof(*out));
    if (C < 1 || C > ORC_MAX_CLASSES || cap < 1 || cap > ORC_MAX_CAP || n_root < 1 || P < 1)
        return -1;
    out->n_classes = C;
    out->cap = cap;
    int64_t node_cap = 2 * n_root + 1;
    if (tree_reserve(out, node_cap, C, cap))
        return -1;

    int32_t *cur = (int32_t *)malloc((size_t)n_root * sizeof(int32_t));
    int32_t *nxt = (int32_t *)malloc((size_t)n_root * sizeof(int32_t));
    orc_pending *lvl = (orc_pending *)malloc((size_t)n_root * sizeof(orc_pending));
    orc_pending *nlv = (orc_pending *)malloc((size_t)n_root * sizeof(orc_pending));
    int32_t *pnnz = (int32_t *)malloc((size_t)P * sizeof(int32_t));
    int32_t *pfeat = (int32_t *)malloc((size_t)P * cap * sizeof(int32_t));
    int8_t *psign = (int8_t *)malloc((size_t)P * cap);
    int32_t *ptr = (int32_t *)malloc((size_t)(P + 1) * sizeof(int32_t));
    int32_t *cfeat = (int32_t *)malloc((size_t)P * cap * sizeof(int32_t));
    int8_t *csign = (int8_t *)malloc((size_t)P * cap);
    int rc = -1;
    if (!cur || !nxt || !lvl || !nlv || !pnnz || !pfeat || !psign || !ptr || !cfeat || !csign)
        goto done;

    memcpy(cur, root_idx, (size_t)n_root * sizeof(int32_t));
    int64_t m = 1, n_nodes = 1;
    lvl[0].off = 0;
    lvl[0].cnt = n_root;
    lvl[0].key = orc_root_key(seed, tree_id);
    lvl[0].depth = 0;
    int64_t level_base = 0;

    while (m > 0) {
        int64_t m_next = 0, next_off = 0;
        for (int64_t j = 0; j < m; j++) {
            int64_t id = level_base + j;
            orc_pending nd = lvl[j];
            int32_t *seg = cur + nd.off;
            int64_t N[ORC_MAX_CLASSES] = {0};
            for (int64_t i = 0; i < nd.cnt; i++)
                N[y[seg[i]]]++;
            int present = 0, maj = 0;
            for (int c = 0; c < C; c++) {
                if (N[c] > 0) present++;
                if (N[c] > N[maj]) maj = c;
            }
            out->left[id] = -1;
            out->right[id] = -1;
            out->depth[id] = nd.depth;
            out->leaf_class[id] = maj;
            out->proj_nnz[id] = 0;
            out->cand[id] = -1;
            out->path[id] = -1;
            out->threshold[id] = 0.0f;
            out->gain[id] = 0.0;
            out->n_samples[id] = nd.cnt;
            for (int c = 0; c < C; c++)
                out->class_counts[id * C + c] = N[c];
            for (int q = 0; q < cap; q++) {
                out->feat[id * cap + q] = 0;
                out->sign[id * cap + q] = 0;
            }
            if (nd.cnt < 2 || present < 2 || (max_depth >= 0 && nd.depth >= max_depth))
                continue;

            if (orc_sample_node(nd.key, P, d, lambda, cap, pnnz, pfeat, psign))
                goto done;
            ptr[0] = 0;
            for (int p = 0; p < P; p++) {
                for (int q = 0; q < pnnz[p]; q++) {
                    cfeat[ptr[p] + q] = pfeat[p * cap + q];
                    csign[ptr[p] + q] = psign[p * cap + q];
                }
                ptr[p + 1] = ptr[p] + pnnz[p];
            }
            orc_split sp;
            if (orc_split_search_rule(X, ld, y, C, seg, nd.cnt, P, ptr, cfeat, csign, B,
                                      sort_below, hist_only, bin_rule, nd.key, 0, criterion, &sp,
                                      NULL, NULL, NULL, NULL, NULL))
                goto done;
            out->path[id] = (int8_t)sp.path;
            if (!sp.valid)
                continue;
            int k = pnnz[sp.proj];
            const int32_t *wf = pfeat + sp.proj * cap;
            const int8_t *ws = psign + sp.proj * cap;
            out->proj_nnz[id] = k;
            for (int q = 0; q < k; q++) {
                out->feat[id * cap + q] = wf[q];
                out->sign[id * cap + q] = ws[q];
            }
            out->cand[id] = sp.cand;
            out->threshold[id] = sp.threshold;
            out->gain[id] = sp.gain;

            /* stable partition into the next level's buffer */
            int32_t *dst = nxt + next_off;
            int64_t nl = 0;
            for (int64_t i = 0; i < nd.cnt; i++)
                if (project(X, ld, seg[i], wf, ws, k) < sp.threshold)
                    dst[nl++] = seg[i];
            int64_t r = nl;
            for (int64_t i = 0; i < nd.cnt; i++)
                if (!(project(X, ld, seg[i], wf, ws, k) < sp.threshold))
                    dst[r++] = seg[i];
            if (nl != sp.n_left)
                goto done; /* cannot happen: the split's left count is the partition's */

            int64_t lid = n_nodes, rid = n_nodes + 1;
            n_nodes += 2;
            out->left[id] = (int32_t)lid;
            out->right[id] = (int32_t)rid;
            nlv[m_next].off = next_off;
            nlv[m_next].cnt = nl;
            nlv[m_next].key = orc_child_key(nd.key, 0);
            nlv[m_next].depth = nd.depth + 1;
            nlv[m_next + 1].off = next_off + nl;
            nlv[m_next + 1].cnt = nd.cnt - nl;
            nlv[m_next + 1].key = orc_child_key(nd.key, 1);
            nlv[m_next + 1].depth = nd.depth + 1;
            m_next += 2;
            next_off += nd.cnt;
        }
        level_base += m;
        m = m_next;
        int32_t *ti = cur; cur = nxt; nxt = ti;
        orc_pending *tl = lvl; lvl = nlv; nlv = tl;
    }
    out->n_nodes = n_nodes;
    rc = 0;
done:
    free(cur); free(nxt); free(lvl); free(nlv); free(pnnz); free(pfeat); free(psign);
    free(ptr); free(cfeat); free(csign);
    if (rc)
        orc_tree_free(out);
    return rc;
}

/* Forest prediction by majority vote of leaf classes (used by accuracy checks). */
void orc_predict_tree(const orc_tree *t, const float *X, int64_t ld, const int32_t *rows,
                      int64_t n, int32_t *cls_out)
{
    for (int64_t i = 0; i < n; i++) {
        int64_t id = 0;
        while (t->left[id] >= 0) {
            float v = project(X, ld, rows[i], t->feat + id * t->cap, t->sign + id * t->cap,
                              t->proj_nnz[id]);
            id = (v < t->threshold[id]) ? t->left[id] : t->right[id];
        }
        cls_out[i] = t->leaf_class[id];
    }
}


/*
 * The same split search with the projections divided into contiguous ranges,
 * one per thread (each range searched by orc_split_search above), and the
 * range results taken in projection order with the same strict comparison,
 * so the result is the single-threaded one.  Used to time the oracle on all
 * host cores; debug outputs are not offered.  Returns 0 or -1.
 */
typedef struct {
    const float *X; int64_t ld; const uint8_t *y; int C; const int32_t *idx; int64_t n;
    int p0, p1; const int32_t *ptr; const int32_t *feat; const int8_t *sign;
    int B, sort_below, hist_only, bin_rule, criterion; uint64_t bin_key;
    orc_split res; int64_t lc[ORC_MAX_CLASSES]; int rc;
} orc_range_job;

static void *orc_range_run(void *arg)
{
    orc_range_job *j = (orc_range_job *)arg;
    j->rc = orc_split_search_rule(j->X, j->ld, j->y, j->C, j->idx, j->n, j->p1 - j->p0,
                                  j->ptr + j->p0, j->feat, j->sign, j->B, j->sort_below,
                                  j->hist_only, j->bin_rule, j->bin_key, j->p0, j->criterion,
                                  &j->res, j->lc, NULL, NULL, NULL, NULL);
    return NULL;
}

int orc_split_search_mt(const float *X, int64_t ld, const uint8_t *y, int C,
                        const int32_t *idx, int64_t n, int P, const int32_t *ptr,
                        const int32_t *feat, const int8_t *sign, int B, int sort_below,
                        int hist_only, int bin_rule, uint64_t bin_key, int criterion,
                        int n_threads, orc_split *out, int64_t *left_counts)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > P) n_threads = P > 0 ? P : 1;
    orc_range_job *jobs = (orc_range_job *)calloc((size_t)n_threads, sizeof(orc_range_job));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    for (int t = 0; t < n_threads; t++) {
        orc_range_job *j = &jobs[t];
        j->X = X; j->ld = ld; j->y = y; j->C = C; j->idx = idx; j->n = n;
        j->p0 = (int)((int64_t)P * t / n_threads);
        j->p1 = (int)((int64_t)P * (t + 1) / n_threads);
        j->ptr = ptr; j->feat = feat; j->sign = sign;
        j->B = B; j->sort_below = sort_below; j->hist_only = hist_only;
        j->bin_rule = bin_rule; j->bin_key = bin_key; j->criterion = criterion;
    }
    int started = 0;
    for (int t = 1; t < n_threads; t++) {
        if (pthread_create(&th[t], NULL, orc_range_run, &jobs[t]) != 0) break;
        started = t;
    }
    orc_range_run(&jobs[0]);
    for (int t = started + 1; t < n_threads; t++) orc_range_run(&jobs[t]);  /* threads that failed to start */
    for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
    int rc = 0;
    memset(out, 0, sizeof(*out));
    out->proj = -1;
    out->cand = -1;
    int64_t bestL[ORC_MAX_CLASSES] = {0};
    double best = 0.0;
    for (int t = 0; t < n_threads; t++) {
        orc_range_job *j = &jobs[t];
        if (j->rc) rc = -1;
        out->path = j->res.path;
        if (j->res.valid && j->res.gain > best) {
            best = j->res.gain;
            *out = j->res;
            out->proj = j->res.proj + j->p0;
            memcpy(bestL, j->lc, sizeof(bestL));
        }
    }
    if (left_counts)
        for (int c = 0; c < C; c++)
            left_counts[c] = bestL[c];
    free(jobs); free(th);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Tree to purity with each level's nodes searched on several threads        */
/* ------------------------------------------------------------------------ */

/*
 * The tree of orc_train_tree (R7, Section 2 item 2), grown on n_threads host
 * threads.  The nodes of one level are independent: a node's split depends
 * only on its own samples and key.  So each level runs in two phases:
 *   A. every node is examined, its projections sampled, its split searched
 *      and its segment stably partitioned in place, in any order on any
 *      thread; nodes of at least big_node samples one at a time with the
 *      projections divided over the threads (orc_split_search_mt), the rest
 *      each on one thread (orc_split_search_rule);
 *   B. one thread takes the results in breadth-first node order, exactly as
 *      orc_train_tree does: records, child ids, next-level offsets and the
 *      copy of each split node's partitioned segment.
 * The tree is the one orc_train_tree grows, field for field.  Returns 0 or -1.
 */
typedef struct {
    orc_split sp;
    int64_t N[ORC_MAX_CLASSES];
    int32_t k, searched, maj;
    int32_t feat[ORC_MAX_CAP];
    int8_t sign[ORC_MAX_CAP];
} orc_node_res;

typedef struct {
    const float *X; int64_t ld; int32_t d; const uint8_t *y; int C;
    int B, sort_below, hist_only, bin_rule, criterion, P, cap, max_depth, n_threads;
    int64_t big_node;
    double lambda;
    int32_t *cur;            /* this level's segments (partitioned in place) */
    const orc_pending *lvl;  /* this level's nodes */
    orc_node_res *res;       /* per node of the level */
    int64_t m;
    int64_t next;            /* next small node to take (guarded by mu) */
    int failed;
    pthread_mutex_t mu;
} orc_level_job;

/* Phase A for node j: counts, leaf tests, sampling, search, in-place stable
 * partition.  tmp holds at least the node's sample count; the work arrays
 * hold P (ptr P+1) and P*cap entries.  threads > 1 divides the projections. */
static int orc_level_node(orc_level_job *L, int64_t j, int threads, int32_t *tmp, int32_t *pnnz,
                          int32_t *pfeat, int8_t *psign, int32_t *ptr, int32_t *cfeat, int8_t *csign)
{
    const orc_pending nd = L->lvl[j];
    orc_node_res *r = &L->res[j];
    int32_t *seg = L->cur + nd.off;
    const int C = L->C, cap = L->cap, P = L->P;
    memset(r, 0, sizeof(*r));
    for (int64_t i = 0; i < nd.cnt; i++)
        r->N[L->y[seg[i]]]++;
    int present = 0, maj = 0;
    for (int c = 0; c < C; c++) {
        if (r->N[c] > 0) present++;
        if (r->N[c] > r->N[maj]) maj = c;
    }
    r->maj = maj;
    r->sp.path = -1;
    if (nd.cnt < 2 || present < 2 || (L->max_depth >= 0 && nd.depth >= L->max_depth))
        return 0;
    if (orc_sample_node(nd.key, P, L->d, L->lambda, cap, pnnz, pfeat, psign))
        return -1;
    ptr[0] = 0;
    for (int p = 0; p < P; p++) {
        for (int q = 0; q < pnnz[p]; q++) {
            cfeat[ptr[p] + q] = pfeat[p * cap + q];
            csign[ptr[p] + q] = psign[p * cap + q];
        }
        ptr[p + 1] = ptr[p] + pnnz[p];
    }
    int rc;
    if (threads > 1)
        rc = orc_split_search_mt(L->X, L->ld, L->y, C, seg, nd.cnt, P, ptr, cfeat, csign, L->B,
                                 L->sort_below, L->hist_only, L->bin_rule, nd.key, L->criterion,
                                 threads, &r->sp, NULL);
    else
        rc = orc_split_search_rule(L->X, L->ld, L->y, C, seg, nd.cnt, P, ptr, cfeat, csign, L->B,
                                   L->sort_below, L->hist_only, L->bin_rule, nd.key, 0,
                                   L->criterion, &r->sp, NULL, NULL, NULL, NULL, NULL);
    if (rc)
        return -1;
    r->searched = 1;
    if (!r->sp.valid)
        return 0;
    int k = pnnz[r->sp.proj];
    const int32_t *wf = pfeat + r->sp.proj * cap;
    const int8_t *ws = psign + r->sp.proj * cap;
    r->k = k;
    for (int q = 0; q < k; q++) {
        r->feat[q] = wf[q];
        r->sign[q] = ws[q];
    }
    int64_t nl = 0;
    for (int64_t i = 0; i < nd.cnt; i++)
        if (project(L->X, L->ld, seg[i], wf, ws, k) < r->sp.threshold)
            tmp[nl++] = seg[i];
    int64_t rr = nl;
    for (int64_t i = 0; i < nd.cnt; i++)
        if (!(project(L->X, L->ld, seg[i], wf, ws, k) < r->sp.threshold))
            tmp[rr++] = seg[i];
    if (nl != r->sp.n_left)
        return -1; /* cannot happen: the split's left count is the partition's */
    memcpy(seg, tmp, (size_t)nd.cnt * sizeof(int32_t));
    return 0;
}

typedef struct {
    orc_level_job *L;
    int32_t *tmp, *pnnz, *pfeat, *ptr, *cfeat;
    int8_t *psign, *csign;
} orc_worker;

static void *orc_level_worker(void *arg)
{
    orc_worker *w = (orc_worker *)arg;
    orc_level_job *L = w->L;
    for (;;) {
        int64_t j = -1;
        pthread_mutex_lock(&L->mu);
        while (L->next < L->m && L->lvl[L->next].cnt >= L->big_node)
            L->next++; /* large nodes were done in phase A's first part */
        if (L->next < L->m && !L->failed)
            j = L->next++;
        pthread_mutex_unlock(&L->mu);
        if (j < 0)
            break;
        if (orc_level_node(L, j, 1, w->tmp, w->pnnz, w->pfeat, w->psign, w->ptr, w->cfeat, w->csign)) {
            pthread_mutex_lock(&L->mu);
            L->failed = 1;
            pthread_mutex_unlock(&L->mu);
        }
    }
    return NULL;
}

int orc_train_tree_mt(const float *X, int64_t ld, int32_t d, const uint8_t *y, int C,
                      const int32_t *root_idx, int64_t n_root, int B, int sort_below,
                      int hist_only, int bin_rule, int criterion, int P, double lambda, int cap,
                      uint64_t seed, int32_t tree_id, int32_t max_depth, int n_threads,
                      int64_t big_node, orc_tree *out)
{
    memset(out, 0, sizeof(*out));
    if (C < 1 || C > ORC_MAX_CLASSES || cap < 1 || cap > ORC_MAX_CAP || n_root < 1 || P < 1)
        return -1;
    if (n_threads < 1)
        n_threads = 1;
    out->n_classes = C;
    out->cap = cap;
    if (tree_reserve(out, 2 * n_root + 1, C, cap))
        return -1;

    int32_t *cur = (int32_t *)malloc((size_t)n_root * sizeof(int32_t));
    int32_t *nxt = (int32_t *)malloc((size_t)n_root * sizeof(int32_t));
    orc_pending *lvl = (orc_pending *)malloc((size_t)n_root * sizeof(orc_pending));
    orc_pending *nlv = (orc_pending *)malloc((size_t)n_root * sizeof(orc_pending));
    orc_node_res *res = NULL;
    int64_t res_cap = 0;
    orc_worker *wk = (orc_worker *)calloc((size_t)n_threads, sizeof(orc_worker));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    int rc = -1;
    if (!cur || !nxt || !lvl || !nlv || !wk || !th)
        goto done;
    for (int t = 0; t < n_threads; t++) {
        wk[t].tmp = (int32_t *)malloc((size_t)n_root * sizeof(int32_t));
        wk[t].pnnz = (int32_t *)malloc((size_t)P * sizeof(int32_t));
        wk[t].pfeat = (int32_t *)malloc((size_t)P * cap * sizeof(int32_t));
        wk[t].psign = (int8_t *)malloc((size_t)P * cap);
        wk[t].ptr = (int32_t *)malloc((size_t)(P + 1) * sizeof(int32_t));
        wk[t].cfeat = (int32_t *)malloc((size_t)P * cap * sizeof(int32_t));
        wk[t].csign = (int8_t *)malloc((size_t)P * cap);
        if (!wk[t].tmp || !wk[t].pnnz || !wk[t].pfeat || !wk[t].psign || !wk[t].ptr ||
            !wk[t].cfeat || !wk[t].csign)
            goto done;
    }

    memcpy(cur, root_idx, (size_t)n_root * sizeof(int32_t));
    int64_t m = 1, n_nodes = 1, level_base = 0;
    lvl[0].off = 0;
    lvl[0].cnt = n_root;
    lvl[0].key = orc_root_key(seed, tree_id);
    lvl[0].depth = 0;

    while (m > 0) {
        if (m > res_cap) {
            orc_node_res *q = (orc_node_res *)realloc(res, (size_t)m * sizeof(orc_node_res));
            if (!q)
                goto done;
            res = q;
            res_cap = m;
        }
        orc_level_job L;
        memset(&L, 0, sizeof(L));
        L.X = X; L.ld = ld; L.d = d; L.y = y; L.C = C;
        L.B = B; L.sort_below = sort_below; L.hist_only = hist_only; L.bin_rule = bin_rule;
        L.criterion = criterion; L.P = P; L.cap = cap; L.max_depth = max_depth;
        L.n_threads = n_threads; L.big_node = big_node; L.lambda = lambda;
        L.cur = cur; L.lvl = lvl; L.res = res; L.m = m;
        pthread_mutex_init(&L.mu, NULL);
        /* phase A, large nodes: one at a time, projections over the threads */
        int fail = 0;
        for (int64_t j = 0; j < m && !fail; j++)
            if (lvl[j].cnt >= big_node)
                fail = orc_level_node(&L, j, n_threads, wk[0].tmp, wk[0].pnnz, wk[0].pfeat,
                                      wk[0].psign, wk[0].ptr, wk[0].cfeat, wk[0].csign);
        /* phase A, the other nodes: one per thread at a time */
        int started = 0;
        if (!fail) {
            for (int t = 0; t < n_threads; t++)
                wk[t].L = &L;
            for (int t = 1; t < n_threads && m > 1; t++) {
                if (pthread_create(&th[t], NULL, orc_level_worker, &wk[t]) != 0)
                    break;
                started = t;
            }
            orc_level_worker(&wk[0]);
            for (int t = 1; t <= started; t++)
                pthread_join(th[t], NULL);
            fail = L.failed;
        }
        pthread_mutex_destroy(&L.mu);
        if (fail)
            goto done;

        /* phase B: records and the next level, in node order */
        int64_t m_next = 0, next_off = 0;
        for (int64_t j = 0; j < m; j++) {
            int64_t id = level_base + j;
            const orc_pending nd = lvl[j];
            const orc_node_res *r = &res[j];
            out->left[id] = -1;
            out->right[id] = -1;
            out->depth[id] = nd.depth;
            out->leaf_class[id] = r->maj;
            out->proj_nnz[id] = 0;
            out->cand[id] = -1;
            out->path[id] = r->searched ? (int8_t)r->sp.path : (int8_t)-1;
            out->threshold[id] = 0.0f;
            out->gain[id] = 0.0;
            out->n_samples[id] = nd.cnt;
            for (int c = 0; c < C; c++)
                out->class_counts[id * C + c] = r->N[c];
            for (int q = 0; q < cap; q++) {
                out->feat[id * cap + q] = 0;
                out->sign[id * cap + q] = 0;
            }
            if (!r->searched || !r->sp.valid)
                continue;
            out->proj_nnz[id] = r->k;
            for (int q = 0; q < r->k; q++) {
                out->feat[id * cap + q] = r->feat[q];
                out->sign[id * cap + q] = r->sign[q];
            }
            out->cand[id] = r->sp.cand;
            out->threshold[id] = r->sp.threshold;
            out->gain[id] = r->sp.gain;
            memcpy(nxt + next_off, cur + nd.off, (size_t)nd.cnt * sizeof(int32_t));
            int64_t nl = r->sp.n_left;
            int64_t lid = n_nodes, rid = n_nodes + 1;
            n_nodes += 2;
            out->left[id] = (int32_t)lid;
            out->right[id] = (int32_t)rid;
            nlv[m_next].off = next_off;
            nlv[m_next].cnt = nl;
            nlv[m_next].key = orc_child_key(nd.key, 0);
            nlv[m_next].depth = nd.depth + 1;
            nlv[m_next + 1].off = next_off + nl;
            nlv[m_next + 1].cnt = nd.cnt - nl;
            nlv[m_next + 1].key = orc_child_key(nd.key, 1);
            nlv[m_next + 1].depth = nd.depth + 1;
            m_next += 2;
            next_off += nd.cnt;
        }
        level_base += m;
        m = m_next;
        int32_t *ti = cur; cur = nxt; nxt = ti;
        orc_pending *tl = lvl; lvl = nlv; nlv = tl;
    }
    out->n_nodes = n_nodes;
    rc = 0;
done:
    if (wk)
        for (int t = 0; t < n_threads; t++) {
            free(wk[t].tmp); free(wk[t].pnnz); free(wk[t].pfeat); free(wk[t].psign);
            free(wk[t].ptr); free(wk[t].cfeat); free(wk[t].csign);
        }
    free(wk); free(th); free(res);
    free(cur); free(nxt); free(lvl); free(nlv);
    if (rc)
        orc_tree_free(out);
    return rc;
}
