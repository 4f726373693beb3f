/*
 * soforest.h -- C ABI of the B300 (sm_103a) sparse-oblique split-search library.
 *
 * The library computes, on one GPU, the per-node split search of sparse
 * oblique forest training as stated in "Vectorized Adaptive Histograms for
 * Sparse Oblique Forests" (Section 3, steps 1-3; Section 3.1 the
 * sort/histogram switch by node cardinality; Section 3.3 the GPU offload,
 * whose two kernels take a list of projection non-zeros and return the best
 * projection and its split), plus the stable partition of the node's samples
 * and a breadth-first tree grown to purity (Section 2, item 2).
 *
 * Conventions shared by every call:
 *   - Every pointer documented "device" is CUDA device memory owned by the
 *     caller; the library never frees it.  Pointers documented "host" are
 *     ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered; those that return results into host
 *     memory synchronise the stream before returning.
 *   - Arguments are validated on the host before any launch; a bad argument
 *     returns SO_EINVAL and launches nothing.  Device-side consistency checks
 *     report SO_EINTERNAL.  CUDA errors report SO_ECUDA.  so_last_error()
 *     returns a thread-local message for the last failure.
 *   - No C++ exception crosses this boundary.
 *   - Feature matrices are column-major: X[f*ld + i] is feature f of sample i.
 *     Values must be finite.  Labels are uint8 in [0, n_classes), n_classes
 *     in 1..8.
 *   - A projection is a sparse row of +-1 weights over distinct features
 *     listed in ascending order.  Its value for a sample is computed in float,
 *     starting from +0 and adding (or subtracting) the features in that order,
 *     one round-to-nearest addition each, no fused multiply-add.
 *   - Results are bit-identical to the plain CPU definition of the method:
 *     bins, histograms, chosen splits (projection, candidate, threshold bits,
 *     double gain bits) and tree arrays.
 */
#ifndef SOFOREST_H
#define SOFOREST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SO_OK = 0,
    SO_EINVAL = 1,     /* bad argument, found on the host before any launch */
    SO_ENOMEM = 2,     /* device or host allocation failed / workspace too small */
    SO_ECUDA = 3,      /* a CUDA runtime call failed */
    SO_ETIMEOUT = 4,   /* reserved for a bounded device-side wait that gives up; no
                          call returns it: no kernel here waits on another */
    SO_EINTERNAL = 5   /* a device-side consistency check failed */
} so_status;

/* Training data, device resident (the paper preloads the whole table once,
 * Section 3.3).  X: device, column-major, X[f*ld + i], f < d, i < n.
 * y: device, n labels in [0, n_classes).
 * Xr: optional device row-major copy of the same values, Xr[i*d + f], or
 * NULL.  When given, the min/max pass reads the feature rows of scattered
 * samples from it, and so does the exact path for nodes of more than 128
 * samples. One sample's features share DRAM sectors, where X costs one
 * sector per (sample, feature). Results do not change. */
typedef struct {
    const float *X;
    int64_t n;          /* samples, 1 .. 2^31-1 */
    int32_t d;          /* features, >= 1 */
    int64_t ld;         /* leading dimension, >= n */
    const uint8_t *y;
    int32_t n_classes;  /* 1..8 */
    const float *Xr;    /* optional row-major copy [n][d], or NULL */
} so_dataset;

/* Sparse projections in CSR form (Section 3: "a sparse list" of non-zero
 * offsets with random weights).  For a batch of m nodes the rows are
 * node-major: row q = node*n_proj + p, so ptr has m*n_proj + 1 entries.
 * All three arrays are device memory.  feat values are distinct within a row,
 * ascending, in [0, d); sign values are +1 or -1; 1 <= row length <= 32. */
typedef struct {
    int32_t n_proj;        /* projections per node, 1..1024 */
    const int32_t *ptr;    /* [rows + 1] */
    const int32_t *feat;   /* [ptr[rows]] */
    const int8_t *sign;    /* [ptr[rows]] */
    int32_t max_nnz;       /* upper bound of every row length (selects the kernel
                              variant), 1..32; 0 = unknown, taken as 32.  A row
                              longer than this marks its node malformed. */
} so_projs;

/* Histogram boundary rules (so_split_params.bin_rule). */
enum { SO_BINS_EQUAL_WIDTH = 0, SO_BINS_RANDOM_WIDTH = 1 };

/* Split criteria (so_split_params.criterion). */
enum { SO_CRIT_GINI = 0, SO_CRIT_ENTROPY = 1 };

/* Split-search parameters.
 *  n_bins       bins per projection, 2..256 (Section 3.2 uses 256).
 *  sort_below   T: nodes with fewer than T samples take the exact sort path
 *               (Section 3.1); 0..2048.
 *  hist_only    nonzero: every node takes the histogram path.
 *  rescore_rel_eps  relative window of the double-precision re-score of
 *               float near-ties; <= 0 selects the default 4e-6.  Values below
 *               the float error bound of the gain are raised to that bound.
 *  bin_rule     where the B-1 boundaries t_1..t_{B-1} of a projection with
 *               node range [min, max] sit.  Under both rules a value v falls
 *               in bin #{j : t_j <= v}, candidate b sends bins <= b left
 *               (exactly v < t_{b+1}) and its threshold is t_{b+1}.
 *               SO_BINS_EQUAL_WIDTH: t_j = min + j*w, w = (max-min)/B (float).
 *               SO_BINS_RANDOM_WIDTH: boundaries at random intervals, the
 *               YDF default the paper's Section 1 footnote names.  For the
 *               node key K and projection p, a splitmix64 generator with state
 *               splitmix64((K ^ 0x6A09E667F3BCC908) + p*0xD2B74407B1CE6E93)
 *               draws B-1 outputs r; their top 23 bits u = r >> 41, sorted
 *               ascending, place t_j = min + f_j*(max-min) with
 *               f_j = (2u+1)*2^-24 (float, two roundings).
 *  criterion    SO_CRIT_GINI: Gini decrease sum_c D_c^2 / (n^2 nL nR),
 *               D_c = n L_c - N_c nL.  SO_CRIT_ENTROPY: information gain in
 *               nats (the entropy criterion of YDF, Section 3 step 3):
 *               (f(n) - sum_c f(N_c) + sum_c f(L_c) - f(nL) + sum_c f(R_c)
 *               - f(nR)) / n with f(x) = x ln x, in double in that order, 0
 *               when every D_c is 0; ln x = e ln2 + 2s sum_{k<12} s^2k/(2k+1)
 *               with x = 2^e m, m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1)
 *               (so the bits are the same on any IEEE machine).  Either way
 *               the best split maximises the double gain (ties to the lowest
 *               projection, then candidate) and is valid iff that gain is > 0.
 *  bin_keys     SO_BINS_RANDOM_WIDTH: device uint64 [m], the key of each node
 *               of the call (node j of a batch reads bin_keys[j]; a one-node
 *               call reads bin_keys[0]); the same keys so_sample_projections
 *               takes.  Ignored (may be NULL) for equal width.
 *  proj_per_cta projections whose histograms (all n_bins bins of each) one
 *               CTA holds in shared memory per histogram work item; 0 = the
 *               most that fit (at most 64), else 1..64 (capped at what fits).
 *  chunk        samples per histogram work item; 0 = 16384, else
 *               512..16384.  Neither changes any result (integer counts),
 *               only the work decomposition; so_autotune picks both. */
typedef struct {
    int32_t n_bins;
    int32_t sort_below;
    int32_t hist_only;
    float rescore_rel_eps;
    int32_t bin_rule;
    int32_t criterion;
    const uint64_t *bin_keys;
    int32_t proj_per_cta;
    int32_t chunk;
} so_split_params;

/* Result of one node's split search.
 *  valid      1 iff a split with criterion gain > 0 exists.
 *  proj       winning projection (row within the node), or -1.
 *  path       0 histogram, 1 exact sort: the path the node's size selects
 *             (also reported for nodes of fewer than 2 samples, which are
 *             never valid); -2: a projection row of the node is malformed and
 *             the node was skipped.
 *  cand       histogram path: bin b (bins <= b go left); sort path: sorted
 *             position i (the i+1 smallest values go left); -1 if invalid.
 *  threshold  samples with projected value < threshold go left.
 *  gain       the criterion's gain (Gini decrease or information gain, see
 *             so_split_params) evaluated in double (bit-identical to the CPU
 *             definition).
 *  n_left / n_right  child sizes (counting repeated samples). */
typedef struct {
    int32_t valid;
    int32_t proj;
    int32_t path;
    int32_t cand;
    float threshold;
    double gain;
    int64_t n_left;
    int64_t n_right;
} so_split;

/* Fills the optional row-major copy of a feature matrix (so_dataset.Xr):
 * Xr[i*d + f] = X[f*ld + i] for i < n, f < d.  X, Xr: device; Xr holds n*d
 * floats and is owned by the caller.  Asynchronous on `stream`. */
so_status so_row_major(const float *X, int64_t n, int32_t d, int64_t ld, float *Xr, void *stream);

/* Best split of ONE node (the paper's node-at-a-time GPU call, Section 3.3).
 *  idx        device, n_node sample indices (repeats allowed, e.g. bootstrap).
 *  projs      n_proj rows for this node.
 *  out_host   host, receives the result; the call synchronises `stream`.
 *  workspace  device scratch of ws_bytes, or NULL to use the library's
 *             internal arena (kept until so_shutdown()).  Size it with
 *             so_split_search_ws_bytes(1, n_node, ...).
 *  left_counts_host  host [n_classes] class counts of the left child, or NULL. */
so_status so_split_search(const so_dataset *ds, const int32_t *idx, int64_t n_node,
                          const so_projs *projs, const so_split_params *params,
                          so_split *out_host, int64_t *left_counts_host,
                          void *workspace, size_t ws_bytes, void *stream);

/* Best split of m nodes at once (the batched frontier): node j owns
 * idx[node_off[j] .. node_off[j+1]).  Small and large nodes take their own
 * paths in the same call.  Asynchronous; nothing is read back.
 *  node_off        device int64 [m+1], non-decreasing, node_off[0] >= 0,
 *                  node_off[m] <= n_total (the length of idx).
 *  out_dev         device so_split [m].
 *  left_counts_dev device int64 [m*n_classes] or NULL.
 *  workspace       as above, sized by so_split_search_ws_bytes(m, n_total, ...);
 *                  for m > 1 it includes a [n_proj][n_total] float buffer in
 *                  which the min/max pass keeps the histogram-path samples'
 *                  projected values for the histogram pass. */
so_status so_split_search_batch(const so_dataset *ds, const int32_t *idx, int64_t n_total,
                                const int64_t *node_off, int32_t m, const so_projs *projs,
                                const so_split_params *params, so_split *out_dev,
                                int64_t *left_counts_dev, void *workspace, size_t ws_bytes,
                                void *stream);

/* so_split_search without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code running inside another framework's memory pool that owns
 * the device memory, processes held to a fixed device-memory budget, and
 * latency-critical loops where an allocation (and the device synchronisation
 * cudaMalloc/cudaFree can imply) is not acceptable.  Same arguments and result
 * as so_split_search, minus the workspace.
 *
 * Scratch: a statically allocated 8 MiB device array inside the library (every
 * GPU that loads the library holds it until the process exits).  A node whose
 * scratch (about n_proj * n_bins * n_classes * 4 bytes of histograms plus a
 * few KiB) exceeds 8 MiB is rejected with SO_EINVAL before any launch.  The
 * first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it until
 * so_shutdown; after a cudaDeviceReset call so_shutdown before the next call,
 * so that the address is looked up again.  Every call on a device shares the
 * array and leaves its contents behind (the kernels initialise what they
 * read); calls that overlap on the GPU, from any stream or thread, race on
 * it.  Keep tracing (so_profile_enable) off: tracing creates CUDA events.
 * The call synchronises `stream` to return the split on the host, so it
 * cannot be made while `stream` is being captured into a CUDA graph.
 * Argument errors and CUDA errors are reported as by so_split_search. */
so_status so_split_search_noalloc(const so_dataset *ds, const int32_t *idx, int64_t n_node,
                                  const so_projs *projs, const so_split_params *params,
                                  so_split *out_host, int64_t *left_counts_host, void *stream);

/* Device workspace bytes needed by the two calls above. */
size_t so_split_search_ws_bytes(int32_t m, int64_t n_total, int32_t n_proj, int32_t n_classes,
                                const so_split_params *params);

/* Stable partition of one node's samples (left = value < threshold, in
 * input order, then right in input order), in place.
 *  idx_inout  device [n_node]; feat/sign device [nnz] (one projection row).
 *  n_left_out host; the call synchronises `stream`.  Uses the internal arena. */
so_status so_partition(const so_dataset *ds, int32_t *idx_inout, int64_t n_node,
                       const int32_t *feat, const int8_t *sign, int32_t nnz, float threshold,
                       int64_t *n_left_out, void *stream);

/* Stable partition of m nodes' segments at once (the batched frontier).
 * Node j with splits[j].valid moves idx_in[node_off[j]..node_off[j+1]) to
 * idx_out at the same offsets, left part first; invalid nodes are copied
 * unchanged.  projs are the same rows as given to so_split_search_batch.
 * Asynchronous.  idx_in and idx_out must not overlap. */
so_status so_partition_batch(const so_dataset *ds, const int32_t *idx_in, int32_t *idx_out,
                             int64_t n_total, const int64_t *node_off, int32_t m,
                             const so_projs *projs, const so_split *splits_dev, void *stream);

/* Per-node projection sampling on the device (Section 3: the projection
 * matrix; Appendix A: distinct features by Floyd's algorithm).  For node j
 * with 64-bit key keys[j] and projection p: a splitmix64 stream seeded from
 * (key, p) draws nnz = min(cap, d, 1 + Poisson(lambda)) by inverse CDF, then
 * nnz distinct features by Floyd's algorithm (sorted ascending), then one
 * sign bit per feature.  Outputs use fixed slots of width cap:
 *  nnz_out  device int32 [m*n_proj]
 *  feat_out device int32 [m*n_proj*cap]  (slot q*cap .. q*cap+nnz-1)
 *  sign_out device int8  [m*n_proj*cap]
 * keys: device uint64 [m].  cap in 1..32, lambda >= 0.  Asynchronous. */
so_status so_sample_projections(int32_t m, const uint64_t *keys, int32_t n_proj, int32_t d,
                                double lambda, int32_t cap, int32_t *nnz_out, int32_t *feat_out,
                                int8_t *sign_out, void *stream);

/* The histogram stage alone for m nodes, every node on the histogram path
 * (Section 3 step 2; the paper's first GPU kernel).  For inspection and
 * testing of the intermediate results.
 *  params      n_bins, bin_rule and bin_keys are used; the rest is ignored.
 *  minmax_dev  device float [m*n_proj*2]: (min, max) of each projection.
 *  hist_dev    device int32 [m*n_proj*n_bins*n_classes] class counts per bin.
 *  gain32_dev  device float [m*n_proj*(n_bins-1)] float Gini gain of every
 *              candidate without the 1/n^2 factor, sum_c D_c^2 / (nL nR)
 *              (-1 where a side is empty), or NULL; Gini whatever
 *              params->criterion says.
 *  bounds_dev  device float [m*n_proj*(n_bins-1)] boundaries t_1..t_{B-1}
 *              of every projection, or NULL.
 * Asynchronous; uses the internal arena. */
so_status so_histograms(const so_dataset *ds, const int32_t *idx, int64_t n_total,
                        const int64_t *node_off, int32_t m, const so_projs *projs,
                        const so_split_params *params, float *minmax_dev, int32_t *hist_dev,
                        float *gain32_dev, float *bounds_dev, void *stream);

/* Tree growth parameters.
 *  n_bins, sort_below, hist_only, rescore_rel_eps, bin_rule, criterion,
 *             proj_per_cta, chunk  as in so_split_params, except that chunk 0
 *             means 4096 here (a tree's histogram nodes are mostly gathered
 *             nodes of a few thousand samples); random-width boundaries use the
 *             tree's node keys.
 *  n_proj     projections sampled per node, 1..1024.
 *  lambda, nnz_cap  nnz law of a projection: min(nnz_cap, d, 1+Poisson(lambda)).
 *  seed, tree_id    root key = splitmix64(seed ^ tree_id*0x9E3779B97F4A7C15);
 *             child key = splitmix64(2*key + side), side 0 left, 1 right.
 *  max_depth  -1 grows to purity; otherwise nodes at this depth are leaves. */
typedef struct {
    int32_t n_bins;
    int32_t sort_below;
    int32_t hist_only;
    float rescore_rel_eps;
    int32_t n_proj;
    double lambda;
    int32_t nnz_cap;
    uint64_t seed;
    int32_t tree_id;
    int32_t max_depth;
    int32_t bin_rule;
    int32_t criterion;
    int32_t proj_per_cta;
    int32_t chunk;
} so_tree_params;

/* A trained tree in breadth-first order (children appended level by level in
 * parent order, left before right).  Host arrays allocated by the library;
 * release with so_tree_free().  Per node i:
 *  left/right   child ids or -1 for a leaf; depth (root 0);
 *  leaf_class   majority class (ties to the lowest id);
 *  proj_nnz, feat[i*cap..], sign[i*cap..]  the split's projection (nnz 0 for leaves);
 *  cand, path   as in so_split (path -1: never searched, i.e. the node was
 *               pure, had fewer than 2 samples or sat at max_depth);
 *  threshold, gain  as in so_split (0 for leaves);
 *  n_samples, class_counts[i*n_classes..]  node population. */
typedef struct {
    int64_t n_nodes;
    int32_t n_classes;
    int32_t cap;
    int32_t *left, *right, *depth, *leaf_class, *proj_nnz, *feat, *cand;
    int8_t *sign, *path;
    float *threshold;
    int64_t *n_samples, *class_counts;
    double *gain;
} so_tree;

/* Grows one tree to purity (Section 2, item 2), level by level: every node of
 * a depth is searched in one batched pass (sampling, min/max, histograms or
 * exact sort, Gini scan, partition), then the next frontier is built on the
 * device.  root_idx: device [n_root] (repeats allowed).  out: host, filled on
 * success.  Synchronises `stream`; uses the internal arena. */
so_status so_train_tree(const so_dataset *ds, const int32_t *root_idx, int64_t n_root,
                        const so_tree_params *params, so_tree *out, void *stream);

void so_tree_free(so_tree *tree);

/* ---- forest inference ----------------------------------------------------
 * A forest on the device: the trees' node arrays concatenated, tree t owning
 * nodes [tree_off[t], tree_off[t+1]); child ids are local to their tree (as
 * in so_tree), -1 for a leaf.  All arrays device, caller-owned:
 *  tree_off [n_trees+1] int64; left, right, leaf_class, proj_nnz [n_nodes]
 *  int32; feat [n_nodes*cap] int32 and sign [n_nodes*cap] int8 (a node's
 *  projection, ascending features); threshold [n_nodes] float. */
typedef struct {
    int32_t n_trees;
    int32_t n_classes;     /* 1..8 */
    int32_t cap;           /* slots per node in feat/sign, 1..32 */
    const int64_t *tree_off;
    const int32_t *left, *right, *leaf_class, *proj_nnz, *feat;
    const int8_t *sign;
    const float *threshold;
} so_forest;

/* Forest prediction (the forest's use, Section 4's accuracy evaluation):
 * every tree routes sample i from its root -- at an internal node the
 * projection value of Section 3 step 1 (float, +0 start, ascending features,
 * one rounding per term) goes left iff it is below the threshold -- and votes
 * its leaf's class.  votes: device [n*n_classes] int32 or NULL; pred: device
 * [n] int32, the class with most votes (ties to the lowest id).
 * X: device, column-major X[f*ld + i], i < n, f < d; every feature id in the
 * forest must be < d (checked on the device: a node with a bad feature or a
 * child outside its tree makes the call return SO_EINTERNAL).  A route
 * longer than 2^20 nodes stops (SO_EINTERNAL).  Synchronises `stream`. */
so_status so_predict(const float *X, int64_t n, int32_t d, int64_t ld, const so_forest *forest,
                     int32_t *votes, int32_t *pred, void *stream);

/* The start-up crossover microbenchmark of Section 3.1: on this GPU, for node
 * sizes s = 32 .. 2047, times one batched split search of many s-sample nodes
 * drawn from ds on the exact path and on the histogram path (n_proj sampled
 * projections per node with nnz = min(nnz_cap, d, 1+Poisson(lambda))), and
 * writes into params->sort_below the smallest measured size at which the
 * histogram path is no slower per node (2048 if it never is).  Then times the
 * histogram path for proj_per_cta in {16, 32, 64} (those that fit) and chunk
 * in {4096, 8192, 16384} on two workloads -- one node of min(n, 2^20)
 * bootstrap-like samples and a batch of up to 128 gathered nodes of 2048
 * samples -- each the better of two timings, and writes into
 * params->proj_per_cta and params->chunk the pair with the least sum of its
 * times relative to each workload's fastest.  Other fields of params are kept.  Times per size go to times_ms_host [2*n_sizes] when
 * not NULL (exact, histogram), with the sizes in sizes_host [n_sizes];
 * n_sizes_out receives the count (at most 16).  The timed searches use
 * params->n_bins and params->bin_rule (random width with keys of their own;
 * params->bin_keys is not read).  Takes well under a second; synchronises
 * `stream`; uses the internal arena. */
so_status so_autotune(const so_dataset *ds, int32_t n_proj, double lambda, int32_t nnz_cap,
                      so_split_params *params, int32_t *sizes_host, float *times_ms_host,
                      int32_t *n_sizes_out, void *stream);

/* ---- tracing ------------------------------------------------------------
 * Per-stage timing (the paper instruments every node, Section 3).  When
 * enabled, each kernel launch group records a CUDA event pair on its stream.
 * so_profile_read() waits for the recorded events, writes up to max_entries
 * (stage name, launches, total milliseconds) and resets the totals; it
 * returns the number of entries written. */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} so_profile_entry;

void so_profile_enable(int on);
int so_profile_read(so_profile_entry *out, int max_entries);

/* Number of kernels this library has launched in this process. */
long long so_launch_count(void);

/* Thread-local description of the last failure on this thread ("" if none). */
const char *so_last_error(void);

/* Releases the internal arena on every device the library touched. */
void so_shutdown(void);

/* Library version string. */
const char *so_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SOFOREST_H */
