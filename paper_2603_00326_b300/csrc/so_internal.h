// so_internal.h -- host-side interface between the C ABI layer (so_api.cu) and
// the kernels (so_kernels.cu).  Not installed; not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <new>
#include <cuda_runtime.h>

#include "../../include/soforest.h"

namespace sof {

constexpr int kMaxClasses = 8;     // labels in [0, 8)
constexpr int kMaxBins = 256;      // equal-width bins per projection
constexpr int kMaxCap = 32;        // non-zeros per projection row
constexpr int kMaxProj = 1024;     // projections per node
constexpr int kMaxSortBelow = 2048;  // largest exact-path node + 1
constexpr int kSortRegMax = 128;     // exact-path nodes sorted by one warp in registers
constexpr int kRwRow = 256;          // random-width table row: B-1 boundaries (padded) or guide cells
constexpr int kRwCells = 256;        // guide cells per projection

// 4-lane int64 vector carried through the generic device scans.
struct V4 {
  long long x, y, z, w;
};

struct DatasetView {
  const float* X;
  int64_t n;
  int64_t ld;
  const uint8_t* y;
  int32_t d;
  int32_t C;
  const float* Xr = nullptr;  // optional row-major copy [n][d]
};

// Projection rows q = node*P + p: features feat[beg[q] .. end[q]).
// CSR input: beg = ptr, end = ptr + 1.  Sampled slots: beg[q] = q*cap.
struct ProjView {
  const int32_t* beg;
  const int32_t* end;
  const int32_t* feat;
  const int8_t* sign;
  int32_t P;
};

// Bump allocator over one device buffer (256-byte aligned pieces).
struct Carver {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  bool dry = false;  // sizing pass: count only
  template <typename T>
  T* take(size_t count) {
    const size_t off = (used + 255) & ~size_t(255);
    const size_t bytes = count * sizeof(T);
    used = off + bytes;
    if (dry || base == nullptr) return nullptr;
    if (used > cap) return nullptr;
    return reinterpret_cast<T*>(base + off);
  }
  bool ok() const { return dry || used <= cap; }
};

// Histogram-path work decomposition (chosen by the host; the autotuner may
// change them).
struct HistTuning {
  int32_t chunk = 16384;  // samples per work item (S)
  int32_t pgroup = 8;     // projections per work item of the general kernels (one warp each)
  int32_t staged_pg = 0;  // projections per work item of the staged kernels (0: the most that fit)
};

// Random-width boundary tables of the histogram nodes (one row of kRwRow per
// histogram slot h and projection p, row h*P + p):
//  t   boundaries t_1..t_{B-1}, ascending, padded with +inf;
//  g   guide of cell c: lo | (k << 8), lo = number of boundaries whose cell
//      is below c, k = number of boundaries in cell c (cells of the monotone
//      map v -> clamp(floor(fma(v, s, o)), 0, kRwCells-1));
//  so  (s, o) of that map; s < 0 marks a projection without a guide (zero or
//      ill-conditioned range), binned by binary search.
struct RwTables {
  float* t = nullptr;
  uint16_t* g = nullptr;
  float2* so = nullptr;
};

// Everything one batched split search needs.
struct SearchArgs {
  DatasetView ds;
  const int32_t* idx = nullptr;
  int64_t n_total = 0;
  const int64_t* node_off = nullptr;  // device [m+1]
  int32_t m = 0;
  ProjView pv{};
  int32_t B = 256;
  int32_t T = 1024;
  int32_t hist_only = 0;
  float eps = 4e-6f;
  int32_t max_nnz = kMaxCap;        // upper bound of projection row lengths
  so_split* out = nullptr;          // device [m]
  int64_t* left_counts = nullptr;   // device [m*C] or null
  // inspection outputs (so_histograms): all nodes forced onto the histogram path
  float* minmax_out = nullptr;
  int32_t* hist_out = nullptr;
  float* gain32_out = nullptr;
  float* bounds_out = nullptr;      // [m*P*(B-1)] boundaries (so_histograms)
  HistTuning tune{};
  // SO_BINS_EQUAL_WIDTH or SO_BINS_RANDOM_WIDTH; node keys of the random rule
  int32_t bin_rule = 0;
  const uint64_t* bin_keys = nullptr;  // device [m]
  int32_t criterion = 0;               // SO_CRIT_GINI or SO_CRIT_ENTROPY
  // optional [P][n_total] buffer: the min / max pass stores every
  // histogram-path sample's projected values and the histogram pass reads
  // them back instead of gathering the feature columns again
  float* vbuf = nullptr;
  // projection rows sampled by this library (k_sample: distinct ascending
  // features in [0, d), 1 <= length <= max_nnz), so they need no validation
  int32_t rows_trusted = 0;
  // an upper bound of the nodes' sizes, or -1: below T no node takes the
  // histogram path, so its launches are left out
  int64_t max_nv_hint = -1;
};

// Scratch of the staged-tile histogram kernels (so_hist_staged.cu).
struct StagedScratch {
  int32_t* ng1 = nullptr;      // groups per histogram node (min/max kernel)
  int32_t* gs1 = nullptr;      // [m_hist_cap][P+1] group starts
  int32_t* ng2 = nullptr;      // groups per histogram node (histogram kernel)
  int32_t* gs2 = nullptr;
  int64_t* item_off1 = nullptr;
  int64_t* item_off2 = nullptr;
  V4* item_total = nullptr;
  V4* tiles = nullptr;
  unsigned long long* item_ctr = nullptr;  // [2] dynamic item counters of the two kernels
};

// Device scratch of one search (carved from a workspace).
struct SearchScratch {
  V4* plan_total = nullptr;     // [1]: x=m_hist, y=m_sort, z=n_items
  V4* tiles = nullptr;          // scan tile sums
  int32_t* hist_nodes = nullptr;
  int32_t* sort_nodes = nullptr;
  int64_t* item_off = nullptr;
  uint32_t* mm_keys = nullptr;  // [m_hist_cap*P*2]
  float* max32 = nullptr;       // [m_hist_cap*P]
  int32_t* node_counts = nullptr;  // [m_hist_cap*C]
  int32_t* hist = nullptr;      // [m_hist_cap*P*B*C]
  int32_t* err = nullptr;       // [m+1] per-node bad-input flags
  void* sort_res = nullptr;     // [m*P] per-(exact-path node, projection) results
  int32_t* node_cls = nullptr;  // [m*8] class counts of exact-path nodes
  int64_t* sort_lists = nullptr;  // [2][m*P] exact-path pairs to re-score in double
  int32_t* sort_list_n = nullptr; // [2] their counts
  int64_t m_hist_cap = 0;
  StagedScratch staged;
  RwTables rw;                  // random-width rule only
  double* xlnx = nullptr;       // [2048] x ln x of the entropy criterion
};

// Carves a SearchScratch (dry run gives the size).
void carve_search(Carver& cv, SearchScratch& s, int32_t m, int64_t n_total, int32_t P, int32_t C,
                  int32_t B, int32_t T, int32_t hist_only, int32_t bin_rule = 0);

// Random-width boundaries, guide and cell map of every (histogram node,
// projection), from the node keys and the min / max keys mm.
cudaError_t launch_rw_bounds(const SearchArgs& a, const V4* plan_total, const int32_t* hist_nodes,
                             const uint32_t* mm, const RwTables& rw, cudaStream_t st);

// Whether per-stage tracing is on (so_profile_enable).
bool profiling_on();

// Records a CUDA event pair around a launch group when profiling is on, and
// counts its kernel launches.
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t st, int launches = 1);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t st_;
  int stage_ = -1;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

struct DeviceInfo {
  int device = 0;
  int num_sms = 148;
  int smem_optin = 232448;  // largest shared memory of one CTA (static + dynamic), bytes
};
const DeviceInfo& device_info();

cudaError_t launch_search(const SearchArgs& a, const SearchScratch& s, cudaStream_t st);

// exact path: one warp per (node, projection); res holds m*P per-projection
// results (sort_res_bytes() each), indexed by node
// Split criterion of the scoring kernels.
struct Crit {
  int ent;            // 0: Gini decrease; 1: information gain
  float eps;          // Gini: relative re-score window (above three times the key's relative error)
  const double* tab;  // information gain: x ln x for x < 2048 (device), or null
};

cudaError_t launch_sort_warp(const SearchArgs& a, const Crit& cr, const V4* plan_total, const int32_t* tiny,
                             const int32_t* med, void* res, int32_t* node_cls, int64_t* lists, int32_t* list_n,
                             cudaStream_t st);
size_t sort_res_bytes();

// staged-tile histogram path (features up to 65536)
bool staged_supported(int d);
int hist_group_size(int B, int C, bool rw);  // the most projections per staged histogram item
void carve_staged(Carver& cv, StagedScratch& s, int64_t m_hist_cap, int P);
cudaError_t launch_staged(const SearchArgs& a, const V4* plan_total, const int32_t* hist_nodes,
                          int64_t m_hist_cap, const StagedScratch& ss, uint32_t* mm, int32_t* hist,
                          const RwTables& rw, int64_t S, int kmax, cudaStream_t st);

// ---- partition ------------------------------------------------------------
// Per-node instruction for the batched stable partition.
enum PartMode : int32_t { PART_DROP = 0, PART_SPLIT = 1, PART_COPY = 2 };
struct PartNode {
  int64_t beg, end;        // segment in idx_in
  int64_t ones_prefix;     // number of flag-1 elements before beg (whole level)
  int64_t ones;            // flag-1 elements of this node (left size, or size for COPY)
  int64_t dst_one;         // destination of the flag-1 part, -1 = drop
  int64_t dst_zero;        // destination of the flag-0 part, -1 = drop
  int64_t feat_off;        // projection row start in (feat, sign)
  float thr;
  int32_t nnz;
  int32_t mode;
  int32_t pad;
};

struct PartArgs {
  DatasetView ds;
  const int32_t* idx_in;
  int32_t* idx_out;
  int64_t n;                 // elements of the level
  const int64_t* node_off;   // [m+1] segment starts (device), node_off[m] = n
  int32_t m;
  const PartNode* nodes;     // [m]
  const int32_t* feat;
  const int8_t* sign;
  uint8_t* flags;            // [n]
  int64_t* tile_cnt;         // [tiles]
  int64_t* ones_total;       // [1] out: all flag-1 elements
  int64_t n_out;             // length of idx_out (writes outside are refused)
  int32_t* err;
  PartNode* fix_node;        // single-node form: its flag-1 count is only known
                             // after the flags are counted; set it then
};
int64_t part_tiles(int64_t n);
cudaError_t launch_partition(const PartArgs& a, cudaStream_t st);

// PartNode for the batch API / single-node API from split records.
cudaError_t launch_part_nodes_from_splits(const int64_t* node_off, int32_t m, const so_split* splits,
                                          const ProjView pv, PartNode* nodes, V4* tiles,
                                          V4* total, cudaStream_t st);
// Single node with a given projection: ones = computed on device.
cudaError_t launch_part_single(int64_t n, int32_t nnz, float thr, PartNode* node,
                               int64_t* node_off, cudaStream_t st);
cudaError_t launch_fill_off(int64_t* off, int64_t n, cudaStream_t st);
cudaError_t launch_bench_nodes(int32_t m, int32_t s, int64_t n, uint64_t seed, int32_t* idx, int64_t* off,
                               uint64_t* keys, cudaStream_t st);
cudaError_t launch_hist_inspect(const SearchArgs& a, const SearchScratch& s, float* gain_tmp,
                                cudaStream_t st);
// scan tile sums needed for n elements (tile = 512 elements)
inline int64_t scan_tiles_for_host(int64_t n) { return (n + 511) / 512 + 1; }

// ---- sampler ----------------------------------------------------------------
cudaError_t launch_sample(int32_t m, const uint64_t* keys, int32_t P, int32_t d, double lambda,
                          int32_t cap, int32_t* nnz, int32_t* feat, int8_t* sign, int32_t* beg,
                          int32_t* end, cudaStream_t st);

// ---- tree level machinery ---------------------------------------------------
struct TreeDev {
  int32_t *left, *right, *depth, *leaf_class, *proj_nnz, *feat, *cand;
  int8_t *sign, *path;
  float* threshold;
  int64_t *n_samples, *class_counts;
  double* gain;
  int32_t cap, C;
};

struct Frontier {
  int64_t* off;      // [M+1]
  uint64_t* key;     // [M]
  int32_t* id;       // [M]
  int32_t* depth;    // [M]
  int32_t* counts;   // [M*C]
};

struct LevelStats {  // device-resident, read by the host once per level
  long long m_next;
  long long n_next;
  long long new_nodes;
  int err;
  int max_next;  // samples of the next frontier's largest node
};

cudaError_t launch_tree_root(const DatasetView ds, const int32_t* root_idx, int64_t n_root,
                             uint64_t root_key, int32_t max_depth, TreeDev t, Frontier f,
                             LevelStats* stats, cudaStream_t st);
// Copies each searched node's winning projection (from sampled slots) and
// split fields into the tree records.
cudaError_t launch_tree_record_splits(int32_t j0, int32_t mb, const Frontier f, const so_split* splits,
                                      const int32_t* snnz, const int32_t* sfeat, const int8_t* ssign,
                                      int32_t P, int32_t cap, TreeDev t, cudaStream_t st);
cudaError_t launch_tree_level(int32_t m, const Frontier cur, Frontier nxt, const so_split* splits,
                              const int64_t* left_counts, int32_t max_depth, int64_t node_base_next,
                              TreeDev t, PartNode* pnodes, V4* tiles, V4* total, LevelStats* stats,
                              cudaStream_t st);

// ---- argument checks and conventions shared by every entry point ------------
// Sets the thread-local message of so_last_error() and returns st.
so_status fail(so_status st, const char* fmt, ...);
// Each returns SO_OK or SO_EINVAL with a message.  keys_given: the caller
// supplies the random-width node keys through p->bin_keys.
so_status check_dataset(const so_dataset* ds);
so_status check_params(const so_split_params* p, bool keys_given = true);
so_status check_projs(const so_projs* pr);
// Re-score window actually used: eps raised to the float gain's error floor.
float effective_eps(float eps, int C);
// Longest projection row to assume (max_nnz, or the cap when unknown).
int32_t projs_max_nnz(const so_projs* pr);
// The histogram work decomposition a caller (or so_autotune) chose.
void apply_tuning(SearchArgs& a, int32_t proj_per_cta, int32_t chunk);
DatasetView view_of(const so_dataset* ds);
ProjView csr_view(const so_projs* pr);
// Forgets the cached device addresses of the allocation-free entry point's
// static scratch (so_shutdown calls it; the next call looks them up again).
void noalloc_forget();

// Runs an entry point's body; no C++ exception crosses the ABI.
template <typename F>
so_status guarded(F f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fail(SO_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(SO_EINTERNAL, "unexpected exception");
  }
}

}  // namespace sof
