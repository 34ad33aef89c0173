// gapla_internal.cuh - internal data layout and device helpers of the GB300
// layer-assignment library (the public C ABI is include/gapla.h).
//
// HBM layout
//   Grid arrays are stored per preferred direction d (0 = H, 1 = V) as
//   [line][pos][ld]: line = row y (H) or column x (V); pos = GCell edge offset
//   along the line (npos = X for H, Y for V; the last pos is a sentinel used by
//   the demand difference array); ld = index of the layer among the layers of
//   direction d.  All layers of one direction that a segment may take are thus
//   adjacent in memory: the DP reads the congestion prefix of all of them at a
//   segment end with one contiguous load.
//   Per-node tables (A, Cc, M, via stacks) are [node][LD] with LD = the larger
//   per-direction layer count; entries of a son are [son][LD] indexed by the
//   parent's candidate index.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gapla.h"

namespace gapla {

constexpr int kMaxL = LA_MAX_LAYERS;
constexpr int64_t kPenMax = int64_t(1) << 48;

// Nodes are bucketed by (level, class, size class): class = min(sons, 2) +
// 0 for a non-root node with a pin, 3 for a root (roots always hold the driver
// pin), 6 for a node without a pin; size class = ceil(log2(nodes of the node's
// net)), capped at 15.  Inside every (level, class) range the nodes of nets
// with at most 2^k nodes form a prefix, for every k: the batched form splits
// small and large nets at any power of two without re-sorting.
constexpr int kClasses = 9;
__host__ __device__ inline int node_class(bool root, int sons, bool has_pin) {
  return (sons < 2 ? sons : 2) + (root ? 3 : (has_pin ? 0 : 6));
}
constexpr int kSizeClasses = 16;
constexpr int kMinBigSc = 5;  // nets of 17+ nodes get per-net level lists
__host__ __device__ inline int size_class(int64_t m) {
  int s = 0;
  while ((int64_t(1) << s) < m && s < kSizeClasses - 1) ++s;
  return s;
}
__host__ __device__ inline int64_t bucket_key(int64_t h, int cls, int sc) {
  return (h * kClasses + cls) * kSizeClasses + sc;
}

// Device error word: (index << 8) | code, smallest wins (atomicMin).
enum DevErr : int {
  DE_NONE = 0,
  DE_NETPTR = 1,      // net_ptr not increasing / out of range
  DE_PARENT = 2,      // parent id out of order
  DE_COORD = 3,       // x / y outside the grid
  DE_SEGMENT = 4,     // segment not straight or of zero length
  DE_PIN = 5,         // pin layer out of range, or root without a pin
  DE_VALUE = 6,       // negative or non-finite cap / criticality / driver R; cap without a pin
  DE_ASSIGN = 7,      // assignment layer of the wrong direction / stack not covering
  DE_DEGREE = 8,      // more sons than the kernels support
  DE_BATCH = 10,      // batch id out of range
  DE_NOSTACK = 9,     // DP found no valid stack (internal)
};
constexpr unsigned long long kNoErr = ~0ull;

// Everything a kernel needs about the layer stack; passed by value.
struct LayerInfo {
  int L;
  int nld[2];                 // layers per direction
  int lay[2][kMaxL];          // the layers of each direction, ascending
  int ld_of[kMaxL];           // index of layer l within its direction
  int8_t dir[kMaxL];
  uint32_t mask[2];           // bitmask of the layers of each direction
  double unit_r[kMaxL], unit_c[kMaxL], half_c[kMaxL];
  double rbar[2];             // mean unit R of each direction (look-ahead r_est)
  double via_c;
  int32_t nlines[2], npos[2]; // per direction
  int64_t grid_off[2];        // offset of direction d's [line][pos][ld] block (elements)
  int64_t pub_off[kMaxL + 1]; // offset of layer l in the public edge layout
};

// Small per-grid tables every DP/backtrack/demand kernel reads with
// thread-varying indices; kernels copy them to shared memory (load_tables).
// Row stride of the Rvia table: odd, so that the threads of a node, each on
// its own row l, reading column lc hit different shared-memory banks (a
// stride of 16 doubles = 128 bytes would put them all on one bank).
constexpr int kRvStride = kMaxL + 1;
struct DevTables {
  double rv[kMaxL * kRvStride];  // Rvia(a, b) at [a * kRvStride + b]: sum of via R between layers a and b
  double kd[kMaxL];           // 0.0, 1.0, ..., 15.0 (via counts as doubles)
  double unit_r[kMaxL], unit_c[kMaxL], half_c[kMaxL];
  double via_c;
  int64_t grid_off[2];
  int32_t npos[2], nlines[2], nld[2];
  uint32_t mask[2];
  int32_t L, pad_;
  int8_t lay[2][kMaxL];
  int8_t ld_of[kMaxL];
  int8_t dir[kMaxL];
};
static_assert(sizeof(DevTables) % 8 == 0, "DevTables is copied as 8-byte words");

// Segment geometry of a non-root node, packed:
// bit 63: direction, bits 32..47 line, 16..31 lo, 0..15 len.
__host__ __device__ inline uint64_t pack_geo(int d, int line, int lo, int len) {
  return (uint64_t(d) << 63) | (uint64_t(uint32_t(line)) << 32) | (uint64_t(uint32_t(lo)) << 16) |
         uint64_t(uint32_t(len));
}
__host__ __device__ inline int geo_dir(uint64_t g) { return int(g >> 63); }
__host__ __device__ inline int geo_line(uint64_t g) { return int((g >> 32) & 0xFFFF); }
__host__ __device__ inline int geo_lo(uint64_t g) { return int((g >> 16) & 0xFFFF); }
__host__ __device__ inline int geo_len(uint64_t g) { return int(g & 0xFFFF); }

struct Forest {
  int64_t N = 0, V = 0;
  int Hmax = 0;                         // max height (levels 0..Hmax)
  int nbatch = 1;                       // batches; batch k's level h is the global level k (Hmax + 1) + h
  int nlev = 1;                         // global levels: nbatch (Hmax + 1)
  std::vector<int64_t> lvl_off;         // host copy: global level g is [lvl_off[g], lvl_off[g+1])
  std::vector<int64_t> key_off;         // host copy: offsets of the (level, class, size class) buckets
  uint64_t key_hash = 0;                // hash of key_off (a captured round depends on it)
  // Per-net level lists of the nets with size class >= kMinBigSc (input-order
  // slots of the net: bl_nodes[base + j] is the internal id of its j-th node
  // by height; bl_hoff[base + n + h] the start of height h, relative to base).
  int32_t* bl_nodes = nullptr;
  int32_t* bl_hoff = nullptr;
  int32_t* net_H = nullptr;             // [N] height of each net
  int32_t* big_queue = nullptr;         // those nets, size class descending (largest first)
  std::vector<int64_t> big_sc_cnt;      // host: how many of them per size class
  int* queue_ctr = nullptr;             // device work-queue counter
  // Device arrays.  Node ids are int32 (V < 2^31).  After la_load_nets every
  // per-node array is in INTERNAL order: nodes sorted by (level, class), so a
  // level's nodes, their table rows and their sons' rows are contiguous
  // ranges.  lvl_nodes maps internal -> input id (outputs are scattered back
  // through it at the API boundary).
  int64_t* net_ptr = nullptr;           // N + 1 (input ids)
  int32_t* root_of_net = nullptr;       // N: internal id of each net's root
  int32_t* parent_g = nullptr;          // parent id, -1 at roots
  int32_t* net_of = nullptr;            // net of each node
  int8_t* pin = nullptr;
  double* sink_cap = nullptr;
  double* kappa = nullptr;
  double* gk = nullptr;                 // kappa at pin nodes, 0 elsewhere (adjoint seed)
  double* r_drv = nullptr;              // per net
  uint64_t* geo = nullptr;              // packed segment geometry (0 at roots)
  int32_t* child_start = nullptr;       // first son slot in child_list
  int32_t* nch = nullptr;               // number of sons
  int32_t* child_list = nullptr;        // son ids, increasing within a parent
  int32_t* son0 = nullptr;              // internal order: the first son's id (-1 at a leaf)
  int32_t* height = nullptr;
  int32_t* lvl_nodes = nullptr;         // internal -> input node id
  double* W_eq4 = nullptr;
  double* rho_eq4 = nullptr;
  double* W_adj = nullptr;
  double* rho_adj = nullptr;
  double* rho_zero = nullptr;           // [V] zeros: r_est of the look-ahead ablation (allocated on first use)
  bool have_adj = false;
  bool wsum_valid = false;              // W_adj holds the kappa sums below each node (fixed per forest)
  // round tables
  double* A = nullptr;                  // [V][LD]
  double* Cc = nullptr;
  double* M = nullptr;
  double* B = nullptr;                  // look-ahead base fma(w_d r_est(parent), Cc, A)
  double* ncache[2] = {nullptr, nullptr};  // batched form, per weight source: [V][2] per weight set, then [V][2] per round
  double* scache[2] = {nullptr, nullptr};  // and [V][LD][3] per (node, layer) constants
  int8_t* sb = nullptr;                 // [V][LD] chosen stack bottom
  int8_t* st = nullptr;                 // [V][LD] chosen stack top
  int8_t* ent = nullptr;                // [V][LD] layer of this son per parent candidate
  double* Jroot = nullptr;              // [V], valid at roots
  int8_t* layer = nullptr;              // [V]
  int8_t* b = nullptr;
  int8_t* t = nullptr;
  int8_t* layer_old = nullptr;          // [V] the layers a multi-batch round starts from
  bool have_assign = false;
  // Elmore scratch (internal order)
  double* s0 = nullptr;                 // [V]
  double* s1 = nullptr;
  double* s2 = nullptr;
  double* s3 = nullptr;
  double* s4 = nullptr;
  int64_t S = 0;                        // segments (non-root nodes)
  int32_t* seg_node = nullptr;          // [S] the segments' nodes, by (direction, line)
  uint64_t* seg_geo = nullptr;          // [S] their geometry, same order
  int64_t* seg_off = nullptr;           // [lines + 1] first segment of each line (line key as in the scan)
  // [kSizeClasses][Hmax + 1][kClasses] (first node, count) of the nets of at
  // most 2^k nodes, per (level, class): the tail kernels' level ranges (one batch)
  int64_t* range_tab = nullptr;
  double* red = nullptr;                // reduction partials: [red_cap] tof, [red_cap] J
  int red_cap = 0;
};

struct Grid {
  bool loaded = false;
  int X = 0, Y = 0;
  int64_t E = 0;                        // public edge count
  int64_t G = 0;                        // internal element count (both directions)
  LayerInfo li;
  double via_r[kMaxL] = {0};
  double ofw[kMaxL] = {0};
  double rvia[kMaxL * kMaxL] = {0};     // Rvia(a, b) table
  int64_t pen_T[kMaxL * 2 * 129] = {0}; // penalty table
  int32_t* cap = nullptr;               // internal layout, G elements
  int32_t* D = nullptr;
  int32_t* H = nullptr;
  int32_t* diff = nullptr;
  int64_t* P = nullptr;
  int64_t* T_dev = nullptr;             // penalty table on the device
  double* tofT_dev = nullptr;           // ofw_l exp(s over) for over in [-128, 128]
  DevTables tab;                        // host copy
  DevTables* tab_dev = nullptr;
  bool P_valid = false;                 // P holds the prefix of the current (D, H, hist_w)
  double round_hist_w = 1.0;            // hist_w of the last round (la_commit_demand uses it)
  bool fused_scan = false;              // the round's demand update runs inside the line scan
  double P_hist_w = -1.0;
};

// Batched form: small nets (size class <= k) by level waves of class kernels,
// the rest by the persistent block-per-net kernels on a second stream; chosen
// by the autotuner, and the round replayed as a CUDA graph.
struct BatchPlan {
  bool tuned = false;
  int k = kSizeClasses - 1;
  int block = 256, grid = 0;
  bool cached = true;         // read the constant caches (else recompute in the DP)
  int64_t n_big = 0;
  int Hs = 0;                 // highest level with a small-net node
  int tail_h = 1 << 30;       // levels tail_h..Hs (if any) run in one persistent block, not as waves
  int tail_T = 0;             // the task count below which a level joins the tail (0: no tail)
  double best_ms = 0.0;       // tuning time of the chosen plan
  int trials = 0;
  // one graph and one constant cache per weight source (0 Eq. 4, 1 adjoint)
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  double w[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};  // what each graph was captured with
  long long graph_launches[2] = {0, 0};
  uint64_t graph_sig[2] = {0, 0};  // the device addresses and shapes each graph was captured with
  double cache_wd[2] = {-1.0, -1.0}, cache_wcap[2] = {-1.0, -1.0};
};

// The tuner's choice for one forest shape: a forest loaded later whose
// (level, class, size class) bucket offsets are the same reuses it untimed.
struct TuneMemo {
  bool valid = false;
  int L = 0, LD = 0;
  std::vector<int64_t> key_off;
  int k = 0, block = 0, grid = 0;
  bool cached = true;
  int tail_T = 0;
  double best_ms = 0.0;
  int trials = 0;
};

struct Stats {  // device accumulators of one round
  unsigned long long vias, wl, relu;
  unsigned long long wl_layer[kMaxL];
};

}  // namespace gapla

struct la_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool poisoned = false;
  la_status inject = LA_OK;             // la_inject_fault: the failure the next matching step reports
  bool fuse_adjoint = false;            // the backtrack kernels also do the adjoint's top-down step
  std::string err;
  size_t bytes = 0;
  gapla::Grid grid;
  gapla::Forest forest;
  unsigned long long* d_err = nullptr;  // device error word
  gapla::Stats* d_stats = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int LD = 0;
  long long launches = 0;               // kernels launched (host-side count)
  cudaStream_t s2 = nullptr;            // second stream (big-net bucket)
  cudaStream_t s3 = nullptr;            // third stream (a level's several-son, root and no-pin classes)
  cudaEvent_t ev_lfork = nullptr, ev_ljoin = nullptr;
  cudaStream_t s_cap = nullptr;         // stream the batched round is captured on
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  gapla::BatchPlan plan;
  gapla::TuneMemo memo;
  void* alloc_groups = nullptr;         // device allocations, grouped per load
};

namespace gapla {

// ------------------------------- kernels --------------------------------
// k_load.cu
// to_internal: public -> internal (and negative values are reported in err);
// otherwise internal -> public (pub is written).
void launch_grid_to_internal(const LayerInfo& li, int X, int Y, const int32_t* pub, int32_t* inter,
                             bool to_internal, unsigned long long* err, cudaStream_t s);
// d_max: [0] max height, [1] max batch id, [2] set when a net range is bad
void launch_forest_prepare(la_ctx* c, Forest& f, const la_net_desc* d, int* d_max, cudaStream_t s);
// Between two batches of a round: the demand of the nodes [lo, hi) moves from
// their old layers (layer_old, or none) to their new ones, into the
// difference array (global atomics).
void launch_demand_delta(la_ctx* c, int64_t lo, int64_t hi, const int8_t* layer_old, cudaStream_t s);
// batch: the input's per-net batch ids (or null); hmax1 = Hmax + 1; nkeys buckets;
// counts (lvl_cnt non-null, zeroed), then placement (lvl_cursor holding the
// bucket offsets) into in2int[input id] = internal id and key_of[input id] = bucket
void launch_level_sort(Forest& f, const int32_t* batch, int hmax1, int64_t nkeys, int32_t* lvl_cnt,
                       int64_t* lvl_cursor, int32_t* in2int, int32_t* key_of, cudaStream_t s);
// segments by (direction, line): counts (cnt non-null, zeroed), then placement
// (cursor holding the key offsets)
void launch_seg_sort(const Forest& f, int nl0, int nkeys, int32_t* cnt, int64_t* cursor, int32_t* seg_node,
                     uint64_t* seg_geo, cudaStream_t s);
// per-net level lists and the big-net queue (input-order forest `in`, internal ids via in2int)
void launch_net_levels(const Forest& in, const int32_t* in2int, Forest& out, int32_t* sc_cnt, int64_t* sc_cur,
                       cudaStream_t s);
void launch_check_assignment(la_ctx* c, const int8_t* layer, const int8_t* b, const int8_t* t,
                             cudaStream_t s);
// input-order forest `in` (after prepare and level sort) -> internal order `out`,
// out.lvl_nodes[internal id] = input id
void launch_renumber(const Forest& in, const int32_t* in2int, const int32_t* key_of, int64_t nkeys, Forest& out,
                     cudaStream_t s);
// f.son0[v] = f.child_list[f.child_start[v]] (-1 without sons), internal order
void launch_first_son(const Forest& f, cudaStream_t s);
// dst[i] = src[perm[i]] (gather into internal order) or dst[perm[i]] = src[i] (scatter)
void launch_permute8(int64_t V, const int32_t* perm, const int8_t* src, int8_t* dst, bool gather, cudaStream_t s);
void launch_permute64(int64_t V, const int32_t* perm, const double* src, double* dst, bool gather, cudaStream_t s);
// k_round.cu
struct RoundW {
  double w_cong, w_via, w_cap, w_d, hist_w;
};
// from_diff: 0 the prefix of the current D and H; 1 D := the difference
// array's prefix, then H += max(0, D - C) and the statistics; 2 D += that
// prefix (between the batches of a round: H and the statistics untouched);
// 3 the current D as given (a sharded round's summed demand), then
// H += max(0, D - C) and the statistics.  The difference array is cleared in
// modes 1 and 2.
void launch_scan_lines(la_ctx* c, int from_diff, double hist_w, double* red_tof, cudaStream_t s);
// the demand update and the line scan of the end of a round (fused when a
// line's difference array fits in shared memory: prepare_fused_scan at load)
constexpr size_t kFusedLineMaxBytes = 96 * 1024;
size_t fused_line_bytes(const LayerInfo& li);
bool prepare_fused_scan(const LayerInfo& li);
void launch_demand_scan(la_ctx* c, double hist_w, double* red_tof, cudaStream_t s);
// the end of a round that is one shard of a round split by nets: D := the
// demand of this context's nets (global atomics, then a scan); H untouched
void launch_local_demand(la_ctx* c, double hist_w, double* red_tof, cudaStream_t s);
// kmax: nodes of nets up to size class kmax (kSizeClasses - 1 = every node)
// cache: the batched form's constant-cache set to read (0 Eq. 4, 1 adjoint), or
// kNoCache to recompute the constants in the DP (the plain form)
constexpr int kNoCache = -1;
// class_mask: the node classes to launch (bit cls)
constexpr unsigned kAllClasses = (1u << kClasses) - 1u;
void launch_dp_level(la_ctx* c, const RoundW& w, const double* W, const double* rho, int level, int kmax,
                     int cache, cudaStream_t s, unsigned class_mask = kAllClasses);
void launch_backtrack_level(la_ctx* c, int level, int kmax, cudaStream_t s);
// the first n_big nets of the big-net queue, persistent grid
void launch_dp_bignets(la_ctx* c, const RoundW& w, const double* W, const double* rho, int64_t n_big, int grid,
                       int block, int cache, cudaStream_t s);
// The tail of the small-net level waves: levels h0..h1 in one block that
// walks them in order (DP ascending / backtrack descending), any class.
void launch_dp_tail(la_ctx* c, const RoundW& w, const double* W, const double* rho, int h0, int h1, int k, int cache,
                    cudaStream_t s);
void launch_backtrack_tail(la_ctx* c, int h0, int h1, int k, cudaStream_t s);
void launch_backtrack_bignets(la_ctx* c, int64_t n_big, int grid, int block, cudaStream_t s);
void launch_seg_consts(la_ctx* c, const RoundW& w, const double* W, int cache, cudaStream_t s);
void launch_node_round(la_ctx* c, const RoundW& w, const double* rho, int cache, cudaStream_t s);
int bignet_blocks_per_sm(int L, int LD, int block);
void launch_demand(la_ctx* c, cudaStream_t s);
void launch_sum_roots(la_ctx* c, double* part, double* J_out, cudaStream_t s);
int scan_blocks(const LayerInfo& li);
// k_elmore.cu
// R, C in internal order, or scattered to input order when perm != nullptr
void launch_rc_from_assignment(la_ctx* c, double* R, double* C, const int32_t* perm, cudaStream_t s);
// delays from given R_seg, C_seg; every array in input order
void launch_elmore_fwd(la_ctx* c, const double* R, const double* C, double* delay, cudaStream_t s);
// the delays of the current assignment (R_seg, C_seg from its layers), input order
void launch_elmore_assignment(la_ctx* c, double* delay_input_order, cudaStream_t s);
// dL/dR_seg, dL/dC_seg of L = sum g delay from given R_seg, C_seg, g; input order
void launch_elmore_bwd(la_ctx* c, const double* R, const double* C, const double* g, double* dR, double* dC,
                       cudaStream_t s);
// The DP's adjoint weights on the current assignment (R_seg = len x unit R of
// the layer): with_wsum, W_adj = the sums of g = kappa below each node, then
// rho_adj = U_J; else rho_adj = U_J from the W_adj already there.
void launch_reweight(la_ctx* c, bool with_wsum, cudaStream_t s);
// W_adj = the sums of kappa below each node (they depend on the forest only)
void launch_wsum(la_ctx* c, cudaStream_t s);

// error message of calls that have no context (read by la_last_error(NULL))
void set_noctx_error(const std::string& msg);

// small device helpers
__device__ __forceinline__ void dev_error(unsigned long long* err, int code, int64_t index) {
  unsigned long long key = (static_cast<unsigned long long>(index) << 8) | static_cast<unsigned long long>(code);
  atomicMin(err, key);
}
// Order of non-negative doubles through their bit patterns (integer compare,
// no FP64 pipe): a < b  <=>  bits(a) < bits(b) for a, b >= +0, not NaN.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// double(x) for an integer 0 <= x < 2^53, built from its bits (IEEE 754
// binary64): the leading one, at bit p, shifted to the hidden bit 52, which
// carries into the biased exponent 1022 + p written above it.  Exact, and no
// FP64 instruction: GB300 issues FP64 (conversions included) at 1/64 of the
// FP32 rate, so the kernels bound by it convert integers this way.
__device__ __forceinline__ double exact_int_to_double(unsigned long long x) {
  if (x == 0) return 0.0;
  const int p = 63 - __clzll(static_cast<long long>(x));
  return __longlong_as_double(
      static_cast<long long>((x << (52 - p)) + (static_cast<unsigned long long>(1022 + p) << 52)));
}

// Copy the tables to shared memory; every thread of the block must call it.
__device__ __forceinline__ void load_tables(DevTables& s, const DevTables* g) {
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(g);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s);
  for (int i = threadIdx.x; i < int(sizeof(DevTables) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Butterfly warp sum: the same lanes pair up on every run (deterministic).
template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

}  // namespace gapla
