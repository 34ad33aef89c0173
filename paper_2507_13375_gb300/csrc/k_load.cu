// k_load.cu - forest loader and levelisation kernels (Sec. III-B directed
// tree; levels of Alg. 2; edge weights of Eq. 4; look-ahead r_est of Sec. III-D).
#include "gapla_internal.cuh"

namespace gapla {

// Public edge layout <-> internal [d][line][pos][ld] layout, one thread per public edge.
__global__ void k_grid_layout(LayerInfo li, int X, int Y, int64_t E, const int32_t* __restrict__ pub_in,
                              int32_t* __restrict__ int_out, const int32_t* __restrict__ int_in,
                              int32_t* __restrict__ pub_out, unsigned long long* err) {
  int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= E) return;
  int l = 0;
  while (l + 1 < li.L && g >= li.pub_off[l + 1]) ++l;
  const int64_t i = g - li.pub_off[l];
  const int d = li.dir[l];
  const int64_t per = d == 0 ? X - 1 : Y - 1;
  const int64_t line = i / per, e = i % per;
  const int64_t k = li.grid_off[d] + (line * li.npos[d] + e) * li.nld[d] + li.ld_of[l];
  if (pub_in) {
    const int32_t v = pub_in[g];
    if (v < 0) dev_error(err, DE_VALUE, g);
    int_out[k] = v;
  } else {
    pub_out[g] = int_in[k];
  }
}

void launch_grid_to_internal(const LayerInfo& li, int X, int Y, const int32_t* pub, int32_t* inter,
                             bool to_internal, unsigned long long* err, cudaStream_t s) {
  const int64_t E = li.pub_off[li.L];
  if (E == 0) return;
  const int T = 256;
  const int64_t B = (E + T - 1) / T;
  if (to_internal) k_grid_layout<<<(unsigned)B, T, 0, s>>>(li, X, Y, E, pub, inter, nullptr, nullptr, err);
  else k_grid_layout<<<(unsigned)B, T, 0, s>>>(li, X, Y, E, nullptr, nullptr, inter, const_cast<int32_t*>(pub), err);
}

struct PrepArgs {
  int64_t N, V;
  int X, Y, L;
  const int64_t* net_ptr_in;
  const int32_t *x, *y, *parent;
  const int8_t* pin_in;
  const double *cap_in, *kap_in, *rdrv_in;
  int64_t* net_ptr;
  int32_t *parent_g, *net_of, *child_start, *nch, *child_list, *height;
  int8_t* pin;
  double *sink_cap, *kappa, *r_drv, *W, *rho;  // W, rho: Eq. 4 weights and look-ahead r_est
  double rbar[2];                               // mean unit R of each direction
  uint64_t* geo;
  int* hmax;             // [0] max height, [1] max batch id, [2] a bad net range
  const int32_t* batch;  // per net, or null
  unsigned long long* err;
};

__device__ inline bool finite_nonneg(double v) { return v >= 0.0 && v <= 1.7976931348623157e308; }

// Three passes (each error reports its node; the error word keeps the least
// (index, code), so the message names the first bad node of the forest):
//   nets:  the net's node range, driver R and batch; net_of of its nodes;
//   nodes: node fields, parent order, coordinates, the straight segment to the
//          parent and its packed geometry; sons counted per parent (atomics);
//          node-parallel, every array read or written once, coalesced;
//   tree:  one warp per group of nets: son CSR, heights, Eq. 4 weights and r_est.
// The node pass runs only when every net range is good (the ranges are then
// disjoint and cover the nodes), the tree pass only when no check failed.
__device__ __forceinline__ bool net_range_ok(const PrepArgs& a, int64_t n, int64_t base, int64_t end) {
  return base >= 0 && base < end && end <= a.V && (n != 0 || base == 0) && (n != a.N - 1 || end == a.V);
}

// Block-wide maximum of v (every thread of the block calls it), added to *dst
// with one atomic per block: a per-net atomic on one address serialises.
__device__ __forceinline__ void block_atomic_max(int* dst, int v) {
  __shared__ int s_m[32];
  v = __reduce_max_sync(~0u, v);
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = s_m[0];
    for (int w = 1; w < int(blockDim.x >> 5); ++w) m = max(m, s_m[w]);
    if (m > 0) atomicMax(dst, m);
  }
}

__global__ void __launch_bounds__(1024) k_prepare_nets(PrepArgs a) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int bmax = 0;
  if (n < a.N) {
    const int64_t base = a.net_ptr_in[n], end = a.net_ptr_in[n + 1];
    if (!net_range_ok(a, n, base, end)) {
      dev_error(a.err, DE_NETPTR, n);
      a.hmax[2] = 1;
    } else {
      if (!finite_nonneg(a.rdrv_in[n])) dev_error(a.err, DE_VALUE, base);
      if (a.batch) {
        const int bt = a.batch[n];
        if (bt < 0 || bt >= LA_MAX_BATCHES) dev_error(a.err, DE_BATCH, n);
        else bmax = bt;
      }
      a.net_ptr[n] = base;
      if (n == a.N - 1) a.net_ptr[a.N] = end;
      a.r_drv[n] = a.rdrv_in[n];
      for (int64_t v = base; v < end; ++v) a.net_of[v] = int32_t(n);
    }
  }
  if (a.batch) block_atomic_max(a.hmax + 1, bmax);
}

__global__ void k_prepare_nodes(PrepArgs a) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= a.V || a.hmax[2]) return;
  const int64_t n = a.net_of[v];
  const int64_t base = a.net_ptr_in[n];
  const int64_t i = v - base;
  const int32_t par = a.parent[v];
  const int32_t xv = a.x[v], yv = a.y[v];
  const int pv = a.pin_in[v];
  const double cv = a.cap_in[v], kv = a.kap_in[v];
  a.height[v] = 0;
  a.pin[v] = int8_t(pv);
  a.sink_cap[v] = cv;
  a.kappa[v] = kv;
  a.W[v] = pv >= 0 ? kv : 0.0;  // Eq. 4 starts from the node's own sink criticality
  if (i == 0 ? par != -1 : (par < 0 || par >= i)) { dev_error(a.err, DE_PARENT, v); return; }
  if (xv < 0 || xv >= a.X || yv < 0 || yv >= a.Y) { dev_error(a.err, DE_COORD, v); return; }
  if (pv < -1 || pv >= a.L || (i == 0 && pv < 0)) { dev_error(a.err, DE_PIN, v); return; }
  if (!finite_nonneg(cv) || !finite_nonneg(kv) || (pv < 0 && cv != 0.0)) { dev_error(a.err, DE_VALUE, v); return; }
  if (i == 0) {
    a.parent_g[v] = -1;
    a.geo[v] = 0;
    return;
  }
  const int64_t p = base + par;
  a.parent_g[v] = int32_t(p);
  const int32_t xp = a.x[p], yp = a.y[p];
  const int32_t dx = xv - xp, dy = yv - yp;
  if ((dx == 0) == (dy == 0)) { dev_error(a.err, DE_SEGMENT, v); return; }
  if (xp < 0 || xp >= a.X || yp < 0 || yp >= a.Y) return;  // the parent reports its coordinates
  if (dy == 0) a.geo[v] = pack_geo(0, yv, min(xv, xp), dx < 0 ? -dx : dx);  // row y, edges [min x, max x)
  else a.geo[v] = pack_geo(1, xv, min(yv, yp), dy < 0 ? -dy : dy);           // column x, edges [min y, max y)
  atomicAdd(a.nch + p, 1);
}

// One warp per kTreeNets consecutive nets, over their nodes in chunks of 32
// (lane = node - chunk start).  Sons have larger ids than their parent and
// stay in their net, so
//   forward chunks, ascending lanes:  parents before sons (CSR slots, r_est);
//   backward chunks, descending lanes: sons before parents (heights, W).
// Inside a chunk the sweep passes values by shuffles; a parent in another
// chunk is reached through memory (atomics backward, loads forward).
//   CSR: child_start = the net's base + the exclusive prefix of the son counts
//        inside the net (each net's slots [base, base + m - 1), the last slot
//        base + m - 1 holds -1); sons in id order inside their parent's run.
//   height = 0 at leaves, 1 + max over sons otherwise.
//   Eq. 4: W_v = the largest sink criticality in the subtree of v; r_est of
//        Sec. III-D: r(root) = W_root R_drv, r(v) = r(p) + W_v len_v rbar(dir v).
//        A son replaces W_p only when strictly larger, so W_p is the maximum
//        when it is positive and the node's own value otherwise, in any order.
constexpr int kTreeNets = 16;

__device__ __forceinline__ int prepare_tree_nets(const PrepArgs& a, int64_t n0, int64_t n1) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t lo = a.net_ptr_in[n0], hi = a.net_ptr_in[n1];
  int hmax = 0;
  // son slots: prefix of the counts over the range, plus one unused slot per
  // earlier net of the range; the counts restart as per-parent cursors
  int64_t carry = lo;
  for (int64_t c0 = lo; c0 < hi; c0 += 32) {
    const int64_t v = c0 + lane;
    const bool act = v < hi;
    const int k = act ? a.nch[v] : 0;
    int inc = k;
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(~0u, inc, d);
      if (lane >= d) inc += t;
    }
    if (act) {
      a.child_start[v] = int32_t(carry + inc - k + (a.net_of[v] - n0));
      a.nch[v] = 0;
    }
    carry += __shfl_sync(~0u, inc, 31);
  }
  __syncwarp();
  for (int64_t c0 = lo; c0 < hi; c0 += 32) {
    const int64_t v = c0 + lane;
    const long long p = v < hi ? a.parent_g[v] : -1;
    const bool son = p >= 0;
    const unsigned peers = __match_any_sync(~0u, p);
    int before = 0;
    if (son) {
      before = a.nch[p];
      a.child_list[a.child_start[p] + before + __popc(peers & lt)] = int32_t(v);
    }
    __syncwarp();
    if (son && (peers & lt) == 0) a.nch[p] = before + __popc(peers);
    __syncwarp();
  }
  // heights and W, sons before parents.  W >= 0 (or -0), so its bit pattern
  // as an int64 orders like the value, and only a positive son replaces it:
  // integer compares, off the FP64 pipe.
  for (int64_t c0 = lo + ((hi - 1 - lo) & ~int64_t(31)); c0 >= lo; c0 -= 32) {
    const int64_t v = c0 + lane;
    const bool act = v < hi;
    int h = act ? __ldcg(a.height + v) : 0;
    long long wb = act ? __ldcg(reinterpret_cast<const long long*>(a.W) + v) : 0;
    const int p = act ? a.parent_g[v] : -1;
    const int last = hi - 1 - c0 < 31 ? int(hi - 1 - c0) : 31;
    for (int j = last; j >= 0; --j) {
      const int hj = __shfl_sync(~0u, h, j);
      const long long wj = __shfl_sync(~0u, wb, j);
      const int pj = __shfl_sync(~0u, p, j);
      if (pj >= c0) {
        if (lane == pj - c0) {
          h = max(h, hj + 1);
          if (wj > 0 && wj > wb) wb = wj;
        }
      } else if (pj >= 0 && lane == j) {
        atomicMax(a.height + pj, hj + 1);
        if (wj > 0) atomicMax(reinterpret_cast<long long*>(a.W) + pj, wj);
      }
    }
    if (act) {
      a.height[v] = h;
      reinterpret_cast<long long*>(a.W)[v] = wb;
    }
    hmax = max(hmax, h);
    __syncwarp();
  }
  // r_est, parents before sons: a node in the chunk takes its parent's value
  // (one shuffle from the parent's lane) in the round after the parent's is
  // known; rounds = the depth of the chunk's trees, one FP64 add each.
  for (int64_t c0 = lo; c0 < hi; c0 += 32) {
    const int64_t v = c0 + lane;
    const bool act = v < hi;
    double r = 0.0, t = 0.0;
    int p = -1;
    bool done = true;
    if (act) {
      const double w = __ldcg(a.W + v);
      p = a.parent_g[v];
      if (p < 0) {
        const int nt = a.net_of[v];
        r = w * a.rdrv_in[nt];
        a.child_list[a.net_ptr_in[nt + 1] - 1] = -1;  // the net's unused last slot
      } else {
        const uint64_t g = a.geo[v];
        t = (w * double(geo_len(g))) * a.rbar[geo_dir(g)];
        if (p < c0) r = __ldcg(a.rho + p) + t;
        else done = false;
      }
    }
    const int src = done ? lane : int(p - c0);
    while (__any_sync(~0u, !done)) {
      const double rp = __shfl_sync(~0u, r, src);
      const int pd = __shfl_sync(~0u, int(done), src);
      if (!done && pd) {
        r = rp + t;
        done = true;
      }
    }
    if (act) a.rho[v] = r;
    __syncwarp();
  }
  return hmax;  // the largest height of the range (a root's)
}

__global__ void __launch_bounds__(256) k_prepare_tree(PrepArgs a) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t n0 = w * kTreeNets, n1 = n0 + kTreeNets < a.N ? n0 + kTreeNets : a.N;
  int h = 0;
  if (n0 < a.N && *a.err == kNoErr) h = prepare_tree_nets(a, n0, n1);  // uniform over the warp
  block_atomic_max(a.hmax, h);
}

void launch_forest_prepare(la_ctx* c, Forest& f, const la_net_desc* d, int* d_hmax, cudaStream_t s) {
  PrepArgs a;
  a.N = f.N; a.V = f.V; a.X = c->grid.X; a.Y = c->grid.Y; a.L = c->grid.li.L;
  a.net_ptr_in = d->net_ptr; a.x = d->x; a.y = d->y; a.parent = d->parent; a.pin_in = d->pin_layer;
  a.cap_in = d->sink_cap; a.kap_in = d->kappa; a.rdrv_in = d->r_drv;
  a.net_ptr = f.net_ptr; a.parent_g = f.parent_g; a.net_of = f.net_of; a.child_start = f.child_start;
  a.nch = f.nch; a.child_list = f.child_list; a.height = f.height; a.pin = f.pin; a.sink_cap = f.sink_cap;
  a.kappa = f.kappa; a.r_drv = f.r_drv; a.geo = f.geo; a.W = f.W_eq4; a.rho = f.rho_eq4;
  a.rbar[0] = c->grid.li.rbar[0];
  a.rbar[1] = c->grid.li.rbar[1];
  a.hmax = d_hmax;
  a.batch = d->batch;
  a.err = c->d_err;
  cudaMemsetAsync(f.nch, 0, sizeof(int32_t) * size_t(f.V), s);  // son counts: atomics of the node pass
  k_prepare_nets<<<(unsigned)((f.N + 1023) / 1024), 1024, 0, s>>>(a);
  k_prepare_nodes<<<(unsigned)((f.V + 255) / 256), 256, 0, s>>>(a);
  const int64_t warps = (f.N + kTreeNets - 1) / kTreeNets;
  k_prepare_tree<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(a);
  c->launches += 3;
}

struct BucketIn {
  const int32_t *height, *nch, *parent_g, *net_of;
  const int64_t* net_ptr;
  const int8_t* pin;
  const int32_t* batch;  // per net, or null
  int hmax1;             // Hmax + 1: a batch's span of global levels
};
__device__ __forceinline__ long long node_bucket(int64_t v, const BucketIn& b) {
  const int cls = node_class(b.parent_g[v] < 0, b.nch[v], b.pin[v] >= 0);
  const int n = b.net_of[v];
  const int64_t g = (b.batch ? int64_t(b.batch[n]) * b.hmax1 : 0) + b.height[v];
  return bucket_key(g, cls, size_class(b.net_ptr[n + 1] - b.net_ptr[n]));
}

// Counting sorts by a small integer key (the level buckets, the lines of the
// segments).  Count: per-key totals; place: each node reserves its position
// in its key's run (the runs laid out by the host from the totals).  Within
// a run the order is whatever the atomics give.  With at most kHistMaxKeys
// keys a block keeps its counts in shared memory and adds one total per key
// to global memory (kHistItems nodes per thread); otherwise warps add to
// global counters directly.
constexpr int kHistMaxKeys = 12288;  // 48 KB of shared counters
constexpr int kHistItems = 16;
constexpr int kHistT = 256;

struct LevelKeys {  // key = (global level, class, size class) bucket; out: in2int and the key of each node
  BucketIn b;
  int32_t *in2int, *key_of;
  __device__ long long key(int64_t v) const { return node_bucket(v, b); }
  __device__ void put(int64_t v, int64_t pos, long long k) const {
    in2int[v] = int32_t(pos);
    key_of[v] = int32_t(k);
  }
};

// Segments by (direction, line): key = line for horizontal segments, nlines0 +
// line for vertical ones; roots have no segment.  The demand pass walks them
// in this order, so a warp's atomics land in one or two lines.
__device__ __forceinline__ int seg_key(uint64_t g, int nl0) { return geo_dir(g) == 0 ? geo_line(g) : nl0 + geo_line(g); }
struct SegKeys {
  const int32_t* parent_g;
  const uint64_t* geo;
  int nl0;
  int32_t* seg_node;
  uint64_t* seg_geo;
  __device__ long long key(int64_t v) const { return parent_g[v] >= 0 ? seg_key(geo[v], nl0) : -1; }
  __device__ void put(int64_t v, int64_t pos, long long) const {
    seg_node[pos] = int32_t(v);
    seg_geo[pos] = geo[v];
  }
};

template <class K>
__global__ void __launch_bounds__(kHistT) k_hist_count(int64_t V, K kf, int nkeys, int32_t* __restrict__ cnt) {
  extern __shared__ int s_h[];
  for (int k = threadIdx.x; k < nkeys; k += kHistT) s_h[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t t0 = int64_t(blockIdx.x) * (kHistT * kHistItems) + threadIdx.x;
  for (int it = 0; it < kHistItems; ++it) {
    const int64_t v = t0 + it * kHistT;
    const int key = v < V ? int(kf.key(v)) : -1;
    const unsigned peers = __match_any_sync(~0u, key);
    if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(&s_h[key], __popc(peers));
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nkeys; k += kHistT)
    if (s_h[k]) atomicAdd(&cnt[k], s_h[k]);
}

template <class K>
__global__ void __launch_bounds__(kHistT) k_hist_place(int64_t V, K kf, int nkeys,
                                                       unsigned long long* __restrict__ cursor) {
  extern __shared__ int s_h[];
  for (int k = threadIdx.x; k < nkeys; k += kHistT) s_h[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t t0 = int64_t(blockIdx.x) * (kHistT * kHistItems) + threadIdx.x;
  int key[kHistItems], loc[kHistItems];
#pragma unroll
  for (int it = 0; it < kHistItems; ++it) {
    const int64_t v = t0 + it * kHistT;
    key[it] = v < V ? int(kf.key(v)) : -1;
    const unsigned peers = __match_any_sync(~0u, key[it]);
    const int leader = __ffs(peers) - 1;
    int old = 0;
    if (key[it] >= 0 && lane == leader) old = atomicAdd(&s_h[key[it]], __popc(peers));
    loc[it] = __shfl_sync(~0u, old, leader) + __popc(peers & lt);
  }
  __syncthreads();
  // the block's run of each key: positions < V < 2^31
  for (int k = threadIdx.x; k < nkeys; k += kHistT)
    if (s_h[k]) s_h[k] = int(atomicAdd(&cursor[k], (unsigned long long)s_h[k]));
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kHistItems; ++it)
    if (key[it] >= 0) kf.put(t0 + it * kHistT, int64_t(s_h[key[it]]) + loc[it], key[it]);
}

template <class K>
__global__ void k_glob_count(int64_t V, K kf, int32_t* __restrict__ cnt) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long key = v < V ? kf.key(v) : -1;
  const unsigned peers = __match_any_sync(~0u, key);
  if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[key], __popc(peers));
}

template <class K>
__global__ void k_glob_place(int64_t V, K kf, unsigned long long* __restrict__ cursor) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const long long key = v < V ? kf.key(v) : -1;
  const unsigned peers = __match_any_sync(~0u, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if (key >= 0 && lane == leader) base = atomicAdd(&cursor[key], (unsigned long long)__popc(peers));
  base = __shfl_sync(~0u, base, leader);
  if (key >= 0) kf.put(v, int64_t(base + __popc(peers & ((1u << lane) - 1u))), key);
}

// cnt: nkeys zeroed ints (count), or null; cursor: nkeys int64 holding the
// runs' first positions (place), or null.
template <class K>
static void key_sort(int64_t V, const K& kf, int64_t nkeys, int32_t* cnt, int64_t* cursor, cudaStream_t s) {
  auto* cur = reinterpret_cast<unsigned long long*>(cursor);
  if (nkeys <= kHistMaxKeys) {
    const unsigned B = (unsigned)((V + kHistT * kHistItems - 1) / (kHistT * kHistItems));
    const size_t sm = sizeof(int) * size_t(nkeys);
    if (cnt) k_hist_count<K><<<B, kHistT, sm, s>>>(V, kf, int(nkeys), cnt);
    if (cursor) k_hist_place<K><<<B, kHistT, sm, s>>>(V, kf, int(nkeys), cur);
  } else {
    const unsigned B = (unsigned)((V + 255) / 256);
    if (cnt) k_glob_count<K><<<B, 256, 0, s>>>(V, kf, cnt);
    if (cursor) k_glob_place<K><<<B, 256, 0, s>>>(V, kf, cur);
  }
}

void launch_seg_sort(const Forest& f, int nl0, int nkeys, int32_t* cnt, int64_t* cursor, int32_t* seg_node,
                     uint64_t* seg_geo, cudaStream_t s) {
  key_sort(f.V, SegKeys{f.parent_g, f.geo, nl0, seg_node, seg_geo}, nkeys, cnt, cursor, s);
}

// Level buckets in the input order: out = in2int (input -> internal id) and
// key_of (each node's bucket); the renumbering writes the inverse.
void launch_level_sort(Forest& f, const int32_t* batch, int hmax1, int64_t nkeys, int32_t* lvl_cnt,
                       int64_t* lvl_cursor, int32_t* in2int, int32_t* key_of, cudaStream_t s) {
  BucketIn b{f.height, f.nch, f.parent_g, f.net_of, f.net_ptr, f.pin, batch, hmax1};
  key_sort(f.V, LevelKeys{b, in2int, key_of}, nkeys, lvl_cnt, lvl_cursor, s);
}

// An assignment given by the caller: layers of the right direction (the pin
// layer at roots), stacks holding the junction layer, the pin and every son.
__global__ void k_check_assignment(int64_t V, LayerInfo li, const int32_t* __restrict__ parent_g,
                                   const int8_t* __restrict__ pin, const uint64_t* __restrict__ geo,
                                   const int8_t* __restrict__ layer, const int8_t* __restrict__ b,
                                   const int8_t* __restrict__ t, unsigned long long* err) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int l = layer[v], bb = b[v], tt = t[v];
  const int p = parent_g[v];
  bool ok = l >= 0 && l < li.L && bb >= 0 && bb <= l && l <= tt && tt < li.L;
  if (ok) {
    if (p < 0) ok = (l == pin[v]);
    else ok = (li.dir[l] == geo_dir(geo[v])) && b[p] <= l && l <= t[p];
  }
  if (ok && pin[v] >= 0) ok = bb <= pin[v] && pin[v] <= tt;
  if (!ok) dev_error(err, DE_ASSIGN, v);
}

void launch_check_assignment(la_ctx* c, const int8_t* layer, const int8_t* b, const int8_t* t, cudaStream_t s) {
  Forest& f = c->forest;
  const int T = 256;
  k_check_assignment<<<(unsigned)((f.V + T - 1) / T), T, 0, s>>>(f.V, c->grid.li, f.parent_g, f.pin, f.geo,
                                                                layer, b, t, c->d_err);
  ++c->launches;
}

// Internal order: input node v goes to position i = in2int[v] of the
// (level, class, size class) order, and lvl_nodes[i] = v.  Reads run in input
// order.  Staged form: a block takes the tile of input nodes one block of the
// level sort placed (kHistT x kHistItems nodes), so each key's nodes of the
// tile hold one run of positions; sorting the tile by position in shared
// memory then only needs each key's count and first position, and every
// field is written run by run, coalesced.  Plain form (more than kRnMaxKeys
// keys, or the level sort's global-counter path): each thread writes its
// node's fields where they go.
struct RenumArgs {
  int64_t V;
  const int32_t *in2int, *key_of;
  const int32_t *parent_in, *net_of_in, *child_start_in, *nch_in, *child_list_in;
  const int8_t* pin_in;
  const double *cap_in, *kap_in, *W_in, *rho_in;
  const uint64_t* geo_in;
  int32_t *lvl_nodes, *parent, *net_of, *child_start, *nch, *child_list, *root_of_net;
  int8_t* pin;
  double *cap, *kap, *gk, *W, *rho;
  uint64_t* geo;
};

__global__ void k_renumber(RenumArgs a) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= a.V) return;
  const int i = a.in2int[v];
  const int p = a.parent_in[v];
  a.lvl_nodes[i] = int32_t(v);
  a.parent[i] = p < 0 ? -1 : a.in2int[p];
  if (p < 0) a.root_of_net[a.net_of_in[v]] = i;
  a.net_of[i] = a.net_of_in[v];
  const int8_t pn = a.pin_in[v];
  const double kv = a.kap_in[v];
  a.pin[i] = pn;
  a.cap[i] = a.cap_in[v];
  a.kap[i] = kv;
  a.gk[i] = pn >= 0 ? kv : 0.0;
  a.W[i] = a.W_in[v];
  a.rho[i] = a.rho_in[v];
  a.geo[i] = a.geo_in[v];
  a.child_start[i] = a.child_start_in[v];
  a.nch[i] = a.nch_in[v];
  // son slots keep their place (slot space = input node space); their
  // contents become internal ids, -1 stays -1
  const int c = a.child_list_in[v];
  a.child_list[v] = c < 0 ? -1 : a.in2int[c];
}

constexpr int kRnTile = kHistT * kHistItems;
constexpr int kRnMaxKeys = 6144;  // shared memory: 8 B per key + 12 B per tile node

// One field: load the tile's values (all loads first), stage them at their
// sorted slots, then write the slots in order (consecutive threads,
// consecutive positions inside a run).
template <typename T, typename F>
__device__ __forceinline__ void renumber_field(T* __restrict__ out, F value, const int (&slot)[kHistItems],
                                               const int* s_pos, void* s_stage, int ntile) {
  T* st = reinterpret_cast<T*>(s_stage);
  T val[kHistItems];
#pragma unroll
  for (int it = 0; it < kHistItems; ++it) val[it] = slot[it] >= 0 ? value(it) : T(0);
#pragma unroll
  for (int it = 0; it < kHistItems; ++it)
    if (slot[it] >= 0) st[slot[it]] = val[it];
  __syncthreads();
  for (int t = threadIdx.x; t < ntile; t += kHistT)
    if (s_pos[t] >= 0) out[s_pos[t]] = st[t];
  __syncthreads();
}

__global__ void __launch_bounds__(kHistT, 2) k_renumber_staged(RenumArgs a, int nkeys) {
  extern __shared__ double s_dyn[];
  double* s_stage = s_dyn;                                      // [kRnTile] values
  int* s_pos = reinterpret_cast<int*>(s_stage + kRnTile);       // [kRnTile] positions in slot order
  int* s_cnt = s_pos + kRnTile;                                 // [nkeys] counts, then first slots
  int* s_first = s_cnt + nkeys;                                 // [nkeys] first position of each run
  __shared__ int s_wsum[kHistT / 32];
  const int tid = threadIdx.x;
  for (int k = tid; k < nkeys; k += kHistT) {
    s_cnt[k] = 0;
    s_first[k] = 0x7fffffff;
  }
  for (int t = tid; t < kRnTile; t += kHistT) s_pos[t] = -1;
  const int64_t t0 = int64_t(blockIdx.x) * kRnTile;
  const int ntile = int(a.V - t0 < kRnTile ? a.V - t0 : kRnTile);
  int key[kHistItems], pos[kHistItems];
#pragma unroll
  for (int it = 0; it < kHistItems; ++it) {
    const int j = it * kHistT + tid;
    key[it] = j < ntile ? __ldg(a.key_of + t0 + j) : -1;
    pos[it] = j < ntile ? __ldg(a.in2int + t0 + j) : 0;
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kHistItems; ++it)
    if (key[it] >= 0) {
      atomicAdd(&s_cnt[key[it]], 1);
      atomicMin(&s_first[key[it]], pos[it]);
    }
  __syncthreads();
  // first slot of each key: exclusive prefix of the counts in key order
  const int per = (nkeys + kHistT - 1) / kHistT;
  const int k0 = min(nkeys, tid * per), k1 = min(nkeys, k0 + per);
  int sum = 0;
  for (int k = k0; k < k1; ++k) sum += s_cnt[k];
  const int lane = tid & 31;
  int inc = sum;
  for (int d = 1; d < 32; d <<= 1) {
    const int t = __shfl_up_sync(~0u, inc, d);
    if (lane >= d) inc += t;
  }
  if (lane == 31) s_wsum[tid >> 5] = inc;
  __syncthreads();
  int run = inc - sum;
  for (int w = 0; w < (tid >> 5); ++w) run += s_wsum[w];
  for (int k = k0; k < k1; ++k) {
    const int c = s_cnt[k];
    s_cnt[k] = run;
    run += c;
  }
  __syncthreads();
  int slot[kHistItems];
#pragma unroll
  for (int it = 0; it < kHistItems; ++it) {
    slot[it] = key[it] >= 0 ? s_cnt[key[it]] + pos[it] - s_first[key[it]] : -1;
    if (slot[it] >= ntile) slot[it] = -1;  // not reached: a key's positions in a tile form one run
    if (slot[it] >= 0) s_pos[slot[it]] = pos[it];
  }
  __syncthreads();
  auto vin = [&](int it) { return t0 + it * kHistT + tid; };
  // parents: input ids first (all loads), then their internal ids
  int par[kHistItems];
#pragma unroll
  for (int it = 0; it < kHistItems; ++it) par[it] = slot[it] >= 0 ? __ldg(a.parent_in + vin(it)) : -1;
  unsigned roots = 0;
#pragma unroll
  for (int it = 0; it < kHistItems; ++it)
    if (slot[it] >= 0 && par[it] < 0) roots |= 1u << it;
  renumber_field<int32_t>(a.parent, [&](int it) { return par[it] < 0 ? -1 : __ldg(a.in2int + par[it]); }, slot, s_pos,
                          s_stage, ntile);
  renumber_field<int32_t>(a.lvl_nodes, [&](int it) { return int32_t(vin(it)); }, slot, s_pos, s_stage, ntile);
  renumber_field<int32_t>(a.net_of, [&](int it) { return __ldg(a.net_of_in + vin(it)); }, slot, s_pos, s_stage, ntile);
  renumber_field<int8_t>(a.pin, [&](int it) { return __ldg(a.pin_in + vin(it)); }, slot, s_pos, s_stage, ntile);
  renumber_field<double>(a.cap, [&](int it) { return __ldg(a.cap_in + vin(it)); }, slot, s_pos, s_stage, ntile);
  renumber_field<double>(a.kap, [&](int it) { return __ldg(a.kap_in + vin(it)); }, slot, s_pos, s_stage, ntile);
  renumber_field<double>(a.gk, [&](int it) {
    const int64_t v = vin(it);
    return __ldg(a.pin_in + v) >= 0 ? __ldg(a.kap_in + v) : 0.0;
  }, slot, s_pos, s_stage, ntile);
  renumber_field<double>(a.W, [&](int it) { return __ldg(a.W_in + vin(it)); }, slot, s_pos, s_stage, ntile);
  renumber_field<double>(a.rho, [&](int it) { return __ldg(a.rho_in + vin(it)); }, slot, s_pos, s_stage, ntile);
  renumber_field<uint64_t>(a.geo, [&](int it) { return __ldg(a.geo_in + vin(it)); }, slot, s_pos, s_stage, ntile);
  renumber_field<int32_t>(a.child_start, [&](int it) { return __ldg(a.child_start_in + vin(it)); }, slot, s_pos,
                          s_stage, ntile);
  renumber_field<int32_t>(a.nch, [&](int it) { return __ldg(a.nch_in + vin(it)); }, slot, s_pos, s_stage, ntile);
  // son slots keep their place (slot space = input node space): the tile's
  // slots, contents to internal ids (-1 stays -1); roots name their net's root
  int ch[kHistItems];
#pragma unroll
  for (int it = 0; it < kHistItems; ++it) ch[it] = slot[it] >= 0 ? __ldg(a.child_list_in + vin(it)) : -1;
#pragma unroll
  for (int it = 0; it < kHistItems; ++it) ch[it] = ch[it] < 0 ? -1 : __ldg(a.in2int + ch[it]);
#pragma unroll
  for (int it = 0; it < kHistItems; ++it)
    if (slot[it] >= 0) a.child_list[vin(it)] = ch[it];
#pragma unroll
  for (int it = 0; it < kHistItems; ++it)
    if ((roots >> it) & 1u) a.root_of_net[__ldg(a.net_of_in + vin(it))] = pos[it];
}

void launch_renumber(const Forest& in, const int32_t* in2int, const int32_t* key_of, int64_t nkeys, Forest& out,
                     cudaStream_t s) {
  RenumArgs a;
  a.V = in.V; a.in2int = in2int; a.key_of = key_of;
  a.parent_in = in.parent_g; a.net_of_in = in.net_of; a.child_start_in = in.child_start; a.nch_in = in.nch;
  a.child_list_in = in.child_list; a.pin_in = in.pin; a.cap_in = in.sink_cap; a.kap_in = in.kappa;
  a.W_in = in.W_eq4; a.rho_in = in.rho_eq4; a.geo_in = in.geo;
  a.lvl_nodes = out.lvl_nodes; a.parent = out.parent_g; a.net_of = out.net_of; a.child_start = out.child_start;
  a.nch = out.nch; a.child_list = out.child_list; a.root_of_net = out.root_of_net; a.pin = out.pin;
  a.cap = out.sink_cap; a.kap = out.kappa; a.gk = out.gk; a.W = out.W_eq4; a.rho = out.rho_eq4; a.geo = out.geo;
  if (nkeys <= kRnMaxKeys) {
    // the staged form requires the level sort's tiles, i.e. its shared-counter path
    static_assert(kRnMaxKeys <= kHistMaxKeys, "staged renumbering follows the tiles of the shared-counter sort");
    const size_t sm = size_t(kRnTile) * (sizeof(double) + sizeof(int)) + size_t(nkeys) * 2 * sizeof(int);
    cudaFuncSetAttribute(k_renumber_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    const unsigned B = (unsigned)((in.V + kRnTile - 1) / kRnTile);
    k_renumber_staged<<<B, kHistT, sm, s>>>(a, int(nkeys));
  } else {
    k_renumber<<<(unsigned)((in.V + 255) / 256), 256, 0, s>>>(a);
  }
}

// The first son of every node (internal order), so that a one-son node reaches
// its son's table row in one dependent load instead of two.
__global__ void k_first_son(int64_t V, const int32_t* __restrict__ child_start, const int32_t* __restrict__ nch,
                            const int32_t* __restrict__ child_list, int32_t* __restrict__ son0) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= V) return;
  son0[v] = nch[v] > 0 ? child_list[child_start[v]] : -1;
}

void launch_first_son(const Forest& f, cudaStream_t s) {
  k_first_son<<<(unsigned)((f.V + 255) / 256), 256, 0, s>>>(f.V, f.child_start, f.nch, f.child_list, f.son0);
}

// One thread per net of size class >= kMinBigSc: a stable counting sort of
// its nodes by height (internal ids), and the net's height.
__global__ void k_net_levels(int64_t N, const int64_t* __restrict__ net_ptr, const int32_t* __restrict__ height,
                             const int32_t* __restrict__ in2int, int32_t* __restrict__ nodes,
                             int32_t* __restrict__ hoff, int32_t* __restrict__ net_H, int32_t* __restrict__ sc_cnt) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int64_t base = net_ptr[n], m = net_ptr[n + 1] - base;
  const int H = height[base];
  net_H[n] = H;
  const int sc = size_class(m);
  if (sc < kMinBigSc) return;
  atomicAdd(&sc_cnt[sc], 1);
  int32_t* ho = hoff + base + n;  // H + 2 <= m + 1 slots
  for (int h = 0; h <= H + 1; ++h) ho[h] = 0;
  for (int64_t i = 0; i < m; ++i) ho[height[base + i] + 1] += 1;
  for (int h = 0; h <= H; ++h) ho[h + 1] += ho[h];
  // place (ho[h] advances to the end of height h; shift back afterwards)
  for (int64_t i = 0; i < m; ++i) {
    const int h = height[base + i];
    nodes[base + ho[h]] = in2int[base + i];
    ho[h] += 1;
  }
  for (int h = H; h >= 1; --h) ho[h] = ho[h - 1];
  ho[0] = 0;
}

__global__ void k_big_queue(int64_t N, const int64_t* __restrict__ net_ptr, unsigned long long* __restrict__ cursor,
                            int32_t* __restrict__ queue) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int sc = size_class(net_ptr[n + 1] - net_ptr[n]);
  if (sc < kMinBigSc) return;
  queue[atomicAdd(&cursor[sc], 1ull)] = int32_t(n);
}

void launch_net_levels(const Forest& in, const int32_t* in2int, Forest& out, int32_t* sc_cnt, int64_t* sc_cur,
                       cudaStream_t s) {
  const unsigned B = (unsigned)((in.N + 127) / 128);
  if (sc_cnt) k_net_levels<<<B, 128, 0, s>>>(in.N, in.net_ptr, in.height, in2int, out.bl_nodes, out.bl_hoff,
                                             out.net_H, sc_cnt);
  if (sc_cur) k_big_queue<<<B, 128, 0, s>>>(in.N, in.net_ptr, reinterpret_cast<unsigned long long*>(sc_cur),
                                            out.big_queue);
}

template <typename T>
__global__ void k_permute(int64_t V, const int32_t* __restrict__ perm, const T* __restrict__ src, T* __restrict__ dst,
                          bool gather) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= V) return;
  if (gather) dst[i] = src[perm[i]];
  else dst[perm[i]] = src[i];
}
void launch_permute8(int64_t V, const int32_t* perm, const int8_t* src, int8_t* dst, bool gather, cudaStream_t s) {
  k_permute<int8_t><<<(unsigned)((V + 255) / 256), 256, 0, s>>>(V, perm, src, dst, gather);
}
void launch_permute64(int64_t V, const int32_t* perm, const double* src, double* dst, bool gather, cudaStream_t s) {
  k_permute<double><<<(unsigned)((V + 255) / 256), 256, 0, s>>>(V, perm, src, dst, gather);
}

}  // namespace gapla
