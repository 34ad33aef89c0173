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
  double *sink_cap, *kappa, *gk, *r_drv;
  uint64_t* geo;
  int* hmax;             // [0] max height, [1] max batch id
  const int32_t* batch;  // per net, or null
  unsigned long long* err;
};

__device__ inline bool finite_nonneg(double v) { return v >= 0.0 && v <= 1.7976931348623157e308; }

// One thread per net: validate, then build the net-local structure.  Nodes of
// a net are contiguous and parent < child, so single sweeps in id order (or
// reverse id order) visit parents before children (or children before parents).
__global__ void k_forest_prepare(PrepArgs a) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= a.N) return;
  const int64_t base = a.net_ptr_in[n], end = a.net_ptr_in[n + 1];
  if (!(base >= 0 && base < end && end <= a.V) || (n == 0 && base != 0) || (n == a.N - 1 && end != a.V)) {
    dev_error(a.err, DE_NETPTR, n);
    return;
  }
  const int64_t m = end - base;
  bool bad = false;
  for (int64_t i = 0; i < m; ++i) {
    const int64_t v = base + i;
    const int32_t par = a.parent[v];
    if (i == 0 ? par != -1 : (par < 0 || par >= i)) { dev_error(a.err, DE_PARENT, v); bad = true; break; }
    const int32_t xv = a.x[v], yv = a.y[v];
    if (xv < 0 || xv >= a.X || yv < 0 || yv >= a.Y) { dev_error(a.err, DE_COORD, v); bad = true; break; }
    const int pv = a.pin_in[v];
    if (pv < -1 || pv >= a.L || (i == 0 && pv < 0)) { dev_error(a.err, DE_PIN, v); bad = true; break; }
    if (!finite_nonneg(a.cap_in[v]) || !finite_nonneg(a.kap_in[v]) || (pv < 0 && a.cap_in[v] != 0.0)) {
      dev_error(a.err, DE_VALUE, v);
      bad = true;
      break;
    }
  }
  if (bad) return;
  if (!finite_nonneg(a.rdrv_in[n])) { dev_error(a.err, DE_VALUE, base); return; }
  if (a.batch) {
    const int bt = a.batch[n];
    if (bt < 0 || bt >= LA_MAX_BATCHES) { dev_error(a.err, DE_BATCH, n); return; }
    atomicMax(a.hmax + 1, bt);
  }
  a.net_ptr[n] = base;
  if (n == a.N - 1) a.net_ptr[a.N] = end;
  a.r_drv[n] = a.rdrv_in[n];
  for (int64_t i = 0; i < m; ++i) {
    const int64_t v = base + i;
    a.net_of[v] = int32_t(n);
    a.nch[v] = 0;
    a.height[v] = 0;
    a.pin[v] = a.pin_in[v];
    a.sink_cap[v] = a.cap_in[v];
    a.kappa[v] = a.kap_in[v];
    a.gk[v] = a.pin_in[v] >= 0 ? a.kap_in[v] : 0.0;
  }
  a.parent_g[base] = -1;
  a.geo[base] = 0;
  for (int64_t i = 1; i < m; ++i) {
    const int64_t v = base + i, p = base + a.parent[v];
    a.parent_g[v] = int32_t(p);
    a.nch[p] += 1;
    const int32_t dx = a.x[v] - a.x[p], dy = a.y[v] - a.y[p];
    if ((dx == 0) == (dy == 0)) { dev_error(a.err, DE_SEGMENT, v); return; }
    if (dy == 0) {  // horizontal: row y, edges [min x, max x)
      const int lo = min(a.x[v], a.x[p]);
      a.geo[v] = pack_geo(0, a.y[v], lo, dx < 0 ? -dx : dx);
    } else {        // vertical: column x, edges [min y, max y)
      const int lo = min(a.y[v], a.y[p]);
      a.geo[v] = pack_geo(1, a.x[v], lo, dy < 0 ? -dy : dy);
    }
  }
  // sons: CSR inside the net's own slot range [base, base + m - 1)
  int64_t acc = base;
  for (int64_t i = 0; i < m; ++i) {
    a.child_start[base + i] = int32_t(acc);
    acc += a.nch[base + i];
    a.nch[base + i] = 0;
  }
  for (int64_t i = 1; i < m; ++i) {
    const int64_t v = base + i, p = base + a.parent[v];
    a.child_list[a.child_start[p] + a.nch[p]] = int32_t(v);
    a.nch[p] += 1;
  }
  // height = 0 at leaves, 1 + max over sons otherwise
  for (int64_t i = m - 1; i >= 1; --i) {
    const int64_t v = base + i, p = base + a.parent[v];
    a.height[p] = max(a.height[p], a.height[v] + 1);
  }
  atomicMax(a.hmax, a.height[base]);
}

void launch_forest_prepare(la_ctx* c, Forest& f, const la_net_desc* d, int* d_hmax, cudaStream_t s) {
  PrepArgs a;
  a.N = f.N; a.V = f.V; a.X = c->grid.X; a.Y = c->grid.Y; a.L = c->grid.li.L;
  a.net_ptr_in = d->net_ptr; a.x = d->x; a.y = d->y; a.parent = d->parent; a.pin_in = d->pin_layer;
  a.cap_in = d->sink_cap; a.kap_in = d->kappa; a.rdrv_in = d->r_drv;
  a.net_ptr = f.net_ptr; a.parent_g = f.parent_g; a.net_of = f.net_of; a.child_start = f.child_start;
  a.nch = f.nch; a.child_list = f.child_list; a.height = f.height; a.pin = f.pin; a.sink_cap = f.sink_cap;
  a.kappa = f.kappa; a.gk = f.gk; a.r_drv = f.r_drv; a.geo = f.geo;
  a.hmax = d_hmax;
  a.batch = d->batch;
  a.err = c->d_err;
  const int T = 128;
  k_forest_prepare<<<(unsigned)((f.N + T - 1) / T), T, 0, s>>>(a);
  ++c->launches;
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

// Warp-aggregated counting: lanes with the same bucket add once.
__global__ void k_level_count(int64_t V, BucketIn b, int32_t* __restrict__ cnt) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool act = v < V;
  const long long key = act ? node_bucket(v, b) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  if (act && lane == __ffs(peers) - 1) atomicAdd(&cnt[key], __popc(peers));
}
__global__ void k_level_place(int64_t V, BucketIn b, unsigned long long* __restrict__ cursor,
                              int32_t* __restrict__ out) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool act = v < V;
  const long long key = act ? node_bucket(v, b) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if (act && lane == leader) base = atomicAdd(&cursor[key], (unsigned long long)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  if (act) out[base + __popc(peers & ((1u << lane) - 1u))] = int32_t(v);
}

// Segments by (direction, line): key = line for horizontal segments, nlines0 +
// line for vertical ones; roots have no segment.  The demand pass walks them
// in this order, so a warp's atomics land in one or two lines.
__device__ __forceinline__ int seg_key(uint64_t g, int nl0) { return geo_dir(g) == 0 ? geo_line(g) : nl0 + geo_line(g); }
__global__ void k_seg_count(int64_t V, const int32_t* __restrict__ parent_g, const uint64_t* __restrict__ geo,
                            int nl0, int32_t* __restrict__ cnt) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool act = v < V && parent_g[v] >= 0;
  const int key = act ? seg_key(geo[v], nl0) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  if (act && lane == __ffs(peers) - 1) atomicAdd(&cnt[key], __popc(peers));
}
__global__ void k_seg_place(int64_t V, const int32_t* __restrict__ parent_g, const uint64_t* __restrict__ geo,
                            int nl0, unsigned long long* __restrict__ cursor, int32_t* __restrict__ seg_node,
                            uint64_t* __restrict__ seg_geo) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool act = v < V && parent_g[v] >= 0;
  const uint64_t g = act ? geo[v] : 0;
  const int key = act ? seg_key(g, nl0) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if (act && lane == leader) base = atomicAdd(&cursor[key], (unsigned long long)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  if (act) {
    const unsigned long long pos = base + __popc(peers & ((1u << lane) - 1u));
    seg_node[pos] = int32_t(v);
    seg_geo[pos] = g;
  }
}

void launch_seg_sort(const Forest& f, int nl0, int32_t* cnt, int64_t* cursor, int32_t* seg_node, uint64_t* seg_geo,
                     cudaStream_t s) {
  const int T = 256;
  const unsigned B = (unsigned)((f.V + T - 1) / T);
  if (cnt) k_seg_count<<<B, T, 0, s>>>(f.V, f.parent_g, f.geo, nl0, cnt);
  if (cursor)
    k_seg_place<<<B, T, 0, s>>>(f.V, f.parent_g, f.geo, nl0, reinterpret_cast<unsigned long long*>(cursor), seg_node,
                                seg_geo);
}

// lvl_cnt: one zeroed int per bucket key; lvl_cursor: as many int64 holding
// the bucket offsets on entry.  Within a bucket the order is whatever the
// atomics give: nodes of one level never read each other's results.
void launch_level_sort(Forest& f, const int32_t* batch, int hmax1, int32_t* lvl_cnt, int64_t* lvl_cursor,
                       cudaStream_t s) {
  const int T = 256;
  const unsigned B = (unsigned)((f.V + T - 1) / T);
  BucketIn b{f.height, f.nch, f.parent_g, f.net_of, f.net_ptr, f.pin, batch, hmax1};
  if (lvl_cnt) k_level_count<<<B, T, 0, s>>>(f.V, b, lvl_cnt);
  if (lvl_cursor) k_level_place<<<B, T, 0, s>>>(f.V, b, reinterpret_cast<unsigned long long*>(lvl_cursor), f.lvl_nodes);
}

// Eq. 4 edge weights (max sink criticality below) and the distance-based
// look-ahead r_est = W_root R_drv + sum of W_x len_x rbar(dir x) down to v.
__global__ void k_weights_eq4(int64_t N, LayerInfo li, const int64_t* __restrict__ net_ptr,
                              const int32_t* __restrict__ parent_g, const int8_t* __restrict__ pin,
                              const double* __restrict__ kappa, const double* __restrict__ r_drv,
                              const uint64_t* __restrict__ geo, double* __restrict__ W,
                              double* __restrict__ rho) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int64_t base = net_ptr[n], m = net_ptr[n + 1] - base;
  for (int64_t i = 0; i < m; ++i) W[base + i] = pin[base + i] >= 0 ? kappa[base + i] : 0.0;
  for (int64_t i = m - 1; i >= 1; --i) {
    const int64_t v = base + i, p = parent_g[v];
    if (W[v] > W[p]) W[p] = W[v];
  }
  rho[base] = W[base] * r_drv[n];
  for (int64_t i = 1; i < m; ++i) {
    const int64_t v = base + i, p = parent_g[v];
    const uint64_t g = geo[v];
    rho[v] = rho[p] + (W[v] * double(geo_len(g))) * li.rbar[geo_dir(g)];
  }
}

void launch_weights_eq4(const LayerInfo& li, Forest& f, cudaStream_t s) {
  const int T = 128;
  k_weights_eq4<<<(unsigned)((f.N + T - 1) / T), T, 0, s>>>(f.N, li, f.net_ptr, f.parent_g, f.pin,
                                                          f.kappa, f.r_drv, f.geo, f.W_eq4, f.rho_eq4);
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

// Internal order: thread i is the node at position i of the (level, class)
// sort; in = its input id.
__global__ void k_inverse_perm(int64_t V, const int32_t* __restrict__ int2in, int32_t* __restrict__ in2int) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < V) in2int[int2in[i]] = int32_t(i);
}

struct RenumArgs {
  int64_t V;
  const int32_t *int2in, *in2int;
  const int32_t *parent_in, *net_of_in, *child_start_in, *nch_in, *child_list_in;
  const int8_t* pin_in;
  const double *cap_in, *kap_in, *gk_in, *W_in, *rho_in;
  const uint64_t* geo_in;
  int32_t *parent, *net_of, *child_start, *nch, *child_list, *root_of_net;
  int8_t* pin;
  double *cap, *kap, *gk, *W, *rho;
  uint64_t* geo;
};

__global__ void k_renumber(RenumArgs a) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.V) return;
  const int in = a.int2in[i];
  const int p = a.parent_in[in];
  a.parent[i] = p < 0 ? -1 : a.in2int[p];
  if (p < 0) a.root_of_net[a.net_of_in[in]] = int32_t(i);
  a.net_of[i] = a.net_of_in[in];
  a.pin[i] = a.pin_in[in];
  a.cap[i] = a.cap_in[in];
  a.kap[i] = a.kap_in[in];
  a.gk[i] = a.gk_in[in];
  a.W[i] = a.W_in[in];
  a.rho[i] = a.rho_in[in];
  a.geo[i] = a.geo_in[in];
  // the son slots of a node keep their place; their contents become internal ids
  const int cs = a.child_start_in[in], nc = a.nch_in[in];
  a.child_start[i] = cs;
  a.nch[i] = nc;
  for (int k = 0; k < nc; ++k) a.child_list[cs + k] = a.in2int[a.child_list_in[cs + k]];
}

void launch_inverse_perm(int64_t V, const int32_t* int2in, int32_t* in2int, cudaStream_t s) {
  k_inverse_perm<<<(unsigned)((V + 255) / 256), 256, 0, s>>>(V, int2in, in2int);
}

void launch_renumber(const Forest& in, const int32_t* in2int, Forest& out, cudaStream_t s) {
  const int T = 256;
  const unsigned B = (unsigned)((in.V + T - 1) / T);
  RenumArgs a;
  a.V = in.V; a.int2in = out.lvl_nodes; a.in2int = in2int;
  a.parent_in = in.parent_g; a.net_of_in = in.net_of; a.child_start_in = in.child_start; a.nch_in = in.nch;
  a.child_list_in = in.child_list; a.pin_in = in.pin; a.cap_in = in.sink_cap; a.kap_in = in.kappa; a.gk_in = in.gk;
  a.W_in = in.W_eq4; a.rho_in = in.rho_eq4; a.geo_in = in.geo;
  a.parent = out.parent_g; a.net_of = out.net_of; a.child_start = out.child_start; a.nch = out.nch;
  a.child_list = out.child_list; a.root_of_net = out.root_of_net; a.pin = out.pin; a.cap = out.sink_cap;
  a.kap = out.kappa; a.gk = out.gk; a.W = out.W_eq4; a.rho = out.rho_eq4; a.geo = out.geo;
  k_renumber<<<B, T, 0, s>>>(a);
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
