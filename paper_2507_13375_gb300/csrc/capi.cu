// capi.cu - the C ABI of include/gapla.h: contexts, loading, the round driver
// (Alg. 2: levels 0..max for the DP, max..0 for the backtrack) and the Elmore
// calls.  Host code only; kernels live in k_*.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "gapla_internal.cuh"

using namespace gapla;

namespace {

thread_local std::string g_create_err;

la_status set_err(la_ctx* c, la_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  c->err = buf;
  if (code == LA_ERR_CUDA || code == LA_ERR_TIMEOUT || code == LA_ERR_DEVICE_CHECK) c->poisoned = true;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return set_err(c, LA_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define TRY(expr)                  \
  do {                             \
    la_status s_ = (expr);         \
    if (s_ != LA_OK) return s_;    \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// FNV-1a over the 8 bytes of x.
uint64_t fnv_mix(uint64_t h, uint64_t x) {
  for (int i = 0; i < 8; ++i) {
    h ^= (x >> (8 * i)) & 0xffu;
    h *= 1099511628211ull;
  }
  return h;
}

// Freed device blocks kept for reuse, by exact size.  A reload of a forest of
// the same shape takes every block back (first in, first out among equal
// sizes, so the arrays land at the same addresses), and nothing is allocated
// or freed; a block that stays unused through a whole load is freed.
struct DevPool {
  struct Blk {
    void* p;
    uint64_t gen;
  };
  std::multimap<size_t, Blk> blocks;
  uint64_t gen = 0;
  void* take(size_t b) {
    auto it = blocks.lower_bound(b);
    if (it == blocks.end() || it->first != b) return nullptr;
    void* p = it->second.p;
    blocks.erase(it);
    return p;
  }
  // the block at p of b bytes, if the pool holds it
  void* take_exact(void* p, size_t b) {
    auto r = blocks.equal_range(b);
    for (auto it = r.first; it != r.second; ++it)
      if (it->second.p == p) {
        blocks.erase(it);
        return p;
      }
    return nullptr;
  }
  void put(void* p, size_t b) { blocks.emplace(b, Blk{p, gen}); }
  void free_older_than(uint64_t g) {
    for (auto it = blocks.begin(); it != blocks.end();) {
      if (it->second.gen < g) {
        cudaFree(it->second.p);
        it = blocks.erase(it);
      } else {
        ++it;
      }
    }
  }
  void clear() { free_older_than(UINT64_MAX); }
};

// Device allocations of one load (grid or forest), released together (into
// the pool when there is one).  With a hint (the previous load's list, in
// call order), the i-th allocation takes the block the i-th took last time
// when the pool holds it: a same-shaped reload puts every array at its old
// address.
struct Allocs {
  std::vector<std::pair<void*, size_t>> list;
  size_t bytes = 0;
  DevPool* pool = nullptr;
  DevPool* spare = nullptr;  // another pool, emptied too before an allocation fails
  const std::vector<std::pair<void*, size_t>>* hint = nullptr;
  size_t next = 0;
  template <typename T>
  la_status get(la_ctx* c, T** p, size_t n) {
    size_t b = n * sizeof(T);
    if (b == 0) b = 16;
    b = (b + 255) & ~size_t(255);
    if (c->inject == LA_ERR_OOM) {  // a test's injected allocation failure
      c->inject = LA_OK;
      *p = nullptr;
      return set_err(c, LA_ERR_OOM, "device allocation of %zu bytes failed: injected fault", b);
    }
    void* q = nullptr;
    if (pool && hint && next < hint->size() && (*hint)[next].second == b) q = pool->take_exact((*hint)[next].first, b);
    ++next;
    if (!q && pool) q = pool->take(b);
    if (!q) {
      cudaError_t e = cudaMalloc(&q, b);
      if (e == cudaErrorMemoryAllocation && pool && (!pool->blocks.empty() || (spare && !spare->blocks.empty()))) {
        cudaGetLastError();
        pool->clear();  // give the pooled blocks back and try once more
        if (spare) spare->clear();
        e = cudaMalloc(&q, b);
      }
      if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(c, LA_ERR_OOM, "device allocation of %zu bytes failed: %s", b, cudaGetErrorString(e));
      }
    }
    list.emplace_back(q, b);
    bytes += b;
    *p = static_cast<T*>(q);
    return LA_OK;
  }
  void release() {
    for (auto& x : list) {
      if (pool) pool->put(x.first, x.second);
      else cudaFree(x.first);
    }
    list.clear();
    bytes = 0;
  }
};

}  // namespace

void gapla::set_noctx_error(const std::string& msg) { g_create_err = msg; }

// Allocation groups live beside the context (kept out of the shared header).
// The forest's arrays and the loads' temporaries keep separate pools, so a
// temporary never takes the block an array of the next forest wants.
struct la_ctx_allocs {
  DevPool pool;   // temporaries (and the grid)
  DevPool fpool;  // forest arrays
  Allocs grid, forest;
  la_ctx_allocs() {
    grid.pool = &pool;
    forest.pool = &fpool;
    grid.spare = &fpool;
    forest.spare = &pool;
  }
};
static la_ctx_allocs* allocs_of(la_ctx* c) { return reinterpret_cast<la_ctx_allocs*>(c->alloc_groups); }

static la_status check_ctx(la_ctx* c) {
  if (!c) return LA_ERR_INVALID;
  if (c->poisoned) return set_err(c, LA_ERR_STATE, "context is poisoned by an earlier CUDA/device error: %s", c->err.c_str());
  return LA_OK;
}

static bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

static const char* dev_err_name(int code) {
  switch (code) {
    case DE_NETPTR: return "net_ptr not increasing or out of range";
    case DE_PARENT: return "parent id out of order (need -1 at a net's first node, 0 <= parent < local id elsewhere)";
    case DE_COORD: return "node coordinate outside the grid";
    case DE_SEGMENT: return "tree edge is not a straight horizontal/vertical run of length >= 1";
    case DE_PIN: return "pin layer out of range, or a root without a driver pin";
    case DE_VALUE: return "negative or non-finite value, or a sink cap at a node without a pin";
    case DE_ASSIGN: return "assignment layer of the wrong direction, or a via stack not covering it";
    case DE_DEGREE: return "too many sons";
    case DE_NOSTACK: return "no valid via stack";
    case DE_BATCH: return "batch id out of range";
    default: return "unknown device check";
  }
}

// Sync and read the device error word; returns (code, index) or (0, 0).
static la_status read_dev_err(la_ctx* c, int* code, long long* index) {
  CK(cudaStreamSynchronize(c->stream));
  unsigned long long e = kNoErr;
  CK(cudaMemcpy(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost));
  if (c->inject == LA_ERR_DEVICE_CHECK) {  // a test's injected failures, reported like real ones
    c->inject = LA_OK;
    e = uint64_t(DE_NOSTACK);
  } else if (c->inject == LA_ERR_CUDA || c->inject == LA_ERR_TIMEOUT) {
    const la_status k = c->inject;
    c->inject = LA_OK;
    return set_err(c, k, k == LA_ERR_CUDA ? "cudaStreamSynchronize: injected fault"
                                          : "a bounded device wait ran out: injected fault");
  }
  if (e == kNoErr) {
    *code = 0;
    *index = 0;
  } else {
    *code = int(e & 0xFF);
    *index = (long long)(e >> 8);
  }
  return LA_OK;
}

static la_status reset_dev_err(la_ctx* c) {
  const unsigned long long e = kNoErr;
  CK(cudaMemcpyAsync(c->d_err, &e, sizeof e, cudaMemcpyHostToDevice, c->stream));
  return LA_OK;
}

// ------------------------------------------------------------------------
extern "C" {

la_status la_create(la_ctx** out, int device, void* stream) {
  if (!out) return LA_ERR_INVALID;
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    g_create_err = std::string("no CUDA device ") + std::to_string(device) + ": " + cudaGetErrorString(e);
    return e != cudaSuccess ? LA_ERR_CUDA : LA_ERR_INVALID;
  }
  la_ctx* c = new la_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  c->alloc_groups = new la_ctx_allocs();
  DeviceGuard g(device);
  bool ok = cudaMalloc(&c->d_err, sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&c->d_stats, sizeof(Stats)) == cudaSuccess;
  for (auto& e2 : c->ev) ok = ok && cudaEventCreate(&e2) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&c->s2, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&c->s_cap, cudaStreamNonBlocking) == cudaSuccess &&
       cudaStreamCreateWithFlags(&c->s3, cudaStreamNonBlocking) == cudaSuccess &&
       cudaEventCreateWithFlags(&c->ev_lfork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&c->ev_ljoin, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
       cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    g_create_err = std::string("context set-up failed: ") + cudaGetErrorString(cudaGetLastError());
    la_destroy(c);
    return LA_ERR_CUDA;
  }
  *out = c;
  return LA_OK;
}

la_status la_destroy(la_ctx* c) {
  if (!c) return LA_OK;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  if (la_ctx_allocs* a = allocs_of(c)) {
    a->forest.release();
    a->grid.release();
    a->pool.clear();
    a->fpool.clear();
    delete a;
  }
  if (c->d_err) cudaFree(c->d_err);
  if (c->d_stats) cudaFree(c->d_stats);
  for (auto& e2 : c->ev)
    if (e2) cudaEventDestroy(e2);
  for (auto& e2 : c->plan.exec)
    if (e2) cudaGraphExecDestroy(e2);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->s2) cudaStreamDestroy(c->s2);
  if (c->s_cap) cudaStreamDestroy(c->s_cap);
  if (c->s3) cudaStreamDestroy(c->s3);
  if (c->ev_lfork) cudaEventDestroy(c->ev_lfork);
  if (c->ev_ljoin) cudaEventDestroy(c->ev_ljoin);
  delete c;
  return LA_OK;
}

const char* la_last_error(const la_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

la_status la_set_stream(la_ctx* c, void* stream) {
  if (!c) return LA_ERR_INVALID;
  c->stream = static_cast<cudaStream_t>(stream);
  return LA_OK;
}

la_status la_device_bytes(const la_ctx* c, size_t* bytes) {
  if (!c || !bytes) return LA_ERR_INVALID;
  la_ctx_allocs* a = allocs_of(const_cast<la_ctx*>(c));
  size_t pooled = 0;
  for (const auto& kv : a->pool.blocks) pooled += kv.first;
  for (const auto& kv : a->fpool.blocks) pooled += kv.first;
  *bytes = a->grid.bytes + a->forest.bytes + pooled + sizeof(Stats) + sizeof(unsigned long long);
  return LA_OK;
}

la_status la_launch_count(const la_ctx* c, int64_t* n) {
  if (!c || !n) return LA_ERR_INVALID;
  *n = c->launches;
  return LA_OK;
}

la_status la_inject_fault(la_ctx* c, la_status code) {
  if (!c) return LA_ERR_INVALID;
  if (code != LA_OK && code != LA_ERR_OOM && code != LA_ERR_CUDA && code != LA_ERR_TIMEOUT &&
      code != LA_ERR_DEVICE_CHECK)
    return set_err(c, LA_ERR_INVALID, "la_inject_fault: code %d cannot be injected", int(code));
  c->inject = code;
  return LA_OK;
}

la_status la_check(la_ctx* c) {
  TRY(check_ctx(c));
  DeviceGuard g(c->device);
  int code;
  long long idx;
  TRY(read_dev_err(c, &code, &idx));
  if (code) return set_err(c, LA_ERR_DEVICE_CHECK, "device check failed: %s (index %lld)", dev_err_name(code), idx);
  return LA_OK;
}

// ------------------------------------------------------------------------
la_status la_load_grid(la_ctx* c, const la_grid_desc* gd) {
  TRY(check_ctx(c));
  if (!gd || !gd->dir || !gd->cap || !gd->unit_r || !gd->unit_c || !gd->ofw || (gd->L > 1 && !gd->via_r))
    return set_err(c, LA_ERR_INVALID, "la_load_grid: null pointer in the descriptor");
  const int X = gd->X, Y = gd->Y, L = gd->L;
  if (X < 2 || Y < 2 || X > 16384 || Y > 16384 || L < 2 || L > kMaxL)
    return set_err(c, LA_ERR_INVALID, "la_load_grid: need 2 <= X, Y <= 16384 and 2 <= L <= %d", kMaxL);
  LayerInfo li{};
  li.L = L;
  for (int l = 0; l < L; ++l) {
    const int d = gd->dir[l];
    if (d != 0 && d != 1) return set_err(c, LA_ERR_INVALID, "la_load_grid: dir[%d] must be 0 or 1", l);
    if (!finite_nonneg(gd->unit_r[l]) || !finite_nonneg(gd->unit_c[l]) || !finite_nonneg(gd->ofw[l]))
      return set_err(c, LA_ERR_INVALID, "la_load_grid: unit_r/unit_c/ofw of layer %d must be finite and >= 0", l);
    if (l + 1 < L && !finite_nonneg(gd->via_r[l]))
      return set_err(c, LA_ERR_INVALID, "la_load_grid: via_r[%d] must be finite and >= 0", l);
    li.dir[l] = int8_t(d);
    li.ld_of[l] = li.nld[d];
    li.lay[d][li.nld[d]++] = l;
    li.mask[d] |= 1u << l;
    li.unit_r[l] = gd->unit_r[l];
    li.unit_c[l] = gd->unit_c[l];
    li.half_c[l] = 0.5 * gd->unit_c[l];
  }
  if (li.nld[0] == 0 || li.nld[1] == 0)
    return set_err(c, LA_ERR_INVALID, "la_load_grid: each direction needs at least one layer");
  if (!finite_nonneg(gd->via_c)) return set_err(c, LA_ERR_INVALID, "la_load_grid: via_c must be finite and >= 0");
  li.via_c = gd->via_c;
  for (int d = 0; d < 2; ++d) {
    double s = 0.0;
    int n = 0;
    for (int l = 0; l < L; ++l)
      if (li.dir[l] == d) { s += li.unit_r[l]; ++n; }
    li.rbar[d] = s / n;
  }
  li.nlines[0] = Y; li.npos[0] = X;
  li.nlines[1] = X; li.npos[1] = Y;
  li.grid_off[0] = 0;
  li.grid_off[1] = int64_t(Y) * X * li.nld[0];
  const int64_t G = li.grid_off[1] + int64_t(X) * Y * li.nld[1];
  li.pub_off[0] = 0;
  for (int l = 0; l < L; ++l)
    li.pub_off[l + 1] = li.pub_off[l] + (li.dir[l] == 0 ? int64_t(Y) * (X - 1) : int64_t(X) * (Y - 1));
  for (int l = L; l < kMaxL; ++l) li.pub_off[l + 1] = li.pub_off[L];

  Grid ng;
  ng.X = X; ng.Y = Y; ng.E = li.pub_off[L]; ng.G = G; ng.li = li;
  for (int l = 0; l + 1 < L; ++l) ng.via_r[l] = gd->via_r[l];
  for (int l = 0; l < L; ++l) ng.ofw[l] = gd->ofw[l];
  // Rvia(a, b): the via resistances between the two layers, summed upwards
  for (int a = 0; a < L; ++a)
    for (int b = 0; b < L; ++b) {
      const int lo = std::min(a, b), hi = std::max(a, b);
      double s = 0.0;
      for (int k = lo; k < hi; ++k) s += ng.via_r[k];
      ng.rvia[a * kMaxL + b] = s;
    }
  // congestion penalty table (reading of Eq. 3) and the Eq. 3 overflow table
  std::vector<double> tofT(size_t(L) * 2 * 257);
  for (int l = 0; l < L; ++l)
    for (int si = 0; si < 2; ++si) {
      const double s = si == 0 ? 0.5 : 1.5;
      for (int k = -64; k <= 64; ++k) {
        double v = ng.ofw[l] * std::exp(s * k) * 16777216.0;
        if (v > double(kPenMax)) v = double(kPenMax);
        ng.pen_T[(l * 2 + si) * 129 + (k + 64)] = llround(v);
      }
      for (int o = -128; o <= 128; ++o) tofT[(l * 2 + si) * 257 + (o + 128)] = ng.ofw[l] * std::exp(s * double(o));
    }
  DevTables& t = ng.tab;
  memset(&t, 0, sizeof t);
  for (int a = 0; a < kMaxL; ++a)
    for (int b = 0; b < kMaxL; ++b) t.rv[a * kRvStride + b] = ng.rvia[a * kMaxL + b];
  for (int k = 0; k < kMaxL; ++k) t.kd[k] = double(k);
  for (int l = 0; l < kMaxL; ++l) {
    t.unit_r[l] = li.unit_r[l];
    t.unit_c[l] = li.unit_c[l];
    t.half_c[l] = li.half_c[l];
    t.ld_of[l] = int8_t(l < L ? li.ld_of[l] : 0);
    t.dir[l] = int8_t(l < L ? li.dir[l] : 0);
    t.lay[0][l] = int8_t(li.lay[0][l]);
    t.lay[1][l] = int8_t(li.lay[1][l]);
  }
  t.via_c = li.via_c;
  for (int d = 0; d < 2; ++d) {
    t.grid_off[d] = li.grid_off[d];
    t.npos[d] = li.npos[d];
    t.nlines[d] = li.nlines[d];
    t.nld[d] = li.nld[d];
    t.mask[d] = li.mask[d];
  }
  t.L = L;

  DeviceGuard g(c->device);
  Allocs na;
  la_status st = LA_OK;
  if ((st = na.get(c, &ng.cap, G)) || (st = na.get(c, &ng.D, G)) || (st = na.get(c, &ng.H, G)) ||
      (st = na.get(c, &ng.diff, G)) || (st = na.get(c, &ng.P, G)) || (st = na.get(c, &ng.T_dev, size_t(L) * 2 * 129)) ||
      (st = na.get(c, &ng.tofT_dev, tofT.size())) || (st = na.get(c, &ng.tab_dev, 1))) {
    na.release();
    return st;
  }
  auto fail = [&](la_status s) { na.release(); return s; };
  cudaStream_t s = c->stream;
  if (cudaMemsetAsync(ng.cap, 0, G * 4, s) || cudaMemsetAsync(ng.D, 0, G * 4, s) || cudaMemsetAsync(ng.H, 0, G * 4, s) ||
      cudaMemsetAsync(ng.diff, 0, G * 4, s) || cudaMemsetAsync(ng.P, 0, G * 8, s) ||
      cudaMemcpyAsync(ng.T_dev, ng.pen_T, sizeof(int64_t) * L * 2 * 129, cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(ng.tofT_dev, tofT.data(), sizeof(double) * tofT.size(), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(ng.tab_dev, &ng.tab, sizeof(DevTables), cudaMemcpyHostToDevice, s))
    return fail(set_err(c, LA_ERR_CUDA, "la_load_grid: %s", cudaGetErrorString(cudaGetLastError())));
  if (reset_dev_err(c)) return fail(LA_ERR_CUDA);
  launch_grid_to_internal(li, X, Y, gd->cap, ng.cap, true, c->d_err, s);
  ++c->launches;
  int code;
  long long idx;
  if (cudaGetLastError() != cudaSuccess || read_dev_err(c, &code, &idx) != LA_OK)
    return fail(set_err(c, LA_ERR_CUDA, "la_load_grid: kernel launch failed"));
  if (code) return fail(set_err(c, LA_ERR_INVALID, "la_load_grid: capacity %lld is negative", idx));
  // success: replace the grid, drop the forest and the batched plan
  for (auto& e2 : c->plan.exec)
    if (e2) cudaGraphExecDestroy(e2);
  c->plan = BatchPlan();
  la_ctx_allocs* a = allocs_of(c);
  a->forest.release();
  a->grid.release();
  c->forest = Forest();
  a->grid = na;
  ng.fused_scan = prepare_fused_scan(ng.li);
  c->grid = ng;
  c->grid.loaded = true;
  c->grid.P_valid = false;
  c->LD = std::max(li.nld[0], li.nld[1]);
  return LA_OK;
}

static void plan_from_memo(la_ctx* c);

// ------------------------------------------------------------------------
la_status la_load_nets(la_ctx* c, const la_net_desc* nd) {
  TRY(check_ctx(c));
  if (!c->grid.loaded) return set_err(c, LA_ERR_STATE, "la_load_nets: load the grid first");
  if (!nd || !nd->net_ptr || !nd->x || !nd->y || !nd->parent || !nd->pin_layer || !nd->sink_cap || !nd->kappa ||
      !nd->r_drv)
    return set_err(c, LA_ERR_INVALID, "la_load_nets: null pointer in the descriptor");
  if (nd->num_nets < 1 || nd->num_nodes < nd->num_nets || nd->num_nodes > int64_t(INT32_MAX) - 1)
    return set_err(c, LA_ERR_INVALID, "la_load_nets: need 1 <= num_nets <= num_nodes < 2^31");
  DeviceGuard g(c->device);
  cudaStream_t s = c->stream;
  const int LD = c->LD;
  // tf: the forest in input order (validation, levels, Eq. 4 weights);
  // nf: the same in internal (level, class) order, kept by the context.
  Forest tf, nf;
  tf.N = nf.N = nd->num_nets;
  tf.V = nf.V = nd->num_nodes;
  const size_t N = size_t(nf.N), V = size_t(nf.V);
  la_ctx_allocs* al = allocs_of(c);
  const uint64_t gen0 = ++al->pool.gen;
  al->fpool.gen = gen0;
  Allocs na, ta;  // kept / temporary
  na.pool = &al->fpool;
  ta.pool = &al->pool;
  na.spare = &al->pool;
  ta.spare = &al->fpool;
  std::vector<std::pair<void*, size_t>> prev_list;  // the old forest's arrays, in allocation order
  BatchPlan old_plan;  // the old forest's plan, once the old forest is released
  la_status st = LA_OK;
  auto fail = [&](la_status s2) {
    na.release();
    ta.release();
    for (auto& e2 : old_plan.exec)
      if (e2) cudaGraphExecDestroy(e2);
    return s2;
  };
  auto cuda_fail = [&]() { return fail(set_err(c, LA_ERR_CUDA, "la_load_nets: %s", cudaGetErrorString(cudaGetLastError()))); };
#define GETK(p, n) if (st == LA_OK) st = na.get(c, &(p), (n))
#define GETT(p, n) if (st == LA_OK) st = ta.get(c, &(p), (n))
  // the input-order forest (temporaries); the kept arrays are allocated only
  // once the old forest is released, so that they can take its blocks
  GETT(tf.net_ptr, N + 1); GETT(tf.r_drv, N);
  GETT(tf.parent_g, V); GETT(tf.net_of, V); GETT(tf.pin, V); GETT(tf.sink_cap, V); GETT(tf.kappa, V);
  GETT(tf.geo, V); GETT(tf.child_start, V); GETT(tf.nch, V); GETT(tf.child_list, V);
  GETT(tf.height, V); GETT(tf.W_eq4, V); GETT(tf.rho_eq4, V);
  int* d_hmax = nullptr;  // [0] max height, [1] max batch id, [2] bad net range
  GETT(d_hmax, 3);
  if (st) return fail(st);
  if (reset_dev_err(c) || cudaMemsetAsync(d_hmax, 0, 3 * sizeof(int), s)) return cuda_fail();
  launch_forest_prepare(c, tf, nd, d_hmax, s);
  int code;
  long long idx;
  if (cudaGetLastError() != cudaSuccess) return fail(set_err(c, LA_ERR_CUDA, "la_load_nets: launch failed"));
  if ((st = read_dev_err(c, &code, &idx))) return fail(st);
  if (code) return fail(set_err(c, LA_ERR_INVALID, "la_load_nets: %s (%s %lld)", dev_err_name(code),
                                 code == DE_NETPTR ? "net" : "node", idx));
  // The input is valid: the old forest's blocks go back to the forest pool,
  // where the new forest's arrays find them, each the block the same
  // allocation took last time (same shape: same addresses).  Its batched plan
  // is kept aside until the new forest's plan is known.
  old_plan = c->plan;
  c->plan = BatchPlan();
  prev_list = al->forest.list;
  al->forest.release();
  c->forest = Forest();
  na.hint = &prev_list;
  GETK(nf.net_ptr, N + 1); GETK(nf.r_drv, N);
  if (st) return fail(st);
  if (cudaMemcpyAsync(nf.net_ptr, tf.net_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToDevice, s) ||
      cudaMemcpyAsync(nf.r_drv, tf.r_drv, sizeof(double) * N, cudaMemcpyDeviceToDevice, s))
    return cuda_fail();
  int hb[2] = {0, 0};
  if (cudaMemcpy(hb, d_hmax, sizeof hb, cudaMemcpyDeviceToHost)) return cuda_fail();
  const int hmax = hb[0];
  nf.Hmax = tf.Hmax = hmax;
  nf.nbatch = nd->batch ? hb[1] + 1 : 1;
  nf.nlev = nf.nbatch * (hmax + 1);
  // levels: (global level, class, size class) buckets, global level = batch (Hmax + 1) + height
  if (int64_t(nf.nlev) * kClasses * kSizeClasses > (int64_t(1) << 28))
    return fail(set_err(c, LA_ERR_INVALID, "la_load_nets: %d batches x %d levels is too many buckets", nf.nbatch,
                        hmax + 1));
  int32_t* d_cnt = nullptr;
  int64_t* d_cur = nullptr;
  int32_t* in2int = nullptr;  // input id -> internal id
  int32_t* key_of = nullptr;  // input id -> bucket
  const size_t nbk = size_t(bucket_key(nf.nlev, 0, 0));
  GETT(d_cnt, nbk); GETT(d_cur, nbk); GETT(in2int, V); GETT(key_of, V);
  GETK(nf.lvl_nodes, V);
  if (st) return fail(st);
  tf.lvl_nodes = nf.lvl_nodes;
  if (cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * nbk, s)) return cuda_fail();
  launch_level_sort(tf, nd->batch, hmax + 1, int64_t(nbk), d_cnt, nullptr, nullptr, nullptr, s);
  ++c->launches;
  std::vector<int32_t> cnt(nbk);
  if (cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * nbk, cudaMemcpyDeviceToHost, s) ||
      cudaStreamSynchronize(s))
    return cuda_fail();
  nf.key_off.assign(nbk + 1, 0);
  for (size_t k = 0; k < nbk; ++k) nf.key_off[k + 1] = nf.key_off[k] + cnt[k];
  nf.key_hash = 1469598103934665603ull;
  for (int64_t x : nf.key_off) nf.key_hash = fnv_mix(nf.key_hash, uint64_t(x));
  nf.lvl_off.assign(size_t(nf.nlev) + 1, 0);
  for (int g = 0; g <= nf.nlev; ++g) nf.lvl_off[g] = nf.key_off[size_t(bucket_key(g, 0, 0))];
  if (cudaMemcpyAsync(d_cur, nf.key_off.data(), sizeof(int64_t) * nbk, cudaMemcpyHostToDevice, s)) return cuda_fail();
  launch_level_sort(tf, nd->batch, hmax + 1, int64_t(nbk), nullptr, d_cur, in2int, key_of, s);
  ++c->launches;
  // per-net level lists and the big-net queue, then the internal order
  int32_t* d_sc = nullptr;
  int64_t* d_sccur = nullptr;
  GETT(d_sc, kSizeClasses); GETT(d_sccur, kSizeClasses);
  GETK(nf.bl_nodes, V); GETK(nf.bl_hoff, V + N); GETK(nf.net_H, N); GETK(nf.queue_ctr, 4);
  if (st) return fail(st);
  if (cudaMemsetAsync(d_sc, 0, sizeof(int32_t) * kSizeClasses, s)) return cuda_fail();
  launch_net_levels(tf, in2int, nf, d_sc, nullptr, s);
  ++c->launches;
  std::vector<int32_t> sc_cnt(kSizeClasses);
  if (cudaMemcpyAsync(sc_cnt.data(), d_sc, sizeof(int32_t) * kSizeClasses, cudaMemcpyDeviceToHost, s) ||
      cudaStreamSynchronize(s))
    return cuda_fail();
  {
    // queue order: size class descending (largest nets first)
    std::vector<int64_t> cur(kSizeClasses, 0);
    int64_t acc = 0;
    nf.big_sc_cnt.assign(kSizeClasses, 0);
    for (int sc = kSizeClasses - 1; sc >= kMinBigSc; --sc) {
      cur[sc] = acc;
      acc += sc_cnt[sc];
      nf.big_sc_cnt[sc] = sc_cnt[sc];
    }
    GETK(nf.big_queue, size_t(std::max<int64_t>(acc, 1)));
    if (st) return fail(st);
    if (cudaMemcpyAsync(d_sccur, cur.data(), sizeof(int64_t) * kSizeClasses, cudaMemcpyHostToDevice, s))
      return cuda_fail();
    launch_net_levels(tf, in2int, nf, nullptr, d_sccur, s);
    ++c->launches;
  }
  // internal order
  GETK(nf.root_of_net, N); GETK(nf.parent_g, V); GETK(nf.net_of, V); GETK(nf.pin, V); GETK(nf.sink_cap, V);
  GETK(nf.kappa, V); GETK(nf.gk, V); GETK(nf.geo, V); GETK(nf.child_start, V); GETK(nf.nch, V);
  GETK(nf.child_list, V); GETK(nf.son0, V); GETK(nf.W_eq4, V); GETK(nf.rho_eq4, V);
  GETK(nf.A, V * LD); GETK(nf.Cc, V * LD); GETK(nf.M, V * LD); GETK(nf.B, V * LD); GETK(nf.sb, V * LD);
  GETK(nf.st, V * LD); GETK(nf.ent, V * LD); GETK(nf.Jroot, V); GETK(nf.layer, V); GETK(nf.b, V); GETK(nf.t, V);
  GETK(nf.s0, V); GETK(nf.s1, V); GETK(nf.s2, V); GETK(nf.s3, V); GETK(nf.s4, V); GETK(nf.W_adj, V);
  GETK(nf.rho_adj, V);
  const int nred = std::max(scan_blocks(c->grid.li), int((N + 255) / 256)) + 8;
  GETK(nf.red, size_t(nred) * 2);
#undef GETK
#undef GETT
  if (st) return fail(st);
  nf.red_cap = nred;
  {
    // every array the kernels below and the rounds use must exist
    const void* need[] = {nf.net_ptr, nf.r_drv, nf.lvl_nodes, nf.bl_nodes, nf.bl_hoff, nf.net_H, nf.queue_ctr,
                          nf.big_queue, nf.root_of_net, nf.parent_g, nf.net_of, nf.pin, nf.sink_cap, nf.kappa,
                          nf.gk, nf.geo, nf.child_start, nf.nch, nf.child_list, nf.son0, nf.W_eq4, nf.rho_eq4, nf.A, nf.Cc,
                          nf.M, nf.B, nf.sb, nf.st, nf.ent, nf.Jroot, nf.layer, nf.b, nf.t, nf.s0, nf.s1, nf.s2,
                          nf.s3, nf.s4, nf.W_adj, nf.rho_adj, nf.red, in2int};
    for (const void* q : need)
      if (!q) return fail(set_err(c, LA_ERR_STATE, "la_load_nets: internal allocation missing"));
  }
  launch_renumber(tf, in2int, key_of, int64_t(nbk), nf, s);
  launch_first_son(nf, s);
  c->launches += 2;
  {
    // the segments by (direction, line), for the demand pass
    const int nl0 = c->grid.li.nlines[0], nkeys = nl0 + c->grid.li.nlines[1];
    const size_t S = size_t(nf.V - nf.N);
    int32_t* d_scnt = nullptr;
    int64_t* d_scur = nullptr;
    if ((st = ta.get(c, &d_scnt, size_t(nkeys))) || (st = ta.get(c, &d_scur, size_t(nkeys))) ||
        (st = na.get(c, &nf.seg_node, std::max<size_t>(S, 1))) || (st = na.get(c, &nf.seg_geo, std::max<size_t>(S, 1))))
      return fail(st);
    if (cudaMemsetAsync(d_scnt, 0, sizeof(int32_t) * nkeys, s)) return cuda_fail();
    launch_seg_sort(nf, nl0, nkeys, d_scnt, nullptr, nullptr, nullptr, s);
    std::vector<int32_t> scnt(nkeys);
    if (cudaMemcpyAsync(scnt.data(), d_scnt, sizeof(int32_t) * nkeys, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
      return cuda_fail();
    std::vector<int64_t> scur(nkeys);
    int64_t acc = 0;
    for (int k = 0; k < nkeys; ++k) {
      scur[k] = acc;
      acc += scnt[k];
    }
    if (acc != int64_t(S)) return fail(set_err(c, LA_ERR_STATE, "la_load_nets: segment count mismatch"));
    scur.push_back(acc);
    if ((st = na.get(c, &nf.seg_off, size_t(nkeys) + 1))) return fail(st);
    if (cudaMemcpyAsync(nf.seg_off, scur.data(), sizeof(int64_t) * (nkeys + 1), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d_scur, scur.data(), sizeof(int64_t) * nkeys, cudaMemcpyHostToDevice, s))
      return cuda_fail();
    launch_seg_sort(nf, nl0, nkeys, nullptr, d_scur, nf.seg_node, nf.seg_geo, s);
    c->launches += 2;
    nf.S = int64_t(S);
  }
  if (nf.nbatch == 1) {
    // per split k, level and class: (first node, count) of the nets of at most
    // 2^k nodes (the tail kernels' ranges)
    const size_t H1 = size_t(nf.Hmax) + 1;
    std::vector<int64_t> rt(size_t(kSizeClasses) * H1 * kClasses * 2);
    for (int k = 0; k < kSizeClasses; ++k)
      for (size_t h = 0; h < H1; ++h)
        for (int cls = 0; cls < kClasses; ++cls) {
          const int64_t lo = nf.key_off[size_t(bucket_key(int64_t(h), cls, 0))];
          const int64_t hi = nf.key_off[size_t(bucket_key(int64_t(h), cls, k + 1))];
          const size_t o = ((size_t(k) * H1 + h) * kClasses + cls) * 2;
          rt[o] = lo;
          rt[o + 1] = hi - lo;
        }
    if ((st = na.get(c, &nf.range_tab, rt.size()))) return fail(st);
    if (cudaMemcpyAsync(nf.range_tab, rt.data(), sizeof(int64_t) * rt.size(), cudaMemcpyHostToDevice, s))
      return cuda_fail();
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return cuda_fail();
  ta.release();
  al->pool.free_older_than(gen0);  // blocks no load took since the last one
  al->fpool.free_older_than(gen0);
  al->forest = na;
  al->forest.hint = nullptr;  // the hint names this load's local list
  al->forest.next = 0;
  c->forest = nf;
  plan_from_memo(c);
  // A plan taken from the memo keeps the old graphs: each replays only if the
  // addresses and shapes it was captured with are unchanged (round_signature).
  for (int i = 0; i < 2; ++i) {
    if (c->plan.tuned && old_plan.exec[i]) {
      c->plan.exec[i] = old_plan.exec[i];
      c->plan.graph_launches[i] = old_plan.graph_launches[i];
      c->plan.graph_sig[i] = old_plan.graph_sig[i];
      for (int j = 0; j < 5; ++j) c->plan.w[i][j] = old_plan.w[i][j];
    } else if (old_plan.exec[i]) {
      cudaGraphExecDestroy(old_plan.exec[i]);
    }
  }
  return LA_OK;
}

// ------------------------------------------------------------------------
static la_status check_loaded(la_ctx* c) {
  TRY(check_ctx(c));
  if (!c->grid.loaded || c->forest.V == 0) return set_err(c, LA_ERR_STATE, "load a grid and a forest first");
  return LA_OK;
}

// ---- batched form ----
// Everything a captured round bakes in: the device addresses it reads and
// writes, the forest's shape and the plan.  A graph replays only while this
// is unchanged (a reload of a same-shaped forest gets the same addresses back
// from the pool and keeps its graphs).
static uint64_t round_signature(la_ctx* c, int si, const double* W, const double* rho, bool local) {
  const Forest& f = c->forest;
  const Grid& g = c->grid;
  const BatchPlan& bp = c->plan;
  const void* ptrs[] = {f.bl_nodes, f.bl_hoff, f.net_H, f.big_queue, f.queue_ctr, f.net_ptr, f.root_of_net,
                        f.parent_g, f.net_of, f.pin, f.sink_cap, f.kappa, f.gk, f.r_drv, f.geo, f.child_start,
                        f.nch, f.child_list, f.son0, f.W_eq4, f.rho_eq4, f.W_adj, f.rho_adj, f.A, f.Cc, f.M, f.B,
                        f.ncache[si], f.scache[si], f.sb, f.st, f.ent, f.Jroot, f.layer, f.b, f.t, f.red,
                        f.seg_node, f.seg_geo, f.seg_off, f.range_tab, f.layer_old,
                        g.cap, g.D, g.H, g.diff, g.P, g.T_dev, g.tofT_dev, g.tab_dev, c->d_stats, c->d_err};
  uint64_t h = 1469598103934665603ull;
  for (const void* q : ptrs) h = fnv_mix(h, uint64_t(reinterpret_cast<uintptr_t>(q)));
  h = fnv_mix(h, uint64_t(reinterpret_cast<uintptr_t>(W)));
  h = fnv_mix(h, uint64_t(reinterpret_cast<uintptr_t>(rho)));
  const int64_t vals[] = {f.N, f.V, f.Hmax, f.nbatch, f.red_cap, c->LD, bp.k, bp.block, bp.grid, bp.cached ? 1 : 0,
                          bp.n_big, bp.Hs, bp.tail_h, int64_t(f.key_hash), local ? 1 : 0, c->fuse_adjoint ? 1 : 0};
  for (int64_t x : vals) h = fnv_mix(h, uint64_t(x));
  return h;
}

// tail_T > 0: the top levels whose (node, candidate) task counts are all
// below tail_T go to the one-block tail kernels instead of level waves.
static BatchPlan make_plan(la_ctx* c, int k, int block, bool one_per_sm, int tail_T = 0) {
  Forest& f = c->forest;
  BatchPlan bp;
  bp.k = k;
  bp.block = block;
  for (int sc = std::max(k + 1, kMinBigSc); sc < kSizeClasses; ++sc) bp.n_big += f.big_sc_cnt[sc];
  bp.Hs = 0;
  auto tasks = [&](int h) {
    int64_t n = 0;
    for (int cls = 0; cls < kClasses; ++cls) {
      const int64_t m = f.key_off[size_t(bucket_key(h, cls, k + 1))] - f.key_off[size_t(bucket_key(h, cls, 0))];
      n += m * ((cls >= 3 && cls <= 5) ? 1 : c->LD);
    }
    return n;
  };
  for (int h = f.Hmax; h >= 0; --h) {
    if (tasks(h) > 0) { bp.Hs = h; break; }
  }
  if (tail_T > 0 && f.range_tab) {
    int th = bp.Hs + 1;
    while (th > 0 && tasks(th - 1) < tail_T) --th;
    if (th + 1 <= bp.Hs) {  // at least two levels
      bp.tail_h = th;
      bp.tail_T = tail_T;
    }
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int per_sm = one_per_sm ? 1 : bignet_blocks_per_sm(c->grid.li.L, c->LD, block);
  bp.grid = int(std::min<int64_t>(bp.n_big, int64_t(sms) * per_sm));
  if (bp.grid < 1) bp.grid = 1;
  return bp;
}

// DP and backtrack of the batched form: small nets on `s`, big nets on s2.
static la_status enqueue_batched(la_ctx* c, const BatchPlan& bp, const RoundW& w, const double* W, const double* rho,
                                 int si, cudaStream_t s) {
  const int cache = bp.cached ? si : kNoCache;
  Forest& f = c->forest;
  if (bp.n_big > 0) {
    CK(cudaEventRecord(c->ev_fork, s));
    CK(cudaStreamWaitEvent(c->s2, c->ev_fork, 0));
    CK(cudaMemsetAsync(f.queue_ctr, 0, 2 * sizeof(int), c->s2));
    launch_dp_bignets(c, w, W, rho, bp.n_big, bp.grid, bp.block, cache, c->s2);
    launch_backtrack_bignets(c, bp.n_big, bp.grid, bp.block, c->s2);
    CK(cudaEventRecord(c->ev_join, c->s2));
  }
  const bool tail = bp.tail_h <= bp.Hs;
  const int hw = tail ? bp.tail_h - 1 : bp.Hs;  // the last level-wave level
  // A level's classes are independent: the several-son, root and no-pin
  // classes (latency-bound, small) run on a side branch beside the leaves,
  // one-son and bend classes (FP64-bound, large), joined before the next level.
  constexpr unsigned kSide = (1u << 2) | (1u << 3) | (1u << 4) | (1u << 5) | (1u << 6) | (1u << 8);
  for (int h = 0; h <= hw; ++h) {
    bool side = false;
    for (int cls = 0; cls < kClasses && !side; ++cls)
      side = ((kSide >> cls) & 1u) &&
             f.key_off[size_t(bucket_key(h, cls, bp.k + 1))] > f.key_off[size_t(bucket_key(h, cls, 0))];
    if (!side) {
      launch_dp_level(c, w, W, rho, h, bp.k, cache, s);
      continue;
    }
    CK(cudaEventRecord(c->ev_lfork, s));
    CK(cudaStreamWaitEvent(c->s3, c->ev_lfork, 0));
    launch_dp_level(c, w, W, rho, h, bp.k, cache, c->s3, kSide);
    launch_dp_level(c, w, W, rho, h, bp.k, cache, s, kAllClasses & ~kSide);
    CK(cudaEventRecord(c->ev_ljoin, c->s3));
    CK(cudaStreamWaitEvent(s, c->ev_ljoin, 0));
  }
  if (tail) {
    launch_dp_tail(c, w, W, rho, bp.tail_h, bp.Hs, bp.k, cache, s);
    launch_backtrack_tail(c, bp.tail_h, bp.Hs, bp.k, s);
  }
  for (int h = hw; h >= 0; --h) launch_backtrack_level(c, h, bp.k, s);
  if (bp.n_big > 0) CK(cudaStreamWaitEvent(s, c->ev_join, 0));
  CK(cudaGetLastError());
  return LA_OK;
}

// The batched form of a forest in sequential batches (Sec. III-A): every net
// in the level waves of the class kernels with the constant caches; after
// batch k's DP and backtrack its nets' demand moves from their layers at the
// round's start (layer_old; -1: none) to the new ones and the penalty prefix
// is refreshed, so batch k + 1 sees it.  No persistent kernels and no tuning.
static la_status enqueue_batched_multi(la_ctx* c, const RoundW& w, const double* W, const double* rho, int si,
                                       cudaStream_t s) {
  Forest& f = c->forest;
  const int H1 = f.Hmax + 1;
  for (int k = 0; k < f.nbatch; ++k) {
    const int g0 = k * H1;
    if (f.lvl_off[g0 + H1] == f.lvl_off[g0]) continue;  // an empty batch
    for (int h = 0; h < H1; ++h) launch_dp_level(c, w, W, rho, g0 + h, kSizeClasses - 1, si, s);
    for (int h = H1 - 1; h >= 0; --h) launch_backtrack_level(c, g0 + h, kSizeClasses - 1, s);
    if (k + 1 < f.nbatch) {
      launch_demand_delta(c, f.lvl_off[g0], f.lvl_off[g0 + H1], f.layer_old, s);
      launch_scan_lines(c, 2, w.hist_w, f.red, s);
    }
  }
  CK(cudaGetLastError());
  return LA_OK;
}

// The batched form's constant caches: allocated on first use, refreshed when
// the weight set (W, w_d, w_cap) changes; w_d r_est per round.
static la_status batched_caches(la_ctx* c, const RoundW& w, const double* W, int si, cudaStream_t s) {
  Forest& f = c->forest;
  if (!f.ncache[si]) {
    la_ctx_allocs* a = allocs_of(c);
    TRY(a->forest.get(c, &f.ncache[si], size_t(f.V) * 4));
    TRY(a->forest.get(c, &f.scache[si], size_t(f.V) * c->LD * 3));
  }
  BatchPlan& bp = c->plan;
  if (bp.cache_wd[si] != w.w_d || bp.cache_wcap[si] != w.w_cap) {
    launch_seg_consts(c, w, W, si, s);
    CK(cudaGetLastError());
    bp.cache_wd[si] = w.w_d;
    bp.cache_wcap[si] = w.w_cap;
  }
  return LA_OK;
}

// Autotuner: time the DP + backtrack of every distinct split (size-class
// threshold) and block shape on the loaded forest, keep the fastest.  The
// trials compute the same tables the round computes next.
// One trial of plan b timed the way the round runs it: the DP and backtrack
// captured into a graph, then one untimed replay and the best of three timed
// ones (launched one by one, the same kernels would be timed with the host's
// launch overhead of every small level in them).
static la_status time_plan(la_ctx* c, const BatchPlan& b, const RoundW& w, const double* W, const double* rho,
                           int si, cudaStream_t s, double* ms_out) {
  cudaStream_t cs = c->s_cap;
  const long long l0 = c->launches;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const la_status st = enqueue_batched(c, b, w, W, rho, si, cs);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  c->launches = l0;
  if (st != LA_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    if (st != LA_OK) return st;
    return set_err(c, LA_ERR_CUDA, "la_assign_round: tuner capture failed: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t x = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return set_err(c, LA_ERR_CUDA, "la_assign_round: tuner instantiate: %s", cudaGetErrorString(ei));
  double t = 1e30;
  cudaError_t er = cudaSuccess;
  for (int rep = 0; rep < 4 && er == cudaSuccess; ++rep) {
    float ms = 0.f;
    if ((er = cudaEventRecord(c->ev[1], s)) != cudaSuccess || (er = cudaGraphLaunch(x, s)) != cudaSuccess ||
        (er = cudaEventRecord(c->ev[2], s)) != cudaSuccess || (er = cudaEventSynchronize(c->ev[2])) != cudaSuccess ||
        (er = cudaEventElapsedTime(&ms, c->ev[1], c->ev[2])) != cudaSuccess)
      break;
    if (rep > 0) t = std::min(t, double(ms));
  }
  cudaGraphExecDestroy(x);
  if (er != cudaSuccess) return set_err(c, LA_ERR_CUDA, "la_assign_round: tuner trial: %s", cudaGetErrorString(er));
  *ms_out = t;
  return LA_OK;
}

static la_status autotune(la_ctx* c, const RoundW& w, const double* W, const double* rho, int si, cudaStream_t s) {
  Forest& f = c->forest;
  TRY(batched_caches(c, w, W, si, s));
  launch_node_round(c, w, rho, si, s);
  std::vector<BatchPlan> cand;
  int64_t last_big = -1;
  for (int k = kSizeClasses - 1; k >= kMinBigSc - 1; --k) {
    BatchPlan b = make_plan(c, k, 256, false);
    if (b.n_big == last_big) continue;
    last_big = b.n_big;
    cand.push_back(b);
    if (b.n_big > 0) {
      cand.push_back(make_plan(c, k, 128, false));
      cand.push_back(make_plan(c, k, 256, true));
    }
  }
  // each shape with the constant caches and without
  const size_t nshape = cand.size();
  for (size_t i = 0; i < nshape; ++i) {
    BatchPlan b = cand[i];
    b.cached = false;
    cand.push_back(b);
  }
  double best = 1e30;
  BatchPlan chosen = cand.front();
  for (auto& b : cand) {
    double t = 1e30;
    TRY(time_plan(c, b, w, W, rho, si, s, &t));
    if (t < best) { best = t; chosen = b; }
  }
  (void)f;
  int trials = int(cand.size());
  // then the winner with its top levels in the one-block tail kernels
  for (int T : {2048, 8192, 32768}) {
    BatchPlan b = make_plan(c, chosen.k, chosen.block, false, T);
    if (b.tail_h > b.Hs) continue;
    b.grid = chosen.grid;
    b.cached = chosen.cached;
    double t = 1e30;
    TRY(time_plan(c, b, w, W, rho, si, s, &t));
    ++trials;
    if (t < best) { best = t; chosen = b; }
  }
  chosen.tuned = true;
  chosen.best_ms = best;
  chosen.trials = trials;
  for (int i = 0; i < 2; ++i) {
    chosen.cache_wd[i] = c->plan.cache_wd[i];
    chosen.cache_wcap[i] = c->plan.cache_wcap[i];
  }
  c->plan = chosen;
  TuneMemo& m = c->memo;
  m.valid = true;
  m.L = c->grid.li.L;
  m.LD = c->LD;
  m.key_off = f.key_off;
  m.k = chosen.k;
  m.block = chosen.block;
  m.grid = chosen.grid;
  m.cached = chosen.cached;
  m.tail_T = chosen.tail_T;
  m.best_ms = chosen.best_ms;
  m.trials = chosen.trials;
  return LA_OK;
}

// A forest with the same bucket offsets as the one the memo was tuned on
// takes the memo's plan without new trials.
static void plan_from_memo(la_ctx* c) {
  const TuneMemo& m = c->memo;
  if (!m.valid || m.L != c->grid.li.L || m.LD != c->LD || m.key_off != c->forest.key_off) return;
  BatchPlan b = make_plan(c, m.k, m.block, false, m.tail_T);
  b.grid = m.grid;
  b.cached = m.cached;
  b.tuned = true;
  b.best_ms = m.best_ms;
  b.trials = 0;
  c->plan = b;
}

// The current plan's block and caching with split k and tail threshold T
// (0: no tail); the persistent grid is the tuned one while the split is the
// tuned one, else the occupancy grid of the new split.  The graphs and
// constant caches stay with the plan; a graph replays only if its signature,
// which holds the split and the tail level, still matches.
static void set_shape(la_ctx* c, int k, int T) {
  const BatchPlan& o = c->plan;
  BatchPlan b = make_plan(c, k, o.block, false, T);
  if (k == c->memo.k) b.grid = c->memo.grid;
  b.cached = o.cached;
  b.tuned = o.tuned;
  b.best_ms = o.best_ms;
  b.trials = o.trials;  // the trials that chose the shape (0: the memo's)
  for (int i = 0; i < 2; ++i) {
    b.exec[i] = o.exec[i];
    b.graph_launches[i] = o.graph_launches[i];
    b.graph_sig[i] = o.graph_sig[i];
    for (int j = 0; j < 5; ++j) b.w[i][j] = o.w[i][j];
    b.cache_wd[i] = o.cache_wd[i];
    b.cache_wcap[i] = o.cache_wcap[i];
  }
  c->plan = b;
}

// The round after the penalty prefix, as one CUDA graph (captured once per
// weights and parameter set on the context's own capture stream, replayed on
// the caller's stream every round; the caller's stream may be the legacy
// default stream, which cannot be captured).
static la_status batched_graph(la_ctx* c, const RoundW& w, const double* W, const double* rho, int si,
                               cudaStream_t s_run, bool* captured, bool local) {
  BatchPlan& bp = c->plan;
  cudaStream_t s = c->s_cap;
  const double wv[5] = {w.w_cong, w.w_via, w.w_cap, w.w_d, w.hist_w};
  const uint64_t sig = round_signature(c, si, W, rho, local);
  bool same = bp.exec[si] != nullptr && bp.graph_sig[si] == sig;
  for (int i = 0; i < 5 && same; ++i) same = bp.w[si][i] == wv[i];
  *captured = !same;
  if (!same) {
    if (bp.exec[si]) {
      cudaGraphExecDestroy(bp.exec[si]);
      bp.exec[si] = nullptr;
    }
    const long long l0 = c->launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    la_status st = LA_OK;
    // phase events as external record nodes of the graph (timed on replay)
    auto mark = [&](cudaEvent_t e) {
      if (st == LA_OK && cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) != cudaSuccess) st = LA_ERR_CUDA;
    };
    launch_node_round(c, w, rho, si, s);
    mark(c->ev[1]);
    if (st == LA_OK)
      st = c->forest.nbatch > 1 ? enqueue_batched_multi(c, w, W, rho, si, s) : enqueue_batched(c, bp, w, W, rho, si, s);
    mark(c->ev[3]);
    Forest& f = c->forest;
    if (st == LA_OK) {
      if (local) launch_local_demand(c, w.hist_w, f.red, s);
      else launch_demand_scan(c, w.hist_w, f.red, s);
      launch_sum_roots(c, f.red + f.red_cap, nullptr, s);
    }
    mark(c->ev[4]);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != LA_OK || e != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return set_err(c, LA_ERR_CUDA, "la_assign_round: graph capture failed: %s", cudaGetErrorString(e));
    }
    const cudaError_t ei = cudaGraphInstantiate(&bp.exec[si], g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return set_err(c, LA_ERR_CUDA, "la_assign_round: graph instantiate: %s", cudaGetErrorString(ei));
    bp.graph_launches[si] = c->launches - l0;
    bp.graph_sig[si] = sig;
    c->launches = l0;
    for (int i = 0; i < 5; ++i) bp.w[si][i] = wv[i];
  }
  CK(cudaGraphLaunch(bp.exec[si], s_run));
  c->launches += bp.graph_launches[si];
  return LA_OK;
}

la_status la_assign_round(la_ctx* c, const la_round_params* p, la_round_stats* stats) {
  TRY(check_loaded(c));
  if (!p) return set_err(c, LA_ERR_INVALID, "la_assign_round: null params");
  const double ws[5] = {p->w_cong, p->w_via, p->w_cap, p->w_d, p->hist_w};
  for (double w : ws)
    if (!finite_nonneg(w)) return set_err(c, LA_ERR_INVALID, "la_assign_round: weights must be finite and >= 0");
  if (p->mode != LA_MODE_PLAIN && p->mode != LA_MODE_BATCHED)
    return set_err(c, LA_ERR_INVALID, "la_assign_round: unknown mode %d", p->mode);
  if (p->weights != LA_WEIGHTS_EQ4 && p->weights != LA_WEIGHTS_ADJOINT)
    return set_err(c, LA_ERR_INVALID, "la_assign_round: unknown weights source %d", p->weights);
  Forest& f = c->forest;
  Grid& gr = c->grid;
  if (p->weights == LA_WEIGHTS_ADJOINT && !f.have_adj)
    return set_err(c, LA_ERR_STATE, "la_assign_round: no adjoint weights yet (call la_reweight_adjoint)");
  if (p->no_look_ahead != 0 && p->no_look_ahead != 1)
    return set_err(c, LA_ERR_INVALID, "la_assign_round: no_look_ahead must be 0 or 1");
  if (p->tail_threshold < 0) return set_err(c, LA_ERR_INVALID, "la_assign_round: tail_threshold must be >= 0");
  if (p->local_demand != 0 && p->local_demand != 1)
    return set_err(c, LA_ERR_INVALID, "la_assign_round: local_demand must be 0 or 1");
  if (p->reweight_adjoint != 0 && p->reweight_adjoint != 1)
    return set_err(c, LA_ERR_INVALID, "la_assign_round: reweight_adjoint must be 0 or 1");
  if (p->force_split != 0 && (p->force_split < kMinBigSc - 1 || p->force_split > kSizeClasses - 1))
    return set_err(c, LA_ERR_INVALID, "la_assign_round: force_split must be 0 or in [%d, %d]", kMinBigSc - 1,
                   kSizeClasses - 1);
  const double* W = p->weights == LA_WEIGHTS_ADJOINT ? f.W_adj : f.W_eq4;
  const double* rho = p->weights == LA_WEIGHTS_ADJOINT ? f.rho_adj : f.rho_eq4;
  if (p->no_look_ahead) {
    if (!f.rho_zero) {
      TRY(allocs_of(c)->forest.get(c, &f.rho_zero, size_t(f.V)));
      CK(cudaMemsetAsync(f.rho_zero, 0, sizeof(double) * size_t(f.V), c->stream));
    }
    rho = f.rho_zero;
  }
  DeviceGuard g(c->device);
  cudaStream_t s = c->stream;
  RoundW w{p->w_cong, p->w_via, p->w_cap, p->w_d, p->hist_w};
  if (p->reset) {
    CK(cudaMemsetAsync(gr.D, 0, gr.G * 4, s));
    CK(cudaMemsetAsync(gr.H, 0, gr.G * 4, s));
    CK(cudaMemsetAsync(gr.diff, 0, gr.G * 4, s));
    gr.P_valid = false;
  }
  TRY(reset_dev_err(c));
  const long long launches0 = c->launches;
  double* tof_part = f.red;
  double* J_part = f.red + f.red_cap;
  if (!gr.P_valid || gr.P_hist_w != p->hist_w) launch_scan_lines(c, 0, p->hist_w, tof_part, s);
  const bool batched = p->mode == LA_MODE_BATCHED;
  const int si = p->weights == LA_WEIGHTS_ADJOINT ? 1 : 0;
  if (p->local_demand && f.nbatch > 1)
    return set_err(c, LA_ERR_INVALID, "la_assign_round: sequential batches cannot be split over shards");
  if (batched && f.nbatch > 1) {
    TRY(batched_caches(c, w, W, si, s));
    BatchPlan& bp = c->plan;
    if (!bp.tuned) {  // every net in level waves, caches on; nothing to tune
      bp.k = kSizeClasses - 1;
      bp.block = 256;
      bp.grid = 1;
      bp.cached = true;
      bp.n_big = 0;
      bp.Hs = f.nlev - 1;
      bp.tail_h = 1 << 30;
      bp.tail_T = 0;
      bp.tuned = true;
      bp.trials = 0;
      bp.best_ms = 0.0;
    }
    // the batches' start layers: the previous assignment, or none after a reset
    if (!f.layer_old) TRY(allocs_of(c)->forest.get(c, &f.layer_old, size_t(f.V)));
    if (!p->reset && f.have_assign) CK(cudaMemcpyAsync(f.layer_old, f.layer, size_t(f.V), cudaMemcpyDeviceToDevice, s));
    else CK(cudaMemsetAsync(f.layer_old, 0xFF, size_t(f.V), s));
  } else if (batched) {
    TRY(batched_caches(c, w, W, si, s));
    if (!c->plan.tuned) TRY(autotune(c, w, W, rho, si, s));
    const int T = p->tail_threshold > 0 ? p->tail_threshold : c->memo.tail_T;
    const int k = p->force_split > 0 ? p->force_split : c->memo.k;
    if (T != c->plan.tail_T || k != c->plan.k) set_shape(c, k, T);
  }
  // the statistics count this round only (not the tuner's trial rounds)
  CK(cudaMemsetAsync(c->d_stats, 0, sizeof(Stats), s));
  // The adjoint reweighting of the new assignment in the backtrack (never in
  // the tuner's trials above: their backtracks would overwrite the adjoint
  // weights this round reads).  Its W, the kappa sums, depend on the forest
  // only and are computed once.
  struct FuseOff {
    la_ctx* c;
    ~FuseOff() { c->fuse_adjoint = false; }
  } fuse_off{c};
  if (p->reweight_adjoint) {
    if (!f.wsum_valid) {
      launch_wsum(c, s);
      f.wsum_valid = true;
    }
    c->fuse_adjoint = true;
  }
  bool captured = false;
  CK(cudaEventRecord(c->ev[0], s));
  if (batched) {
    TRY(batched_graph(c, w, W, rho, si, s, &captured, p->local_demand != 0));
  } else if (f.nbatch == 1) {
    CK(cudaEventRecord(c->ev[1], s));
    for (int h = 0; h <= f.Hmax; ++h) launch_dp_level(c, w, W, rho, h, kSizeClasses - 1, kNoCache, s);
    CK(cudaEventRecord(c->ev[2], s));
    for (int h = f.Hmax; h >= 0; --h) launch_backtrack_level(c, h, kSizeClasses - 1, s);
    CK(cudaEventRecord(c->ev[3], s));
    if (p->local_demand) launch_local_demand(c, p->hist_w, tof_part, s);
    else launch_demand_scan(c, p->hist_w, tof_part, s);
    launch_sum_roots(c, J_part, nullptr, s);
    CK(cudaEventRecord(c->ev[4], s));
  } else {
    // Sequential batches (Sec. III-A): batch k's DP and backtrack, then its
    // nets' demand moves from their old layers (none after a reset) to the new
    // ones and the penalty prefix is refreshed (H stays the round's), so batch
    // k + 1 sees it.  The round's end is the single-batch one.
    const int8_t* old = nullptr;
    if (!p->reset && f.have_assign) {
      if (!f.layer_old) TRY(allocs_of(c)->forest.get(c, &f.layer_old, size_t(f.V)));
      CK(cudaMemcpyAsync(f.layer_old, f.layer, size_t(f.V), cudaMemcpyDeviceToDevice, s));
      old = f.layer_old;
    }
    const int H1 = f.Hmax + 1;
    CK(cudaEventRecord(c->ev[1], s));
    for (int k = 0; k < f.nbatch; ++k) {
      const int g0 = k * H1;
      if (f.lvl_off[g0 + H1] == f.lvl_off[g0]) continue;  // an empty batch
      for (int h = 0; h < H1; ++h) launch_dp_level(c, w, W, rho, g0 + h, kSizeClasses - 1, kNoCache, s);
      for (int h = H1 - 1; h >= 0; --h) launch_backtrack_level(c, g0 + h, kSizeClasses - 1, s);
      if (k + 1 < f.nbatch) {
        launch_demand_delta(c, f.lvl_off[g0], f.lvl_off[g0 + H1], old, s);
        launch_scan_lines(c, 2, p->hist_w, tof_part, s);
      }
    }
    CK(cudaEventRecord(c->ev[2], s));
    CK(cudaEventRecord(c->ev[3], s));
    if (p->local_demand) launch_local_demand(c, p->hist_w, tof_part, s);
    else launch_demand_scan(c, p->hist_w, tof_part, s);
    launch_sum_roots(c, J_part, nullptr, s);
    CK(cudaEventRecord(c->ev[4], s));
  }
  CK(cudaGetLastError());
  gr.P_valid = p->local_demand == 0;  // a shard's D is not the round's snapshot until la_commit_demand
  gr.P_hist_w = p->hist_w;
  gr.round_hist_w = p->hist_w;
  f.have_assign = true;
  if (p->reweight_adjoint) f.have_adj = true;
  if (!stats) return LA_OK;
  CK(cudaStreamSynchronize(s));
  int code;
  long long idx;
  TRY(read_dev_err(c, &code, &idx));
  if (code) return set_err(c, LA_ERR_DEVICE_CHECK, "la_assign_round: %s (index %lld)", dev_err_name(code), idx);
  Stats hs;
  CK(cudaMemcpy(&hs, c->d_stats, sizeof hs, cudaMemcpyDeviceToHost));
  const int nsb = scan_blocks(gr.li), njb = int((f.N + 255) / 256);
  std::vector<double> part(size_t(f.red_cap) * 2);
  CK(cudaMemcpy(part.data(), f.red, sizeof(double) * part.size(), cudaMemcpyDeviceToHost));
  double tof = 0.0, J = 0.0;
  for (int i = 0; i < nsb; ++i) tof += part[i];
  for (int i = 0; i < njb; ++i) J += part[f.red_cap + i];
  float ms = 0.f, ms_dp = 0.f, ms_bt = 0.f, ms_dem = 0.f;
  // phase times from events (inside the graph for the batched form); a
  // phase whose events cannot be timed is reported as -1
  auto elapsed = [&](float* out, cudaEvent_t a, cudaEvent_t b) {
    if (cudaEventElapsedTime(out, a, b) != cudaSuccess) {
      cudaGetLastError();
      *out = -1.f;
    }
  };
  elapsed(&ms, c->ev[0], c->ev[4]);
  if (batched) {  // DP and backtrack overlap across the two buckets: reported together
    elapsed(&ms_dp, c->ev[1], c->ev[3]);
  } else {
    elapsed(&ms_dp, c->ev[1], c->ev[2]);
    elapsed(&ms_bt, c->ev[2], c->ev[3]);
  }
  elapsed(&ms_dem, c->ev[3], c->ev[4]);
  memset(stats, 0, sizeof *stats);
  stats->total_cost = J;
  stats->tof = tof;
  stats->relu_overflow = (int64_t)hs.relu;
  stats->vias = (int64_t)hs.vias;
  stats->wl = (int64_t)hs.wl;
  for (int l = 0; l < LA_MAX_LAYERS; ++l) stats->wl_per_layer[l] = (int64_t)hs.wl_layer[l];
  stats->ms = ms;
  stats->ms_dp = ms_dp;
  stats->ms_backtrack = ms_bt;
  stats->ms_demand = ms_dem;
  stats->launches = c->launches - launches0;
  if (batched) {
    stats->batch_split = c->plan.k;
    stats->batch_block = c->plan.block;
    stats->batch_big_nets = c->plan.n_big;
    stats->batch_tune_ms = c->plan.best_ms;
    stats->batch_cached = c->plan.cached ? 1 : 0;
    stats->batch_trials = c->plan.trials;
    stats->batch_levels = c->plan.Hs + 1;
    stats->batch_tail_level = std::min(c->plan.tail_h, c->plan.Hs + 1);
    stats->batch_graph_captured = captured ? 1 : 0;
  }
  return LA_OK;
}

la_status la_commit_demand(la_ctx* c, const int32_t* demand, la_round_stats* stats) {
  TRY(check_loaded(c));
  if (!demand) return set_err(c, LA_ERR_INVALID, "la_commit_demand: null pointer");
  if (!c->forest.have_assign) return set_err(c, LA_ERR_STATE, "la_commit_demand: no round run yet");
  DeviceGuard g(c->device);
  Grid& gr = c->grid;
  Forest& f = c->forest;
  cudaStream_t s = c->stream;
  // stage through the difference array (all zero between rounds) so that a
  // negative entry leaves the snapshot unchanged
  TRY(reset_dev_err(c));
  launch_grid_to_internal(gr.li, gr.X, gr.Y, demand, gr.diff, true, c->d_err, s);
  ++c->launches;
  CK(cudaGetLastError());
  int code;
  long long idx;
  TRY(read_dev_err(c, &code, &idx));
  if (code) {
    CK(cudaMemsetAsync(gr.diff, 0, gr.G * 4, s));
    return set_err(c, LA_ERR_INVALID, "la_commit_demand: demand at edge %lld is negative", idx);
  }
  CK(cudaMemcpyAsync(gr.D, gr.diff, gr.G * 4, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(gr.diff, 0, gr.G * 4, s));
  CK(cudaMemsetAsync(c->d_stats, 0, sizeof(Stats), s));
  launch_scan_lines(c, 3, gr.round_hist_w, f.red, s);
  CK(cudaGetLastError());
  gr.P_valid = true;
  gr.P_hist_w = gr.round_hist_w;
  if (!stats) return LA_OK;
  CK(cudaStreamSynchronize(s));
  Stats hs;
  CK(cudaMemcpy(&hs, c->d_stats, sizeof hs, cudaMemcpyDeviceToHost));
  const int nsb = scan_blocks(gr.li);
  std::vector<double> part(static_cast<size_t>(nsb));
  CK(cudaMemcpy(part.data(), f.red, sizeof(double) * part.size(), cudaMemcpyDeviceToHost));
  double tof = 0.0;
  for (int i = 0; i < nsb; ++i) tof += part[i];
  memset(stats, 0, sizeof *stats);
  stats->tof = tof;
  stats->relu_overflow = (int64_t)hs.relu;
  return LA_OK;
}

la_status la_get_assignment(la_ctx* c, int8_t* layer, int8_t* b, int8_t* t) {
  TRY(check_loaded(c));
  if (!c->forest.have_assign) return set_err(c, LA_ERR_STATE, "no assignment yet");
  DeviceGuard g(c->device);
  Forest& f = c->forest;
  if (layer) { launch_permute8(f.V, f.lvl_nodes, f.layer, layer, false, c->stream); ++c->launches; }
  if (b) { launch_permute8(f.V, f.lvl_nodes, f.b, b, false, c->stream); ++c->launches; }
  if (t) { launch_permute8(f.V, f.lvl_nodes, f.t, t, false, c->stream); ++c->launches; }
  CK(cudaGetLastError());
  return LA_OK;
}

la_status la_set_assignment(la_ctx* c, const int8_t* layer, const int8_t* b, const int8_t* t) {
  TRY(check_loaded(c));
  if (!layer || !b || !t) return set_err(c, LA_ERR_INVALID, "la_set_assignment: null pointer");
  DeviceGuard g(c->device);
  Forest& f = c->forest;
  // gather into internal order in scratch (s0 holds 8 bytes per node), check, then commit
  int8_t* gl = reinterpret_cast<int8_t*>(f.s0);
  int8_t* gb = gl + f.V;
  int8_t* gt = gb + f.V;
  launch_permute8(f.V, f.lvl_nodes, layer, gl, true, c->stream);
  launch_permute8(f.V, f.lvl_nodes, b, gb, true, c->stream);
  launch_permute8(f.V, f.lvl_nodes, t, gt, true, c->stream);
  c->launches += 3;
  TRY(reset_dev_err(c));
  launch_check_assignment(c, gl, gb, gt, c->stream);
  CK(cudaGetLastError());
  int code;
  long long idx;
  TRY(read_dev_err(c, &code, &idx));
  if (code) {
    int32_t in_id = -1;
    CK(cudaMemcpy(&in_id, f.lvl_nodes + idx, sizeof in_id, cudaMemcpyDeviceToHost));
    return set_err(c, LA_ERR_INVALID, "la_set_assignment: %s (node %d)", dev_err_name(code), in_id);
  }
  const size_t V = size_t(f.V);
  CK(cudaMemcpyAsync(f.layer, gl, V, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(f.b, gb, V, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(f.t, gt, V, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  f.have_assign = true;
  return LA_OK;
}

la_status la_get_net_cost(la_ctx* c, double* J) {
  TRY(check_loaded(c));
  if (!J) return set_err(c, LA_ERR_INVALID, "la_get_net_cost: null pointer");
  if (!c->forest.have_assign) return set_err(c, LA_ERR_STATE, "no round run yet");
  DeviceGuard g(c->device);
  launch_sum_roots(c, c->forest.red + c->forest.red_cap, J, c->stream);
  CK(cudaGetLastError());
  return LA_OK;
}

la_status la_get_state(la_ctx* c, int32_t* demand, int32_t* history) {
  TRY(check_ctx(c));
  if (!c->grid.loaded) return set_err(c, LA_ERR_STATE, "load a grid first");
  DeviceGuard g(c->device);
  Grid& gr = c->grid;
  if (demand) launch_grid_to_internal(gr.li, gr.X, gr.Y, demand, gr.D, false, c->d_err, c->stream);
  if (history) launch_grid_to_internal(gr.li, gr.X, gr.Y, history, gr.H, false, c->d_err, c->stream);
  c->launches += (demand != nullptr) + (history != nullptr);
  CK(cudaGetLastError());
  return LA_OK;
}

la_status la_set_state(la_ctx* c, const int32_t* demand, const int32_t* history) {
  TRY(check_ctx(c));
  if (!c->grid.loaded) return set_err(c, LA_ERR_STATE, "load a grid first");
  DeviceGuard g(c->device);
  Grid& gr = c->grid;
  // stage through the difference array (all zero between rounds) so that a
  // negative value leaves the snapshot unchanged
  TRY(reset_dev_err(c));
  int code;
  long long idx;
  const int32_t* src[2] = {demand, history};
  int32_t* dst[2] = {gr.D, gr.H};
  for (int k = 0; k < 2; ++k) {
    if (!src[k]) continue;
    CK(cudaMemsetAsync(gr.diff, 0, gr.G * 4, c->stream));
    launch_grid_to_internal(gr.li, gr.X, gr.Y, src[k], gr.diff, true, c->d_err, c->stream);
    ++c->launches;
    CK(cudaGetLastError());
    TRY(read_dev_err(c, &code, &idx));
    if (code) {
      CK(cudaMemsetAsync(gr.diff, 0, gr.G * 4, c->stream));
      return set_err(c, LA_ERR_INVALID, "la_set_state: value at edge %lld is negative", idx);
    }
    CK(cudaMemcpyAsync(dst[k], gr.diff, gr.G * 4, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemsetAsync(gr.diff, 0, gr.G * 4, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  gr.P_valid = false;
  return LA_OK;
}

// ------------------------------------------------------------------------
static la_status check_assigned(la_ctx* c) {
  TRY(check_loaded(c));
  if (!c->forest.have_assign) return set_err(c, LA_ERR_STATE, "no assignment yet (run a round or la_set_assignment)");
  return LA_OK;
}

la_status la_rc_from_assignment(la_ctx* c, double* R, double* C) {
  TRY(check_assigned(c));
  if (!R || !C) return set_err(c, LA_ERR_INVALID, "la_rc_from_assignment: null pointer");
  DeviceGuard g(c->device);
  launch_rc_from_assignment(c, R, C, c->forest.lvl_nodes, c->stream);
  CK(cudaGetLastError());
  return LA_OK;
}

la_status la_elmore(la_ctx* c, const double* R, const double* C, double* delay) {
  TRY(check_assigned(c));
  if (!R || !C || !delay) return set_err(c, LA_ERR_INVALID, "la_elmore: null pointer");
  DeviceGuard g(c->device);
  launch_elmore_fwd(c, R, C, delay, c->stream);
  CK(cudaGetLastError());
  return LA_OK;
}

la_status la_elmore_assignment(la_ctx* c, double* delay) {
  TRY(check_assigned(c));
  if (!delay) return set_err(c, LA_ERR_INVALID, "la_elmore_assignment: null pointer");
  DeviceGuard g(c->device);
  launch_elmore_assignment(c, delay, c->stream);
  CK(cudaGetLastError());
  return LA_OK;
}

la_status la_elmore_backward(la_ctx* c, const double* R, const double* C, const double* gd, double* dR, double* dC) {
  TRY(check_assigned(c));
  if (!R || !C || !gd || !dR || !dC) return set_err(c, LA_ERR_INVALID, "la_elmore_backward: null pointer");
  DeviceGuard g(c->device);
  launch_elmore_bwd(c, R, C, gd, dR, dC, c->stream);
  CK(cudaGetLastError());
  return LA_OK;
}

la_status la_reweight_adjoint(la_ctx* c) {
  TRY(check_assigned(c));
  DeviceGuard g(c->device);
  Forest& f = c->forest;
  // The adjoint with g = kappa at pins: W = Ws (the kappa sums below, which
  // depend on the forest only: computed once per forest) and r_est = U (the
  // top-down pass over the current assignment's R).
  launch_reweight(c, !f.wsum_valid, c->stream);
  f.wsum_valid = true;
  CK(cudaGetLastError());
  f.have_adj = true;
  return LA_OK;
}

la_status la_get_weights(la_ctx* c, int32_t source, double* W, double* rho) {
  TRY(check_loaded(c));
  Forest& f = c->forest;
  if (source != LA_WEIGHTS_EQ4 && source != LA_WEIGHTS_ADJOINT)
    return set_err(c, LA_ERR_INVALID, "la_get_weights: unknown source %d", source);
  if (source == LA_WEIGHTS_ADJOINT && !f.have_adj) return set_err(c, LA_ERR_STATE, "no adjoint weights yet");
  DeviceGuard g(c->device);
  if (W) { launch_permute64(f.V, f.lvl_nodes, source ? f.W_adj : f.W_eq4, W, false, c->stream); ++c->launches; }
  if (rho) { launch_permute64(f.V, f.lvl_nodes, source ? f.rho_adj : f.rho_eq4, rho, false, c->stream); ++c->launches; }
  CK(cudaGetLastError());
  return LA_OK;
}

}  // extern "C"
