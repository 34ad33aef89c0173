// k_static.cu - la_elmore_static: the Elmore forward pass without any device
// allocation.  Its scratch (a downstream cap and two son links per node, plus
// a small header holding the net-pointer check flag) lives in the fixed
// file-scope device array below, which every GPU that loads the library holds
// until the process exits.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "gapla_internal.cuh"

namespace gapla {

// Header (32 doubles = 256 bytes: the flag word first), then per node
// Cd_J (a double) and the son links head / next (two int32): 16 bytes per
// node, 32 MiB for LA_STATIC_MAX_NODES nodes.
constexpr int64_t kStaticHeader = 32;
static __device__ __align__(256) double g_static_scratch[kStaticHeader + 2 * int64_t(LA_STATIC_MAX_NODES)];

struct RviaTable {
  double rv[kMaxL * kMaxL];  // Rvia(a, b) at a * L + b
};

// net_ptr must rise strictly from 0 to V; otherwise the flag is set and every
// delay is NaN (nets could overlap, so no net's result could be trusted).
__global__ void k_static_check_netptr(int64_t N, int64_t V, const int64_t* __restrict__ net_ptr,
                                      unsigned* __restrict__ flag) {
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n > N) return;
  const int64_t x = net_ptr[n];
  bool bad = x < 0 || x > V;
  if (n == 0) bad = bad || x != 0;
  if (n == N) bad = bad || x != V;
  if (n < N) bad = bad || net_ptr[n + 1] <= x;
  if (bad) atomicOr(flag, 1u);
}

// One thread per net; the nodes of a net are visited in id order (parents
// first) or reverse id order (sons first).  The son lists are built in
// reverse id order, each son put in front of its parent's list, so every list
// runs in increasing id: downstream caps are summed over the sons in that
// order, the order la_elmore and the CPU model use (the results are equal bit
// for bit).  Junction delays are written to `delay` first and the pin terms
// added last.  A node whose parent id is out of order, or whose layer, pin or
// stack is out of range, makes the whole net's delays NaN (no access outside
// the given arrays is made).
__global__ void k_elmore_static(int64_t N, const int64_t* __restrict__ net_ptr, const int32_t* __restrict__ parent,
                                const int8_t* __restrict__ pin, const double* __restrict__ sink_cap,
                                const double* __restrict__ r_drv, const int8_t* __restrict__ layer,
                                const int8_t* __restrict__ b, const int8_t* __restrict__ t, const double* __restrict__ R,
                                const double* __restrict__ C, double* __restrict__ delay, int L, double via_c,
                                const __grid_constant__ RviaTable tab, const unsigned* __restrict__ flag,
                                double* __restrict__ CdJ, int32_t* __restrict__ head, int32_t* __restrict__ next,
                                int64_t V) {
  const double* rv = tab.rv;
  const int64_t gtid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (*flag) {  // malformed net_ptr: every delay is NaN
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = gtid; i < V; i += stride) delay[i] = nan("");
    return;
  }
  const int64_t n = gtid;
  if (n >= N) return;
  const int64_t base = net_ptr[n], m = net_ptr[n + 1] - base;
  bool bad = false;
  // own capacitance at each junction: C_seg/2 (not at the root), vias, pin
  for (int64_t i = 0; i < m && !bad; ++i) {
    const int64_t v = base + i;
    const int p = parent[v], l = layer[v], pv = pin[v], bv = b[v], tv = t[v];
    bad = (i == 0 ? p != -1 : (p < 0 || p >= i)) || l < 0 || l >= L || pv < -1 || pv >= L || bv < 0 || bv > tv ||
          tv >= L;
    double s = i == 0 ? 0.0 : 0.5 * C[v];
    s = s + via_c * double(tv - bv);
    CdJ[v] = s + sink_cap[v];
    head[v] = -1;
  }
  if (bad) {
    for (int64_t i = 0; i < m; ++i) delay[base + i] = nan("");
    return;
  }
  // son lists, increasing local id
  for (int64_t i = m - 1; i >= 1; --i) {
    const int64_t v = base + i, p = base + parent[v];
    next[v] = head[p];
    head[p] = int32_t(i);
  }
  // sons before parents: Cd_J(v) += sum over sons c of (C_seg[c]/2 + Cd_J(c))
  for (int64_t i = m - 1; i >= 0; --i) {
    const int64_t v = base + i;
    double s = CdJ[v];
    for (int32_t c = head[v]; c >= 0; c = next[base + c]) s = s + (0.5 * C[base + c] + CdJ[base + c]);
    CdJ[v] = s;
  }
  // parents before sons: junction delays
  for (int64_t i = 0; i < m; ++i) {
    const int64_t v = base + i;
    double dj;
    if (i == 0) {
      dj = r_drv[n] * CdJ[v];
    } else {
      const int64_t p = base + parent[v];
      const double dX = delay[p] + rv[layer[p] * L + layer[v]] * (0.5 * C[v] + CdJ[v]);
      dj = dX + R[v] * CdJ[v];
    }
    delay[v] = dj;
  }
  // the pin point of each pin node
  for (int64_t i = 0; i < m; ++i) {
    const int64_t v = base + i;
    if (pin[v] >= 0) delay[v] = delay[v] + rv[layer[v] * L + pin[v]] * sink_cap[v];
  }
}

}  // namespace gapla

namespace {
std::mutex g_static_mu;
double* g_static_ptr[64] = {nullptr};  // device address of the scratch, per device
la_status fail_noctx(la_status code, const std::string& msg) {
  gapla::set_noctx_error(msg);
  return code;
}
}  // namespace

extern "C" la_status la_elmore_static(const la_net_desc* nets, const int8_t* layer, const int8_t* b,
                                      const int8_t* t, int32_t L, const double* via_r, double via_c,
                                      const double* R_seg, const double* C_seg, double* delay, void* stream) {
  using namespace gapla;
  if (!nets || !nets->net_ptr || !nets->parent || !nets->pin_layer || !nets->sink_cap || !nets->r_drv || !layer ||
      !b || !t || !R_seg || !C_seg || !delay || (L > 1 && !via_r))
    return fail_noctx(LA_ERR_INVALID, "la_elmore_static: null pointer");
  if (nets->num_nets < 1 || nets->num_nodes < nets->num_nets)
    return fail_noctx(LA_ERR_INVALID, "la_elmore_static: need 1 <= num_nets <= num_nodes");
  if (L < 2 || L > kMaxL) return fail_noctx(LA_ERR_INVALID, "la_elmore_static: need 2 <= L <= 16");
  if (nets->num_nodes > int64_t(LA_STATIC_MAX_NODES))
    return fail_noctx(LA_ERR_INVALID, "la_elmore_static: " + std::to_string(nets->num_nodes) +
                                          " nodes exceed the fixed scratch (at most " +
                                          std::to_string(LA_STATIC_MAX_NODES) + " nodes)");
  if (!(via_c >= 0.0 && std::isfinite(via_c)))
    return fail_noctx(LA_ERR_INVALID, "la_elmore_static: via_c must be finite and >= 0");
  for (int l = 0; l + 1 < L; ++l)
    if (!(via_r[l] >= 0.0 && std::isfinite(via_r[l])))
      return fail_noctx(LA_ERR_INVALID, "la_elmore_static: via_r must be finite and >= 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return fail_noctx(LA_ERR_CUDA, std::string("la_elmore_static: no current CUDA device: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the
    // static array (its host-side name is not a device address)
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p)
        return fail_noctx(LA_ERR_CUDA,
                          std::string("la_elmore_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      g_static_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_static_ptr[dev];
  }
  // Rvia(a, b) travels as a kernel parameter
  RviaTable tab;
  for (int a = 0; a < L; ++a)
    for (int c = 0; c < L; ++c) {
      const int lo = a < c ? a : c, hi = a < c ? c : a;
      double s = 0.0;
      for (int k = lo; k < hi; ++k) s += via_r[k];
      tab.rv[a * L + c] = s;
    }
  const int64_t V = nets->num_nodes, N = nets->num_nets;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* flag = reinterpret_cast<unsigned*>(scratch);
  double* CdJ = scratch + kStaticHeader;
  int32_t* head = reinterpret_cast<int32_t*>(CdJ + V);
  int32_t* next = head + V;
  e = cudaMemsetAsync(flag, 0, sizeof(unsigned), s);  // the flag starts at zero on every call
  if (e != cudaSuccess)
    return fail_noctx(LA_ERR_CUDA, std::string("la_elmore_static: clearing the flag failed: ") + cudaGetErrorString(e));
  k_static_check_netptr<<<(unsigned)((N + 1 + 255) / 256), 256, 0, s>>>(N, V, nets->net_ptr, flag);
  k_elmore_static<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(
      N, nets->net_ptr, nets->parent, nets->pin_layer, nets->sink_cap, nets->r_drv, layer, b, t, R_seg, C_seg,
      delay, L, via_c, tab, flag, CdJ, head, next, V);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail_noctx(LA_ERR_CUDA, std::string("la_elmore_static: launch failed: ") + cudaGetErrorString(e));
  return LA_OK;
}
