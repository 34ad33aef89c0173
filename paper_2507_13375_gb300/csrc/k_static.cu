// k_static.cu - la_elmore_static: the Elmore forward pass without any device
// allocation.  Its scratch (downstream caps and junction delays, 2 doubles per
// node) lives in the fixed file-scope device array below, which every GPU that
// loads the library holds until the process exits.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "gapla_internal.cuh"

namespace gapla {

// 2 * LA_STATIC_MAX_NODES doubles = 32 MiB.
static __device__ __align__(256) double g_static_scratch[2 * LA_STATIC_MAX_NODES];

struct RviaTable {
  double rv[kMaxL * kMaxL];  // Rvia(a, b) at a * L + b
};

// One thread per net; nodes of a net are visited in id order (parents first)
// or reverse id order (sons first), which needs no son lists.  A node whose
// parent id is out of order, or whose layers/pin are out of range, makes the
// whole net's delays NaN (no access outside the given arrays is made).
__global__ void k_elmore_static(int64_t N, const int64_t* __restrict__ net_ptr, const int32_t* __restrict__ parent,
                                const int8_t* __restrict__ pin, const double* __restrict__ sink_cap,
                                const double* __restrict__ r_drv, const int8_t* __restrict__ layer,
                                const int8_t* __restrict__ b, const int8_t* __restrict__ t, const double* __restrict__ R,
                                const double* __restrict__ C, double* __restrict__ delay, int L, double via_c,
                                const __grid_constant__ RviaTable tab, double* __restrict__ CdJ,
                                double* __restrict__ dJ, int64_t V) {
  const double* rv = tab.rv;
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int64_t base = net_ptr[n], end = net_ptr[n + 1];
  if (!(base >= 0 && base < end && end <= V)) return;
  const int64_t m = end - base;
  bool bad = false;
  // own capacitance at each junction: C_seg/2 (not at the root), vias, pin
  for (int64_t i = 0; i < m && !bad; ++i) {
    const int64_t v = base + i;
    const int p = parent[v], l = layer[v], pv = pin[v];
    bad = (i == 0 ? p != -1 : (p < 0 || p >= i)) || l < 0 || l >= L || pv < -1 || pv >= L || b[v] > t[v];
    double s = i == 0 ? 0.0 : 0.5 * C[v];
    s = s + via_c * double(t[v] - b[v]);
    CdJ[v] = s + sink_cap[v];
  }
  if (!bad) {
    // sons before parents: add each son's (C_seg/2 + Cd_J) to its parent
    for (int64_t i = m - 1; i >= 1; --i) {
      const int64_t v = base + i, p = base + parent[v];
      CdJ[p] = CdJ[p] + (0.5 * C[v] + CdJ[v]);
    }
    // parents before sons: junction delays, then the pin point
    for (int64_t i = 0; i < m; ++i) {
      const int64_t v = base + i;
      double dj;
      if (i == 0) {
        dj = r_drv[n] * CdJ[v];
      } else {
        const int64_t p = base + parent[v];
        dj = dJ[p] + rv[layer[p] * L + layer[v]] * (0.5 * C[v] + CdJ[v]) + R[v] * CdJ[v];
      }
      dJ[v] = dj;
      delay[v] = pin[v] >= 0 ? dj + rv[layer[v] * L + pin[v]] * sink_cap[v] : dj;
    }
  } else {
    for (int64_t i = 0; i < m; ++i) delay[base + i] = nan("");
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
  // Rvia(a, b) travels as a kernel parameter; the scratch holds [CdJ V][dJ V]
  RviaTable tab;
  for (int a = 0; a < L; ++a)
    for (int c = 0; c < L; ++c) {
      const int lo = a < c ? a : c, hi = a < c ? c : a;
      double s = 0.0;
      for (int k = lo; k < hi; ++k) s += via_r[k];
      tab.rv[a * L + c] = s;
    }
  const int64_t V = nets->num_nodes, N = nets->num_nets;
  double* CdJ = scratch;
  double* dJ = scratch + V;
  k_elmore_static<<<(unsigned)((N + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      N, nets->net_ptr, nets->parent, nets->pin_layer, nets->sink_cap, nets->r_drv, layer, b, t, R_seg, C_seg,
      delay, L, via_c, tab, CdJ, dJ, V);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail_noctx(LA_ERR_CUDA, std::string("la_elmore_static: launch failed: ") + cudaGetErrorString(e));
  return LA_OK;
}
