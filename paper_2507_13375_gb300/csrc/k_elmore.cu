// k_elmore.cu - Elmore delay on the RC tree of an assignment (Sec. II-C, and the
// worked example d_34 = R_34 (C4 + C5 + C6 + C7) of Sec. III-D) and its adjoint.
//
// RC tree: driver R into the root junction J_root; for a segment v, a via
// resistor Rvia(l_p, l_v) from J_p to X_v (C_seg/2 at X_v), the wire R_seg[v]
// from X_v to J_v (C_seg/2 + vc (t - b) + the pin cap below J_v); at a pin
// node a via resistor Rvia(l_v, p_v) to the pin point holding the sink cap.
// Downstream caps (and adjoint weight sums) bottom-up, delays (and upstream
// weighted resistances) top-down.  Sums over sons run in increasing son id,
// as in the oracle, and every value is the oracle's expression: results are
// equal bit for bit whichever kernel computes a net.
//
// Two kernels share the nets:
//   nets of at most kElmSmall nodes (nearly all nets of the paper-shaped
//   workloads): k_elm_small, in input (net-major) order.  A block stages a
//   group of whole nets in shared memory - the static per-node pack and caps
//   read contiguously, the assignment's bytes and the internal-order weights
//   gathered through the input -> internal map (each gather stream runs
//   monotonically through a (level, class) bucket, so every sector is used) -
//   and one thread sweeps each net in shared memory; outputs in input order
//   are written contiguously, internal-order outputs (the DP's weights) are
//   scattered the same monotone way.
//   larger nets: k_elm_big, one block per net walking the net's level lists
//   (internal order), a barrier between levels.
#include "gapla_internal.cuh"

namespace gapla {

__global__ void k_rc(int64_t V, const DevTables* __restrict__ tab, const int32_t* __restrict__ parent_g,
                     const uint64_t* __restrict__ geo, const int8_t* __restrict__ layer, const int32_t* perm,
                     double* __restrict__ R, double* __restrict__ C) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int64_t o = perm ? perm[v] : v;
  if (parent_g[v] < 0) {
    R[o] = 0.0;
    C[o] = 0.0;
    return;
  }
  const int l = layer[v];
  const double len = double(geo_len(geo[v]));
  R[o] = len * tab->unit_r[l];
  C[o] = len * tab->unit_c[l];
}

void launch_rc_from_assignment(la_ctx* c, double* R, double* C, const int32_t* perm, cudaStream_t s) {
  Forest& f = c->forest;
  k_rc<<<(unsigned)((f.V + 255) / 256), 256, 0, s>>>(f.V, c->grid.tab_dev, f.parent_g, f.geo, f.layer, perm, R, C);
  ++c->launches;
}

// ---------------------------------------------------------------------------
// The input-order pack of the small-net kernel, built once per forest:
// bits 0..31 the node's internal id, 32..47 its segment length, 48..55 pin + 1,
// 56..63 net-local parent id + 1 (0 at a root; nets of at most kElmSmall
// nodes only, larger nets leave the field 0 and are not read through it).
// ---------------------------------------------------------------------------
__global__ void k_elm_pack(int64_t V, const int64_t* __restrict__ net_ptr, const int32_t* __restrict__ net_of,
                           const int32_t* __restrict__ parent_g, const uint64_t* __restrict__ geo,
                           const int8_t* __restrict__ pin, const double* __restrict__ cap,
                           const int32_t* __restrict__ in2int, uint64_t* __restrict__ ep, double* __restrict__ ecap) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const int n = net_of[v];
  const int64_t base = net_ptr[n], m = net_ptr[n + 1] - base;
  const int p = parent_g[v];
  const uint64_t par1 = (p < 0 || m > kElmSmall) ? 0u : uint64_t(p - base + 1);
  ep[v] = uint64_t(uint32_t(in2int[v])) | (uint64_t(geo_len(geo[v])) << 32) | (uint64_t(uint8_t(pin[v] + 1)) << 48) |
          (par1 << 56);
  ecap[v] = cap[v];
}

void launch_elm_pack(const Forest& in, const int32_t* in2int, Forest& out, cudaStream_t s) {
  k_elm_pack<<<(unsigned)((in.V + 255) / 256), 256, 0, s>>>(in.V, in.net_ptr, in.net_of, in.parent_g, in.geo, in.pin,
                                                            in.sink_cap, in2int, out.ep, out.ecap);
}

// What one pass computes.
enum ElmMode : int {
  EM_FWD_ASSIGN = 0,   // delays of the assignment (R, C from the layers), input order
  EM_FWD_GIVEN = 1,    // delays from given R_seg, C_seg (input order)
  EM_REWEIGHT_WS = 2,  // W = sum of g below (g = kappa at pins), then r_est = U_J: DP weights, internal order
  EM_REWEIGHT_U = 3,   // r_est = U_J from the W already there
  EM_BWD_GIVEN = 4,    // dL/dR_seg, dL/dC_seg from given R_seg, C_seg, g (input order)
};
__host__ __device__ constexpr bool em_needs_cd(int m) { return m == EM_FWD_ASSIGN || m == EM_FWD_GIVEN || m == EM_BWD_GIVEN; }
__host__ __device__ constexpr bool em_needs_ws(int m) { return m == EM_REWEIGHT_WS || m == EM_BWD_GIVEN; }
__host__ __device__ constexpr bool em_fwd(int m) { return m == EM_FWD_ASSIGN || m == EM_FWD_GIVEN; }
__host__ __device__ constexpr bool em_given(int m) { return m == EM_FWD_GIVEN || m == EM_BWD_GIVEN; }

struct ElmArgs {
  int64_t N;
  const int64_t* net_ptr;          // input ids
  const uint64_t* ep;              // input-order pack (small nets)
  const double* ecap;              // input-order sink caps
  const double* r_drv;             // per net
  // internal order
  const int32_t *parent_g, *child_start, *nch, *child_list, *net_of, *lvl_nodes;
  const uint64_t* geo;
  const int8_t *layer, *b, *t, *pin;
  const double *sink_cap, *gk;
  // given R_seg, C_seg, g (input order), or null
  const double *R, *C, *g;
  const DevTables* tab;
  // outputs: delay, dR, dC input order; W, rho internal order
  double *delay, *dR, *dC, *W, *rho;
  // big-net scratch, internal order
  double *CdJ, *X, *UJ;
};

// ---------------------------------------------------------------------------
// Small nets: block of kElmT threads, groups of kElmT nets, at most kElmCap
// nodes staged per pass (kElmCap / kElmT slots per thread, every load of a
// thread's slots issued before the first use).  Shared memory holds only what
// the mode reads: R_seg and C_seg as the segment length (times the layer's
// unit R and C, the expressions of la_rc_from_assignment) unless given.
// ---------------------------------------------------------------------------
constexpr int kElmT = 128, kElmCap = 1024, kElmSlots = kElmCap / kElmT;

template <int MODE>
struct ElmSmem {
  static constexpr bool kGiven = em_given(MODE), kCd = em_needs_cd(MODE), kWs = em_needs_ws(MODE);
  static constexpr bool kW = MODE == EM_REWEIGHT_WS || MODE == EM_REWEIGHT_U || MODE == EM_BWD_GIVEN;
  static constexpr bool kIid = MODE == EM_REWEIGHT_WS || MODE == EM_REWEIGHT_U;
  static constexpr bool kLinks = kCd || kWs;
  double x[kElmCap];                       // Cd_J, then junction delay, then delay; or U_J
  double w[kW ? kElmCap : 1];              // g, then the sums of g below
  double u[MODE == EM_BWD_GIVEN ? kElmCap : 1];
  double R[kGiven ? kElmCap : 1], C[kGiven ? kElmCap : 1];
  double cap[kCd ? kElmCap : 1];
  double rv[kMaxL * kMaxL], ur[kMaxL], uc[kMaxL];
  int64_t base[kElmT];
  int32_t iid[kIid ? kElmCap : 1];
  int32_t off[kElmT + 1];                  // staged offsets of the pass's nets (off[cnt] = total)
  int32_t wsum[kElmT / 32];
  uint16_t len[kGiven ? 1 : kElmCap];
  int8_t par[kElmCap], lay[kElmCap], netof[kElmCap];
  int8_t pin[em_fwd(MODE) ? kElmCap : 1], nv[kCd ? kElmCap : 1];
  int8_t head[kLinks ? kElmCap : 1], next[kLinks ? kElmCap : 1];
};

template <int MODE>
__global__ void __launch_bounds__(kElmT) k_elm_small(ElmArgs a) {
  using SM = ElmSmem<MODE>;
  extern __shared__ __align__(16) unsigned char s_raw[];
  SM& S = *reinterpret_cast<SM*>(s_raw);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int i = tid; i < kMaxL * kMaxL; i += kElmT) S.rv[i] = a.tab->rv[i];
  if (tid < kMaxL) {
    S.ur[tid] = a.tab->unit_r[tid];
    S.uc[tid] = a.tab->unit_c[tid];
  }
  const double vc = a.tab->via_c;
  for (int64_t g0 = int64_t(blockIdx.x) * kElmT; g0 < a.N; g0 += int64_t(gridDim.x) * kElmT) {
    const int ng = int(a.N - g0 < kElmT ? a.N - g0 : int64_t(kElmT));
    int k = 0;  // nets of the group done
    while (k < ng) {
      // the pass: nets g0 + k + j, j < cnt, whose sizes sum to at most kElmCap
      const int j = tid;
      int m = 0;
      int64_t nb = 0;
      if (k + j < ng) {
        const int64_t n = g0 + k + j;
        nb = a.net_ptr[n];
        const int64_t mm = a.net_ptr[n + 1] - nb;
        m = mm <= kElmSmall ? int(mm) : 0;  // larger nets: the block-per-net kernel
      }
      int incl = m;  // inclusive block scan of m
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) S.wsum[wid] = incl;
      __syncthreads();
      for (int w2 = 0; w2 < wid; ++w2) incl += S.wsum[w2];
      const bool fits = (k + j < ng) && incl <= kElmCap;
      const int cnt = __syncthreads_count(fits);  // a prefix of the threads (sizes <= kElmSmall <= kElmCap)
      const int o = incl - m;
      if (j < cnt) {
        S.off[j] = o;
        S.base[j] = nb;
        if (j == cnt - 1) S.off[cnt] = incl;
        for (int i = 0; i < m; ++i) S.netof[o + i] = int8_t(j);
      }
      __syncthreads();
      const int total = S.off[cnt];
      // stage: slot q = tid + u kElmT holds node q of the pass
      {
        int64_t gid[kElmSlots];
        uint64_t e[kElmSlots];
#pragma unroll
        for (int u = 0; u < kElmSlots; ++u) {
          const int q = tid + u * kElmT;
          gid[u] = -1;
          if (q < total) {
            const int jj = S.netof[q];
            gid[u] = S.base[jj] + (q - S.off[jj]);
          }
        }
#pragma unroll
        for (int u = 0; u < kElmSlots; ++u) e[u] = gid[u] >= 0 ? a.ep[gid[u]] : 0;
        double c1[kElmSlots], c2[kElmSlots], c3[kElmSlots];
#pragma unroll
        for (int u = 0; u < kElmSlots; ++u) {
          c1[u] = c2[u] = c3[u] = 0.0;
          if (gid[u] >= 0) {
            if constexpr (SM::kCd) c1[u] = a.ecap[gid[u]];
            if constexpr (SM::kGiven) {
              c2[u] = a.R[gid[u]];
              c3[u] = a.C[gid[u]];
            }
          }
        }
        int8_t l1[kElmSlots], nv1[kElmSlots];
        double w1[kElmSlots];
#pragma unroll
        for (int u = 0; u < kElmSlots; ++u) {
          l1[u] = 0;
          nv1[u] = 0;
          w1[u] = 0.0;
          if (gid[u] >= 0) {
            const int32_t iv = int32_t(uint32_t(e[u]));
            l1[u] = a.layer[iv];
            if constexpr (SM::kCd) nv1[u] = int8_t(a.t[iv] - a.b[iv]);
            if constexpr (MODE == EM_REWEIGHT_WS) w1[u] = a.gk[iv];
            if constexpr (MODE == EM_REWEIGHT_U) w1[u] = a.W[iv];
            if constexpr (MODE == EM_BWD_GIVEN) w1[u] = a.g[gid[u]];
          }
        }
#pragma unroll
        for (int u = 0; u < kElmSlots; ++u) {
          const int q = tid + u * kElmT;
          if (gid[u] >= 0) {
            S.par[q] = int8_t(int((e[u] >> 56) & 0xFF) - 1);
            S.lay[q] = l1[u];
            if constexpr (em_fwd(MODE)) S.pin[q] = int8_t(int((e[u] >> 48) & 0xFF) - 1);
            if constexpr (SM::kCd) {
              S.cap[q] = c1[u];
              S.nv[q] = nv1[u];
            }
            if constexpr (SM::kGiven) {
              S.R[q] = c2[u];
              S.C[q] = c3[u];
            } else {
              S.len[q] = uint16_t((e[u] >> 32) & 0xFFFF);
            }
            if constexpr (SM::kW) S.w[q] = w1[u];
            if constexpr (SM::kIid) S.iid[q] = int32_t(uint32_t(e[u]));
          }
        }
      }
      __syncthreads();
      if (j < cnt && m > 0) {
        const int64_t n = g0 + k + j;
        // R_seg, C_seg of local node i (0 at the root)
        auto segR = [&](int i) -> double {
          if constexpr (SM::kGiven) return S.R[o + i];
          else return i == 0 ? 0.0 : double(S.len[o + i]) * S.ur[S.lay[o + i]];
        };
        auto segC = [&](int i) -> double {
          if constexpr (SM::kGiven) return S.C[o + i];
          else return i == 0 ? 0.0 : double(S.len[o + i]) * S.uc[S.lay[o + i]];
        };
        if constexpr (SM::kLinks) {
          // son lists in increasing local id
          for (int i = 0; i < m; ++i) S.head[o + i] = -1;
          for (int i = m - 1; i >= 1; --i) {
            const int p = S.par[o + i];
            S.next[o + i] = S.head[o + p];
            S.head[o + p] = int8_t(i);
          }
          // sons before parents: Cd_J and the sums of g below
          for (int i = m - 1; i >= 0; --i) {
            if constexpr (SM::kCd) {
              double sum = i == 0 ? 0.0 : 0.5 * segC(i);
              sum = sum + vc * double(S.nv[o + i]);
              sum = sum + S.cap[o + i];
              for (int c = S.head[o + i]; c >= 0; c = S.next[o + c]) sum = sum + (0.5 * segC(c) + S.x[o + c]);
              S.x[o + i] = sum;
            }
            if constexpr (SM::kWs) {
              double w = S.w[o + i];
              for (int c = S.head[o + i]; c >= 0; c = S.next[o + c]) w = w + S.w[o + c];
              S.w[o + i] = w;
            }
          }
        }
        const double rd = a.r_drv[n];
        if constexpr (em_fwd(MODE)) {
          // parents before sons: junction delays (over Cd_J), then the pin points
          S.x[o] = rd * S.x[o];
          for (int i = 1; i < m; ++i) {
            const int p = S.par[o + i];
            const double cd = S.x[o + i];
            const double dX = S.x[o + p] + S.rv[S.lay[o + p] * kMaxL + S.lay[o + i]] * (0.5 * segC(i) + cd);
            S.x[o + i] = dX + segR(i) * cd;
          }
          for (int i = 0; i < m; ++i) {
            const int pn = S.pin[o + i];
            if (pn >= 0) S.x[o + i] = S.x[o + i] + S.rv[S.lay[o + i] * kMaxL + pn] * S.cap[o + i];
          }
        } else {
          // parents before sons: U_J (r_est of the next round), and dR, dC
          double* U = MODE == EM_BWD_GIVEN ? S.u : S.x;
          U[o] = rd * S.w[o];
          if constexpr (MODE == EM_BWD_GIVEN) {
            S.R[o] = 0.0;  // dR, dC of the root
            S.C[o] = 0.0;
          }
          for (int i = 1; i < m; ++i) {
            const int p = S.par[o + i];
            const double w = S.w[o + i];
            const double UX = U[o + p] + S.rv[S.lay[o + p] * kMaxL + S.lay[o + i]] * w;
            const double uj = UX + segR(i) * w;
            U[o + i] = uj;
            if constexpr (MODE == EM_BWD_GIVEN) {
              S.R[o + i] = S.x[o + i] * w;  // dR = Cd_J Ws (R_seg of this node no longer needed)
              S.C[o + i] = 0.5 * (UX + uj);
            }
          }
        }
      }
      __syncthreads();
      // write the pass's results
#pragma unroll
      for (int u = 0; u < kElmSlots; ++u) {
        const int q = tid + u * kElmT;
        if (q < total) {
          if constexpr (SM::kIid) {
            const int32_t iv = S.iid[q];
            if constexpr (MODE == EM_REWEIGHT_WS) a.W[iv] = S.w[q];
            a.rho[iv] = S.x[q];
          } else {
            const int jj = S.netof[q];
            const int64_t gid = S.base[jj] + (q - S.off[jj]);
            if constexpr (em_fwd(MODE)) {
              a.delay[gid] = S.x[q];
            } else {
              a.dR[gid] = S.R[q];
              a.dC[gid] = S.C[q];
            }
          }
        }
      }
      __syncthreads();
      k += cnt;
    }
  }
}

// ---------------------------------------------------------------------------
// Large nets: one block per net (the nets of more than kElmSmall nodes, at
// the head of the big-net queue, largest first), the net's nodes level by
// level from its level lists (internal ids).  Per node the expressions of the
// small-net kernel.
// ---------------------------------------------------------------------------
struct BigNets {
  const int32_t* queue;
  int64_t n_big;
  const int32_t *bl_nodes, *bl_hoff, *net_H;
};

__device__ __forceinline__ double big_r(const ElmArgs& a, int MODE_GIVEN, int v) {
  if (MODE_GIVEN) return a.R[a.lvl_nodes[v]];
  return a.parent_g[v] < 0 ? 0.0 : double(geo_len(a.geo[v])) * a.tab->unit_r[a.layer[v]];
}
__device__ __forceinline__ double big_c(const ElmArgs& a, int MODE_GIVEN, int v) {
  if (MODE_GIVEN) return a.C[a.lvl_nodes[v]];
  return a.parent_g[v] < 0 ? 0.0 : double(geo_len(a.geo[v])) * a.tab->unit_c[a.layer[v]];
}

template <int MODE>
__global__ void __launch_bounds__(128) k_elm_big(ElmArgs a, BigNets bn) {
  constexpr int GV = em_given(MODE) ? 1 : 0;
  const double vc = a.tab->via_c;
  double* Ws = MODE == EM_BWD_GIVEN ? a.X : a.W;   // sums of g below (internal order)
  double* U = MODE == EM_BWD_GIVEN ? a.UJ : a.rho; // U_J (internal order)
  for (int64_t q = blockIdx.x; q < bn.n_big; q += gridDim.x) {
    const int n = bn.queue[q];
    const int64_t base = a.net_ptr[n];
    const int32_t* ho = bn.bl_hoff + base + n;
    const int H = bn.net_H[n];
    if constexpr (em_needs_cd(MODE) || em_needs_ws(MODE)) {
      for (int h = 0; h <= H; ++h) {
        const int lo = ho[h], cnt = ho[h + 1] - lo;
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
          const int v = bn.bl_nodes[base + lo + i];
          const int cs = a.child_start[v], nc = a.nch[v];
          if constexpr (em_needs_cd(MODE)) {
            double s = a.parent_g[v] < 0 ? 0.0 : 0.5 * big_c(a, GV, v);
            s = s + vc * double(a.t[v] - a.b[v]);
            s = s + a.sink_cap[v];
            for (int jj = 0; jj < nc; ++jj) {
              const int c = a.child_list[cs + jj];
              s = s + (0.5 * big_c(a, GV, c) + a.CdJ[c]);
            }
            a.CdJ[v] = s;
          }
          if constexpr (em_needs_ws(MODE)) {
            double w = MODE == EM_BWD_GIVEN ? a.g[a.lvl_nodes[v]] : a.gk[v];
            for (int jj = 0; jj < nc; ++jj) w = w + Ws[a.child_list[cs + jj]];
            Ws[v] = w;
          }
        }
        __syncthreads();
      }
    }
    for (int h = H; h >= 0; --h) {
      const int lo = ho[h], cnt = ho[h + 1] - lo;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int v = bn.bl_nodes[base + lo + i];
        const int p = a.parent_g[v];
        const int lv = a.layer[v];
        if constexpr (em_fwd(MODE)) {
          double dj;
          if (p < 0) {
            dj = a.r_drv[n] * a.CdJ[v];
          } else {
            const double dX = a.X[p] + a.tab->rv[a.layer[p] * kMaxL + lv] * (0.5 * big_c(a, GV, v) + a.CdJ[v]);
            dj = dX + big_r(a, GV, v) * a.CdJ[v];
          }
          a.X[v] = dj;
          const int pn = a.pin[v];
          a.delay[a.lvl_nodes[v]] = pn >= 0 ? dj + a.tab->rv[lv * kMaxL + pn] * a.sink_cap[v] : dj;
        } else {
          const double w = Ws[v];
          if (p < 0) {
            U[v] = a.r_drv[n] * w;
            if constexpr (MODE == EM_BWD_GIVEN) {
              a.dR[a.lvl_nodes[v]] = 0.0;
              a.dC[a.lvl_nodes[v]] = 0.0;
            }
          } else {
            const double UX = U[p] + a.tab->rv[a.layer[p] * kMaxL + lv] * w;
            const double uj = UX + big_r(a, GV, v) * w;
            U[v] = uj;
            if constexpr (MODE == EM_BWD_GIVEN) {
              a.dR[a.lvl_nodes[v]] = a.CdJ[v] * w;
              a.dC[a.lvl_nodes[v]] = 0.5 * (UX + uj);
            }
          }
        }
      }
      __syncthreads();
    }
  }
}

static ElmArgs elm_args(la_ctx* c) {
  Forest& f = c->forest;
  ElmArgs a{};
  a.N = f.N;
  a.net_ptr = f.net_ptr; a.ep = f.ep; a.ecap = f.ecap; a.r_drv = f.r_drv;
  a.parent_g = f.parent_g; a.child_start = f.child_start; a.nch = f.nch; a.child_list = f.child_list;
  a.net_of = f.net_of; a.lvl_nodes = f.lvl_nodes; a.geo = f.geo;
  a.layer = f.layer; a.b = f.b; a.t = f.t; a.pin = f.pin; a.sink_cap = f.sink_cap; a.gk = f.gk;
  a.tab = c->grid.tab_dev;
  a.CdJ = f.s0; a.X = f.s1; a.UJ = f.s2;
  return a;
}

// The nets of more than kElmSmall nodes (size class above log2 kElmSmall):
// the head of the big-net queue, which runs by size class, largest first.
static int64_t big_elm_nets(const Forest& f) {
  int64_t n = 0;
  for (int sc = 0; sc < kSizeClasses; ++sc)
    if ((int64_t(1) << sc) > kElmSmall) n += f.big_sc_cnt[sc];
  return n;
}

// The small-net kernel on the context's stream and, beside it on the second
// stream, the block-per-net kernel of the large nets (latency-bound level
// walks that overlap the small nets' bandwidth-bound sweep).
template <int MODE>
static void elm_launch(la_ctx* c, const ElmArgs& a, cudaStream_t s) {
  Forest& f = c->forest;
  const size_t smem = sizeof(ElmSmem<MODE>);
  cudaFuncSetAttribute(k_elm_small<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_elm_small<MODE>, kElmT, smem);
  const int64_t groups = (f.N + kElmT - 1) / kElmT;
  const int grid = int(std::min<int64_t>(groups, int64_t(sms) * std::max(per_sm, 1) * 4));
  const int64_t nb = big_elm_nets(f);
  if (nb > 0) {
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(c->s2, c->ev_fork, 0);
    BigNets bn{f.big_queue, nb, f.bl_nodes, f.bl_hoff, f.net_H};
    k_elm_big<MODE><<<(unsigned)std::min<int64_t>(nb, int64_t(sms) * 16), 128, 0, c->s2>>>(a, bn);
    ++c->launches;
  }
  k_elm_small<MODE><<<grid, kElmT, smem, s>>>(a);
  ++c->launches;
  if (nb > 0) {
    cudaEventRecord(c->ev_join, c->s2);
    cudaStreamWaitEvent(s, c->ev_join, 0);
  }
}

void launch_elmore_fwd(la_ctx* c, const double* R, const double* C, double* delay, cudaStream_t s) {
  ElmArgs a = elm_args(c);
  a.R = R;
  a.C = C;
  a.delay = delay;
  elm_launch<EM_FWD_GIVEN>(c, a, s);
}

void launch_elmore_assignment(la_ctx* c, double* delay, cudaStream_t s) {
  ElmArgs a = elm_args(c);
  a.delay = delay;
  elm_launch<EM_FWD_ASSIGN>(c, a, s);
}

void launch_elmore_bwd(la_ctx* c, const double* R, const double* C, const double* g, double* dR, double* dC,
                       cudaStream_t s) {
  ElmArgs a = elm_args(c);
  a.R = R;
  a.C = C;
  a.g = g;
  a.dR = dR;
  a.dC = dC;
  elm_launch<EM_BWD_GIVEN>(c, a, s);
}

void launch_reweight(la_ctx* c, bool with_wsum, cudaStream_t s) {
  Forest& f = c->forest;
  ElmArgs a = elm_args(c);
  a.W = f.W_adj;
  a.rho = f.rho_adj;
  if (with_wsum) elm_launch<EM_REWEIGHT_WS>(c, a, s);
  else elm_launch<EM_REWEIGHT_U>(c, a, s);
}

}  // namespace gapla
