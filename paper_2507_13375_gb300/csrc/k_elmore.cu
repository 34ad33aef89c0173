// k_elmore.cu - Elmore delay on the RC tree of an assignment (Sec. II-C, and the
// worked example d_34 = R_34 (C4 + C5 + C6 + C7) of Sec. III-D) and its adjoint.
//
// RC tree: driver R into the root junction J_root; for a segment v, a via
// resistor Rvia(l_p, l_v) from J_p to X_v (C_seg/2 at X_v), the wire R_seg[v]
// from X_v to J_v (C_seg/2 + vc (t - b) + the pin cap below J_v); at a pin
// node a via resistor Rvia(l_v, p_v) to the pin point holding the sink cap.
// Level passes in internal order: downstream caps bottom-up (levels
// ascending), delays and upstream weighted resistances top-down (levels
// descending); every thread one node, its sons' values gathered.  Sums over
// sons run in son order, and every value is the oracle's expression, so the
// results equal the oracle's bit for bit.  On GB300 these passes are bound by
// FP64 issue (1/64 of FP32), not by HBM: each value is computed once - the
// bottom-up pass keeps every node's C_seg / 2 and R_seg for its parent and
// for the top-down pass, and via counts come from a table of doubles.
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
  const double len = exact_int_to_double(unsigned(geo_len(geo[v])));
  R[o] = len * tab->unit_r[l];
  C[o] = len * tab->unit_c[l];
}

void launch_rc_from_assignment(la_ctx* c, double* R, double* C, const int32_t* perm, cudaStream_t s) {
  Forest& f = c->forest;
  k_rc<<<(unsigned)((f.V + 255) / 256), 256, 0, s>>>(f.V, c->grid.tab_dev, f.parent_g, f.geo, f.layer, perm, R, C);
  ++c->launches;
}

struct ElmArgs {
  const int32_t *parent_g, *child_start, *nch, *child_list, *son0, *net_of;
  const uint64_t* geo;  // R or C null: R_seg / C_seg from the geometry and the layer
  const int32_t* out_perm;  // k_elm_delay: delay[out_perm[v]] (input order), or delay[v]
  int64_t base, count;
  const int8_t *layer, *b, *t, *pin;
  const double *sink_cap, *r_drv, *R, *C, *g;
  const DevTables* tab;
  double *CdJ, *Ws, *dJ, *delay, *UJ, *dR, *dC;
  double *CX, *RS;  // forward: C_seg / 2 + Cd_J and R_seg of every node, kept by the bottom-up pass
  double vck[kMaxL];  // via_c x k, k = 0 .. kMaxL - 1 (the products the expressions take)
};

// 0.5 x: exact for a finite x >= 0, by one less in the exponent where the
// result stays normal (GB300 issues FP64 at 1/64 of FP32; this is integer).
__device__ __forceinline__ double half_exact(double x) {
  const long long b = __double_as_longlong(x);
  const long long e = b >> 52;  // biased exponent (x >= 0)
  return (e >= 2 && e < 2047) ? __longlong_as_double(b - (1LL << 52)) : 0.5 * x;
}

// R_seg and C_seg of node v: the given arrays, or the assignment's len x unit
// R / unit C of v's layer (the expressions of k_rc; 0 at roots).
__device__ __forceinline__ double seg_r(const ElmArgs& a, int v) {
  if (a.R) return a.R[v];
  return a.parent_g[v] < 0 ? 0.0 : exact_int_to_double(unsigned(geo_len(a.geo[v]))) * a.tab->unit_r[a.layer[v]];
}
__device__ __forceinline__ double seg_c(const ElmArgs& a, int v) {
  if (a.C) return a.C[v];
  return a.parent_g[v] < 0 ? 0.0 : exact_int_to_double(unsigned(geo_len(a.geo[v]))) * a.tab->unit_c[a.layer[v]];
}

// Bottom-up: Cd_J(v) = C_seg[v]/2 + vc (t - b) + Cs_v + sum over sons of
// (C_seg[c]/2 + Cd_J(c)); with g, also Ws(v) = g_v + sum over sons of Ws(c).
// With CX (the forward pass) the node's C_seg/2 + Cd_J, and with RS its
// R_seg, are kept for its parent and for the top-down pass (the values the
// expressions would compute again).  A node without a pin has Cs = 0, and
// s + 0.0 = s for the s >= 0 here, so that term is added at pins only.
__global__ void k_elm_up(ElmArgs a) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.count) return;
  const int v = int(a.base + i);
  const double hcv = a.parent_g[v] < 0 ? 0.0 : half_exact(seg_c(a, v));
  if (a.RS) a.RS[v] = seg_r(a, v);
  double s = hcv;
  s = s + a.vck[a.t[v] - a.b[v]];
  if (a.pin[v] >= 0) s = s + a.sink_cap[v];
  // the first son straight from son0 (one dependent load instead of two),
  // the others from the son list
  const int nc = a.nch[v];
  const int c0 = a.son0[v];
  if (nc > 0) s = s + (a.CX ? a.CX[c0] : half_exact(seg_c(a, c0)) + a.CdJ[c0]);
  const int cs = nc > 1 ? a.child_start[v] : 0;
  for (int j = 1; j < nc; ++j) {
    const int c = a.child_list[cs + j];
    s = s + (a.CX ? a.CX[c] : half_exact(seg_c(a, c)) + a.CdJ[c]);
  }
  a.CdJ[v] = s;
  if (a.CX) a.CX[v] = hcv + s;
  if (a.Ws) {
    double w = a.g[v];
    if (nc > 0) w = w + a.Ws[c0];
    for (int j = 1; j < nc; ++j) w = w + a.Ws[a.child_list[cs + j]];
    a.Ws[v] = w;
  }
}

// Bottom-up sums of g alone: Ws(v) = g_v + sum over sons of Ws(c) (the
// expression of k_elm_up, without the caps, which need an assignment).
__global__ void k_wsum(ElmArgs a) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.count) return;
  const int v = int(a.base + i);
  const int nc = a.nch[v];
  double w = a.g[v];
  if (nc > 0) w = w + a.Ws[a.son0[v]];
  const int cs = nc > 1 ? a.child_start[v] : 0;
  for (int j = 1; j < nc; ++j) w = w + a.Ws[a.child_list[cs + j]];
  a.Ws[v] = w;
}

// Top-down forward: delay at junctions, then at the pin point.
__global__ void k_elm_delay(ElmArgs a) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.count) return;
  const int v = int(a.base + i);
  const int p = a.parent_g[v];
  const int lv = a.layer[v];
  double dj;
  if (p < 0) {
    dj = a.r_drv[a.net_of[v]] * a.CdJ[v];
  } else {
    const double cx = a.CX ? a.CX[v] : half_exact(seg_c(a, v)) + a.CdJ[v];
    const double dX = a.dJ[p] + a.tab->rv[a.layer[p] * kRvStride + lv] * cx;
    dj = dX + (a.RS ? a.RS[v] : seg_r(a, v)) * a.CdJ[v];
  }
  a.dJ[v] = dj;
  const int pin = a.pin[v];
  a.delay[a.out_perm ? a.out_perm[v] : v] = pin >= 0 ? dj + a.tab->rv[lv * kRvStride + pin] * a.sink_cap[v] : dj;
}

// Top-down adjoint: U_J(root) = R_drv Ws(root); U_X(v) = U_J(p) + Rvia Ws(v);
// U_J(v) = U_X(v) + R_seg[v] Ws(v); dR = Cd_J Ws; dC = (U_X + U_J) / 2.
__global__ void k_elm_adj(ElmArgs a) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= a.count) return;
  const int v = int(a.base + i);
  const int p = a.parent_g[v];
  if (p < 0) {
    a.UJ[v] = a.r_drv[a.net_of[v]] * a.Ws[v];
    if (a.dR) { a.dR[v] = 0.0; a.dC[v] = 0.0; }
    return;
  }
  const double w = a.Ws[v];
  const int lv = a.layer[v];
  const double Rv = seg_r(a, v);
  const double UX = a.UJ[p] + a.tab->rv[a.layer[p] * kRvStride + lv] * w;
  const double uj = UX + Rv * w;
  a.UJ[v] = uj;
  if (a.dR) {
    a.dR[v] = a.CdJ[v] * w;
    a.dC[v] = half_exact(UX + uj);
  }
}

static ElmArgs elm_args(la_ctx* c, const double* R, const double* C) {
  Forest& f = c->forest;
  ElmArgs a{};
  a.parent_g = f.parent_g; a.child_start = f.child_start; a.nch = f.nch; a.child_list = f.child_list;
  a.son0 = f.son0;
  a.net_of = f.net_of; a.layer = f.layer; a.b = f.b; a.t = f.t; a.pin = f.pin; a.sink_cap = f.sink_cap;
  a.r_drv = f.r_drv; a.R = R; a.C = C; a.tab = c->grid.tab_dev; a.geo = f.geo;
  for (int k = 0; k < kMaxL; ++k) a.vck[k] = c->grid.li.via_c * double(k);
  return a;
}

template <typename K>
static void per_level(la_ctx* c, ElmArgs a, K kernel, bool ascending, cudaStream_t s) {
  Forest& f = c->forest;
  for (int q = 0; q < f.nlev; ++q) {  // global levels: every batch's levels, ascending within it
    const int h = ascending ? q : f.nlev - 1 - q;
    a.base = f.lvl_off[h];
    a.count = f.lvl_off[h + 1] - f.lvl_off[h];
    if (a.count == 0) continue;
    kernel<<<(unsigned)((a.count + 255) / 256), 256, 0, s>>>(a);
    ++c->launches;
  }
}

// Given R_seg, C_seg (input order): gathered into internal order (s3, s4);
// delays written in input order.
void launch_elmore_fwd(la_ctx* c, const double* R, const double* C, double* delay, cudaStream_t s) {
  Forest& f = c->forest;
  launch_permute64(f.V, f.lvl_nodes, R, f.s3, true, s);
  launch_permute64(f.V, f.lvl_nodes, C, f.s4, true, s);
  c->launches += 2;
  ElmArgs a = elm_args(c, f.s3, f.s4);
  a.CdJ = f.s0;
  a.dJ = f.s1;
  a.CX = f.s2;
  a.delay = delay;
  a.out_perm = f.lvl_nodes;
  per_level(c, a, k_elm_up, true, s);
  per_level(c, a, k_elm_delay, false, s);
}

// The delays of the current assignment, with R_seg and C_seg from the layers,
// written in input order.
void launch_elmore_assignment(la_ctx* c, double* delay_input_order, cudaStream_t s) {
  Forest& f = c->forest;
  ElmArgs a = elm_args(c, nullptr, nullptr);
  a.CdJ = f.s0;
  a.dJ = f.s1;
  a.CX = f.s2;
  a.RS = f.s3;
  a.delay = delay_input_order;
  a.out_perm = f.lvl_nodes;
  per_level(c, a, k_elm_up, true, s);
  per_level(c, a, k_elm_delay, false, s);
}

// Given R_seg, C_seg and g (input order): gathered into internal order (s3,
// s4 and the DP's A table, free between rounds); dR, dC through the Cc and M
// tables, scattered to input order.
void launch_elmore_bwd(la_ctx* c, const double* R, const double* C, const double* g, double* dR, double* dC,
                       cudaStream_t s) {
  Forest& f = c->forest;
  double* gi = f.A;
  double* dRi = f.Cc;
  double* dCi = f.M;
  launch_permute64(f.V, f.lvl_nodes, R, f.s3, true, s);
  launch_permute64(f.V, f.lvl_nodes, C, f.s4, true, s);
  launch_permute64(f.V, f.lvl_nodes, g, gi, true, s);
  ElmArgs a = elm_args(c, f.s3, f.s4);
  a.g = gi;
  a.CdJ = f.s0;
  a.Ws = f.s1;
  a.UJ = f.s2;
  a.dR = dRi;
  a.dC = dCi;
  per_level(c, a, k_elm_up, true, s);
  per_level(c, a, k_elm_adj, false, s);
  launch_permute64(f.V, f.lvl_nodes, dRi, dR, false, s);
  launch_permute64(f.V, f.lvl_nodes, dCi, dC, false, s);
  c->launches += 5;
}

// The DP's adjoint weights on the current assignment (R_seg = len x unit R of
// the layer): with_wsum, W_adj = the sums of g = kappa below each node and
// rho_adj = U_J; else rho_adj = U_J from the W_adj already there (the sums
// depend on the forest only).
void launch_reweight(la_ctx* c, bool with_wsum, cudaStream_t s) {
  Forest& f = c->forest;
  ElmArgs a = elm_args(c, nullptr, nullptr);
  a.Ws = f.W_adj;
  a.UJ = f.rho_adj;
  if (with_wsum) {
    a.g = f.gk;
    a.CdJ = f.s0;
    per_level(c, a, k_elm_up, true, s);
  }
  per_level(c, a, k_elm_adj, false, s);
}

void launch_wsum(la_ctx* c, cudaStream_t s) {
  Forest& f = c->forest;
  ElmArgs a = elm_args(c, nullptr, nullptr);
  a.g = f.gk;
  a.Ws = f.W_adj;
  per_level(c, a, k_wsum, true, s);
}

}  // namespace gapla
