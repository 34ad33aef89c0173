// k_round.cu - one layer-assignment round on the GPU: congestion penalty and
// line prefix (reading of Eq. 3), the bottom-up DP of Alg. 3 (Kernel 1 and
// Kernel 2 fused: per node and parent-edge layer, enumerate the via stacks,
// let every son take its best layer by look-ahead cost (Sec. III-D), keep the
// stack of least f'), the top-down backtrack of Alg. 4, and the demand / via
// update of the demand map D (Alg. 2).
//
// Arithmetic is FP64 with the oracle's expression trees: nvcc --fmad=false,
// fma() exactly where the oracle calls fma().  Minima over non-negative
// doubles compare their bit patterns as int64 (exact, and it keeps the
// comparisons off the FP64 pipe, which GB300 runs at 1/64 of FP32).
#include <algorithm>
#include <cfloat>
#include <climits>

#include "gapla_internal.cuh"

namespace gapla {

// ---------------------------------------------------------------------------
// Penalty + prefix per line.  One block per (direction, line).  The block
// walks the line in rows of kScanT edge positions, thread j on position
// row*kScanT + j for every layer of the direction (so a warp reads 32 * nld
// contiguous elements).  Per row and layer: a warp shuffle scan, the warp
// totals through shared memory (double-buffered by row parity, so one
// barrier per scan), and the carry of the rows before.  from_diff = 1 also
// folds the demand difference array into D (and clears it), updates
// H += max(0, D - C) and accumulates the overflow statistics of the new demand.
// ---------------------------------------------------------------------------
struct ScanArgs {
  int32_t *cap, *D, *H, *diff;
  int64_t* P;
  const int64_t* T;         // [L][2][129]
  const double* tofT;       // [L][2][257] = ofw_l exp(s over), over in [-128, 128]
  int64_t HW;
  int from_diff;
  double* tof_part;         // one per block
  unsigned long long* relu;
  // fused demand: the segments of line g are seg_node / seg_geo[seg_off[g] ..
  // seg_off[g + 1]); their layers; WL per layer into stats
  const int64_t* seg_off;
  const int32_t* seg_node;
  const uint64_t* seg_geo;
  const int8_t* layer;
  Stats* stats;
};

constexpr int kScanT = 256, kScanW = kScanT / 32;

template <typename Tv>
__device__ __forceinline__ Tv warp_incl_scan(Tv x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Tv y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// NLD bounds the layers of one direction (4, 6, 8 or 16 variants).
// The direction's penalty table sits in shared memory (it is on the path from
// D to the second scan); every global load of a row is issued before the
// row's first barrier.
// FUSED: the demand update of the round, too.  The block first adds its own
// line's segments (+1 at the first edge, -1 past the last) into the line's
// difference array in dynamic shared memory (shared atomics, integer: exact in
// any order), then scans it: no global difference array and no global atomics.
template <int NLD, bool FUSED>
__global__ void __launch_bounds__(kScanT, (NLD <= 8 ? 3 : 1)) k_scan_lines(const DevTables* __restrict__ tab, ScanArgs a) {
  extern __shared__ int32_t s_line[];  // FUSED: [npos][nld] difference array of this line
  __shared__ int32_t s_wd[2][kScanW][NLD];
  __shared__ int64_t s_wp[2][kScanW][NLD];
  __shared__ int64_t s_T[NLD][2][129];
  __shared__ int s_lay[NLD];
  __shared__ int32_t s_cD[2][NLD];  // carries into the row: D and P per layer
  __shared__ int64_t s_cP[2][NLD];
  __shared__ double s_tof[kScanW];
  __shared__ unsigned long long s_relu[kScanW];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gl = blockIdx.x;
  const int nl0 = tab->nlines[0];
  const int d = gl < nl0 ? 0 : 1;
  const int64_t line = gl - (d ? nl0 : 0);
  const int nld = tab->nld[d], npos = tab->npos[d];
  const int64_t base = tab->grid_off[d] + line * npos * nld;
  for (int i = threadIdx.x; i < nld * 2 * 129; i += kScanT) {
    const int q = i / 258, r = i - q * 258;
    (&s_T[q][0][0])[r] = a.T[int(tab->lay[d][q]) * 258 + r];
  }
  if (threadIdx.x < NLD) {
    s_lay[threadIdx.x] = tab->lay[d][threadIdx.x];
    s_cD[0][threadIdx.x] = 0;
    s_cP[0][threadIdx.x] = 0;
  }
  __shared__ unsigned long long s_wl[kMaxL];
  __shared__ int8_t s_ldof[kMaxL];
  if constexpr (FUSED) {
    if (threadIdx.x < kMaxL) {
      s_wl[threadIdx.x] = 0;
      s_ldof[threadIdx.x] = tab->ld_of[threadIdx.x];
    }
    for (int i = threadIdx.x; i < npos * nld; i += kScanT) s_line[i] = 0;
  }
  __syncthreads();
  if constexpr (FUSED) {
    // four segments per thread per step, every load issued before the first
    // atomic; the step count is the same in every lane
    constexpr int kU = 4;
    const int64_t k0 = a.seg_off[gl], k1 = a.seg_off[gl + 1];
    for (int64_t kb = k0; kb < k1; kb += kU * kScanT) {
      int vq[kU];
      uint64_t gq[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t k = kb + u * kScanT + threadIdx.x;
        vq[u] = k < k1 ? __ldcs(a.seg_node + k) : -1;
        gq[u] = k < k1 ? __ldcs(reinterpret_cast<const unsigned long long*>(a.seg_geo) + k) : 0;
      }
      int lq[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) lq[u] = vq[u] >= 0 ? int(a.layer[vq[u]]) : -1;
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int l = lq[u];
        const unsigned len = l >= 0 ? unsigned(geo_len(gq[u])) : 0u;
        if (l >= 0) {
          const int ld = s_ldof[l], lo = geo_lo(gq[u]);
          atomicAdd(&s_line[lo * nld + ld], 1);
          atomicAdd(&s_line[(lo + int(len)) * nld + ld], -1);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, l);
        const unsigned wsum = __reduce_add_sync(peers, len);
        if (l >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s_wl[l], (unsigned long long)wsum);
      }
    }
    __syncthreads();
  }
  double tof = 0.0;
  unsigned long long relu = 0;
  int buf = 0;
  for (int r0 = 0; r0 < npos; r0 += kScanT, buf ^= 1) {
    const int pos = r0 + int(threadIdx.x);
    const bool valid = pos < npos;
    const bool edge = pos < npos - 1;
    const int64_t row = base + int64_t(pos) * nld;
    int32_t Dv[NLD], cv[NLD], hv[NLD];
#pragma unroll
    for (int q = 0; q < NLD; ++q) {
      if (q < nld) {
        if constexpr (FUSED) Dv[q] = valid ? s_line[pos * nld + q] : 0;
        else Dv[q] = (a.from_diff == 1 || a.from_diff == 2) ? (valid ? a.diff[row + q] : 0) : (edge ? a.D[row + q] : 0);
        cv[q] = edge ? a.cap[row + q] : 0;
        hv[q] = edge ? a.H[row + q] : 0;
      }
    }
    if (a.from_diff == 1 || a.from_diff == 2) {
#pragma unroll
      for (int q = 0; q < NLD; ++q) {
        if (q < nld) {
          if (!FUSED && valid) a.diff[row + q] = 0;
          Dv[q] = warp_incl_scan<int32_t>(Dv[q], lane);
          if (lane == 31) s_wd[buf][w][q] = Dv[q];
        }
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NLD; ++q) {
        if (q < nld) {
          int32_t off = s_cD[buf][q], tot = off;
#pragma unroll
          for (int w2 = 0; w2 < kScanW; ++w2) {
            const int32_t x = s_wd[buf][w2][q];
            if (w2 < w) off += x;
            tot += x;
          }
          Dv[q] += off;
          if (threadIdx.x == 0) s_cD[buf ^ 1][q] = tot;
          if (!FUSED && a.from_diff == 2 && edge) Dv[q] += a.D[row + q];  // a batch's change on top
          if (edge) a.D[row + q] = Dv[q];
        }
      }
    }
    int64_t pex[NLD];
#pragma unroll
    for (int q = 0; q < NLD; ++q) {
      if (q < nld) {
        int64_t pen = 0;
        if (edge) {
          const int32_t c = cv[q];
          int32_t h = hv[q];
          const int si = c > 0 ? 0 : 1;
          if (a.from_diff == 1 || a.from_diff == 3) {
            const int32_t over = Dv[q] - c;
            const int l = s_lay[q];
            if (over > 0) { h += over; a.H[row + q] = h; relu += (unsigned long long)over; }
            if (over >= -128 && over <= 128) tof += a.tofT[(l * 2 + si) * 257 + (over + 128)];
            else tof += a.tofT[(l * 2 + si) * 257 + 128] * exp((si ? 1.5 : 0.5) * double(over));
          }
          int kk = Dv[q] + 1 - c;
          kk = kk < -64 ? -64 : (kk > 64 ? 64 : kk);
          const int64_t tv = s_T[q][si][kk + 64];
          if (h > 0 && a.HW > 0 && int64_t(h) > (kPenMax - tv) / a.HW) pen = kPenMax;
          else pen = tv + a.HW * int64_t(h);
          if (pen > kPenMax) pen = kPenMax;
        }
        const int64_t incl = warp_incl_scan<int64_t>(pen, lane);
        pex[q] = incl - pen;
        if (lane == 31) s_wp[buf][w][q] = incl;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NLD; ++q) {
      if (q < nld) {
        int64_t off = s_cP[buf][q], tot = off;
#pragma unroll
        for (int w2 = 0; w2 < kScanW; ++w2) {
          const int64_t x = s_wp[buf][w2][q];
          if (w2 < w) off += x;
          tot += x;
        }
        if (valid) a.P[row + q] = off + pex[q];
        if (threadIdx.x == 0) s_cP[buf ^ 1][q] = tot;
      }
    }
  }
  // deterministic block reduction of the statistics
  tof = warp_sum(tof);
  relu = warp_sum(relu);
  if (lane == 0) { s_tof[w] = tof; s_relu[w] = relu; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    unsigned long long r = 0;
    for (int w2 = 0; w2 < kScanW; ++w2) { t += s_tof[w2]; r += s_relu[w2]; }
    a.tof_part[blockIdx.x] = t;
    if (r) atomicAdd(a.relu, r);
  }
  if constexpr (FUSED) {
    if (threadIdx.x < kMaxL && s_wl[threadIdx.x]) {
      atomicAdd(&a.stats->wl_layer[threadIdx.x], s_wl[threadIdx.x]);
      atomicAdd(&a.stats->wl, s_wl[threadIdx.x]);
    }
  }
}

int scan_blocks(const LayerInfo& li) { return li.nlines[0] + li.nlines[1]; }

static ScanArgs scan_args(la_ctx* c, int from_diff, double hist_w, double* tof_part) {
  Grid& g = c->grid;
  Forest& f = c->forest;
  ScanArgs a;
  a.cap = g.cap; a.D = g.D; a.H = g.H; a.diff = g.diff; a.P = g.P; a.T = g.T_dev; a.tofT = g.tofT_dev;
  a.HW = llround(hist_w * 16777216.0);
  a.from_diff = from_diff;
  a.tof_part = tof_part;
  a.relu = &c->d_stats->relu;
  a.seg_off = f.seg_off; a.seg_node = f.seg_node; a.seg_geo = f.seg_geo; a.layer = f.layer;
  a.stats = c->d_stats;
  return a;
}

template <bool FUSED>
static void scan_launch(la_ctx* c, const ScanArgs& a, size_t dyn, cudaStream_t s) {
  Grid& g = c->grid;
  const int nb = scan_blocks(g.li), nmax = std::max(g.li.nld[0], g.li.nld[1]);
  if (nmax <= 4) k_scan_lines<4, FUSED><<<nb, kScanT, dyn, s>>>(g.tab_dev, a);
  else if (nmax <= 6) k_scan_lines<6, FUSED><<<nb, kScanT, dyn, s>>>(g.tab_dev, a);
  else if (nmax <= 8) k_scan_lines<8, FUSED><<<nb, kScanT, dyn, s>>>(g.tab_dev, a);
  else k_scan_lines<kMaxL, FUSED><<<nb, kScanT, dyn, s>>>(g.tab_dev, a);
  ++c->launches;
}

void launch_scan_lines(la_ctx* c, int from_diff, double hist_w, double* tof_part, cudaStream_t s) {
  scan_launch<false>(c, scan_args(c, from_diff, hist_w, tof_part), 0, s);
}

// The line's difference array in shared memory: the longest line of either
// direction times its layers.
size_t fused_line_bytes(const LayerInfo& li) {
  return size_t(std::max(int64_t(li.npos[0]) * li.nld[0], int64_t(li.npos[1]) * li.nld[1])) * sizeof(int32_t);
}

bool prepare_fused_scan(const LayerInfo& li) {
  const size_t bytes = fused_line_bytes(li);
  if (bytes > kFusedLineMaxBytes) return false;
  const int nmax = std::max(li.nld[0], li.nld[1]);
  cudaError_t e;
  if (nmax <= 4) e = cudaFuncSetAttribute(k_scan_lines<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  else if (nmax <= 6) e = cudaFuncSetAttribute(k_scan_lines<6, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  else if (nmax <= 8) e = cudaFuncSetAttribute(k_scan_lines<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  else e = cudaFuncSetAttribute(k_scan_lines<kMaxL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Between the batches of a round: node v's segment leaves its old layer (-1
// at the first edge, +1 past the last) and takes its new one (+1, -1), in the
// difference array (global atomics; integer, exact in any order).
__global__ void __launch_bounds__(256) k_demand_delta(int64_t lo, int64_t hi, const DevTables* __restrict__ tab,
                                                      const int32_t* __restrict__ parent_g,
                                                      const uint64_t* __restrict__ geo,
                                                      const int8_t* __restrict__ layer,
                                                      const int8_t* __restrict__ layer_old,
                                                      int32_t* __restrict__ diff) {
  const int64_t v = lo + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= hi || parent_g[v] < 0) return;
  const uint64_t g = geo[v];
  const int d = geo_dir(g), nld = tab->nld[d];
  const int64_t at = tab->grid_off[d] + (int64_t(geo_line(g)) * tab->npos[d] + geo_lo(g)) * nld;
  const int64_t span = int64_t(geo_len(g)) * nld;
  const int ln = tab->ld_of[layer[v]];
  atomicAdd(diff + at + ln, 1);
  atomicAdd(diff + at + span + ln, -1);
  if (layer_old && layer_old[v] >= 0) {  // -1: the node had no layer before this round
    const int lold = tab->ld_of[layer_old[v]];
    atomicAdd(diff + at + lold, -1);
    atomicAdd(diff + at + span + lold, 1);
  }
}

void launch_demand_delta(la_ctx* c, int64_t lo, int64_t hi, const int8_t* layer_old, cudaStream_t s) {
  if (hi <= lo) return;
  Forest& f = c->forest;
  k_demand_delta<<<(unsigned)((hi - lo + 255) / 256), 256, 0, s>>>(lo, hi, c->grid.tab_dev, f.parent_g, f.geo,
                                                                    f.layer, layer_old, c->grid.diff);
  ++c->launches;
}

// After the backtrack: demand, D, H += max(0, D - C), the statistics and the
// next penalty prefix.  Fused into the line scan when a line fits in shared
// memory; otherwise global atomics into the difference array, then the scan.
void launch_demand_scan(la_ctx* c, double hist_w, double* tof_part, cudaStream_t s) {
  Grid& g = c->grid;
  if (g.fused_scan) {
    scan_launch<true>(c, scan_args(c, 1, hist_w, tof_part), fused_line_bytes(g.li), s);
  } else {
    launch_demand(c, s);
    launch_scan_lines(c, 1, hist_w, tof_part, s);
  }
}

void launch_local_demand(la_ctx* c, double hist_w, double* tof_part, cudaStream_t s) {
  Grid& g = c->grid;
  cudaMemsetAsync(g.D, 0, size_t(g.G) * sizeof(int32_t), s);
  launch_demand(c, s);
  launch_scan_lines(c, 2, hist_w, tof_part, s);
}

// ---------------------------------------------------------------------------
// DP over one level (Alg. 3).  One launch per (level, node class): DEG = 0
// (leaf), 1 (one son), 2 (two or more sons); ROOT: one thread per root (its
// junction is on the driver pin layer), otherwise one thread per (node, layer
// of its segment's direction).
//
// FP64 economy (GB300 issues FP64 at 1/64 of FP32): every value is the
// oracle's expression, but each is computed once.  A node writes, besides its
// entry A, Cc, M, the look-ahead base B = fma(w_d r_est(parent), Cc, A) that
// every candidate layer of its parent would otherwise recompute; the parent's
// key for son layer lc is then one fma(M, Rvia(l, lc), B).  Minima compare
// the bit patterns of non-negative doubles as integers.
// ---------------------------------------------------------------------------
struct DPArgs {
  int LD;
  int ld_magic;          // ceil(2^16 / LD): t / LD = (t ld_magic) >> 16 for 0 <= t < 256
  int64_t base;          // first node of the (level, class) bucket
  int64_t count;
  const int32_t *parent_g, *child_start, *nch, *child_list, *son0;
  const int8_t* pin;
  const double *sink_cap, *kappa, *W, *rho;
  const uint64_t* geo;
  const int64_t* P;
  const DevTables* tab;
  double *A, *Cc, *M, *B, *Jroot;
  int8_t *sb, *st, *ent;
  double w_cong_s, w_cap, w_d, sigma0;
  unsigned long long* err;
  // batched form only (else null): per node {w_d W, w_d kappa} (per weight
  // set) and {w_d r_est, sigma} (per round), and per (node, layer)
  // {alpha = w_d W R, gamma = fma(alpha, C/2, w_cap C), C}
  const double* ncache;
  const double* nround;
  const double* scache;
};

// double(K) for the penalty sum K of a segment: built from K's bits where
// that is exact (0 <= K < 2^53, which every sum of the non-negative penalties
// below 2^53 is), else the conversion.
__device__ __forceinline__ double penalty_to_double(long long K) {
  if (K >= 0 && K < (1LL << 53)) return exact_int_to_double(static_cast<unsigned long long>(K));
  return double(K);
}

// Float bounds of FP64 values, for an exact argmin filter on the FP32 pipe.
// f32_lo(x): the largest float <= x for x >= 0 (the double's bits truncated
// to a float's: 0 below 2^-126, FLT_MAX from 2^128 on).  f32_up(lo): a float
// >= every x whose lower bound is lo (the next float up; FLT_MIN above a 0).
// Integer instructions only.
__device__ __forceinline__ float f32_lo(double x) {
  const unsigned hi = unsigned(__double2hiint(x)), lo = unsigned(__double2loint(x));
  const unsigned e = hi >> 20;  // biased exponent (the sign bit is 0)
  if (e <= 1023u - 127u) return 0.0f;
  if (e >= 1023u + 128u) return FLT_MAX;
  return __uint_as_float(((hi - ((1023u - 127u) << 20)) << 3) | (lo >> 29));
}
__device__ __forceinline__ float f32_up(float lo) {
  return lo == 0.0f ? FLT_MIN : __uint_as_float(__float_as_uint(lo) + 1u);
}

// Sons of a several-son node whose choices per stack top are recorded.
constexpr int kRecSons = 4;

// (fp, k, b) lexicographic order of Kernel 2 (least f', fewest vias, lowest b).
__device__ __forceinline__ bool stack_better(long long f, int k, int b, long long bf, int bk, int bb) {
  return f < bf || (f == bf && (k < bk || (k == bk && b < bb)));
}

// Round constants of the tail terms at a node without a pin: fma(k, s, 0.0)
// is the rounded product k s, the same for every such node.
struct RoundTabs {
  double tS[kMaxL];  // (via count) x sigma0, sigma0 = w_via + w_cap vc
  double tC[kMaxL];  // (via count) x vc
};
__device__ __forceinline__ void load_round_tabs(RoundTabs& rt, const DPArgs& a, double via_c) {
  if (threadIdx.x < kMaxL) {
    rt.tS[threadIdx.x] = double(threadIdx.x) * a.sigma0;
    rt.tC[threadIdx.x] = double(threadIdx.x) * via_c;
  }
}

// The work of one thread: node v, candidate index ldi (0 at a root).
// CACHED: read the batched form's constant caches instead of recomputing.
// PINK: 1 the node has a pin, 0 it has none, 2 read it (mixed classes).
// STAGED (one son, not a root): the son and its table row (B, M, A, Cc) come
// in `so`, already copied to shared memory by the node's threads, with float
// bounds of B and M, and the block's float bounds of the Rvia table.
struct Son1 {
  int c, dc;
  const double *B, *M, *A, *Cc;
  const float *Blo, *Bup, *Mlo, *Mup;  // f32_lo / f32_up of the son's B and M
  const float *rlo, *rup;              // of Rvia(a, b), at [a * kRvStride + b]
  long long* K;                        // the thread's son keys by son layer index, stride 256 (shared memory)
  // the thread's own node data, loaded before the block's barrier: geometry,
  // pin, sink cap; cached: {w_d W, w_d kappa}, {w_d r_est, sigma}, the
  // parent's w_d r_est, {alpha, gamma, C} (else W, kappa, r_est, the parent's
  // r_est); the two prefix values of the segment on the candidate layer
  uint64_t gv;
  int pin;
  double Cs, nc0, nc1, nr0, nr1, rp, sc0, sc1, sc2;
  long long Kseg;  // P[end] - P[start]: the segment's penalty sum on the candidate layer
  // several sons, staged (SSON): son j < kStageSons of the thread's node in
  // shared memory, its id at sc[j * 32], direction at sd[j * 32], B and M
  // rows at sB / sM + (j * LDM + jj) * 32 (the pointers already offset by
  // the node's lane)
  const int* sc;
  const int8_t* sd;
  const double *sB, *sM;
};

// Sons of a several-son node staged in shared memory by its block (the
// first kStageSons of each node; most several-son nodes have two).
constexpr int kStageSons = 2;
// One son of a several-son node in the scan of the stacks with bottom b: its
// keys on its own direction's layers go to keyL by layer ([t][thread], the
// other layers hold LLONG_MAX), then for every top t = hi_req + i (i < nt) its
// least key in [b, t] is added to S[i] (FIRST: the first son sets S[i]) and
// its layer recorded in chj[t] (chj non-null).  Ascending layers: the lowest
// layer keeps a tie.  The loop over tops ends at the last one, so threads
// with the same hi_req run it the same number of times.
template <int LMAX, int LDM, bool FIRST>
__device__ __forceinline__ void son_scan(const DevTables& s, const double* rvl, int dc, const double* Bc,
                                         const double* Mc, int str, int b, int hi_req, int nt, long long* keyL,
                                         int8_t* chj, double (&S)[LMAX], unsigned& okm) {
  const int nldc = s.nld[dc];
#pragma unroll
  for (int t = 0; t < LMAX; ++t) keyL[t * 256] = LLONG_MAX;
#pragma unroll
  for (int jj = 0; jj < LDM; ++jj) {
    if (jj < nldc) {
      const int lc = s.lay[dc][jj];
      keyL[lc * 256] = dbits(fma(Mc[jj * str], rvl[lc], Bc[jj * str]));
    }
  }
  long long rbits = LLONG_MAX;
  int rlay = 0;
  for (int lc = b; lc < hi_req; ++lc) {
    const long long kk = keyL[lc * 256];
    if (kk < rbits) { rbits = kk; rlay = lc; }
  }
#pragma unroll
  for (int i = 0; i < LMAX; ++i) {
    if (i >= nt) break;
    const int t = hi_req + i;
    const long long kk = keyL[t * 256];
    if (kk < rbits) { rbits = kk; rlay = t; }
    if (rbits == LLONG_MAX) okm &= ~(1u << i);
    else S[i] = FIRST ? __longlong_as_double(rbits) : S[i] + __longlong_as_double(rbits);
    if (chj) chj[t * 256] = int8_t(rlay);
  }
}

// Son j of a several-son node: its id, direction and B, M rows (stride str):
// staged in shared memory for j < kStageSons (SSON), else from the tables.
template <int LDM, bool SSON>
__device__ __forceinline__ void son_row(const DPArgs& a, const Son1& so, int cs, int j, int& c, int& dc,
                                        const double*& Bc, const double*& Mc, int& str) {
  if (SSON && j < kStageSons) {
    c = so.sc[j * 32];
    dc = so.sd[j * 32];
    Bc = so.sB + j * LDM * 32;
    Mc = so.sM + j * LDM * 32;
    str = 32;
  } else {
    c = a.child_list[cs + j];
    dc = geo_dir(a.geo[c]);
    Bc = a.B + int64_t(c) * a.LD;
    Mc = a.M + int64_t(c) * a.LD;
    str = 1;
  }
}

template <int LMAX, int LDM, int DEG, bool ROOT, bool CACHED, int PINK, bool STAGED = false, bool SSON = false>
__device__ __forceinline__ void dp_node(const DPArgs& a, const DevTables& s, const RoundTabs& rt, int L, int v,
                                        int ldi, const Son1& so = Son1{}, long long* keybuf = nullptr,
                                        int8_t* chbuf = nullptr) {
  static_assert(!STAGED || (DEG == 1 && !ROOT), "staged son rows are for one-son non-root nodes");
  static_assert(!SSON || (DEG == 2 && !ROOT), "staged sons are for several-son non-root nodes");
  const int LD = a.LD;
  const int pin = PINK == 0 ? -1 : (STAGED ? so.pin : a.pin[v]);
  const uint64_t gv = STAGED ? so.gv : a.geo[v];
  const int d = geo_dir(gv);
  int l;
  if constexpr (ROOT) {
    l = pin;
  } else {
    if (ldi >= s.nld[d]) return;
    l = s.lay[d][ldi];
  }
  const double* rvl = &s.rv[l * kRvStride];
  const double* nc = CACHED ? a.ncache + 2 * int64_t(v) : nullptr;
  const double wd_rho = CACHED ? (STAGED ? so.nr0 : a.nround[2 * int64_t(v)]) : a.w_d * (STAGED ? so.nr0 : a.rho[v]);
  const double sigma_v = CACHED ? (STAGED ? so.nr1 : a.nround[2 * int64_t(v) + 1]) : fma(wd_rho, s.via_c, a.sigma0);
  double Cs = 0.0, sinkf = 0.0, z = 0.0;  // a node without a pin: all exactly 0
  if (PINK == 1 || (PINK == 2 && pin >= 0)) {
    Cs = STAGED ? so.Cs : a.sink_cap[v];
    sinkf = ((CACHED ? (STAGED ? so.nc1 : nc[1]) : a.w_d * (STAGED ? so.nc1 : a.kappa[v])) * rvl[pin]) * Cs;
    if constexpr (!STAGED) z = fma(wd_rho, Cs, sinkf);  // staged: only where the filter falls back
  }
  const int lo_req = pin >= 0 ? min(l, pin) : l;
  const int hi_req = pin >= 0 ? max(l, pin) : l;
  const int cs = a.child_start[v];

  int bb = lo_req, bt = hi_req;
  long long bfp = LLONG_MAX;
  double sg = 0.0, sc = 0.0;
  if constexpr (DEG == 0) {
    // a leaf: every stack costs tail(t - b); the smallest one wins
    bfp = dbits(fma(s.kd[hi_req - lo_req], sigma_v, z));
  } else if constexpr (DEG == 1) {
    // One son: only a stack that is the hull of (junction, pin, son layer
    // lc), with lc the son's own least key inside it, can win (a larger stack
    // with the same choice costs more and loses ties on t - b): evaluate those.
    // The son's layers ascend with j, so the hull of candidate j covers a run
    // of indices: [p, q) (the layers in [lo_req, hi_req]) widened down to j or
    // up to j.  j is its own least key there (ties to the lower index) iff
    //   j in [p, q): j is the first least key of [p, q);
    //   j < p:       key[j] <= every key of (j, q);
    //   j >= q:      key[j] <  every key of [p, j).
    int c, dc;
    const double *Bc, *Mc, *Ac, *Ccc;
    if constexpr (STAGED) {
      c = so.c; dc = so.dc; Bc = so.B; Mc = so.M; Ac = so.A; Ccc = so.Cc;
    } else {
      c = a.child_list[cs];
      dc = geo_dir(a.geo[c]);
      Bc = a.B + int64_t(c) * LD; Mc = a.M + int64_t(c) * LD;
      Ac = a.A + int64_t(c) * LD; Ccc = a.Cc + int64_t(c) * LD;
    }
    const int nldc = s.nld[dc];
    int bj = -1;
    if constexpr (STAGED) {
      // Exact filter on the FP32 pipe.  With f_j = RN(key_j + tail(via count
      // of the hull of l, the pin and the son layer j)), every stack costs at
      // least the f_j of its son's choice j (the tails grow with the via
      // count), so if one f_j is below every other, its hull is the stack
      // Kernel 2 picks, with j the son's choice in it (a larger stack with
      // the same choice costs no less and has more vias).  Bounds of every
      // f_j from float bounds of the operands with directed rounding
      // (everything is >= 0, and RN is monotone); if they separate one j
      // from the rest it is the winner, else the FP64 search below decides.
      const float slo = f32_lo(sigma_v), sup = f32_up(slo);
      float zlo = 0.0f, zup = 0.0f;
      if constexpr (PINK == 1) {
        const float wlo = f32_lo(wd_rho), clo = f32_lo(Cs), flo = f32_lo(sinkf);
        zlo = __fmaf_rd(wlo, clo, flo);
        zup = __fmaf_ru(f32_up(wlo), f32_up(clo), f32_up(flo));
      }
      const float* rlo = so.rlo + l * kRvStride;
      const float* rup = so.rup + l * kRvStride;
      // Only the least lower bound can win: a j whose upper bound is below
      // every other lower bound has the least lower bound itself.  So the
      // lower bounds of every j, then the upper bound of the first least one
      // (jlo) against the second least lower bound (lo2).
      float lo1 = INFINITY, lo2 = INFINITY;
      int jlo = -1;
#pragma unroll
      for (int j = 0; j < LDM; ++j) {
        if (j < nldc) {
          const int lc = s.lay[dc][j];
          const float kf = float(max(hi_req, lc) - min(lo_req, lc));
          const float klo = __fmaf_rd(so.Mlo[j], rlo[lc], so.Blo[j]);
          const float tlo = PINK == 1 ? __fmaf_rd(kf, slo, zlo) : __fmul_rd(kf, slo);
          const float flo = __fadd_rd(klo, tlo);
          if (flo < lo1) { lo2 = lo1; lo1 = flo; jlo = j; } else if (flo < lo2) { lo2 = flo; }
        }
      }
      if (jlo >= 0) {
        const int lc = s.lay[dc][jlo];
        const float kf = float(max(hi_req, lc) - min(lo_req, lc));
        const float kup = __fmaf_ru(so.Mup[jlo], rup[lc], so.Bup[jlo]);
        const float tup = PINK == 1 ? __fmaf_ru(kf, sup, zup) : __fmul_ru(kf, sup);
        if (__fadd_ru(kup, tup) < lo2) {
          bj = jlo;
          bb = min(lo_req, lc);
          bt = max(hi_req, lc);
        }
      }
    }
    if (bj < 0) {
      if constexpr (STAGED && PINK == 1) z = fma(wd_rho, Cs, sinkf);
      long long key[LDM];
      int p = 0, q = 0;  // son layer indices [p, q) lie in [lo_req, hi_req]
#pragma unroll
      for (int j = 0; j < LDM; ++j) {
        if (j < nldc) {
          const int lc = s.lay[dc][j];
          p += lc < lo_req;
          q += lc <= hi_req;
          key[j] = dbits(fma(Mc[j], rvl[lc], Bc[j]));
          if constexpr (STAGED && PINK == 0) so.K[j * 256] = key[j];
        }
      }
      long long inmin = LLONG_MAX;
      int m = -1;
#pragma unroll
      for (int j = 0; j < LDM; ++j)
        if (j >= p && j < q && key[j] < inmin) { inmin = key[j]; m = j; }
      unsigned cons = m >= 0 ? 1u << m : 0u;
      long long run = inmin;
#pragma unroll
      for (int j = LDM - 1; j >= 0; --j)
        if (j < p) {
          if (key[j] <= run) cons |= 1u << j;
          run = min(run, key[j]);
        }
      run = inmin;
#pragma unroll
      for (int j = 0; j < LDM; ++j)
        if (j >= q && j < nldc) {
          if (key[j] < run) cons |= 1u << j;
          run = min(run, key[j]);
        }
      int bk = INT_MAX;
      bj = 0;
      if constexpr (STAGED && PINK == 0) {
        // the consistent candidates only, lowest index first (a warp issues
        // the most any of its threads has, not the union of theirs)
        for (unsigned mm = cons; mm; mm &= mm - 1u) {
          const int j = __ffs(mm) - 1;
          const int lcj = s.lay[dc][j];
          const int b0 = min(lo_req, lcj), t0 = max(hi_req, lcj);
          const long long f = dbits(__longlong_as_double(so.K[j * 256]) + fma(s.kd[t0 - b0], sigma_v, 0.0));
          if (stack_better(f, t0 - b0, b0, bfp, bk, bb)) { bfp = f; bk = t0 - b0; bb = b0; bt = t0; bj = j; }
        }
      } else {
#pragma unroll
        for (int j = 0; j < LDM; ++j) {
          if ((cons >> j) & 1u) {
            const int lcj = s.lay[dc][j];
            const int b0 = min(lo_req, lcj), t0 = max(hi_req, lcj);
            const long long f = dbits(__longlong_as_double(key[j]) + fma(s.kd[t0 - b0], sigma_v, z));
            if (stack_better(f, t0 - b0, b0, bfp, bk, bb)) { bfp = f; bk = t0 - b0; bb = b0; bt = t0; bj = j; }
          }
        }
      }
      if (bfp == LLONG_MAX) {  // cannot happen (the least key overall is consistent); report it
        dev_error(a.err, DE_NOSTACK, v);
        return;
      }
    }
    const int lc = s.lay[dc][bj];
    a.ent[int64_t(c) * LD + ldi] = int8_t(lc);
    sg = fma(Mc[bj], rvl[lc], Ac[bj]);
    sc = Ccc[bj];
  } else {
    // Two or more sons: every stack [b, t] with b <= lo_req <= hi_req <= t;
    // S[t] accumulates, son by son in order, the son's least key in [b, t].
    // A son's keys are computed on its own direction's layers only and put
    // in shared memory by layer, [t][thread] (conflict-free), for the scan
    // over t (keybuf: LMAX x 256 entries, from the kernel).  With one stack
    // bottom only (lo_req = 0: a pin on layer 0, or a root on it) and at most
    // kRecSons sons, each son's least layer for every top t is recorded
    // (chbuf: kRecSons x LMAX x 256 bytes) and read back for the winner.
    long long* keyL = keybuf + threadIdx.x;
    const int nc = a.nch[v];
    int8_t* chL = chbuf ? chbuf + threadIdx.x : nullptr;
    const bool rec = chL != nullptr && lo_req == 0 && nc <= kRecSons;
    const int nt = L - hi_req;  // stack tops hi_req + i, i < nt
    int bk = INT_MAX;
    for (int b = 0; b <= lo_req; ++b) {
      double S[LMAX];
      unsigned okm = ~0u;  // bit i: every son has a layer in [b, hi_req + i]
#pragma unroll
      for (int i = 0; i < LMAX; ++i) S[i] = 0.0;
      for (int j = 0; j < nc; ++j) {
        int c, dc, str;
        const double *Bc, *Mc;
        son_row<LDM, SSON>(a, so, cs, j, c, dc, Bc, Mc, str);
        if (j == 0)
          son_scan<LMAX, LDM, true>(s, rvl, dc, Bc, Mc, str, b, hi_req, nt, keyL, rec ? chL : nullptr, S, okm);
        else
          son_scan<LMAX, LDM, false>(s, rvl, dc, Bc, Mc, str, b, hi_req, nt, keyL,
                                     rec ? chL + j * LMAX * 256 : nullptr, S, okm);
      }
#pragma unroll
      for (int i = 0; i < LMAX; ++i) {
        if (i >= nt) break;
        if ((okm >> i) & 1u) {
          const int t = hi_req + i;
          const long long f = dbits(S[i] + fma(s.kd[t - b], sigma_v, z));
          if (stack_better(f, t - b, b, bfp, bk, bb)) { bfp = f; bk = t - b; bb = b; bt = t; }
        }
      }
    }
    // each son's layer inside the winning stack (its own layers, ascending:
    // the lowest layer wins ties)
    for (int j = 0; j < nc; ++j) {
      int c, dc, str;
      const double *Bc, *Mc;
      son_row<LDM, SSON>(a, so, cs, j, c, dc, Bc, Mc, str);
      const int nldc = s.nld[dc];
      long long rbits = LLONG_MAX;
      int rj = -1;
      if (rec) {
        rj = s.ld_of[chL[(j * LMAX + bt) * 256]];
      } else {
#pragma unroll
        for (int jj = 0; jj < LDM; ++jj) {
          if (jj < nldc) {
            const int lc = s.lay[dc][jj];
            if (lc >= bb && lc <= bt) {
              const long long kb = dbits(fma(Mc[jj * str], rvl[lc], Bc[jj * str]));
              if (rj < 0 || kb < rbits) { rj = jj; rbits = kb; }
            }
          }
        }
      }
      if (rj < 0) {  // cannot happen for a valid stack; report instead of indexing with -1
        dev_error(a.err, DE_NOSTACK, v);
        return;
      }
      const int rl = s.lay[dc][rj];
      a.ent[int64_t(c) * LD + ldi] = int8_t(rl);
      const double g = fma(Mc[rj * str], rvl[rl], a.A[int64_t(c) * LD + rj]);
      sg = j == 0 ? g : sg + g;
      sc = j == 0 ? a.Cc[int64_t(c) * LD + rj] : sc + a.Cc[int64_t(c) * LD + rj];
    }
  }

  // the table entry of the winning stack (0.0 + x == x for the x >= 0 here)
  const int kk = bt - bb;
  double fv, cv;
  if constexpr (PINK == 0) {
    fv = DEG == 0 ? rt.tS[kk] : sg + rt.tS[kk];
    cv = DEG == 0 ? rt.tC[kk] : sc + rt.tC[kk];
  } else {
    fv = DEG == 0 ? fma(s.kd[kk], a.sigma0, sinkf) : sg + fma(s.kd[kk], a.sigma0, sinkf);
    cv = DEG == 0 ? fma(s.kd[kk], s.via_c, Cs) : sc + fma(s.kd[kk], s.via_c, Cs);
  }
  const int64_t o = int64_t(v) * LD + ldi;
  a.sb[o] = int8_t(bb);
  a.st[o] = int8_t(bt);
  if constexpr (ROOT) {
    a.Jroot[v] = __longlong_as_double(bfp);
  } else {
    const int len = geo_len(gv), line = geo_line(gv), lo = geo_lo(gv);
    double C, wdW, alpha, gamma;
    if constexpr (CACHED && STAGED) {
      alpha = so.sc0;
      gamma = so.sc1;
      C = so.sc2;
      wdW = so.nc0;
    } else if constexpr (CACHED) {
      const double* sc3 = a.scache + 3 * o;
      alpha = sc3[0];
      gamma = sc3[1];
      C = sc3[2];
      wdW = nc[0];
    } else {
      const double lenf = exact_int_to_double(unsigned(len));
      const double R = lenf * s.unit_r[l];
      C = lenf * s.unit_c[l];
      const double Ch = lenf * s.half_c[l];
      wdW = a.w_d * (STAGED ? so.nc0 : a.W[v]);
      alpha = wdW * R;
      gamma = fma(alpha, Ch, a.w_cap * C);
    }
    int64_t K;
    if constexpr (STAGED) {
      K = so.Kseg;
    } else {
      const int nldd = s.nld[d];
      const int64_t pb = s.grid_off[d] + int64_t(line) * s.npos[d] * nldd + ldi;
      K = a.P[pb + int64_t(lo + len) * nldd] - a.P[pb + int64_t(lo) * nldd];
    }
    const double seg = fma(a.w_cong_s, penalty_to_double(K), gamma);
    const double Av = fma(alpha, cv, fv + seg);
    const double ccv = C + cv;
    a.A[o] = Av;
    a.Cc[o] = ccv;
    a.M[o] = wdW * ccv;
    double rp;
    if constexpr (STAGED) {
      rp = CACHED ? so.rp : a.w_d * so.rp;
    } else {
      const int p = a.parent_g[v];
      rp = CACHED ? a.nround[2 * int64_t(p)] : a.w_d * a.rho[p];
    }
    a.B[o] = fma(rp, ccv, Av);
  }
}

// Leaves and one-son nodes fit 64 registers (4 blocks of 256 per SM), the
// bends 48 (5 blocks); the several-sons case keeps 3 blocks (capping it at
// 5 blocks of 32 x LD threads spilled and ran 15% slower).
template <int LMAX, int LDM, int DEG, bool ROOT, bool CACHED, int PINK>
__global__ void __launch_bounds__(256, (DEG == 1 && !ROOT && PINK == 0 ? 5 : (DEG <= 1 ? 4 : 3))) k_dp_level(LayerInfo li, DPArgs a) {
  __shared__ DevTables s;
  __shared__ RoundTabs rt;
  if constexpr (DEG == 1 && !ROOT) {
    // whole nodes per block (256 / LD of them): the node's threads copy the
    // son's table row to shared memory, one entry each per array, with
    // float bounds of its B and M; the block's threads bound the Rvia table.
    // The node's own loads and its son's row are issued before the block
    // copies the grid tables, so that their latencies overlap (the line
    // geometry of the prefix index comes from the kernel's LayerInfo).
    __shared__ double s_son[4][256];
    __shared__ float s_sf[4][256];
    __shared__ float s_rf[2][kMaxL * kRvStride];  // odd row stride: a node's threads (rows l) on distinct banks
    __shared__ long long s_key[PINK == 0 ? LDM : 1][256];
    const int LD = a.LD, npb = 256 / LD;
    // threadIdx.x / LD as a multiply and shift (exact below 256 for LD <= 16)
    const int gi = int((threadIdx.x * unsigned(a.ld_magic)) >> 16), ldi = int(threadIdx.x) - gi * LD;
    const int64_t node_i = int64_t(blockIdx.x) * npb + gi;
    const bool in = gi < npb && node_i < a.count;
    const int v = int(a.base + (in ? node_i : 0));
    Son1 so{};
    so.K = &s_key[0][threadIdx.x];
    so.rlo = s_rf[0];
    so.rup = s_rf[1];
    double Bo = 0.0, Mo = 0.0, Ao = 0.0, Cco = 0.0;
    if (in) {
      const uint64_t gv = a.geo[v];
      const int d = geo_dir(gv);
      const int nldd = d ? li.nld[1] : li.nld[0];
      so.gv = gv;
      so.pin = PINK == 0 ? -1 : a.pin[v];
      if constexpr (PINK == 1) so.Cs = a.sink_cap[v];
      const int p = a.parent_g[v];
      if constexpr (CACHED) {
        so.nc0 = a.ncache[2 * int64_t(v)];
        so.nc1 = a.ncache[2 * int64_t(v) + 1];
        so.nr0 = a.nround[2 * int64_t(v)];
        so.nr1 = a.nround[2 * int64_t(v) + 1];
        so.rp = a.nround[2 * int64_t(p)];
      } else {
        so.nc0 = a.W[v];
        so.nc1 = a.kappa[v];
        so.nr0 = a.rho[v];
        so.rp = a.rho[p];
      }
      if (ldi < nldd) {
        if constexpr (CACHED) {
          const double* sc3 = a.scache + 3 * (int64_t(v) * LD + ldi);
          so.sc0 = sc3[0];
          so.sc1 = sc3[1];
          so.sc2 = sc3[2];
        }
        const int64_t pb = (d ? li.grid_off[1] : li.grid_off[0]) +
                           int64_t(geo_line(gv)) * (d ? li.npos[1] : li.npos[0]) * nldd + ldi;
        so.Kseg = a.P[pb + int64_t(geo_lo(gv) + geo_len(gv)) * nldd] - a.P[pb + int64_t(geo_lo(gv)) * nldd];
      }
      so.c = a.son0[v];
      so.dc = geo_dir(a.geo[so.c]);
      const int64_t o = int64_t(so.c) * LD + ldi;
      Bo = a.B[o];
      Mo = a.M[o];
      Ao = a.A[o];
      Cco = a.Cc[o];
    }
    load_round_tabs(rt, a, li.via_c);
    load_tables(s, a.tab);
    for (int i = threadIdx.x; i < kMaxL * kRvStride; i += blockDim.x) {
      const float r = f32_lo(s.rv[i]);
      s_rf[0][i] = r;
      s_rf[1][i] = f32_up(r);
    }
    if (in) {
      s_son[0][threadIdx.x] = Bo;
      s_son[1][threadIdx.x] = Mo;
      s_son[2][threadIdx.x] = Ao;
      s_son[3][threadIdx.x] = Cco;
      const float bl = f32_lo(Bo), ml = f32_lo(Mo);
      s_sf[0][threadIdx.x] = bl;
      s_sf[1][threadIdx.x] = f32_up(bl);
      s_sf[2][threadIdx.x] = ml;
      s_sf[3][threadIdx.x] = f32_up(ml);
      const int r0 = gi * LD;
      so.B = &s_son[0][r0]; so.M = &s_son[1][r0]; so.A = &s_son[2][r0]; so.Cc = &s_son[3][r0];
      so.Blo = &s_sf[0][r0]; so.Bup = &s_sf[1][r0]; so.Mlo = &s_sf[2][r0]; so.Mup = &s_sf[3][r0];
    }
    __syncthreads();
    if (!in) return;
    dp_node<LMAX, LDM, DEG, ROOT, CACHED, PINK, true>(a, s, rt, li.L, v, ldi, so);
  } else if constexpr (DEG == 2 && !ROOT && LDM <= 8) {
    // 32 nodes per block of 32 x LD threads, warp w evaluating candidate
    // index w of each: a warp's threads share l, so the scans over the stack
    // tops above it have one length per warp.  Where the static shared
    // memory allows it, warp j < kStageSons first copies son j of every
    // node (id, direction, B and M rows) to shared memory: the sons' rows
    // are gathered at once, before the grid tables, instead of one son after
    // another inside the search.
    constexpr bool kSt = size_t(LMAX) * 256 * 8 + size_t(kRecSons) * LMAX * 256 + 2 * kStageSons * LDM * 32 * 8 +
                             sizeof(DevTables) + sizeof(RoundTabs) + 512 <= 48 * 1024;
    const int ldi = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    const int64_t node_i = int64_t(blockIdx.x) * 32 + lane;
    const bool in = node_i < a.count;
    __shared__ long long s_keyL[LMAX * 256];
    __shared__ int8_t s_ch[kRecSons * LMAX * 256];
    __shared__ double s_sr[kSt ? 2 * kStageSons * LDM * 32 : 1];
    __shared__ int s_sc[kSt ? kStageSons * 32 : 1];
    __shared__ int8_t s_sd[kSt ? kStageSons * 32 : 1];
    Son1 so{};
    if constexpr (kSt) {
      // warp w stages sons w, w + LD, ... (a block of one warp stages both)
      for (int j = ldi; j < kStageSons; j += a.LD) {
        int c = -1;
        if (in) {
          const int v = int(a.base + node_i);
          if (a.nch[v] > j) c = a.child_list[a.child_start[v] + j];
        }
        s_sc[j * 32 + lane] = c;
        if (c >= 0) {
          const int dc = geo_dir(a.geo[c]);
          const double* Bc = a.B + int64_t(c) * a.LD;
          const double* Mc = a.M + int64_t(c) * a.LD;
          double rb[LDM], rm[LDM];
#pragma unroll
          for (int jj = 0; jj < LDM; ++jj) {
            rb[jj] = jj < a.LD ? Bc[jj] : 0.0;
            rm[jj] = jj < a.LD ? Mc[jj] : 0.0;
          }
          s_sd[j * 32 + lane] = int8_t(dc);
#pragma unroll
          for (int jj = 0; jj < LDM; ++jj) {
            s_sr[(j * LDM + jj) * 32 + lane] = rb[jj];
            s_sr[((kStageSons + j) * LDM + jj) * 32 + lane] = rm[jj];
          }
        }
      }
      so.sc = s_sc + lane;
      so.sd = s_sd + lane;
      so.sB = s_sr + lane;
      so.sM = s_sr + kStageSons * LDM * 32 + lane;
    }
    load_round_tabs(rt, a, li.via_c);
    load_tables(s, a.tab);
    if (!in) return;
    dp_node<LMAX, LDM, DEG, ROOT, CACHED, PINK, false, kSt>(a, s, rt, li.L, int(a.base + node_i), ldi, so, s_keyL,
                                                            s_ch);
  } else {
    load_round_tabs(rt, a, li.via_c);
    load_tables(s, a.tab);
    // a node's candidate layers side by side (they share its sons' rows)
    const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t node_i = ROOT ? k : k / a.LD;
    const int ldi = ROOT ? 0 : int(k - node_i * a.LD);
    if (node_i >= a.count) return;
    __shared__ long long s_keyL[DEG == 2 ? LMAX * 256 : 1];
    __shared__ int8_t s_ch[DEG == 2 ? kRecSons * LMAX * 256 : 1];
    dp_node<LMAX, LDM, DEG, ROOT, CACHED, PINK>(a, s, rt, li.L, int(a.base + node_i), ldi, Son1{}, s_keyL, s_ch);
  }
}


// Any node: pick its class at run time (used where classes mix).
template <int LMAX, int LDM, bool CACHED>
__device__ void dp_node_any(const DPArgs& a, const DevTables& s, const RoundTabs& rt, int L, int v, int ldi,
                            long long* keybuf) {
  const int nc = a.nch[v];
  if (a.parent_g[v] < 0) {
    if (ldi != 0) return;
    if (nc == 0) dp_node<LMAX, LDM, 0, true, CACHED, 2>(a, s, rt, L, v, 0);
    else if (nc == 1) dp_node<LMAX, LDM, 1, true, CACHED, 2>(a, s, rt, L, v, 0);
    else dp_node<LMAX, LDM, 2, true, CACHED, 2>(a, s, rt, L, v, 0, Son1{}, keybuf);
  } else {
    if (nc == 0) dp_node<LMAX, LDM, 0, false, CACHED, 2>(a, s, rt, L, v, ldi);
    else if (nc == 1) dp_node<LMAX, LDM, 1, false, CACHED, 2>(a, s, rt, L, v, ldi);
    else dp_node<LMAX, LDM, 2, false, CACHED, 2>(a, s, rt, L, v, ldi, Son1{}, keybuf);
  }
}

struct BtArgs {
  int LD;
  const DevTables* tab;
  const int32_t* parent_g;
  const int8_t *pin, *ent, *sb, *st;
  int8_t *layer, *b, *t;
  Stats* stats;
  // the adjoint reweighting fused into the backtrack (UJ null: not fused)
  const uint64_t* geo;
  const int32_t* net_of;
  const double *r_drv, *Ws;
  double* UJ;
};

// Alg. 4 at node v: its layer from its parent's choice, its stack; returns
// the stack's via count t - b (the round's via statistic).  With a.UJ, also
// the top-down step of the adjoint reweighting on the new layers, in the
// expressions of the separate pass (k_elm_adj with g = kappa):
// U_J(root) = R_drv Ws; U_J(v) = (U_J(p) + Rvia(l_p, l_v) Ws(v)) + R_seg(v) Ws(v),
// the parent's U_J written by the level (or barrier step) before.
__device__ __forceinline__ int backtrack_node(const BtArgs& a, const int8_t* ld_of, int v) {
  const int gp = a.parent_g[v];
  int l, idx, lp = 0;
  if (gp < 0) {
    l = a.pin[v];
    idx = 0;
  } else {
    lp = a.layer[gp];
    const int pidx = a.parent_g[gp] < 0 ? 0 : ld_of[lp];
    l = a.ent[int64_t(v) * a.LD + pidx];
    idx = ld_of[l];
  }
  a.layer[v] = int8_t(l);
  const int bv = a.sb[int64_t(v) * a.LD + idx], tv = a.st[int64_t(v) * a.LD + idx];
  a.b[v] = int8_t(bv);
  a.t[v] = int8_t(tv);
  if (a.UJ != nullptr) {
    const double w = a.Ws[v];
    if (gp < 0) {
      a.UJ[v] = a.r_drv[a.net_of[v]] * w;
    } else {
      const double Rv = exact_int_to_double(unsigned(geo_len(a.geo[v]))) * a.tab->unit_r[l];
      const double UX = a.UJ[gp] + a.tab->rv[lp * kRvStride + l] * w;
      a.UJ[v] = UX + Rv * w;
    }
  }
  return tv - bv;
}

// The block's via counts into the round's statistics: warp sums, then one
// atomic per block (every thread of the block calls it; blockDim a multiple
// of 32, at most 1024).
__device__ __forceinline__ void add_vias(Stats* stats, unsigned vias) {
  __shared__ unsigned s_w[32];
  const unsigned w = __reduce_add_sync(0xffffffffu, vias);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sum = 0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) sum += s_w[i];
    if (sum) atomicAdd(&stats->vias, sum);
  }
}

// Large nets (batched form): a persistent grid takes nets from a work queue
// (largest first); a block walks its net's levels, the (node, layer) tasks of
// a level spread over its threads, __syncthreads between levels.  No wait
// crosses blocks.
struct BigArgs {
  const int32_t* queue;
  int64_t n_big;
  const int64_t* net_ptr;
  const int32_t *bl_nodes, *bl_hoff, *net_H;
  int* ctr;
};

template <int LMAX, int LDM, bool CACHED>
__global__ void __launch_bounds__(256) k_dp_bignets(LayerInfo li, DPArgs a, BigArgs g) {
  __shared__ DevTables s;
  __shared__ RoundTabs rt;
  __shared__ int s_q;
  __shared__ long long s_keyL[LMAX * 256];  // blockDim <= 256
  load_round_tabs(rt, a, li.via_c);
  load_tables(s, a.tab);
  const int LD = a.LD;
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(g.ctr, 1);
    __syncthreads();
    const int q = s_q;
    __syncthreads();
    if (q >= g.n_big) return;
    const int n = g.queue[q];
    const int64_t base = g.net_ptr[n];
    const int32_t* ho = g.bl_hoff + base + n;
    const int H = g.net_H[n];
    for (int h = 0; h <= H; ++h) {
      const int lo = ho[h], cnt = ho[h + 1] - lo;
      for (int t = threadIdx.x; t < cnt * LD; t += blockDim.x)
        dp_node_any<LMAX, LDM, CACHED>(a, s, rt, li.L, g.bl_nodes[base + lo + t / LD], t % LD, s_keyL);
      __syncthreads();
    }
  }
}

// One block walks levels h0..h1 of the small-net waves (the tail where every
// level has few tasks): each level's (node, candidate layer) tasks over the
// block's threads, the class chosen per node, __syncthreads between levels.
// ranges: [level][class] (first node, count).  No wait crosses blocks.
template <int LMAX, int LDM, bool CACHED>
__global__ void __launch_bounds__(256, 1) k_dp_tail(LayerInfo li, DPArgs a, const int64_t* __restrict__ ranges,
                                                    int h0, int h1) {
  __shared__ DevTables s;
  __shared__ RoundTabs rt;
  __shared__ long long s_keyL[LMAX * 256];  // blockDim = 256
  __shared__ int64_t s_lo[kClasses], s_n[kClasses];
  load_round_tabs(rt, a, li.via_c);
  load_tables(s, a.tab);
  const int LD = a.LD;
  for (int h = h0; h <= h1; ++h) {
    if (threadIdx.x < kClasses) {
      s_lo[threadIdx.x] = ranges[(int64_t(h) * kClasses + threadIdx.x) * 2];
      s_n[threadIdx.x] = ranges[(int64_t(h) * kClasses + threadIdx.x) * 2 + 1];
    }
    __syncthreads();
    int64_t total = 0;
#pragma unroll
    for (int cls = 0; cls < kClasses; ++cls) total += s_n[cls] * ((cls >= 3 && cls <= 5) ? 1 : LD);
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
      int64_t r = t;
      int cls = 0;
      while (cls < kClasses - 1 && r >= s_n[cls] * ((cls >= 3 && cls <= 5) ? 1 : LD)) {
        r -= s_n[cls] * ((cls >= 3 && cls <= 5) ? 1 : LD);
        ++cls;
      }
      const int ldc = (cls >= 3 && cls <= 5) ? 1 : LD;
      dp_node_any<LMAX, LDM, CACHED>(a, s, rt, li.L, int(s_lo[cls] + r / ldc), int(r % ldc), s_keyL);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_backtrack_bignets(BtArgs a, BigArgs g) {
  __shared__ int s_q;
  __shared__ int8_t s_ld[kMaxL];
  if (threadIdx.x < kMaxL) s_ld[threadIdx.x] = a.tab->ld_of[threadIdx.x];
  unsigned vias = 0;
  for (;;) {
    if (threadIdx.x == 0) s_q = atomicAdd(g.ctr, 1);
    __syncthreads();
    const int q = s_q;
    __syncthreads();
    if (q >= g.n_big) break;
    const int n = g.queue[q];
    const int64_t base = g.net_ptr[n];
    const int32_t* ho = g.bl_hoff + base + n;
    for (int h = g.net_H[n]; h >= 0; --h) {
      const int lo = ho[h], cnt = ho[h + 1] - lo;
      for (int t = threadIdx.x; t < cnt; t += blockDim.x)
        vias += backtrack_node(a, s_ld, g.bl_nodes[base + lo + t]);
      __syncthreads();
    }
  }
  add_vias(a.stats, vias);
}

template <int LMAX, int LDM, int DEG, bool ROOT, int PINK>
static void dp_launch(la_ctx* c, const DPArgs& a, cudaStream_t s) {
  int T = 256;
  unsigned B;
  if (DEG == 1 && !ROOT) {
    const int64_t npb = T / a.LD;  // whole nodes per block
    B = (unsigned)((a.count + npb - 1) / npb);
  } else if (DEG == 2 && !ROOT && LDM <= 8) {  // 32 nodes per block, a warp per candidate index
    T = 32 * a.LD;
    B = (unsigned)((a.count + 31) / 32);
  } else {
    const int64_t threads = ROOT ? a.count : a.count * a.LD;
    B = (unsigned)((threads + T - 1) / T);
  }
  if (a.scache) k_dp_level<LMAX, LDM, DEG, ROOT, true, PINK><<<B, T, 0, s>>>(c->grid.li, a);
  else k_dp_level<LMAX, LDM, DEG, ROOT, false, PINK><<<B, T, 0, s>>>(c->grid.li, a);
  ++c->launches;
}

// class -> kernel (node_class: 0-2 pin, 3-5 root, 6-8 no pin; sons 0, 1, 2+)
template <int LMAX, int LDM>
static void dp_launch_class(la_ctx* c, const DPArgs& a, int cls, cudaStream_t s) {
  switch (cls) {
    case 0: dp_launch<LMAX, LDM, 0, false, 1>(c, a, s); break;
    case 1: dp_launch<LMAX, LDM, 1, false, 1>(c, a, s); break;
    case 2: dp_launch<LMAX, LDM, 2, false, 1>(c, a, s); break;
    case 3: dp_launch<LMAX, LDM, 0, true, 1>(c, a, s); break;
    case 4: dp_launch<LMAX, LDM, 1, true, 1>(c, a, s); break;
    case 5: dp_launch<LMAX, LDM, 2, true, 1>(c, a, s); break;
    case 6: dp_launch<LMAX, LDM, 0, false, 0>(c, a, s); break;
    case 7: dp_launch<LMAX, LDM, 1, false, 0>(c, a, s); break;
    default: dp_launch<LMAX, LDM, 2, false, 0>(c, a, s); break;
  }
}

// Layer-count variants: LMAX bounds L, LDM the layers of one direction (half
// of LMAX when the directions alternate).
static void dp_launch_any(la_ctx* c, const DPArgs& a, int cls, cudaStream_t s) {
  const int L = c->grid.li.L, LD = c->LD;
  if (L <= 6) {
    if (LD <= 3) dp_launch_class<6, 3>(c, a, cls, s);
    else dp_launch_class<6, 6>(c, a, cls, s);
  } else if (L <= 12) {
    if (LD <= 6) dp_launch_class<12, 6>(c, a, cls, s);
    else dp_launch_class<12, 12>(c, a, cls, s);
  } else {
    if (LD <= 8) dp_launch_class<16, 8>(c, a, cls, s);
    else dp_launch_class<16, 16>(c, a, cls, s);
  }
}

static DPArgs dp_args(la_ctx* c, const RoundW& w, const double* W, const double* rho) {
  Forest& f = c->forest;
  DPArgs a;
  a.LD = c->LD;
  a.ld_magic = (65536 + c->LD - 1) / c->LD;
  a.parent_g = f.parent_g; a.child_start = f.child_start; a.nch = f.nch; a.child_list = f.child_list;
  a.son0 = f.son0;
  a.pin = f.pin; a.sink_cap = f.sink_cap; a.kappa = f.kappa; a.W = W; a.rho = rho; a.geo = f.geo;
  a.P = c->grid.P; a.tab = c->grid.tab_dev;
  a.A = f.A; a.Cc = f.Cc; a.M = f.M; a.B = f.B; a.Jroot = f.Jroot; a.sb = f.sb; a.st = f.st; a.ent = f.ent;
  a.w_cong_s = w.w_cong * 0x1.0p-24;
  a.w_cap = w.w_cap;
  a.w_d = w.w_d;
  a.sigma0 = w.w_via + w.w_cap * c->grid.li.via_c;
  a.err = c->d_err;
  a.base = 0;
  a.count = 0;
  a.ncache = nullptr;
  a.nround = nullptr;
  a.scache = nullptr;
  return a;
}

void launch_dp_level(la_ctx* c, const RoundW& w, const double* W, const double* rho, int level, int kmax,
                     int cache, cudaStream_t s, unsigned class_mask) {
  Forest& f = c->forest;
  DPArgs a = dp_args(c, w, W, rho);
  if (cache >= 0) {
    a.ncache = f.ncache[cache];
    a.nround = f.ncache[cache] + 2 * f.V;
    a.scache = f.scache[cache];
  }
  for (int cls = 0; cls < kClasses; ++cls) {
    if (!((class_mask >> cls) & 1u)) continue;
    const int64_t lo = f.key_off[size_t(bucket_key(level, cls, 0))];
    const int64_t hi = f.key_off[size_t(bucket_key(level, cls, kmax + 1))];
    const int64_t n = hi - lo;
    if (n == 0) continue;
    a.base = lo;
    a.count = n;
    dp_launch_any(c, a, cls, s);
  }
}

// ---------------------------------------------------------------------------
// Backtrack (Alg. 4): top-down, one thread per node of the level.
// ---------------------------------------------------------------------------
// Up to kClasses node ranges of one level (the small-net prefixes of its
// class buckets), one thread per node.
struct Ranges {
  int64_t lo[kClasses], cnt[kClasses];
  int64_t total;
};

__global__ void __launch_bounds__(256) k_backtrack_level(Ranges r, BtArgs a) {
  __shared__ int8_t s_ld[kMaxL];
  if (threadIdx.x < kMaxL) s_ld[threadIdx.x] = a.tab->ld_of[threadIdx.x];
  __syncthreads();
  int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  unsigned vias = 0;
  if (j < r.total) {
    int k = 0;
    while (k < kClasses - 1 && j >= r.cnt[k]) j -= r.cnt[k++];
    vias = backtrack_node(a, s_ld, int(r.lo[k] + j));
  }
  add_vias(a.stats, vias);
}

__global__ void __launch_bounds__(256) k_backtrack_tail(BtArgs a, const int64_t* __restrict__ ranges, int h0,
                                                         int h1) {
  __shared__ int8_t s_ld[kMaxL];
  __shared__ int64_t s_lo[kClasses], s_n[kClasses];
  if (threadIdx.x < kMaxL) s_ld[threadIdx.x] = a.tab->ld_of[threadIdx.x];
  unsigned vias = 0;
  for (int h = h1; h >= h0; --h) {
    if (threadIdx.x < kClasses) {
      s_lo[threadIdx.x] = ranges[(int64_t(h) * kClasses + threadIdx.x) * 2];
      s_n[threadIdx.x] = ranges[(int64_t(h) * kClasses + threadIdx.x) * 2 + 1];
    }
    __syncthreads();
    int64_t total = 0;
#pragma unroll
    for (int cls = 0; cls < kClasses; ++cls) total += s_n[cls];
    for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
      int64_t r = t;
      int cls = 0;
      while (cls < kClasses - 1 && r >= s_n[cls]) r -= s_n[cls++];
      vias += backtrack_node(a, s_ld, int(s_lo[cls] + r));
    }
    __syncthreads();
  }
  add_vias(a.stats, vias);
}

static BtArgs bt_args(la_ctx* c) {
  Forest& f = c->forest;
  BtArgs a{c->LD, c->grid.tab_dev, f.parent_g, f.pin, f.ent, f.sb, f.st, f.layer, f.b, f.t, c->d_stats,
           f.geo, f.net_of, f.r_drv, f.W_adj, nullptr};
  if (c->fuse_adjoint) a.UJ = f.rho_adj;
  return a;
}

void launch_backtrack_level(la_ctx* c, int level, int kmax, cudaStream_t s) {
  Forest& f = c->forest;
  Ranges r{};
  for (int cls = 0; cls < kClasses; ++cls) {
    r.lo[cls] = f.key_off[size_t(bucket_key(level, cls, 0))];
    r.cnt[cls] = f.key_off[size_t(bucket_key(level, cls, kmax + 1))] - r.lo[cls];
    r.total += r.cnt[cls];
  }
  if (r.total == 0) return;
  k_backtrack_level<<<(unsigned)((r.total + 255) / 256), 256, 0, s>>>(r, bt_args(c));
  ++c->launches;
}

static BigArgs big_args(la_ctx* c, int64_t n_big, int slot) {
  Forest& f = c->forest;
  return BigArgs{f.big_queue, n_big, f.net_ptr, f.bl_nodes, f.bl_hoff, f.net_H, f.queue_ctr + slot};
}

void launch_backtrack_bignets(la_ctx* c, int64_t n_big, int grid, int block, cudaStream_t s) {
  if (n_big == 0) return;
  k_backtrack_bignets<<<grid, block, 0, s>>>(bt_args(c), big_args(c, n_big, 1));
  ++c->launches;
}

void launch_backtrack_tail(la_ctx* c, int h0, int h1, int k, cudaStream_t s) {
  Forest& f = c->forest;
  const int64_t* ranges = f.range_tab + int64_t(k) * (f.Hmax + 1) * kClasses * 2;
  k_backtrack_tail<<<1, 256, 0, s>>>(bt_args(c), ranges, h0, h1);
  ++c->launches;
}

void launch_dp_tail(la_ctx* c, const RoundW& w, const double* W, const double* rho, int h0, int h1, int k, int cache,
                    cudaStream_t s) {
  Forest& f = c->forest;
  DPArgs a = dp_args(c, w, W, rho);
  const bool cached = cache >= 0;
  if (cached) {
    a.ncache = f.ncache[cache];
    a.nround = f.ncache[cache] + 2 * f.V;
    a.scache = f.scache[cache];
  }
  const int64_t* ranges = f.range_tab + int64_t(k) * (f.Hmax + 1) * kClasses * 2;
  const int L = c->grid.li.L, LD = c->LD;
#define TAIL(LM, LDM_)                                                                                \
  do {                                                                                                \
    if (cached) k_dp_tail<LM, LDM_, true><<<1, 256, 0, s>>>(c->grid.li, a, ranges, h0, h1);           \
    else k_dp_tail<LM, LDM_, false><<<1, 256, 0, s>>>(c->grid.li, a, ranges, h0, h1);                 \
  } while (0)
  if (L <= 6) {
    if (LD <= 3) TAIL(6, 3);
    else TAIL(6, 6);
  } else if (L <= 12) {
    if (LD <= 6) TAIL(12, 6);
    else TAIL(12, 12);
  } else {
    if (LD <= 8) TAIL(16, 8);
    else TAIL(16, 16);
  }
#undef TAIL
  ++c->launches;
}

void launch_dp_bignets(la_ctx* c, const RoundW& w, const double* W, const double* rho, int64_t n_big, int grid,
                       int block, int cache, cudaStream_t s) {
  if (n_big == 0) return;
  DPArgs a = dp_args(c, w, W, rho);
  const bool cached = cache >= 0;
  if (cached) {
    a.ncache = c->forest.ncache[cache];
    a.nround = c->forest.ncache[cache] + 2 * c->forest.V;
    a.scache = c->forest.scache[cache];
  }
  const int L = c->grid.li.L, LD = c->LD;
  BigArgs g = big_args(c, n_big, 0);
#define BIG(LM, LDM_)                                                                   \
  do {                                                                                 \
    if (cached) k_dp_bignets<LM, LDM_, true><<<grid, block, 0, s>>>(c->grid.li, a, g);  \
    else k_dp_bignets<LM, LDM_, false><<<grid, block, 0, s>>>(c->grid.li, a, g);        \
  } while (0)
  if (L <= 6) {
    if (LD <= 3) BIG(6, 3);
    else BIG(6, 6);
  } else if (L <= 12) {
    if (LD <= 6) BIG(12, 6);
    else BIG(12, 12);
  } else {
    if (LD <= 8) BIG(16, 8);
    else BIG(16, 16);
  }
#undef BIG
  ++c->launches;
}

// Batched form: values that do not change between rounds of one weight set,
// computed once (the same expressions the DP evaluates otherwise).  W of the
// adjoint mode is the criticality below each node, which depends only on the
// forest, so it is the same after every la_reweight_adjoint.
__global__ void k_seg_consts(int64_t V, int LD, const DevTables* __restrict__ tab, const uint64_t* __restrict__ geo,
                             const int32_t* __restrict__ parent_g, const int8_t* __restrict__ pin,
                             const double* __restrict__ W, const double* __restrict__ kappa, double w_d, double w_cap,
                             double* __restrict__ ncache, double* __restrict__ scache) {
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t v = k / LD;
  const int ldi = int(k - v * LD);
  if (v >= V) return;
  const double wdW = w_d * W[v];
  if (ldi == 0) {
    ncache[2 * v] = wdW;
    ncache[2 * v + 1] = pin[v] >= 0 ? w_d * kappa[v] : 0.0;
  }
  const uint64_t g = geo[v];
  const int d = geo_dir(g);
  if (parent_g[v] < 0 || ldi >= tab->nld[d]) return;
  const int l = tab->lay[d][ldi];
  const double len = double(geo_len(g));
  const double R = len * tab->unit_r[l];
  const double C = len * tab->unit_c[l];
  const double Ch = len * tab->half_c[l];
  const double alpha = wdW * R;
  double* o = scache + 3 * (v * LD + ldi);
  o[0] = alpha;
  o[1] = fma(alpha, Ch, w_cap * C);
  o[2] = C;
}

// Batched form, every round: w_d r_est and sigma = fma(w_d r_est, vc, w_via + w_cap vc) per node.
__global__ void k_node_round(int64_t V, const double* __restrict__ rho, double w_d, double via_c, double sigma0,
                             double* __restrict__ nround) {
  const int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const double wd_rho = w_d * rho[v];
  nround[2 * v] = wd_rho;
  nround[2 * v + 1] = fma(wd_rho, via_c, sigma0);
}

void launch_seg_consts(la_ctx* c, const RoundW& w, const double* W, int cache, cudaStream_t s) {
  Forest& f = c->forest;
  const int64_t threads = f.V * c->LD;
  k_seg_consts<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(f.V, c->LD, c->grid.tab_dev, f.geo, f.parent_g, f.pin,
                                                                W, f.kappa, w.w_d, w.w_cap, f.ncache[cache],
                                                                f.scache[cache]);
  ++c->launches;
}

void launch_node_round(la_ctx* c, const RoundW& w, const double* rho, int cache, cudaStream_t s) {
  Forest& f = c->forest;
  k_node_round<<<(unsigned)((f.V + 255) / 256), 256, 0, s>>>(f.V, rho, w.w_d, c->grid.li.via_c,
                                                             w.w_via + w.w_cap * c->grid.li.via_c,
                                                             f.ncache[cache] + 2 * f.V);
  ++c->launches;
}

// Resident blocks per SM of the big-net kernels (for a persistent grid).
int bignet_blocks_per_sm(int L, int LD, int block) {
  int n = 0;
  auto occ = [&](const void* k) { cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, 0); };
  if (L <= 6) occ(LD <= 3 ? (const void*)k_dp_bignets<6, 3, true> : (const void*)k_dp_bignets<6, 6, true>);
  else if (L <= 12) occ(LD <= 6 ? (const void*)k_dp_bignets<12, 6, true> : (const void*)k_dp_bignets<12, 12, true>);
  else occ(LD <= 8 ? (const void*)k_dp_bignets<16, 8, true> : (const void*)k_dp_bignets<16, 16, true>);
  return n > 0 ? n : 1;
}

// ---------------------------------------------------------------------------
// Demand: +1 at the segment's first edge and -1 past its last edge in the
// difference array of its line and layer (the line scan folds it into D),
// plus wirelength per layer (the vias are counted by the backtrack).  Integer
// atomics: exact in any order.
// ---------------------------------------------------------------------------
// Thread i: the i-th segment in (direction, line) order: +1 at its first edge
// and -1 past its last edge, in the difference array of its line and layer.
// A warp's segments lie on one or two lines, so its atomics land in a few L2
// sectors.  The segment data is read with streaming loads (each byte once).
__global__ void __launch_bounds__(256) k_demand(int64_t S, int L, const DevTables* __restrict__ tab,
                                                const int32_t* __restrict__ seg_node,
                                                const uint64_t* __restrict__ seg_geo,
                                                const int8_t* __restrict__ layer, int32_t* __restrict__ diff,
                                                Stats* stats) {
  __shared__ unsigned long long s_wl[kMaxL];
  __shared__ int64_t s_off[2];
  __shared__ int32_t s_npos[2], s_nld[2];
  __shared__ int8_t s_ld[kMaxL];
  if (threadIdx.x < kMaxL) {
    s_wl[threadIdx.x] = 0;
    s_ld[threadIdx.x] = tab->ld_of[threadIdx.x];
  }
  if (threadIdx.x < 2) {
    s_off[threadIdx.x] = tab->grid_off[threadIdx.x];
    s_npos[threadIdx.x] = tab->npos[threadIdx.x];
    s_nld[threadIdx.x] = tab->nld[threadIdx.x];
  }
  __syncthreads();
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  unsigned len = 0;
  int l = -1;
  if (i < S) {
    const int v = __ldcs(seg_node + i);
    const uint64_t g = __ldcs(reinterpret_cast<const unsigned long long*>(seg_geo) + i);
    l = layer[v];
    const int d = geo_dir(g);
    len = unsigned(geo_len(g));
    const int nld = s_nld[d];
    const int64_t base = s_off[d] + (int64_t(geo_line(g)) * s_npos[d] + geo_lo(g)) * nld + s_ld[l];
    atomicAdd(diff + base, 1);
    atomicAdd(diff + base + int64_t(len) * nld, -1);
  }
  // warp sums first: one shared atomic per warp and layer
  const unsigned peers = __match_any_sync(0xffffffffu, l);
  const unsigned wl = __reduce_add_sync(peers, len);
  if (l >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s_wl[l], (unsigned long long)wl);
  __syncthreads();
  if (threadIdx.x < L && s_wl[threadIdx.x]) {
    atomicAdd(&stats->wl_layer[threadIdx.x], s_wl[threadIdx.x]);
    atomicAdd(&stats->wl, s_wl[threadIdx.x]);
  }
}

void launch_demand(la_ctx* c, cudaStream_t s) {
  Forest& f = c->forest;
  const int T = 256;
  if (f.S == 0) return;
  k_demand<<<(unsigned)((f.S + T - 1) / T), T, 0, s>>>(f.S, c->grid.li.L, c->grid.tab_dev, f.seg_node, f.seg_geo,
                                                     f.layer, c->grid.diff, c->d_stats);
  ++c->launches;
}

// Per-block partial sums of the root costs J_n, in net order (deterministic).
__global__ void __launch_bounds__(256) k_sum_roots(int64_t N, const int32_t* __restrict__ root_of_net,
                                                   const double* __restrict__ Jroot, double* __restrict__ part,
                                                   double* __restrict__ J_out) {
  __shared__ double s_p[8];
  const int64_t n = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  double x = 0.0;
  if (n < N) {
    x = Jroot[root_of_net[n]];
    if (J_out) J_out[n] = x;
  }
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) s_p[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += s_p[w];
    part[blockIdx.x] = t;
  }
}

void launch_sum_roots(la_ctx* c, double* part, double* J_out, cudaStream_t s) {
  Forest& f = c->forest;
  k_sum_roots<<<(unsigned)((f.N + 255) / 256), 256, 0, s>>>(f.N, f.root_of_net, f.Jroot, part, J_out);
  ++c->launches;
}

}  // namespace gapla
