/* la_oracle.c - plain FP64 CPU oracle of the GAP-LA layer-assignment round.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library never
 * calls it and shares no code with it.
 *
 * It is written for a reader checking it against the paper (arxiv 2507.13375):
 *   - one net at a time, nodes in net-local order (parent < child), so a loop
 *     from the last node to the first visits children before parents
 *     (the bottom-up "level 0 -> max" pass of Alg. 2), and a loop from the
 *     first node visits parents first (the top-down pass of Alg. 2 / Alg. 4);
 *   - Alg. 3 as printed: for every parent-edge layer l, every via stack
 *     [b, t] containing l is enumerated; each son takes its legal layer of
 *     least look-ahead cost inside [b, t] (Kernel 1); then the stack of least
 *     f' is kept (Kernel 2);
 *   - no blocking, fusion or reordering.  Threads only split the nets.
 *
 * Exact readings (where the paper is silent):
 *   Tree / RC model.  Non-root v has a straight segment e_v of length len_v
 *   (GCell edges) to its parent.  On layer l: R_v(l) = len_v r_l,
 *   C_v(l) = len_v c_l, pi-model (half the cap at each end, Sec. III-B).
 *   Rvia(a, b) = sum of vr_k for k from min(a,b) to max(a,b)-1.  The junction
 *   of v is on its parent-edge layer l (the driver pin layer at a root); each
 *   son c is reached through Rvia(l, l_c); a pin at v through Rvia(l, p_v).
 *   A via stack [b, t] holds t-b vias of cap vc each, lumped at the junction.
 *   Weights.  Eq. 4 with "downstream subtree": W_v = max sink criticality in
 *   the subtree of v.  r_est_v = W_root R_drv + sum over the segments x on the
 *   path root..v (including e_v) of W_x len_x rbar(dir x), rbar = mean unit R of
 *   the layers of that direction (Sec. III-D, "node distances and average unit
 *   resistance"; the W factor makes the estimate the weighted upstream R).
 *   Costs (per son c, son layer lc, parent junction layer l):
 *     A_c(lc)  = f_c(lc) + w_cong 2^-24 K_c(lc) + w_cap C_c(lc)
 *                + w_d W_c R_c(lc) (C_c(lc)/2 + c_c(lc))
 *     Cc_c(lc) = C_c(lc) + c_c(lc),   M_c(lc) = w_d W_c Cc_c(lc)
 *     g_c(l, lc)   = A_c(lc) + M_c(lc) Rvia(l, lc)
 *     key_c(l, lc) = g_c(l, lc) + w_d r_est_v Cc_c(lc)     (look-ahead, Sec. III-D)
 *   Node v, layer l, stack [b, t] (k = t - b vias, sons at lc*):
 *     f  = sum_c g_c + (w_via + w_cap vc) k + [pin] w_d kappa_v Rvia(l, p_v) Cs_v
 *     c  = sum_c Cc_c + vc k + Cs_v
 *     f' = f + w_d r_est_v c                                (Sec. III-D)
 *   Ties: a son takes the lowest layer; a stack wins by (f', t-b, b) lowest.
 *   The root's junction is the driver pin layer; J_n = f' at the root.
 *   Congestion penalty (reading of Eq. 3 as a per-edge cost, integer-exact):
 *     k = clamp(D + 1 - C, -64, 64); s = 0.5 if C > 0 else 1.5;
 *     T_l[k] = llround(min(ofw_l e^{s k} 2^24, 2^48));
 *     pen = min(T_l[k] + llround(hist_w 2^24) H, 2^48);  K_v(l) = sum of pen
 *     over the GCell edges of e_v on layer l.
 *
 * Rounding order is fixed (same expression trees in every implementation that
 * is compared with this one): the sums over sons run in net-local son order
 * starting from 0.0; products associate left to right as written; fma() is
 * used exactly where written below.  Build with -ffp-contract=off.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_MAXL 16
#define PEN_MAX (1ll << 48)

typedef struct {
  int32_t X, Y, L;
  const int8_t* dir;
  const int32_t* cap;  /* public edge layout */
  const double *unit_r, *unit_c, *via_r;
  double via_c;
  const double* ofw;
} or_grid;

typedef struct {
  int64_t num_nets, num_nodes;
  const int64_t* net_ptr;
  const int32_t *x, *y, *parent;
  const int8_t* pin_layer;
  const double *sink_cap, *kappa, *r_drv;
} or_forest;

typedef struct {
  double w_cong, w_via, w_cap, w_d, hist_w;
} or_weights;

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */
static int64_t layer_edges(const or_grid* g, int l) {
  return g->dir[l] == 0 ? (int64_t)g->Y * (g->X - 1) : (int64_t)g->X * (g->Y - 1);
}
static int64_t layer_offset(const or_grid* g, int l) {
  int64_t off = 0;
  for (int k = 0; k < l; k++) off += layer_edges(g, k);
  return off;
}
int64_t or_num_edges(const or_grid* g) { return layer_offset(g, g->L); }

/* Rvia(a, b): sum of the via resistances between layers a and b. */
static double rvia(const or_grid* g, int a, int b) {
  int lo = a < b ? a : b, hi = a < b ? b : a;
  double s = 0.0;
  for (int k = lo; k < hi; k++) s += g->via_r[k];
  return s;
}

/* Segment of non-root node v (global id), to its parent (global id p). */
typedef struct { int dir, line, lo, hi, len; } seg_t;
static seg_t segment_of(const or_forest* f, int64_t v, int64_t p) {
  seg_t s;
  if (f->y[v] == f->y[p]) { /* horizontal: row y, edges [min x, max x) */
    s.dir = 0; s.line = f->y[v];
    s.lo = f->x[v] < f->x[p] ? f->x[v] : f->x[p];
    s.hi = f->x[v] < f->x[p] ? f->x[p] : f->x[v];
  } else {                  /* vertical: column x, edges [min y, max y) */
    s.dir = 1; s.line = f->x[v];
    s.lo = f->y[v] < f->y[p] ? f->y[v] : f->y[p];
    s.hi = f->y[v] < f->y[p] ? f->y[p] : f->y[v];
  }
  s.len = s.hi - s.lo;
  return s;
}
/* Index of GCell edge e of line `line` on layer l (public layout). */
static int64_t edge_index(const or_grid* g, int l, int line, int e) {
  int64_t per_line = g->dir[l] == 0 ? g->X - 1 : g->Y - 1;
  return layer_offset(g, l) + (int64_t)line * per_line + e;
}

/* ------------------------------------------------------------------------ */
/* Congestion penalty (reading of Eq. 3)                                     */
/* ------------------------------------------------------------------------ */
/* T[l][sidx][k + 64]: sidx 0 for s = 0.5 (C > 0), 1 for s = 1.5 (C = 0). */
void or_penalty_table(const or_grid* g, int64_t* T /* L*2*129 */) {
  for (int l = 0; l < g->L; l++)
    for (int si = 0; si < 2; si++) {
      double s = si == 0 ? 0.5 : 1.5;
      for (int k = -64; k <= 64; k++) {
        double v = g->ofw[l] * exp(s * k) * 16777216.0;
        if (v > (double)PEN_MAX) v = (double)PEN_MAX;
        T[((int64_t)l * 2 + si) * 129 + (k + 64)] = llround(v);
      }
    }
}

/* pen[e] for every edge, from the snapshot (D, H). */
void or_penalty(const or_grid* g, const int32_t* D, const int32_t* H, double hist_w, int64_t* pen) {
  int64_t T[OR_MAXL * 2 * 129];
  or_penalty_table(g, T);
  int64_t HW = llround(hist_w * 16777216.0);
  for (int l = 0; l < g->L; l++) {
    int64_t off = layer_offset(g, l), ne = layer_edges(g, l);
    for (int64_t i = 0; i < ne; i++) {
      int64_t e = off + i;
      int32_t c = g->cap[e];
      int64_t k = (int64_t)D[e] + 1 - c;
      if (k < -64) k = -64;
      if (k > 64) k = 64;
      int64_t t = T[((int64_t)l * 2 + (c > 0 ? 0 : 1)) * 129 + (k + 64)];
      int64_t p;
      if (H[e] > 0 && HW > 0 && (int64_t)H[e] > (PEN_MAX - t) / HW) p = PEN_MAX;
      else p = t + HW * (int64_t)H[e];
      if (p > PEN_MAX) p = PEN_MAX;
      pen[e] = p;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Edge weights (Eq. 4) and look-ahead upstream resistance (Sec. III-D)      */
/* ------------------------------------------------------------------------ */
static double rbar(const or_grid* g, int d) {
  double s = 0.0;
  int n = 0;
  for (int l = 0; l < g->L; l++)
    if (g->dir[l] == d) { s += g->unit_r[l]; n++; }
  return n ? s / n : 0.0;
}

void or_weights_eq4(const or_grid* g, const or_forest* f, double* W, double* rho) {
  double rb[2] = {rbar(g, 0), rbar(g, 1)};
  for (int64_t n = 0; n < f->num_nets; n++) {
    int64_t base = f->net_ptr[n], m = f->net_ptr[n + 1] - base;
    for (int64_t i = 0; i < m; i++) W[base + i] = f->pin_layer[base + i] >= 0 ? f->kappa[base + i] : 0.0;
    for (int64_t i = m - 1; i >= 1; i--) { /* children before parents */
      int64_t p = base + f->parent[base + i];
      if (W[base + i] > W[p]) W[p] = W[base + i];
    }
    rho[base] = W[base] * f->r_drv[n];
    for (int64_t i = 1; i < m; i++) { /* parents before children */
      int64_t v = base + i, p = base + f->parent[v];
      seg_t s = segment_of(f, v, p);
      rho[v] = rho[p] + (W[v] * (double)s.len) * rb[s.dir];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* The DP (Alg. 3), root selection and backtrack (Alg. 4)                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  const or_grid* g;
  const or_forest* f;
  const or_weights* w;
  const int64_t* pen;
  const double *W, *rho;
  int64_t net_lo, net_hi;
  int8_t *layer, *bo, *to;
  double* J;
  double *A_out, *Cc_out; /* optional, V*L */
  int err;
} dp_job;

typedef struct {
  int64_t cap;
  double *A, *Cc, *M;      /* [node*L + l] */
  int8_t *sb, *st;         /* chosen stack per (node, l) */
  int8_t* ent;             /* [son*L + l]: son layer when the parent's junction is on l */
  int32_t *son_ptr, *son_list;
  int32_t* choice;         /* per son, scratch */
  int32_t* best_choice;
  int8_t* sdir;            /* direction of each node's segment (-1 at the root) */
} dp_scratch;

static void scratch_reserve(dp_scratch* s, int64_t m, int L) {
  if (m <= s->cap) return;
  int64_t c = s->cap ? s->cap : 64;
  while (c < m) c *= 2;
  s->A = realloc(s->A, c * L * sizeof(double));
  s->Cc = realloc(s->Cc, c * L * sizeof(double));
  s->M = realloc(s->M, c * L * sizeof(double));
  s->sb = realloc(s->sb, c * L);
  s->st = realloc(s->st, c * L);
  s->ent = realloc(s->ent, c * L);
  s->son_ptr = realloc(s->son_ptr, (c + 1) * sizeof(int32_t));
  s->son_list = realloc(s->son_list, c * sizeof(int32_t));
  s->choice = realloc(s->choice, c * sizeof(int32_t));
  s->best_choice = realloc(s->best_choice, c * sizeof(int32_t));
  s->sdir = realloc(s->sdir, c);
  s->cap = c;
}
static void scratch_free(dp_scratch* s) {
  free(s->A); free(s->Cc); free(s->M); free(s->sb); free(s->st); free(s->ent);
  free(s->son_ptr); free(s->son_list); free(s->choice); free(s->best_choice); free(s->sdir);
}

/* K_v(l): congestion of segment e_v on layer l = sum of pen over its edges. */
static int64_t seg_congestion(const or_grid* g, const int64_t* pen, seg_t s, int l) {
  int64_t K = 0;
  for (int e = s.lo; e < s.hi; e++) K += pen[edge_index(g, l, s.line, e)];
  return K;
}

static void dp_net(dp_job* job, dp_scratch* S, int64_t n) {
  const or_grid* g = job->g;
  const or_forest* f = job->f;
  const or_weights* w = job->w;
  const int L = g->L;
  const int64_t base = f->net_ptr[n], m = f->net_ptr[n + 1] - base;
  scratch_reserve(S, m, L);
  /* sons of each node, in increasing net-local id */
  for (int64_t i = 0; i <= m; i++) S->son_ptr[i] = 0;
  for (int64_t i = 1; i < m; i++) S->son_ptr[f->parent[base + i] + 1]++;
  for (int64_t i = 0; i < m; i++) S->son_ptr[i + 1] += S->son_ptr[i];
  {
    int32_t* fill = S->choice; /* reuse as a cursor */
    for (int64_t i = 0; i < m; i++) fill[i] = S->son_ptr[i];
    for (int64_t i = 1; i < m; i++) S->son_list[fill[f->parent[base + i]]++] = (int32_t)i;
  }
  S->sdir[0] = -1;
  for (int64_t i = 1; i < m; i++) S->sdir[i] = (int8_t)segment_of(f, base + i, base + f->parent[base + i]).dir;
  const double vc = g->via_c;
  const double sigma0 = w->w_via + w->w_cap * vc;
  const double wcong_s = w->w_cong * 0x1.0p-24;

  /* bottom-up: children (higher local id) before parents */
  for (int64_t i = m - 1; i >= 0; i--) {
    const int64_t v = base + i;
    const int is_root = (i == 0);
    const int pin = f->pin_layer[v];
    const double Cs = f->sink_cap[v];
    const double kap = f->kappa[v];
    const double wd_rho = w->w_d * job->rho[v];
    const double sigma_v = fma(wd_rho, vc, sigma0);
    seg_t sg = {0, 0, 0, 0, 0};
    if (!is_root) sg = segment_of(f, v, base + f->parent[v]);
    const int s0 = S->son_ptr[i], s1 = S->son_ptr[i + 1];
    for (int l = 0; l < L; l++) {
      S->A[i * L + l] = NAN; S->Cc[i * L + l] = NAN; S->M[i * L + l] = NAN;
      S->sb[i * L + l] = -1; S->st[i * L + l] = -1;
    }
    for (int l = 0; l < L; l++) {
      /* candidate junction layers: the segment's direction, or the driver pin layer */
      if (is_root ? (l != pin) : (g->dir[l] != sg.dir)) continue;
      const double sinkf = pin >= 0 ? ((w->w_d * kap) * rvia(g, l, pin)) * Cs : 0.0;
      const double z = fma(wd_rho, Cs, sinkf);
      int found = 0, best_b = 0, best_t = 0;
      double best_fp = 0.0;
      /* Kernel 1: every stack [b, t] holding l (and the pin) */
      for (int b = 0; b <= l; b++) {
        for (int t = l; t < L; t++) {
          if (pin >= 0 && !(b <= pin && pin <= t)) continue;
          double skey = 0.0;
          int ok = 1;
          for (int si = s0; si < s1; si++) {
            const int64_t c = S->son_list[si];
            int lc_best = -1;
            double key_best = 0.0;
            for (int lc = b; lc <= t; lc++) {
              if (g->dir[lc] != S->sdir[c]) continue; /* not a layer of son c's direction */
              const double Bc = fma(wd_rho, S->Cc[c * L + lc], S->A[c * L + lc]);
              const double key = fma(S->M[c * L + lc], rvia(g, l, lc), Bc);
              if (lc_best < 0 || key < key_best) { lc_best = lc; key_best = key; }
            }
            if (lc_best < 0) { ok = 0; break; }
            S->choice[si] = lc_best;
            skey = skey + key_best;
          }
          if (!ok) continue;
          const int k = t - b;
          const double fp = skey + fma((double)k, sigma_v, z);
          /* Kernel 2: least f', then fewest vias, then lowest b */
          int better = !found || fp < best_fp ||
                       (fp == best_fp && (k < best_t - best_b || (k == best_t - best_b && b < best_b)));
          if (better) {
            found = 1; best_fp = fp; best_b = b; best_t = t;
            for (int si = s0; si < s1; si++) S->best_choice[si] = S->choice[si];
          }
        }
      }
      if (!found) { job->err = 1; return; }
      /* the winning stack's table entry */
      double sg_sum = 0.0, sc_sum = 0.0;
      for (int si = s0; si < s1; si++) {
        const int64_t c = S->son_list[si];
        const int lc = S->best_choice[si];
        sg_sum = sg_sum + fma(S->M[c * L + lc], rvia(g, l, lc), S->A[c * L + lc]);
        sc_sum = sc_sum + S->Cc[c * L + lc];
        S->ent[c * L + l] = (int8_t)lc;
      }
      const int k = best_t - best_b;
      const double fv = sg_sum + fma((double)k, sigma0, sinkf);
      const double cv = sc_sum + fma((double)k, vc, Cs);
      S->sb[i * L + l] = (int8_t)best_b;
      S->st[i * L + l] = (int8_t)best_t;
      if (is_root) {
        job->J[n] = best_fp;
      } else {
        const double R = (double)sg.len * g->unit_r[l];
        const double C = (double)sg.len * g->unit_c[l];
        const double Ch = (double)sg.len * (0.5 * g->unit_c[l]);
        const double wdW = w->w_d * job->W[v];
        const double alpha = wdW * R;
        const double gamma = fma(alpha, Ch, w->w_cap * C);
        const int64_t K = seg_congestion(g, job->pen, sg, l);
        const double seg = fma(wcong_s, (double)K, gamma);
        S->A[i * L + l] = fma(alpha, cv, fv + seg);
        S->Cc[i * L + l] = C + cv;
        S->M[i * L + l] = wdW * S->Cc[i * L + l];
      }
    }
  }
  /* Alg. 4: top-down backtrack from the root's junction on the pin layer */
  {
    const int lr = f->pin_layer[base];
    job->layer[base] = (int8_t)lr;
    job->bo[base] = S->sb[0 * L + lr];
    job->to[base] = S->st[0 * L + lr];
    for (int64_t i = 1; i < m; i++) {
      const int64_t p = f->parent[base + i];
      const int lp = job->layer[base + p];
      const int l = S->ent[i * L + lp];
      job->layer[base + i] = (int8_t)l;
      job->bo[base + i] = S->sb[i * L + l];
      job->to[base + i] = S->st[i * L + l];
    }
  }
  if (job->A_out)
    for (int64_t i = 0; i < m; i++)
      for (int l = 0; l < L; l++) {
        job->A_out[(base + i) * L + l] = S->A[i * L + l];
        job->Cc_out[(base + i) * L + l] = S->Cc[i * L + l];
      }
}

static void* dp_worker(void* arg) {
  dp_job* job = (dp_job*)arg;
  dp_scratch S;
  memset(&S, 0, sizeof S);
  for (int64_t n = job->net_lo; n < job->net_hi && !job->err; n++) dp_net(job, &S, n);
  scratch_free(&S);
  return NULL;
}

static int n_threads(int req) {
  if (req > 0) return req > 512 ? 512 : req;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n < 1 ? 1 : (n > 512 ? 512 : (int)n);
}

/* The DP + backtrack for nets [net_lo, net_hi).  Outputs at those nets' nodes.
 * Returns the number of threads used, or -1 on an internal error. */
int or_dp(const or_grid* g, const or_forest* f, const or_weights* w, const int64_t* pen,
          const double* W, const double* rho, int64_t net_lo, int64_t net_hi, int threads,
          int8_t* layer, int8_t* b, int8_t* t, double* J, double* A_out, double* Cc_out) {
  int T = n_threads(threads);
  int64_t nn = net_hi - net_lo;
  if (nn < T) T = nn > 0 ? (int)nn : 1;
  dp_job* jobs = calloc(T, sizeof(dp_job));
  pthread_t* th = calloc(T, sizeof(pthread_t));
  for (int k = 0; k < T; k++) {
    dp_job* j = &jobs[k];
    j->g = g; j->f = f; j->w = w; j->pen = pen; j->W = W; j->rho = rho;
    j->net_lo = net_lo + nn * k / T; j->net_hi = net_lo + nn * (k + 1) / T;
    j->layer = layer; j->bo = b; j->to = t; j->J = J; j->A_out = A_out; j->Cc_out = Cc_out;
    pthread_create(&th[k], NULL, dp_worker, j);
  }
  int err = 0;
  for (int k = 0; k < T; k++) { pthread_join(th[k], NULL); err |= jobs[k].err; }
  free(jobs); free(th);
  return err ? -1 : T;
}

/* ------------------------------------------------------------------------ */
/* Demand, vias, history and the overflow statistics (Eq. 2, Eq. 3)          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t vias, wl, relu_overflow;
  double tof;
  int64_t wl_per_layer[OR_MAXL];
} or_stats;

/* D = demand of the assignment (one unit per segment per GCell edge),
 * H_out = H_in + max(0, D - C), and the statistics. */
void or_demand(const or_grid* g, const or_forest* f, const int8_t* layer, const int8_t* b,
               const int8_t* t, const int32_t* H_in, int32_t* D, int32_t* H_out, or_stats* st) {
  const int64_t E = or_num_edges(g);
  memset(D, 0, E * sizeof(int32_t));
  memset(st, 0, sizeof *st);
  for (int64_t n = 0; n < f->num_nets; n++) {
    int64_t base = f->net_ptr[n], m = f->net_ptr[n + 1] - base;
    st->vias += (int64_t)(t[base] - b[base]);
    for (int64_t i = 1; i < m; i++) {
      int64_t v = base + i;
      seg_t s = segment_of(f, v, base + f->parent[v]);
      int l = layer[v];
      for (int e = s.lo; e < s.hi; e++) D[edge_index(g, l, s.line, e)] += 1;
      st->wl += s.len;
      st->wl_per_layer[l] += s.len;
      st->vias += (int64_t)(t[v] - b[v]);
    }
  }
  for (int l = 0; l < g->L; l++) {
    int64_t off = layer_offset(g, l), ne = layer_edges(g, l);
    for (int64_t i = 0; i < ne; i++) {
      int64_t e = off + i;
      int64_t over = (int64_t)D[e] - g->cap[e];
      if (over > 0) st->relu_overflow += over;
      H_out[e] = H_in[e] + (over > 0 ? (int32_t)over : 0);
      double s = g->cap[e] > 0 ? 0.5 : 1.5;
      st->tof += g->ofw[l] * exp(s * (double)over);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Elmore delay (Sec. II-C, the d_34 example of Sec. III-D) and its adjoint  */
/* ------------------------------------------------------------------------ */
/* R_seg = len r_l, C_seg = len c_l on the assigned layer; 0 at roots. */
void or_rc_from_assignment(const or_grid* g, const or_forest* f, const int8_t* layer,
                           double* R_seg, double* C_seg) {
  for (int64_t n = 0; n < f->num_nets; n++) {
    int64_t base = f->net_ptr[n], m = f->net_ptr[n + 1] - base;
    R_seg[base] = 0.0; C_seg[base] = 0.0;
    for (int64_t i = 1; i < m; i++) {
      int64_t v = base + i;
      seg_t s = segment_of(f, v, base + f->parent[v]);
      R_seg[v] = (double)s.len * g->unit_r[layer[v]];
      C_seg[v] = (double)s.len * g->unit_c[layer[v]];
    }
  }
}

/* Sons of every node of net n, in increasing net-local id (CSR, local ids). */
typedef struct { int64_t cap; int32_t *ptr, *list, *fill; } son_lists;
static void sons_of_net(const or_forest* f, int64_t n, son_lists* S) {
  int64_t base = f->net_ptr[n], m = f->net_ptr[n + 1] - base;
  if (m + 1 > S->cap) {
    S->cap = 2 * (m + 1);
    S->ptr = realloc(S->ptr, S->cap * sizeof(int32_t));
    S->list = realloc(S->list, S->cap * sizeof(int32_t));
    S->fill = realloc(S->fill, S->cap * sizeof(int32_t));
  }
  for (int64_t i = 0; i <= m; i++) S->ptr[i] = 0;
  for (int64_t i = 1; i < m; i++) S->ptr[f->parent[base + i] + 1]++;
  for (int64_t i = 0; i < m; i++) S->ptr[i + 1] += S->ptr[i];
  for (int64_t i = 0; i < m; i++) S->fill[i] = S->ptr[i];
  for (int64_t i = 1; i < m; i++) S->list[S->fill[f->parent[base + i]]++] = (int32_t)i;
}

/* Downstream cap at every junction of net n, children before parents:
 * Cd_J(v) = C_seg[v]/2 + vc (t-b) + Cs_v + sum over sons c, in son order,
 * of (C_seg[c]/2 + Cd_J(c)).  (No segment at the root.) */
static void elmore_cdown(const or_grid* g, const or_forest* f, int64_t n, const son_lists* S,
                         const int8_t* b, const int8_t* t, const double* C_seg, double* CdJ) {
  int64_t base = f->net_ptr[n], m = f->net_ptr[n + 1] - base;
  for (int64_t i = m - 1; i >= 0; i--) {
    int64_t v = base + i;
    double s = (i == 0) ? 0.0 : 0.5 * C_seg[v];
    s = s + g->via_c * (double)(t[v] - b[v]);
    s = s + f->sink_cap[v];
    for (int32_t k = S->ptr[i]; k < S->ptr[i + 1]; k++) {
      int64_t c = base + S->list[k];
      s = s + (0.5 * C_seg[c] + CdJ[c]);
    }
    CdJ[v] = s;
  }
}

void or_elmore(const or_grid* g, const or_forest* f, const int8_t* layer, const int8_t* b,
               const int8_t* t, const double* R_seg, const double* C_seg, double* delay,
               double* CdJ /* scratch V */, double* dJ /* scratch V */) {
  son_lists S = {0, NULL, NULL, NULL};
  for (int64_t n = 0; n < f->num_nets; n++) {
    int64_t base = f->net_ptr[n], m = f->net_ptr[n + 1] - base;
    sons_of_net(f, n, &S);
    elmore_cdown(g, f, n, &S, b, t, C_seg, CdJ);
    dJ[base] = f->r_drv[n] * CdJ[base];
    for (int64_t i = 1; i < m; i++) {
      int64_t v = base + i, p = base + f->parent[v];
      double dX = dJ[p] + rvia(g, layer[p], layer[v]) * (0.5 * C_seg[v] + CdJ[v]);
      dJ[v] = dX + R_seg[v] * CdJ[v];
    }
    for (int64_t i = 0; i < m; i++) {
      int64_t v = base + i;
      int pin = f->pin_layer[v];
      delay[v] = pin >= 0 ? dJ[v] + rvia(g, layer[v], pin) * f->sink_cap[v] : dJ[v];
    }
  }
  free(S.ptr); free(S.list); free(S.fill);
}

/* Adjoint: with Ws(v) = g_v + sum of Ws over sons (children before parents),
 * dR_seg[v] = Cd_J(v) Ws(v);  U_J(root) = R_drv Ws(root);
 * U_X(v) = U_J(p) + Rvia(l_p, l_v) Ws(v);  U_J(v) = U_X(v) + R_seg[v] Ws(v);
 * dC_seg[v] = (U_X(v) + U_J(v)) / 2.  Wsum and U_J are returned too. */
void or_elmore_backward(const or_grid* g, const or_forest* f, const int8_t* layer, const int8_t* b,
                        const int8_t* t, const double* R_seg, const double* C_seg, const double* gd,
                        double* dR, double* dC, double* Wsum, double* UJ, double* CdJ /* scratch */) {
  son_lists S = {0, NULL, NULL, NULL};
  for (int64_t n = 0; n < f->num_nets; n++) {
    int64_t base = f->net_ptr[n], m = f->net_ptr[n + 1] - base;
    sons_of_net(f, n, &S);
    elmore_cdown(g, f, n, &S, b, t, C_seg, CdJ);
    for (int64_t i = m - 1; i >= 0; i--) {
      int64_t v = base + i;
      double s = gd[v];
      for (int32_t k = S.ptr[i]; k < S.ptr[i + 1]; k++) s = s + Wsum[base + S.list[k]];
      Wsum[v] = s;
    }
    dR[base] = 0.0; dC[base] = 0.0;
    UJ[base] = f->r_drv[n] * Wsum[base];
    for (int64_t i = 1; i < m; i++) {
      int64_t v = base + i, p = base + f->parent[v];
      dR[v] = CdJ[v] * Wsum[v];
      double UX = UJ[p] + rvia(g, layer[p], layer[v]) * Wsum[v];
      UJ[v] = UX + R_seg[v] * Wsum[v];
      dC[v] = 0.5 * (UX + UJ[v]);
    }
  }
  free(S.ptr); free(S.list); free(S.fill);
}

/* ------------------------------------------------------------------------ */
/* Net ordering (Sec. III-A, Alg. 1) and pin weights (Sec. III-C)            */
/* ------------------------------------------------------------------------ */
/* Pin weight of Sec. III-C, read as the logistic of the slack ratio (the
 * printed form is garbled; the text says the weight is about 1 for a pin at
 * the worst slack): x = slack / WNS with WNS < 0 the worst slack,
 * w = 1 / (1 + e^{-k (x - b)}); 0 at a node without a pin. */
void or_logistic_pin_weight(int64_t V, const int8_t* pin_layer, const double* slack, double wns, double k,
                            double b, double* w) {
  for (int64_t v = 0; v < V; v++) {
    if (pin_layer[v] < 0) { w[v] = 0.0; continue; }
    double x = slack[v] / wns;
    w[v] = 1.0 / (1.0 + exp(-k * (x - b)));
  }
}

/* Alg. 1's partition of the nets into batches (Divide, then Partition):
 *   C = the largest criticality; the critical nets (crit >= critical_frac C,
 *   C > 0) go by criticality interval: [C, C] first, then [C/2, C),
 *   [C/4, C/2), ... (interval k >= 1 holds C 2^-k <= crit < C 2^-(k-1));
 *   then, with slack given and WNS = the least slack < 0, the other nets with
 *   slack <= slack_ratio WNS by slack interval: slack = WNS first, then the
 *   edges e_j = WNS (1 - j^2 / 100) (interval j >= 1 holds
 *   e_(j-1) < slack <= e_j: 0.99 WNS, 0.96 WNS, ...);
 *   every other net last.
 * Batch ids number the non-empty intervals in that order from 0.  Returns
 * the number of batches. */
int32_t or_partition_batches(int64_t N, const double* crit, const double* slack, double critical_frac,
                             double slack_ratio, int32_t* batch) {
  double C = 0.0, wns = 0.0;
  for (int64_t n = 0; n < N; n++) if (crit[n] > C) C = crit[n];
  if (slack) for (int64_t n = 0; n < N; n++) if (slack[n] < wns) wns = slack[n];
  int used[256] = {0};
  for (int64_t n = 0; n < N; n++) {
    int id = 255;  /* the rest */
    if (C > 0.0 && crit[n] >= critical_frac * C) {
      int k = 0;
      if (crit[n] != C) {
        k = 1;
        while (crit[n] < ldexp(C, -k)) k++;
      }
      id = k < 127 ? k : 127;
    } else if (slack && wns < 0.0 && slack[n] <= slack_ratio * wns) {
      int j = 0;
      if (slack[n] != wns) {
        j = 1;
        while (!(slack[n] <= wns * (1.0 - (double)(j * j) / 100.0))) j++;
      }
      id = 128 + (j < 126 ? j : 126);
    }
    batch[n] = id;
    used[id] = 1;
  }
  int32_t map[256], nb = 0;
  for (int i = 0; i < 256; i++) map[i] = used[i] ? nb++ : -1;
  for (int64_t n = 0; n < N; n++) batch[n] = map[batch[n]];
  return nb;
}
