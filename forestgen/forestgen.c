/* forestgen.c - seeded synthetic inputs for layer assignment: a GCell grid with
 * per-layer edge capacities, and a forest of 2D routing trees (one per net).
 *
 * This module is input data only.  It holds none of the layer-assignment
 * arithmetic (no costs, no delays, no DP).  Both the CUDA library's tests and
 * the CPU oracle consume what it writes.
 *
 * Trees.  The input of layer assignment is a 2D GCell-level routing solution
 * (Sec. II-D).  Here each net's 2D route is a rectilinear minimum spanning
 * tree over its pins (Prim on Manhattan distance from pin 0, the driver).  Each
 * MST edge is drawn as an "L": first the horizontal leg from the parent end,
 * then the vertical leg.  A bend node is inserted at the corner, so every tree
 * edge is a straight H or V segment.  That is the layer-assignment directed
 * tree of Sec. III-B / Fig. 5: layer changes happen only at nodes.
 *
 * Output CSR (per net, nodes numbered so that parent < child):
 *   net_ptr[N+1]  int64   node range of each net
 *   x, y          int32   GCell coordinates of each node
 *   parent        int32   net-local parent index, -1 for the root (local 0)
 *   pin_layer     int8    pin layer (0 for every pin here), -1 for a bend
 *   sink_cap      f64     sink pin capacitance (fF), 0 for bends / pure driver
 *   kappa         f64     sink criticality, 0 for bends / pure driver
 *   r_drv[N]      f64     driver resistance (ohm)
 * Pins falling in one GCell are merged into the first of them: their sink
 * caps add up and their criticality is the maximum.
 *
 * Random numbers: a counter-based generator.  Every entity (a net, a grid
 * edge, a cluster centre) owns a stream keyed by (seed, stream tag, index),
 * so the output does not depend on the thread count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
  int32_t X, Y, L;
  int32_t cap_lo, cap_hi;   /* capacity: uniform integer in [cap_lo, cap_hi]      */
  double block_frac;        /* probability that a (layer, edge) capacity is halved */
  int64_t num_nets;
  int32_t pin_dist;         /* 0: uniform int [pin_a, pin_b]
                               1: 2 + Geometric(pin_p) failures, capped at pin_b
                               2: Zipf(exponent pin_p) on [pin_a, pin_b]           */
  int32_t pin_a, pin_b;
  double pin_p;
  int32_t clustered;        /* 0: pins uniform on the grid; 1: Gaussian mixture   */
  int32_t n_centres;
  double sigma;
  double rdrv_lo, rdrv_hi;  /* driver R, uniform                                 */
  double csink_lo, csink_hi;/* sink pin cap, uniform                             */
  double kappa_lo, kappa_hi;/* sink criticality, uniform                         */
  uint64_t seed;
  int32_t threads;          /* 0: all online CPUs                                */
} fg_params;

enum { ST_CAP = 1, ST_NET = 2, ST_CENTRE = 3 };

/* ---- counter-based random numbers (SplitMix64 finaliser as the mixer) ---- */
static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
typedef struct { uint64_t key, ctr; } rng_t;
static rng_t rng_make(uint64_t seed, uint64_t tag, uint64_t index) {
  rng_t r;
  r.key = mix64(mix64(seed ^ mix64(tag)) ^ mix64(index + 0x632BE59BD9B4E019ull));
  r.ctr = 0;
  return r;
}
static inline uint64_t rng_u64(rng_t* r) { return mix64(r->key + (r->ctr++) * 0xD1B54A32D192ED03ull); }
static inline double rng_u01(rng_t* r) { return (double)(rng_u64(r) >> 11) * 0x1.0p-53; }
static inline int32_t rng_int(rng_t* r, int32_t lo, int32_t hi) {
  return lo + (int32_t)(rng_u64(r) % (uint64_t)(hi - lo + 1));
}
static inline double rng_unif(rng_t* r, double lo, double hi) { return lo + (hi - lo) * rng_u01(r); }
static double rng_normal(rng_t* r) { /* Box-Muller, cosine branch */
  double u1 = 1.0 - rng_u01(r), u2 = rng_u01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static int n_threads(int32_t req) {
  if (req > 0) return req;
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n < 1 ? 1 : (n > 256 ? 256 : (int)n);
}

/* ---------------------------- grid capacity ---------------------------- */
/* Public edge layout, layer by layer: an H layer (even l) is [y][x] with
 * X-1 edges per row, a V layer (odd l) is [x][y] with Y-1 edges per column. */
int64_t fg_grid_edges(int32_t X, int32_t Y, int32_t L) {
  int64_t e = 0;
  for (int l = 0; l < L; l++) e += (l % 2 == 0) ? (int64_t)Y * (X - 1) : (int64_t)X * (Y - 1);
  return e;
}
typedef struct { const fg_params* p; int32_t* cap; int64_t lo, hi; } cap_job;
static void* cap_worker(void* arg) {
  cap_job* j = (cap_job*)arg;
  for (int64_t g = j->lo; g < j->hi; g++) {
    rng_t r = rng_make(j->p->seed, ST_CAP, (uint64_t)g);
    int32_t c = rng_int(&r, j->p->cap_lo, j->p->cap_hi);
    if (rng_u01(&r) < j->p->block_frac) c = c / 2;
    j->cap[g] = c;
  }
  return NULL;
}
void fg_grid_cap(const fg_params* p, int32_t* cap) {
  int64_t E = fg_grid_edges(p->X, p->Y, p->L);
  int T = n_threads(p->threads);
  pthread_t th[256];
  cap_job jobs[256];
  for (int t = 0; t < T; t++) {
    jobs[t].p = p; jobs[t].cap = cap;
    jobs[t].lo = E * t / T; jobs[t].hi = E * (t + 1) / T;
    pthread_create(&th[t], NULL, cap_worker, &jobs[t]);
  }
  for (int t = 0; t < T; t++) pthread_join(th[t], NULL);
}

/* ------------------------------ nets ------------------------------------ */
typedef struct {
  int64_t n_nodes, cap_nodes;
  int32_t *x, *y, *parent;
  int8_t* pin_layer;
  double *sink_cap, *kappa;
  int64_t* net_nodes; /* node count of each net of the chunk */
  double* r_drv;
} chunk_buf;

static void buf_reserve(chunk_buf* b, int64_t extra) {
  if (b->n_nodes + extra <= b->cap_nodes) return;
  int64_t nc = b->cap_nodes ? b->cap_nodes : 1024;
  while (nc < b->n_nodes + extra) nc *= 2;
  b->x = realloc(b->x, nc * sizeof(int32_t));
  b->y = realloc(b->y, nc * sizeof(int32_t));
  b->parent = realloc(b->parent, nc * sizeof(int32_t));
  b->pin_layer = realloc(b->pin_layer, nc * sizeof(int8_t));
  b->sink_cap = realloc(b->sink_cap, nc * sizeof(double));
  b->kappa = realloc(b->kappa, nc * sizeof(double));
  b->cap_nodes = nc;
}

typedef struct { int32_t x, y, idx; } pin_key;
static int cmp_pin(const void* a, const void* b) {
  const pin_key *p = (const pin_key*)a, *q = (const pin_key*)b;
  if (p->x != q->x) return p->x < q->x ? -1 : 1;
  if (p->y != q->y) return p->y < q->y ? -1 : 1;
  return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

typedef struct {
  const fg_params* p;
  const int32_t* centres; /* 2 * n_centres */
  const double* zipf_cdf; /* pin_b - pin_a + 1 entries, or NULL */
  int64_t net_lo, net_hi;
  chunk_buf out;
} net_job;

static int32_t draw_pins(const fg_params* p, const double* zcdf, rng_t* r) {
  if (p->pin_dist == 0) return rng_int(r, p->pin_a, p->pin_b);
  if (p->pin_dist == 1) {
    int32_t k = 0;
    while (2 + k < p->pin_b && rng_u01(r) >= p->pin_p) k++;
    return 2 + k;
  }
  /* Zipf by inverse CDF over the tabulated support */
  double u = rng_u01(r);
  int32_t lo = 0, hi = p->pin_b - p->pin_a;
  while (lo < hi) {
    int32_t mid = (lo + hi) / 2;
    if (zcdf[mid] > u) hi = mid; else lo = mid + 1;
  }
  return p->pin_a + lo;
}

static int32_t clampi(int32_t v, int32_t lo, int32_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void* net_worker(void* arg) {
  net_job* j = (net_job*)arg;
  const fg_params* p = j->p;
  int64_t nn = j->net_hi - j->net_lo;
  j->out.net_nodes = malloc((nn > 0 ? nn : 1) * sizeof(int64_t));
  j->out.r_drv = malloc((nn > 0 ? nn : 1) * sizeof(double));
  int32_t cap_pins = 0;
  int32_t *px = NULL, *py = NULL, *rep = NULL, *par = NULL, *key = NULL, *node_of = NULL, *uniq = NULL;
  double *pc = NULL, *pk = NULL;
  char* in_tree = NULL;
  pin_key* keys = NULL;
  for (int64_t n = j->net_lo; n < j->net_hi; n++) {
    rng_t r = rng_make(p->seed, ST_NET, (uint64_t)n);
    int32_t np = draw_pins(p, j->zipf_cdf, &r);
    if (np > cap_pins) {
      cap_pins = np;
      px = realloc(px, np * sizeof(int32_t)); py = realloc(py, np * sizeof(int32_t));
      rep = realloc(rep, np * sizeof(int32_t)); par = realloc(par, np * sizeof(int32_t));
      key = realloc(key, np * sizeof(int32_t)); node_of = realloc(node_of, np * sizeof(int32_t));
      uniq = realloc(uniq, np * sizeof(int32_t));
      pc = realloc(pc, np * sizeof(double)); pk = realloc(pk, np * sizeof(double));
      in_tree = realloc(in_tree, np); keys = realloc(keys, np * sizeof(pin_key));
    }
    j->out.r_drv[n - j->net_lo] = rng_unif(&r, p->rdrv_lo, p->rdrv_hi);
    int32_t cx = 0, cy = 0;
    if (p->clustered) {
      int32_t c = rng_int(&r, 0, p->n_centres - 1);
      cx = j->centres[2 * c]; cy = j->centres[2 * c + 1];
    }
    for (int32_t i = 0; i < np; i++) {
      if (p->clustered) {
        double zx = rng_normal(&r), zy = rng_normal(&r);
        px[i] = clampi((int32_t)llround(cx + p->sigma * zx), 0, p->X - 1);
        py[i] = clampi((int32_t)llround(cy + p->sigma * zy), 0, p->Y - 1);
      } else {
        px[i] = rng_int(&r, 0, p->X - 1);
        py[i] = rng_int(&r, 0, p->Y - 1);
      }
      if (i == 0) { pc[i] = 0.0; pk[i] = 0.0; }
      else { pc[i] = rng_unif(&r, p->csink_lo, p->csink_hi); pk[i] = rng_unif(&r, p->kappa_lo, p->kappa_hi); }
    }
    /* merge pins that share a GCell into the lowest-index one */
    for (int32_t i = 0; i < np; i++) { keys[i].x = px[i]; keys[i].y = py[i]; keys[i].idx = i; }
    qsort(keys, np, sizeof(pin_key), cmp_pin);
    for (int32_t a = 0; a < np;) {
      int32_t b = a;
      while (b < np && keys[b].x == keys[a].x && keys[b].y == keys[a].y) b++;
      int32_t first = keys[a].idx; /* sorted by idx within a run */
      for (int32_t k = a; k < b; k++) rep[keys[k].idx] = first;
      a = b;
    }
    int32_t m = 0;
    for (int32_t i = 0; i < np; i++) {
      if (rep[i] == i) uniq[m++] = i;
      else { pc[rep[i]] += pc[i]; if (pk[i] > pk[rep[i]]) pk[rep[i]] = pk[i]; }
    }
    /* Prim over the unique pins (positions in uniq order; uniq[0] = pin 0) */
    for (int32_t a = 0; a < m; a++) { in_tree[a] = 0; key[a] = INT32_MAX; par[a] = -1; }
    buf_reserve(&j->out, 2 * (int64_t)m);
    int64_t base = j->out.n_nodes, cnt = 0;
    int32_t cur = 0;
    in_tree[0] = 1;
    /* emit root */
    {
      int32_t i = uniq[0];
      j->out.x[base] = px[i]; j->out.y[base] = py[i]; j->out.parent[base] = -1;
      j->out.pin_layer[base] = 0; j->out.sink_cap[base] = pc[i]; j->out.kappa[base] = pk[i];
      node_of[0] = 0; cnt = 1;
    }
    for (int32_t step = 1; step < m; step++) {
      int32_t ic = uniq[cur];
      for (int32_t a = 0; a < m; a++) {
        if (in_tree[a]) continue;
        int32_t ia = uniq[a];
        int32_t d = abs(px[ia] - px[ic]) + abs(py[ia] - py[ic]);
        if (d < key[a]) { key[a] = d; par[a] = cur; }
      }
      int32_t best = -1;
      for (int32_t a = 0; a < m; a++)
        if (!in_tree[a] && (best < 0 || key[a] < key[best])) best = a;
      in_tree[best] = 1;
      int32_t ib = uniq[best], ipar = uniq[par[best]];
      int32_t pnode = node_of[par[best]];
      if (px[ib] != px[ipar] && py[ib] != py[ipar]) {
        int64_t v = base + cnt;
        j->out.x[v] = px[ib]; j->out.y[v] = py[ipar]; j->out.parent[v] = pnode;
        j->out.pin_layer[v] = -1; j->out.sink_cap[v] = 0.0; j->out.kappa[v] = 0.0;
        pnode = (int32_t)cnt;
        cnt++;
      }
      int64_t v = base + cnt;
      j->out.x[v] = px[ib]; j->out.y[v] = py[ib]; j->out.parent[v] = pnode;
      j->out.pin_layer[v] = 0; j->out.sink_cap[v] = pc[ib]; j->out.kappa[v] = pk[ib];
      node_of[best] = (int32_t)cnt;
      cnt++;
      cur = best;
    }
    j->out.n_nodes += cnt;
    j->out.net_nodes[n - j->net_lo] = cnt;
  }
  free(px); free(py); free(rep); free(par); free(key); free(node_of); free(uniq);
  free(pc); free(pk); free(in_tree); free(keys);
  return NULL;
}

typedef struct {
  int T;
  int64_t num_nets, num_nodes;
  net_job* jobs;
} fg_handle;

fg_handle* fg_generate(const fg_params* p) {
  fg_handle* h = calloc(1, sizeof(fg_handle));
  int T = n_threads(p->threads);
  if (p->num_nets < T * 64) T = (int)(p->num_nets / 64) + 1;
  h->T = T;
  h->num_nets = p->num_nets;
  h->jobs = calloc(T, sizeof(net_job));
  int32_t* centres = NULL;
  if (p->clustered) {
    centres = malloc(2 * sizeof(int32_t) * p->n_centres);
    for (int32_t c = 0; c < p->n_centres; c++) {
      rng_t r = rng_make(p->seed, ST_CENTRE, (uint64_t)c);
      centres[2 * c] = rng_int(&r, 0, p->X - 1);
      centres[2 * c + 1] = rng_int(&r, 0, p->Y - 1);
    }
  }
  double* zcdf = NULL;
  if (p->pin_dist == 2) {
    int32_t K = p->pin_b - p->pin_a + 1;
    zcdf = malloc(K * sizeof(double));
    double s = 0.0;
    for (int32_t k = 0; k < K; k++) { s += pow((double)(p->pin_a + k), -p->pin_p); zcdf[k] = s; }
    for (int32_t k = 0; k < K; k++) zcdf[k] /= s;
    zcdf[K - 1] = 2.0; /* guard: u < 1 always lands inside the support */
  }
  pthread_t th[256];
  for (int t = 0; t < T; t++) {
    net_job* j = &h->jobs[t];
    j->p = p; j->centres = centres; j->zipf_cdf = zcdf;
    j->net_lo = p->num_nets * t / T; j->net_hi = p->num_nets * (t + 1) / T;
    pthread_create(&th[t], NULL, net_worker, j);
  }
  for (int t = 0; t < T; t++) pthread_join(th[t], NULL);
  free(centres); free(zcdf);
  for (int t = 0; t < T; t++) h->num_nodes += h->jobs[t].out.n_nodes;
  return h;
}
int64_t fg_num_nodes(const fg_handle* h) { return h->num_nodes; }
int64_t fg_num_nets(const fg_handle* h) { return h->num_nets; }

void fg_export(const fg_handle* h, int64_t* net_ptr, int32_t* x, int32_t* y, int32_t* parent,
               int8_t* pin_layer, double* sink_cap, double* kappa, double* r_drv) {
  int64_t node_off = 0, net_off = 0;
  net_ptr[0] = 0;
  for (int t = 0; t < h->T; t++) {
    const net_job* j = &h->jobs[t];
    int64_t nn = j->net_hi - j->net_lo, nv = j->out.n_nodes;
    memcpy(x + node_off, j->out.x, nv * sizeof(int32_t));
    memcpy(y + node_off, j->out.y, nv * sizeof(int32_t));
    memcpy(parent + node_off, j->out.parent, nv * sizeof(int32_t));
    memcpy(pin_layer + node_off, j->out.pin_layer, nv * sizeof(int8_t));
    memcpy(sink_cap + node_off, j->out.sink_cap, nv * sizeof(double));
    memcpy(kappa + node_off, j->out.kappa, nv * sizeof(double));
    memcpy(r_drv + net_off, j->out.r_drv, nn * sizeof(double));
    int64_t acc = node_off;
    for (int64_t k = 0; k < nn; k++) { acc += j->out.net_nodes[k]; net_ptr[net_off + k + 1] = acc; }
    node_off += nv; net_off += nn;
  }
}

void fg_free(fg_handle* h) {
  if (!h) return;
  for (int t = 0; t < h->T; t++) {
    chunk_buf* b = &h->jobs[t].out;
    free(b->x); free(b->y); free(b->parent); free(b->pin_layer); free(b->sink_cap);
    free(b->kappa); free(b->net_nodes); free(b->r_drv);
  }
  free(h->jobs);
  free(h);
}
