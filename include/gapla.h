/* gapla.h - C ABI of the GB300 (sm_103a) layer-assignment library.
 *
 * What it computes (arxiv 2507.13375, GAP-LA):
 *   Layer assignment takes a GCell grid with per-layer edge capacities and a
 *   2D GCell routing tree per net, and gives every straight 2D segment a metal
 *   layer of its direction, keeping the planar projection (Sec. II-B, II-D).
 *   One round = the bottom-up tree DP of Alg. 3 with the look-ahead cost of
 *   Sec. III-D, the top-down backtrack of Alg. 4, and the demand/via update of
 *   the demand map D against the capacity map C of Alg. 2.  The Elmore RC-tree
 *   delay of Sec. III-D (d_34 = R_34 (C4+C5+C6+C7)) and its adjoint are exposed
 *   for timing sensitivities.
 *
 * Conventions for every call:
 *   - Every call returns la_status; LA_OK = 0.  On failure la_last_error(ctx)
 *     holds a one-line message.  Invalid input (LA_ERR_INVALID) leaves the
 *     context as it was.  After LA_ERR_CUDA, LA_ERR_TIMEOUT or
 *     LA_ERR_DEVICE_CHECK the context is poisoned: every later call except
 *     la_destroy / la_last_error returns LA_ERR_STATE.
 *   - "device" pointers are CUDA device memory owned by the caller (for
 *     example torch tensors on the context's device); "host" pointers are
 *     ordinary host memory owned by the caller.  The library never frees or
 *     keeps a caller pointer after the call returns, except where stated.
 *   - Work is enqueued on the context's stream (la_create / la_set_stream);
 *     calls return once the work is enqueued, unless stated otherwise.  The
 *     library owns its context and the device memory it allocates for the
 *     loaded grid, forest and round tables (la_device_bytes reports it).
 *   - Node order: every per-node array is in the caller's input node order
 *     (net-major, net-local ids as given in la_net_desc).
 *
 * Layers are 0-based.  dir[l] = 0 means horizontal (H), 1 vertical (V).
 * Public edge layout ("E entries"): layer by layer; an H layer is [y][x] with
 * X-1 edges per row, a V layer is [x][y] with Y-1 edges per column.
 */
#ifndef GAPLA_H
#define GAPLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LA_OK = 0,
  LA_ERR_INVALID = 1,      /* bad argument or malformed input; nothing changed      */
  LA_ERR_CUDA = 2,         /* a CUDA runtime call failed                            */
  LA_ERR_OOM = 3,          /* device allocation failed                              */
  LA_ERR_STATE = 4,        /* call out of order, or context poisoned                */
  LA_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out                    */
  LA_ERR_DEVICE_CHECK = 6  /* a kernel's own bounds/consistency check failed        */
} la_status;

#define LA_MAX_LAYERS 16

typedef struct la_ctx la_ctx;

/* Create a context on CUDA device `device`, enqueuing on `stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
la_status la_create(la_ctx** out, int device, void* stream);
/* Destroy a context and free every device allocation it owns.  NULL is a no-op. */
la_status la_destroy(la_ctx* ctx);
/* Last error message of `ctx` (or of the last failed la_create on this thread
 * when ctx is NULL).  Valid until the next call on the same context. */
const char* la_last_error(const la_ctx* ctx);
/* Change the stream later calls enqueue on. */
la_status la_set_stream(la_ctx* ctx, void* stream);
/* Device bytes currently held by the context. */
la_status la_device_bytes(const la_ctx* ctx, size_t* bytes);
/* Synchronise the stream and check the device error word; LA_OK if clean. */
la_status la_check(la_ctx* ctx);
/* Number of CUDA kernels this context has launched since it was created. */
la_status la_launch_count(const la_ctx* ctx, int64_t* launches);
/* Failure-path hook for tests: the next step of the context that can fail in
 * the given way reports `code` from the host side, exactly as the real
 * failure would be reported; nothing is changed on the device and nothing
 * faults there.  LA_ERR_OOM: the next device allocation of the context fails.
 * LA_ERR_CUDA, LA_ERR_TIMEOUT, LA_ERR_DEVICE_CHECK: the next read of the
 * context's device error word (la_check, la_load_grid, la_load_nets,
 * la_assign_round with stats, la_set_assignment, la_set_state) reports that
 * error, which poisons the context.  LA_OK clears a pending fault; any other
 * code is LA_ERR_INVALID.  The paper has no counterpart. */
la_status la_inject_fault(la_ctx* ctx, la_status code);

/* ---------------------------------------------------------------------------
 * Grid: the GCell grid graph with per-layer edge capacity (Sec. II-A, Alg. 2
 * inputs r, c, vr, X, Y, L, C) and the overflow weight ofw(l) of Eq. 3.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t X, Y, L;         /* 2 <= X, Y <= 16384; 2 <= L <= LA_MAX_LAYERS           */
  const int8_t* dir;       /* host, L: preferred direction, 0 = H, 1 = V            */
  const int32_t* cap;      /* device, E entries, public edge layout, each >= 0      */
  const double* unit_r;    /* host, L: wire resistance per GCell edge (ohm), >= 0    */
  const double* unit_c;    /* host, L: wire capacitance per GCell edge (fF), >= 0    */
  const double* via_r;     /* host, L-1: resistance of the via between l and l+1     */
  double via_c;            /* capacitance of one via (fF), >= 0                      */
  const double* ofw;       /* host, L: overflow weight of Eq. 3, >= 0                */
} la_grid_desc;

/* Load (or replace) the grid.  Copies `cap` into the library's internal
 * layout; resets the demand snapshot D and the history H to zero.  Any loaded
 * forest is dropped.  Errors: LA_ERR_INVALID for sizes/values out of range. */
la_status la_load_grid(la_ctx* ctx, const la_grid_desc* grid);

/* ---------------------------------------------------------------------------
 * Nets: the layer-assignment directed tree of Sec. III-B (Fig. 5): each net's
 * 2D route with extra nodes at bends, so that every tree edge is a straight
 * horizontal or vertical run of GCell edges.  Node 0 of a net is its root and
 * carries the driver pin; parent[v] < v inside a net.
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t num_nets;        /* N >= 1                                                */
  int64_t num_nodes;       /* V = net_ptr[N]                                        */
  const int64_t* net_ptr;  /* device, N+1: nodes of net n are [net_ptr[n], net_ptr[n+1]) */
  const int32_t* x;        /* device, V: GCell column, 0 <= x < X                    */
  const int32_t* y;        /* device, V: GCell row,    0 <= y < Y                    */
  const int32_t* parent;   /* device, V: net-local parent id; -1 exactly at local 0  */
  const int8_t* pin_layer; /* device, V: layer of the node's pin, -1 = no pin; the
                              root must have one (the driver pin)                    */
  const double* sink_cap;  /* device, V: sink pin capacitance (fF) >= 0; exactly 0 at
                              a node without a pin                                  */
  const double* kappa;     /* device, V: sink criticality >= 0 (edge weights, Eq. 4) */
  const double* r_drv;     /* device, N: driver resistance (ohm) >= 0                */
  const int32_t* batch;    /* device, N, or null: the net's batch, 0 <= batch <
                              LA_MAX_BATCHES.  A round assigns the batches one
                              after the other in increasing id; each sees the
                              demand the batches before it committed (the
                              sequential batches of Sec. III-A).  Null: one batch,
                              every net against one snapshot.  In LA_MODE_BATCHED
                              the batches run as level waves of the class kernels
                              with the constant caches, the whole round in one
                              CUDA graph (no persistent kernels, no tuning:
                              tail_threshold and force_split are not used).      */
} la_net_desc;
#define LA_MAX_BATCHES 4096

/* Load the forest (after la_load_grid).  Validates it on the device (parent
 * order, straight segments of length >= 1 inside the grid, pins in range),
 * levelises every tree (level = height above the deepest leaf, Alg. 2) and
 * builds the children lists, segment geometry, and the Eq. 4 edge weights W
 * and the look-ahead upstream resistances r_est (Sec. III-D).  Synchronises
 * the stream.  LA_ERR_INVALID if the forest is malformed (message names the
 * first bad node); the forest loaded before stays loaded, and so it does after
 * an allocation failure (LA_ERR_OOM) before the new forest has passed
 * validation.  After any later error the context holds no forest.  A forest of the same shape as the one
 * before reuses its device blocks and, with the batched form, its tuned plan
 * and captured rounds. */
la_status la_load_nets(la_ctx* ctx, const la_net_desc* nets);

/* ---------------------------------------------------------------------------
 * One layer-assignment round (Alg. 2 over one batch holding every net).
 * ------------------------------------------------------------------------- */
enum { LA_MODE_PLAIN = 0,     /* one kernel launch per tree level (Alg. 2 as printed) */
       LA_MODE_BATCHED = 1 }; /* size-bucketed persistent kernels                     */
enum { LA_WEIGHTS_EQ4 = 0,     /* W = max sink criticality below (Eq. 4), r_est from
                                  distance x average unit R (Sec. III-D)              */
       LA_WEIGHTS_ADJOINT = 1 };/* W and r_est from the last la_reweight_adjoint        */

typedef struct {
  double w_cong;           /* congestion weight w^cong (Alg. 2)                      */
  double w_via;            /* cost per via                                           */
  double w_cap;            /* capacitance weight w^cap (Alg. 2)                      */
  double w_d;              /* delay weight w^d (Alg. 2, Sec. III-D)                  */
  double hist_w;           /* weight of the overflow history in the penalty          */
  int32_t mode;            /* LA_MODE_*                                              */
  int32_t weights;         /* LA_WEIGHTS_*                                           */
  int32_t reset;           /* 1: start from D = 0 and H = 0 (first round)            */
  int32_t no_look_ahead;   /* 1: r_est = 0 for every node, the look-ahead ablation
                            * of the paper's Table VII ("w/o ahead"); W unchanged   */
  int32_t tail_threshold;  /* batched form: 0 = the tuner's plan; T > 0 = the tuned
                            * plan's split and block with the top small-net levels
                            * whose (node, candidate) task counts are all below T
                            * in the one-block tail kernels.  Results do not
                            * depend on it; < 0 is LA_ERR_INVALID                */
  int32_t force_split;     /* batched form: 0 = the tuner's split; k in [4, 15] =
                            * nets of more than 2^k nodes in the persistent
                            * block-per-net kernels, the rest in level waves
                            * (the tuned block and caching kept).  Results do
                            * not depend on it; other values are
                            * LA_ERR_INVALID                                     */
  int32_t local_demand;    /* 1: one shard of a round split over several
                            * contexts by nets (one per GPU): the round ends
                            * with D = the demand of this context's nets only
                            * (H, tof and the overflow statistics untouched);
                            * the caller sums D over the shards (la_get_state,
                            * an all-reduce) and hands the sum to
                            * la_commit_demand before the next round.  0: the
                            * round ends with D, H and the statistics of the
                            * whole forest                                      */
  int32_t reweight_adjoint;/* 1: the round also leaves the adjoint weights of
                            * its new assignment, as la_reweight_adjoint called
                            * after it would (bit for bit; the top-down pass is
                            * done by the backtrack kernels), so that the next
                            * round can take LA_WEIGHTS_ADJOINT.  0: it leaves
                            * the weights as they were.  Other values are
                            * LA_ERR_INVALID                                     */
} la_round_params;

typedef struct {
  double total_cost;       /* sum over nets of the root look-ahead cost J_n          */
  double tof;              /* Eq. 3 total overflow over every (layer, edge)          */
  int64_t relu_overflow;   /* Eq. 2 total overflow, sum of max(0, D - C)             */
  int64_t vias;            /* sum over nodes of t - b                                */
  int64_t wl;              /* GCell edges of wire                                    */
  int64_t wl_per_layer[LA_MAX_LAYERS];
  double ms;               /* device time of the round (CUDA events on the stream)   */
  double ms_dp;            /*   of which the bottom-up DP, all levels (Alg. 3)       */
  double ms_backtrack;     /*   the top-down backtrack, all levels (Alg. 4)          */
  double ms_demand;        /*   demand + line scan (D, H and the next penalty prefix) */
  int64_t launches;        /* kernels this round launched                            */
  /* batched form only: the autotuner's choice (nets with at most 2^split nodes
   * run as level waves, larger ones in the persistent block-per-net kernels) */
  int32_t batch_split, batch_block;
  int64_t batch_big_nets;
  int32_t batch_cached;    /* 1: round-invariant constants cached per weight set  */
  int32_t batch_trials;    /* plans timed to choose it; 0: taken untimed from the
                            * tuning memo (an earlier forest with the same level,
                            * class and size-class bucket offsets)                */
  double batch_tune_ms;    /* its DP + backtrack time when it was chosen         */
  int32_t batch_levels;    /* levels of the small nets (the level waves + tail)   */
  int32_t batch_tail_level;/* first level run by the one-block tail kernels
                            * (= batch_levels: no tail)                          */
  int32_t batch_graph_captured; /* 1: this round captured its CUDA graph (first
                            * round of a weight source, or new addresses, shape,
                            * plan or weights); 0: it replayed the kept graph    */
} la_round_stats;

/* Run one round against the current snapshot (D, H): every net sees the same
 * snapshot.  Afterwards D is the demand of the new assignment and
 * H += max(0, D - C).  If `stats` is non-NULL the call synchronises and fills
 * it; with NULL it only enqueues.  Weights must be >= 0 and finite. */
la_status la_assign_round(la_ctx* ctx, const la_round_params* params, la_round_stats* stats);

/* Ends a round run with local_demand = 1 once the demand of every shard has
 * been summed (Alg. 2 over one demand map, the nets split between contexts):
 * D := demand (device, E entries, public layout, each >= 0), then
 * H += max(0, D - C), the Eq. 2 / Eq. 3 statistics and the penalty prefix of
 * the next round, with the round's hist_w.  Every shard calls it with the same
 * sum, so every shard holds the same snapshot afterwards.  If `stats` is
 * non-NULL the call synchronises and fills tof and relu_overflow (the other
 * fields are zero).  LA_ERR_INVALID for a negative entry (the snapshot is then
 * unchanged); LA_ERR_STATE before any round. */
la_status la_commit_demand(la_ctx* ctx, const int32_t* demand, la_round_stats* stats);

/* Copy the last round's assignment out (device, V each): layer[v] = layer of
 * v's junction (its segment's layer; the driver pin layer at a root), and the
 * via stack [b[v], t[v]] at v.  Any pointer may be NULL. */
la_status la_get_assignment(la_ctx* ctx, int8_t* layer, int8_t* b, int8_t* t);
/* Set the assignment (device, V each, same meaning) that la_rc_from_assignment,
 * la_elmore* and la_reweight_adjoint use.  Checked on the device: layers of the
 * right direction, stacks holding the junction layer, the pin and every child's
 * layer.  Synchronises. */
la_status la_set_assignment(la_ctx* ctx, const int8_t* layer, const int8_t* b, const int8_t* t);
/* Per-net root look-ahead cost J_n of the last round (device, N). */
la_status la_get_net_cost(la_ctx* ctx, double* J);
/* Copy the snapshot out / in (device, E entries each, public layout): demand D
 * and overflow history H.  la_set_state makes (D, H) the snapshot of the next
 * round.  Either pointer may be NULL (NULL in set = leave unchanged). */
la_status la_get_state(la_ctx* ctx, int32_t* demand, int32_t* history);
la_status la_set_state(la_ctx* ctx, const int32_t* demand, const int32_t* history);

/* ---------------------------------------------------------------------------
 * Elmore delay on the RC tree of the current assignment (Sec. II-C, III-D):
 * driver resistance into the root junction; per segment v a via resistor
 * from the parent junction to the segment start (C_seg/2 there), the wire
 * R_seg to v's junction (C_seg/2 plus the via caps there), and at a pin node a
 * via resistor to the pin point holding the sink cap.
 * All arrays: device, V entries, input node order; root entries of R_seg and
 * C_seg are ignored.
 * ------------------------------------------------------------------------- */
/* R_seg[v] = len_v * unit_r[layer v], C_seg[v] = len_v * unit_c[layer v]
 * (0 at roots). */
la_status la_rc_from_assignment(la_ctx* ctx, double* R_seg, double* C_seg);
/* delay[v] = Elmore delay at v's pin point (pin nodes) or junction (others). */
la_status la_elmore(la_ctx* ctx, const double* R_seg, const double* C_seg, double* delay);
/* Adjoint of la_elmore: given g = dL/d delay, writes dL/dR_seg and dL/dC_seg
 * (0 at roots).  Recomputes the downstream caps net by net instead of keeping
 * them from the forward pass. */
la_status la_elmore_backward(la_ctx* ctx, const double* R_seg, const double* C_seg,
                             const double* grad_delay, double* dR_seg, double* dC_seg);

/* The Elmore delays of the current assignment (after a round or
 * la_set_assignment): the RC tree of la_rc_from_assignment's R_seg and C_seg,
 * built from the layers inside the level passes, without the R / C arrays.
 * Equal bit for bit to la_elmore(la_rc_from_assignment(...)).
 *   delay: device, V, input order (written). */
la_status la_elmore_assignment(la_ctx* ctx, double* delay);
/* Timing sensitivities for the next round: with g = kappa on the current
 * assignment's RC tree, W[v] = sum of kappa below v (dT/dR = W * Cdown) and
 * r_est[v] = sum over resistors above v's junction of R * W (dT/dC at v).
 * Later rounds with weights = LA_WEIGHTS_ADJOINT use them. */
la_status la_reweight_adjoint(la_ctx* ctx);
/* Copy the DP weights out (device, V each): W[v] and r_est[v] of the given
 * source (LA_WEIGHTS_EQ4 or LA_WEIGHTS_ADJOINT). */
la_status la_get_weights(la_ctx* ctx, int32_t source, double* W, double* rho);

/* ---------------------------------------------------------------------------
 * Net ordering (Sec. III-A) and pin weights (Sec. III-C).  Context-free: they
 * run on the calling thread's current CUDA device, on `stream`.
 * ------------------------------------------------------------------------- */
/* Pin weights of Sec. III-C: weight[v] = 1 / (1 + e^{-k (slack[v] / wns - b)})
 * at pin nodes (pin_layer[v] >= 0), 0 elsewhere; the paper's k = 10, b = 0.3.
 * The printed formula is garbled (1 / (1 + k (x - b)) would not be near 1 at
 * the worst slack, as the text says the weight is); the logistic is the
 * reading taken.  Passed as la_net_desc.kappa, Eq. 4 then takes the largest
 * weight below each node as its edge weight.
 *   pin_layer: device, V; slack: device, V (the pins' slack; others unread);
 *   wns: the worst negative slack, finite and < 0 (else LA_ERR_INVALID);
 *   weight: device, V, written.  Enqueues only. */
la_status la_logistic_pin_weight(const int8_t* pin_layer, const double* slack, int64_t V, double wns, double k,
                                 double b, double* weight, void* stream);
/* Alg. 1's partition of the nets into batches (Divide, then Partition):
 *   C = the largest criticality; the critical nets (crit >= critical_frac C,
 *   C > 0) first, by criticality interval: [C, C], then [C/2, C), [C/4, C/2),
 *   ... (interval k >= 1 holds C 2^-k <= crit < C 2^-(k-1));
 *   then, with slack given and WNS = the least slack < 0, the other nets with
 *   slack <= slack_ratio WNS, by slack interval: slack = WNS, then
 *   e_(j-1) < slack <= e_j for the edges e_j = WNS (1 - j^2 / 100)
 *   (0.99 WNS, 0.96 WNS, ...);
 *   every other net last.
 * The batch ids number the non-empty intervals in that order from 0 (a
 * forest's la_net_desc.batch).  The paper counts critical paths through a net
 * as its criticality and takes its worst pin slack as its slack; both come
 * from the caller (static timing analysis is outside this library).
 *   crit: device, N, finite and >= 0; slack: device, N, finite, or NULL;
 *   critical_frac, slack_ratio in (0, 1] (the paper's 0.7 for the slack);
 *   batch: device, N, written; num_batches: host, written.
 * Synchronises the stream; allocates and frees a small scratch buffer.
 * LA_ERR_INVALID for a negative or non-finite input (batch is then undefined). */
la_status la_partition_batches(const double* crit, const double* slack, int64_t N, double critical_frac,
                               double slack_ratio, int32_t* batch, int32_t* num_batches, void* stream);

/* Measurement helper (the paper has no counterpart): the rate of FP64 fused
 * multiply-adds this GPU sustains, from a kernel of independent FMA chains on
 * every SM (about 40 G FMAs, timed with CUDA events on `stream` after a
 * warm-up launch).  The tree DP is bound by FP64 arithmetic on GB300, so its
 * roofline is reported against this rate beside the nominal pipe peak.
 * `device` becomes current for the call and the previous device is restored;
 * allocates and frees a small output buffer; synchronises the stream.
 *   dfma_per_s: host, written with the FMAs per second. */
la_status la_probe_fp64(int device, void* stream, double* dfma_per_s);

/* ---------------------------------------------------------------------------
 * Allocation-free Elmore forward pass.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at all,
 * for example code whose device memory is entirely owned by another
 * allocator, or code on a latency-critical path that must not call
 * cudaMalloc (which may synchronise the device and takes unbounded time).
 *
 * It computes what la_elmore computes (delay[v] at v's pin point for pin
 * nodes, at its junction otherwise), with the same expressions in the same
 * order (downstream caps summed over the sons in increasing id), so the two
 * agree bit for bit; it takes the forest and the assignment directly, without
 * a context, and its own code allocates nothing.  Its scratch (16 bytes per
 * node: a downstream cap and two son links, plus a 256-byte header) is a fixed
 * device array compiled into the library, LA_STATIC_MAX_NODES nodes large
 * (32 MiB), which every GPU that has loaded the library's device code holds
 * until the process exits.
 *   nets:           device pointers; net_ptr, parent, pin_layer, sink_cap and
 *                   r_drv are read (x, y, kappa are not)
 *   layer, b, t:    device, V: junction layers and via stacks (input order,
 *                   as la_get_assignment returns them)
 *   L, via_r, via_c: the layer count, host via_r[L-1] and the via cap
 *   R_seg, C_seg:   device, V (root entries ignored); delay: device, V output
 *   stream:         cudaStream_t to enqueue on (NULL = legacy default stream)
 * Runs on the calling thread's current CUDA device; all pointers must be on
 * it.  The first call on a device does a one-time set-up there: with CUDA's
 * lazy module loading the runtime loads the library's device code and commits
 * the fixed array at that point (an allocation by the CUDA runtime, which may
 * synchronise), and the call looks up the array's device address
 * (cudaGetSymbolAddress).  Make one warm-up call per device before any
 * latency-critical use and before any stream capture.  Every call uses the
 * same scratch, which keeps the last call's contents (each call clears the
 * flag word it needs), so calls that overlap on the GPU (other streams, other
 * host threads) race.  Returns LA_ERR_INVALID for more than
 * LA_STATIC_MAX_NODES nodes or bad arguments (la_last_error(NULL) says
 * which).  Malformed input is reported in the output instead of faulting: if
 * net_ptr does not rise strictly from 0 to num_nodes every delay is NaN; a net
 * whose parent ids are out of order, or whose layers, pins or stacks are out
 * of range, gets NaN delays and the other nets are computed as usual. */
#define LA_STATIC_MAX_NODES (1 << 21)
la_status la_elmore_static(const la_net_desc* nets, const int8_t* layer, const int8_t* b, const int8_t* t,
                           int32_t L, const double* via_r, double via_c, const double* R_seg,
                           const double* C_seg, double* delay, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GAPLA_H */
