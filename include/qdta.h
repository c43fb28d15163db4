/*
 * qdta.h -- C ABI of libqdta, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of quasi-dynamic traffic assignment (QDTA) from
 * Chan et al., "Quasi-Dynamic Traffic Assignment using High Performance
 * Computing", arXiv 2104.12911.
 *
 * Units and formats used by every call:
 *   - nodes 0..V-1; links 0..L-1 sorted by (tail, head); link id = position;
 *   - link times are int32 counts of the graph's time quantum (e.g. 0.01 s),
 *     at least 1; distances are int64 counts of the quantum;
 *   - trip amounts and all-or-nothing link flows are int64 fixed point with
 *     32 fractional bits (1 trip = 2^32);
 *   - FW link flows are float64 trips in the interval; capacities float64
 *     vehicles per hour;
 *   - every sum over links (objective, slopes, gap) is the exact sum of the
 *     per-link terms each rounded to nearest-even at 2^-32, so results do not
 *     depend on reduction order (and match the CPU oracle bit for bit).
 *
 * Memory: arguments named *_host are host memory; every other array is
 * device memory on the graph's device, read or written in stream order on
 * `stream` (a cudaStream_t passed as void*, NULL = legacy default stream).
 * The caller owns all arrays it passes.  A graph handle owns a device copy
 * of the network plus a grow-only workspace and must be used from one host
 * thread / one stream at a time.
 *
 * Errors: every call returns a status (QDTA_OK = 0; negative = error, the
 * outputs are undefined; positive = QDTA_ENOTCONV, the outputs are valid but
 * the tolerance was not met within max_iter).  qdta_last_error() returns a
 * thread-local message describing the last failure.  No C++ exception
 * crosses this interface.
 */
#ifndef QDTA_H
#define QDTA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QDTA_OK 0
#define QDTA_EINVAL (-1)     /* invalid argument or graph */
#define QDTA_ENOMEM (-2)     /* device allocation failed */
#define QDTA_ECUDA (-3)      /* CUDA runtime error */
#define QDTA_ETIMEOUT (-4)   /* a bounded device wait or loop gave up */
#define QDTA_ENONFINITE (-5) /* a NaN/inf flow, capacity or cost, or a term beyond 2^68 */
#define QDTA_EUNREACH (-6)   /* a destination is unreachable from an origin */
#define QDTA_EOVERFLOW (-7)  /* a distance exceeded the packed range: 2^(64-ceil(log2(L+1))), or 2^61
                                 for rank-keyed keys (graphs above 10,240 nodes, all degrees <= 4) */
#define QDTA_ENOTCONV 1      /* valid result, tolerance not met within max_iter */

#define QDTA_TO_ROOT 0   /* dist/parent toward the root (destination trees, reverse graph) */
#define QDTA_FROM_ROOT 1 /* dist/parent from the root (origin trees, forward graph) */

#define QDTA_STEP_MSA 0       /* alpha_k = 1/(k+1) (method of successive averages) */
#define QDTA_STEP_PAPER_QN3 1 /* quasi-Newton on three objective values per sweep (Alg. 8-9, Eq. 9) */
#define QDTA_STEP_SWEEP8 2    /* bracketing on the exact slope at eight step sizes per sweep */
#define QDTA_STEP_EXACT 3     /* Newton on the exact slope to |d alpha| < 1e-14 (used by the adjoint) */

#define QDTA_STOP_NONE 0      /* run exactly max_iter steps */
#define QDTA_STOP_PAPER_OBJ 1 /* |C(f) - C(f_new)| / C(f) < tol (Section 4, Converged) */
#define QDTA_STOP_REL_GAP 2   /* -1e-12 <= (sum c f - sum c g) / sum c f <= tol: a negative gap
                                 (possible with truncated loading, Eq. 2) does not stop */

/* Objective (Section 3 names both; the paper solves the user equilibrium).
 * QDTA_OBJ_SO minimises the total cost sum f c(f): routing on the quantised
 * marginal costs c + f c', line search and PAPER_OBJ stop on the total cost,
 * REL_GAP on the marginal costs; loading and truncation keep the link times. */
#define QDTA_OBJ_UE 0
#define QDTA_OBJ_SO 1

/* Truncation rule of Eq. 2 (how a trip that does not finish its interval
 * is carried to the next one).  Both rules load the same links: link a of a
 * trip's path is loaded in the interval the trip enters it, i.e. iff the
 * elapsed time on reaching its tail is < dt.
 *  QDTA_TRUNC_NODE: the trip waits at the first node whose elapsed time is
 *    >= dt (it may overshoot dt by up to one link).
 *  QDTA_TRUNC_CARRY: Section 3.4's alternative -- a trip whose next link
 *    would end after dt stays on that link, carrying the fraction of it
 *    covered, f = floor((dt - elapsed) 2^32 / q) in units of 2^-32.  In the
 *    next interval it first covers the rest of the link at that interval's
 *    time q, q - round(q f / 2^32) quanta (halves up), or, when the rest
 *    exceeds dt, stays on it with f + floor(dt 2^32 / q); from the head it is
 *    rerouted.  A link longer than dt is crossed over several intervals.
 *    Residual trips on a link merge per (root, link) with the amount-weighted
 *    mean fraction (floor, exact integers). */
#define QDTA_TRUNC_NODE 0
#define QDTA_TRUNC_CARRY 1

#define QDTA_SCHEDULE_PLAIN 0 /* host launch loop, one host sync per decision */
#define QDTA_SCHEDULE_GRAPH 1 /* whole FW loop in one CUDA graph with device-side control */

#define QDTA_DIST_INF INT64_MAX

typedef struct qdta_graph qdta_graph;
typedef struct qdta_tape qdta_tape;

/* Network description (host arrays, copied by qdta_graph_create).
 * Section 3.1: G = (V, A) with capacity C_a and free-flow time c_{0,a}. */
typedef struct {
  int32_t n_nodes;             /* V >= 1 */
  int32_t n_links;             /* L >= 0, L < 2^24 */
  const int32_t *tail;         /* [L] nondecreasing */
  const int32_t *head;         /* [L], ties in tail sorted by head */
  const int32_t *fftime_q;     /* [L] free-flow time in quanta, >= 1 */
  const double *capacity_vph;  /* [L] > 0, finite */
  double alpha;                /* BPR alpha (Eq. 1), >= 0 */
  int32_t beta;                /* BPR beta (Eq. 1), integer in [1, 16] */
  double quantum_s;            /* seconds per time quantum, > 0 */
} qdta_graph_desc;

/* Demand of one interval, grouped by destination root (device arrays).
 * Item k carries amount_fx[k] trips from node src[k] to node roots[root_idx[k]]
 * (d_{p,q}(i) of Section 3.1). */
typedef struct {
  int32_t n_roots;
  const int32_t *roots;      /* [n_roots] destination nodes */
  int64_t n_items;
  const int32_t *root_idx;   /* [n_items] in [0, n_roots) */
  const int32_t *src;        /* [n_items] origin nodes */
  const int64_t *amount_fx;  /* [n_items] >= 0 */
  /* Trips carried on a link (QDTA_TRUNC_CARRY residuals; both nullable):
   * carry_link[k] >= 0 puts item k on that link, whose tail must be src[k],
   * having covered the fraction carry_frac[k] / 2^32 of it
   * (0 <= carry_frac < 2^32); -1 (or NULL) starts the item at src[k]. */
  const int64_t *carry_frac;
  const int32_t *carry_link;
} qdta_od;

typedef struct {
  int32_t step;        /* QDTA_STEP_* */
  int32_t stop;        /* QDTA_STOP_* */
  int32_t max_iter;    /* FW steps after the initial all-or-nothing, >= 0 */
  int32_t ls_max;      /* L of Alg. 8: at most ls_max - 1 quasi-Newton sweeps; sweep cap otherwise */
  double tol;          /* T0 of the stop rule */
  double ls_dx;        /* finite-difference step of Eq. 9 */
  double ls_t1;        /* T1 of Alg. 8 (relative slope: |C'| < T1 |C|) */
  double ls_t2;        /* T2 of Alg. 8 / bracket width of SWEEP8 */
  int32_t schedule;    /* QDTA_SCHEDULE_* */
  int32_t record_tape; /* qdta_assign_interval: keep what qdta_backward needs (QDTA_OBJ_UE only) */
  int32_t objective;   /* QDTA_OBJ_UE (the paper's user equilibrium) or QDTA_OBJ_SO */
  int32_t truncation;  /* QDTA_TRUNC_NODE or QDTA_TRUNC_CARRY (qdta_run_day's residual demand) */
} qdta_params;

typedef struct {
  int32_t iterations;  /* accepted FW steps */
  int32_t aon_calls;   /* shortest-path batches (all-or-nothing assignments) run */
  int32_t ls_passes;   /* link sweeps spent in line searches */
  int32_t converged;   /* 1 if the stop rule was met */
  double rel_gap;      /* last measured gap (relative objective change in PAPER_OBJ mode) */
  double objective;    /* Beckmann objective of the returned flows (quanta x trips) */
  int64_t n_items;     /* demand items solved (after merging residual demand) */
  double dual_gap;     /* last relative duality gap (sum c f - sum c g) / sum c f, any stop rule */
} qdta_stats;

/* Output buffer for residual demand (device arrays, caller-owned). */
typedef struct {
  int64_t capacity;    /* entries available */
  int32_t *root_idx;   /* [capacity] */
  int32_t *src;        /* [capacity] stop node s, the new origin */
  int64_t *amount_fx;  /* [capacity] */
  int64_t count;       /* written by the library (host field): entries produced */
  int64_t *carry_frac; /* [capacity] covered fractions (0 at a node); required with QDTA_TRUNC_CARRY */
  int32_t *carry_link; /* [capacity] carrying link, -1 at a node; required with QDTA_TRUNC_CARRY */
} qdta_residual;

/* Per-kernel CUDA-event timings accumulated while profiling is enabled
 * (plain schedule only; graph launches record nothing here). */
typedef struct {
  int64_t sssp_launches;
  double sssp_ms;
  int64_t sssp_roots;       /* roots solved by those launches */
  int64_t load_launches;
  double load_ms;
  int64_t sweep_launches;
  double sweep_ms;
  int64_t kernel_launches;  /* all kernels this library launched (process-wide, any schedule;
                               graph schedules count each captured kernel once) */
  int64_t sssp_rounds;      /* frontier rounds summed over the roots solved */
  int64_t sssp_relaxations; /* link relaxations summed over the roots solved */
  int64_t sssp_cell_activations; /* cell activations (cell-partitioned kernel) */
  int64_t sssp_redo_batches; /* 32-bit-key batches rerun with 64-bit keys (a distance >= 2^29 quanta) */
} qdta_profile;

/* ---------------------------------------------------------------------- */

/* Copy the network to `device` and build its forward/reverse adjacency.
 * Section 3.1 (graph, c_0, C), Eq. 1 (alpha, beta).  Returns QDTA_EINVAL on
 * unsorted links, ids out of range, fftime_q < 1, capacity <= 0 or not
 * finite, beta outside [1, 16], L >= 2^24. */
int qdta_graph_create(const qdta_graph_desc *desc, int device, qdta_graph **out);
int qdta_graph_destroy(qdta_graph *g);

/* Replace the link capacities C_a (Eq. 1, vehicles per hour) of an existing
 * graph by capacity_vph [L], a DEVICE array on `stream`, without rebuilding
 * the graph (for repeated solves over changing capacities, e.g. a training
 * loop differentiating through qdta_assign_interval).  Every value must be
 * finite and > 0: otherwise QDTA_EINVAL and the graph keeps its capacities.
 * Later calls on the graph use the new values; a tape recorded earlier keeps
 * the capacities of its own solve.  Synchronises `stream`. */
int qdta_graph_set_capacity(qdta_graph *g, const double *capacity_vph, void *stream);

/* Batched single-source shortest paths (the Get_shortest_path of Alg. 3 and
 * Alg. 7, for all nodes at once).  For each root r and node v:
 * TO_ROOT: dist = shortest time v -> roots[r]; parent = the smallest link id
 * among the links leaving v that begin a shortest path to the root.
 * FROM_ROOT: dist = shortest time roots[r] -> v; parent = the smallest link
 * id among the links entering v that end a shortest path from the root.
 * parent = -1 at the root and at unreachable nodes (dist = QDTA_DIST_INF).
 * cost_q [L] int32 >= 1; roots [R]; parent_link [R*V] row-major by root;
 * dist [R*V] or NULL.  QDTA_EOVERFLOW if a distance exceeds the packed range.
 * Results do not depend on the launch shape the handle uses (see
 * qdta_autotune): the parent rule is order-free. */
int qdta_sssp_batch(qdta_graph *g, const int32_t *cost_q, const int32_t *roots, int32_t R,
                    int32_t direction, int32_t *parent_link, int64_t *dist, void *stream);

/* All-or-nothing loading with route truncation (Alg. 3, Eq. 2, Eq. 5).
 * For every item, walk src -> root along parent_link (destination trees of
 * qdta_sssp_batch with QDTA_TO_ROOT, one row per od->roots entry), adding
 * cost_q to the elapsed time; link a is loaded iff the elapsed time at its
 * tail is < dt_q; the walk stops at the first node whose elapsed time is
 * >= dt_q or at the root.  flow_fx [L] is ACCUMULATED (integer atomics, so
 * the result is exact and order-free).  stop_node [n_items] (nullable)
 * receives each item's stop node s.  dt_q = INT64_MAX disables truncation.
 * QDTA_EUNREACH if some root is unreachable from its item's origin. */
int qdta_load_aon(qdta_graph *g, const int32_t *cost_q, const int32_t *parent_link,
                  const qdta_od *od, int64_t dt_q, int64_t *flow_fx, int32_t *stop_node,
                  void *stream);

/* BPR link costs (Eq. 1): c_a = c0_a (1 + alpha (f_a / (C_a dt_h))^beta) in
 * quanta, with f_a trips in an interval of dt_s seconds (dt_h = dt_s/3600),
 * evaluated in float64 without contraction, x^beta as x*x*...*x.
 * cost_s [L] (nullable) = c_a * quantum_s; cost_q [L] = clamp(floor(c_a + 0.5),
 * 1, 2^31-1).  QDTA_ENONFINITE on a NaN/inf flow. */
int qdta_bpr_costs(qdta_graph *g, const double *flow, double dt_s, double *cost_s,
                   int32_t *cost_q, void *stream);

/* Step size of one FW iteration (Alg. 8 with Alg. 9 / Eq. 7-9, or the
 * SWEEP8 / EXACT / MSA rules): minimise C(f + alpha (g - f)) over [0, 1]
 * with C the Beckmann objective (Eq. 6), or the total cost sum f c(f) when
 * p->objective is QDTA_OBJ_SO.  flow [L] f, aon_fx [L] g in fixed
 * point, fw_iter = k >= 1 (the k-th step; Alg. 8 starts from 2/(2+k-1)).
 * alpha_out_host, passes_out_host (nullable) are host scalars; the call
 * synchronises `stream`. */
int qdta_line_search(qdta_graph *g, const double *flow, const int64_t *aon_fx, double dt_s,
                     int32_t fw_iter, const qdta_params *p, double *alpha_out_host,
                     int32_t *passes_out_host, void *stream);

/* One interval's static assignment by Frank-Wolfe (Alg. 2 / Alg. 6):
 * initial all-or-nothing at free flow, then repeat {BPR costs; batched
 * shortest paths; truncated loading; step size; convex update} until the
 * stop rule holds or max_iter steps were taken (for QDTA_OBJ_SO the paths
 * follow marginal costs and the step minimises the total cost; see
 * QDTA_OBJ_SO).  flow_out [L] receives f.
 * In PAPER_OBJ mode the iterate before the step that met the test is
 * returned (the pseudo-code breaks before h = h_new).  stats_host
 * (nullable).  With p->record_tape, *tape_out receives a tape for
 * qdta_backward (the od arrays must stay alive and unchanged until the tape
 * is destroyed; QDTA_EINVAL with QDTA_OBJ_SO).  Synchronises `stream`.  An interval with no items returns
 * zero flows, converged. */
int qdta_assign_interval(qdta_graph *g, const qdta_od *od, double dt_s, const qdta_params *p,
                         double *flow_out, qdta_stats *stats_host, qdta_tape **tape_out,
                         void *stream);

/* One independent network / interval of a batch (device arrays). */
typedef struct {
  qdta_graph *graph;
  qdta_od od;
  double dt_s;
  double *flow_out;  /* [L of graph] */
} qdta_instance;

/* Many independent intervals (e.g. different networks) solved together:
 * with QDTA_SCHEDULE_GRAPH all instances run as parallel branches of one
 * CUDA graph launch; with QDTA_SCHEDULE_PLAIN one after another.  Every
 * graph must live on the same device and appear once (each handle holds one
 * workspace).  stats_host [n_inst] (nullable).  Synchronises. */
int qdta_assign_batch(const qdta_instance *inst, int32_t n_inst, const qdta_params *p,
                      qdta_stats *stats_host, void *stream);

/* A day of N intervals (Alg. 1 / Alg. 5): for each interval i,
 * d(i) = d_o(i) + d_r(i) (items merged by (root, origin), amounts summed),
 * FW solve, then Residual_demand (Alg. 4): every path of every accepted
 * all-or-nothing step is re-truncated with the final costs, weighted by its
 * step weight; the truncated link flows form h(i) and the remainders form
 * d_r(i+1).  d_orig_host [N] is a HOST array of qdta_od whose arrays are on
 * the device; all share one root (zone) list: d_orig_host[0].roots with
 * n_roots entries, and root_idx index it.  resid_in (nullable, device items
 * over the same roots) is added to the first interval, so that a day can be
 * resumed from a saved residual.  flow_out [N*L] receives h(i) row by row
 * (trips, float64).  stats_host [N] (nullable).  resid_out (nullable)
 * receives the residual left after the last interval.  Synchronises. */
int qdta_run_day(qdta_graph *g, const qdta_od *d_orig_host, int32_t N, double dt_s,
                 const qdta_params *p, const qdta_od *resid_in, double *flow_out,
                 qdta_stats *stats_host, qdta_residual *resid_out, void *stream);

/* Adjoint of the interval solve recorded in `tape` (not in the paper): the
 * FW iteration is unrolled with the shortest-path trees and truncation
 * masks held fixed (they are piecewise constant in the inputs); trees are
 * recomputed from the taped int32 link times, not stored.  MSA steps are
 * constants; line-search steps are differentiated through their optimality
 * condition C'(alpha) = 0 (zero derivative when alpha is clipped to 0 or 1).
 * dL_dflow [L] = dL/df of the returned flows; dL_ddemand [n_items] receives
 * dL/d(amount in trips) per item (a path-sum gather along the trees, the
 * transpose of loading); dL_dcap [L] dL/dC (vehicles per hour).  Synchronises. */
int qdta_backward(qdta_tape *tape, const double *dL_dflow, double *dL_ddemand, double *dL_dcap,
                  void *stream);
int qdta_tape_destroy(qdta_tape *tape);
/* iterations recorded (K) and items of the taped interval */
int qdta_tape_info(const qdta_tape *tape, int32_t *K_out_host, int64_t *n_items_out_host);

/* Batched shortest paths that allocate no device memory.
 *
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc at the moment they need shortest paths -- for example a process
 * whose device memory is reserved up front by another allocator (a caching
 * pool that holds all free memory, so a fresh cudaMalloc fails), or a
 * latency-critical loop that must not stall in CUDA's allocator.
 * qdta_sssp_batch, by contrast, grows a workspace with cudaMalloc the first
 * time it sees a larger graph.
 *
 * Same arguments, results and error codes as qdta_sssp_batch, for graphs
 * with at most QDTA_NOALLOC_MAX_LINKS links whose per-root state fits in
 * shared memory (at most 10,240 nodes); larger graphs are rejected with
 * QDTA_EINVAL and a message saying which limit was exceeded.  The graph
 * handle must already exist (qdta_graph_create allocates).  The only scratch
 * is a file-scope device array of QDTA_NOALLOC_MAX_LINKS 16-byte entries
 * (1 MiB), which every GPU that loads the library keeps until the process
 * exits.  The first call on a device looks up that array's device address;
 * make it before any stream capture.  Every call shares the array and
 * rewrites the part it uses before reading it, so calls that overlap on the
 * GPU (different streams or threads on one device) race and must be
 * serialised by the caller.  Synchronises `stream`. */
#define QDTA_NOALLOC_MAX_LINKS 65536
int qdta_sssp_batch_noalloc(qdta_graph *g, const int32_t *cost_q, const int32_t *roots, int32_t R,
                            int32_t direction, int32_t *parent_link, int64_t *dist, void *stream);

/* ---- launch-shape autotuning ----------------------------------------------
 * The paper fixes its decomposition by hand (Section 5: processes per node x
 * threads per process, with the routing of Alg. 7 partitioned over threads).
 * On one GPU the equivalent choice is the shape of the batched shortest-path
 * launch, and it is made by measurement: qdta_autotune times every candidate
 * shape on one caller-supplied batch and keeps the fastest in the handle;
 * later qdta_sssp_batch / qdta_assign_* / qdta_run_day calls use it.  Every
 * candidate computes identical distances and parents (the tie rule is
 * order-free), so tuning changes time only.
 *
 * Candidates: for graphs whose per-root state fits in shared memory, only the
 * shared-memory kernel; otherwise the global-memory Bellman-Ford with
 * launch shape {512 threads x 2 CTAs per SM, 256 threads x 4 CTAs per SM,
 * whichever fit in shared memory} x adjacency layout {32-bit rank keys,
 * 64-bit rank keys, four-slot, compressed; the first three only when every
 * degree is <= 4}, the 32-bit rank-keyed kernel also in further shapes
 * (five CTAs per SM with 256 or 192 threads, 5 or 6 frontier nodes in flight
 * per lane group, one lane per node, an L2 prefetch of key blocks, 288
 * threads x 4 CTAs), plus the cell-partitioned kernel.  Offers are applied
 * as "read the neighbour's key, then a non-returning atomicMin"
 * (QDTA_BF_RELAX selects the others).  Within a batch the resident CTAs take
 * roots from an atomic counter, longest first by the rounds each root took
 * in the handle's previous batch (QDTA_BF_DYNAMIC=0, QDTA_BF_LPT=0 turn this
 * off); the order does not change the results.
 *
 * cost_q [L] int32 and roots [R] int32 are device arrays as for
 * qdta_sssp_batch; parent_scratch is a caller-owned device array of R*V int32
 * that receives the trees (contents unspecified afterwards).  Each candidate
 * runs once untimed and then `reps` times between CUDA events on `stream`.
 * The handle's current choice is kept unless another candidate is at least
 * 2 % faster (closer timings are within run-to-run noise).  The report
 * (host) lists every candidate with its mean milliseconds per batch; `best`
 * indexes the one kept.  Errors: QDTA_EINVAL for bad arguments;
 * a failing candidate (e.g. QDTA_ENOMEM) aborts the tuning, restores the
 * previous choice and returns its code.  Synchronises `stream`.  Not to be
 * called during stream capture.
 *
 * Tuning cache per graph signature and GPU model, opt-in through the
 * environment variable QDTA_TUNE_CACHE: "mem" keeps each choice for the rest
 * of the process; a file path also reads earlier choices from that file and
 * appends new ones.  The key is a hash of the GPU model (name, SM count), the
 * network (nodes, links, tails, heads, free-flow times) and the direction; a
 * hit applies the stored choice without timing and sets `cached`. */
#define QDTA_TUNE_MAX 24
typedef struct qdta_tune_entry {
  char kernel[40];     /* kernel name, as qdta_sssp_kernel_name reports it */
  int32_t ctas_per_sm; /* resident CTAs (one root each) per SM */
  int32_t valid;       /* 1 when timed */
  float ms;            /* mean milliseconds per batch */
} qdta_tune_entry;
typedef struct qdta_tune_report {
  int32_t n;    /* candidates timed */
  int32_t best; /* index of the candidate kept */
  qdta_tune_entry entry[QDTA_TUNE_MAX];
  int32_t cached; /* 1: the choice came from the tuning cache (entry[0], nothing timed) */
} qdta_tune_report;
int qdta_autotune(qdta_graph *g, const int32_t *cost_q, const int32_t *roots, int32_t R, int32_t direction,
                  int32_t reps, int32_t *parent_scratch, qdta_tune_report *out_host, void *stream);

/* Scenario metrics of assigned intervals (Section 7.1, the paper's comparison
 * of a static and a quasi-dynamic morning peak): vehicle kilometres
 * travelled, average volume over capacity and vehicle hours of delay per
 * functional class, over the links that carry flow, and the same for the
 * congested subset (volume over capacity >= congested_voc; the paper uses
 * 1.0).  flows [N*L] float64 (N <= 65535): trips of interval i on link a at i*L + a,
 * e.g. the h(i) rows qdta_run_day writes; length_m [L] float64; link_class
 * [L] int32, links outside [0, n_classes) not counted; n_classes in [1,
 * QDTA_METRIC_MAX_CLASSES].  With x = f / (C dt_h) and c(f) per Eq. 1,
 * out [N*n_classes*QDTA_METRICS] float64, row (i, k) =
 *   links with f > 0, VMT = sum f len / 1000 (veh-km), mean x,
 *   VHD = sum f (c(f) - c0) * quantum_s / 3600 (veh-h),
 *   congested links, congested length (km), congested VMT, congested mean x.
 * Sums are exact fixed-point sums (the result does not depend on the launch
 * shape).  QDTA_ENONFINITE on a non-finite flow.  Synchronises `stream`. */
#define QDTA_METRICS 8
#define QDTA_METRIC_MAX_CLASSES 16
int qdta_interval_metrics(qdta_graph *g, const double *flows, int32_t N, double dt_s, const double *length_m,
                          const int32_t *link_class, int32_t n_classes, double congested_voc, double *out,
                          void *stream);

/* Enable / read / reset per-kernel event timings (plain schedule). */
int qdta_profile_enable(qdta_graph *g, int32_t on);
int qdta_profile_read(qdta_graph *g, qdta_profile *out_host);

/* Message of the last failing call on this host thread (never NULL). */
const char *qdta_last_error(void);
/* Library version string. */
const char *qdta_version(void);

/* Name of the shortest-path kernel qdta_sssp_batch launches on this graph in
 * this direction (it depends on the node count, the degree bound and the
 * QDTA_SSSP / QDTA_BF_* environment).  A static string; "" with QDTA_EINVAL
 * set for a NULL graph or a bad direction.  No device work. */
const char *qdta_sssp_kernel_name(const qdta_graph *g, int32_t direction);

#ifdef __cplusplus
}
#endif
#endif /* QDTA_H */
