// qdta_internal.cuh -- device arithmetic, kernel parameter blocks and host
// launchers shared by the two translation units of libqdta.
//
// Floating point: every FP64 operation that must agree bit for bit with the
// CPU reference goes through an explicitly rounded intrinsic (__dmul_rn,
// __dadd_rn, ...), so no multiply-add is ever contracted (the library is also
// compiled with -fmad=false).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qdta {

typedef __int128 i128;
typedef unsigned __int128 u128;

// status bits written by kernels (OR-ed into a device word)
enum : unsigned {
  ST_NONFINITE = 1u,   // NaN/inf input or term, or a fixed-point term >= 2^68
  ST_UNREACH = 2u,     // a walk met a node without parent before its root
  ST_OVERFLOW = 4u,    // a distance exceeded the packed range
  ST_TIMEOUT = 8u,     // a bounded loop hit its limit
  ST_CAPACITY = 16u,   // an output buffer was too small
  ST_K32 = 32u,        // a 32-bit-key batch has a node at distance >= 2^29 (offered only dropped
                       // offers; redone with 64-bit keys; not an error)
  ST_BADARG = 64u,     // a device array argument held an invalid value
};

constexpr int SSSP_THREADS = 256;
constexpr int LINK_THREADS = 256;
constexpr int MAX_SLOTS = 8;    // step sizes evaluated per sweep
constexpr int NSUM = MAX_SLOTS + 2;  // + gap sums A, B

// --------------------------------------------------------------------------
// exact-rounding helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dvd(double a, double b) { return __ddiv_rn(a, b); }

__device__ __forceinline__ double powi(double x, int n) {
  double p = x;
  for (int i = 1; i < n; ++i) p = mul(p, x);
  return p;
}

// fixed point of a trip amount: (double)amount_fx * 2^-32
__device__ __forceinline__ double fx64_to_double(long long v) {
  return mul(__ll2double_rn(v), 0x1p-32);
}

// round_to_nearest_even(v * 2^32) as a 128-bit integer, from the bits of v.
// |v| >= 2^68 or non-finite sets *bad and yields 0.
__device__ __forceinline__ i128 fx_of(double v, unsigned *bad) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  int e = (int)((bits >> 52) & 0x7ffu);
  if (e == 0x7ff) { *bad |= ST_NONFINITE; return 0; }
  if (e == 0) return 0;  // zero or subnormal: far below 2^-33
  long long m = (long long)((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  int sh = e - 1043;     // v * 2^32 = m * 2^sh
  i128 r;
  if (sh >= 0) {
    if (sh > 47) { *bad |= ST_NONFINITE; return 0; }
    r = (i128)m << sh;
  } else {
    int s = -sh;
    if (s > 60) {
      r = 0;
    } else {
      long long q = m >> s;
      long long rem = m - (q << s);
      long long half = 1ll << (s - 1);
      if (rem > half || (rem == half && (q & 1))) ++q;
      r = q;
    }
  }
  return (bits >> 63) ? -r : r;
}

// nearest double to a 128-bit integer (ties to even), built from its bits
__device__ __forceinline__ double i128_to_double(i128 s) {
  if (s == 0) return 0.0;
  bool neg = s < 0;
  u128 u = neg ? (u128)(-s) : (u128)s;
  unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
  int nb = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
  double r;
  if (nb <= 53) {
    r = __ull2double_rn(lo);
  } else {
    int sh = nb - 53;
    unsigned long long m = (unsigned long long)(u >> sh);
    u128 rem = u & (((u128)1 << sh) - 1);
    u128 half = (u128)1 << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
      ++m;
      if (m == (1ull << 53)) { m >>= 1; ++sh; }
    }
    double scale = __longlong_as_double((long long)(1023 + sh) << 52);
    r = mul(__ull2double_rn(m), scale);
  }
  return neg ? -r : r;
}

__device__ __forceinline__ double fx_to_double(i128 s) { return mul(i128_to_double(s), 0x1p-32); }

// --------------------------------------------------------------------------
// link cost model (Eq. 1) and its integral (Eq. 6), per-link constants:
//   inv = 1 / (C dt_h), kb = (alpha C dt_h) / (beta + 1)
// --------------------------------------------------------------------------
struct LinkConst {
  double inv;
  double kb;
};

__device__ __forceinline__ LinkConst link_const(double cap, double dt_h, double alpha, int beta) {
  double cp = mul(cap, dt_h);
  LinkConst k;
  k.inv = dvd(1.0, cp);
  k.kb = dvd(mul(alpha, cp), (double)(beta + 1));
  return k;
}

__device__ __forceinline__ double link_cost(double c0, double inv, double alpha, int beta, double t) {
  double x = mul(t, inv);
  double p = powi(x, beta);
  double w = mul(alpha, p);
  double u = add(1.0, w);
  return mul(c0, u);
}

// System optimum: marginal cost m = c + t c' = c0 (1 + alpha (beta+1) x^beta)
// and its derivative c0 alpha beta (beta+1) x^(beta-1) / cp; the objective
// term is the total cost t c(t).  Same operation order as the CPU oracle.
__device__ __forceinline__ double link_marginal(double c0, double inv, double alpha, int beta, double t) {
  double x = mul(t, inv);
  double p = powi(x, beta);
  double k = mul(alpha, (double)(beta + 1));
  double w = mul(k, p);
  double u = add(1.0, w);
  return mul(c0, u);
}

__device__ __forceinline__ double link_marginal_dt(double c0, double inv, double alpha, int beta, double t) {
  double x = mul(t, inv);
  double p = beta > 1 ? powi(x, beta - 1) : 1.0;
  double w = mul(c0, alpha);
  w = mul(w, (double)beta);
  w = mul(w, (double)(beta + 1));
  w = mul(w, p);
  return mul(w, inv);
}

__device__ __forceinline__ double link_cost_dt(double c0, double inv, double alpha, int beta, double t) {
  double x = mul(t, inv);
  double p = beta > 1 ? powi(x, beta - 1) : 1.0;
  double w = mul(c0, alpha);
  w = mul(w, (double)beta);
  w = mul(w, p);
  return mul(w, inv);
}

__device__ __forceinline__ double beckmann(double c0, double inv, double kb, int beta, double t) {
  double x = mul(t, inv);
  double p = powi(x, beta + 1);
  double w = mul(kb, p);
  double u = add(t, w);
  return mul(c0, u);
}

// t = f + alpha (g - f), the same three roundings as the flow update
__device__ __forceinline__ double step_flow(double f, double g, double alpha) {
  double d = sub(g, f);
  double s = mul(alpha, d);
  return add(f, s);
}

__device__ __forceinline__ int quantize(double c, unsigned *bad) {
  if (isnan(c)) { *bad |= ST_NONFINITE; return 2147483647; }
  double r = floor(add(c, 0.5));
  if (r < 1.0) return 1;
  if (r > 2147483647.0) return 2147483647;
  return (int)r;
}

// --------------------------------------------------------------------------
// device-side controller of one interval solve (single thread updates it)
// --------------------------------------------------------------------------
enum SumKind : int { K_PHI = 0, K_DPHI = 1, K_DDPHI = 2 };

enum LsState : int {
  LS_IDLE = 0,
  LS_GAPONLY = 1,   // MSA (or QN with ls_max <= 1): the sweep only measures the gap
  LS_QN = 2,
  LS_SW_FIRST = 3,
  LS_SW_NEXT = 4,
  LS_EX_END = 5,
  LS_EX_NEWTON = 6,
  LS_OBJ = 7,       // PAPER_OBJ test: phi(0) vs phi(alpha*)
};

struct Plan {
  int n;              // slots in use (0..MAX_SLOTS)
  int want_gap;       // also compute sum fx(q f) and sum q g_fx
  int kind[MAX_SLOTS];
  double alpha[MAX_SLOTS];
};

struct Ctl {
  // parameters
  int step, stop, max_iter, ls_max;
  double tol, dx, t1, t2;
  // loop state
  int k;              // FW step in progress (1-based)
  int fw_continue;    // 0 once the loop is over
  int need_sweep;     // 1 while the line search wants another sweep
  int do_update;      // 1 if the step of iteration k is applied
  int converged;
  int notconv;
  int iterations, aon_calls, ls_passes;
  int ls_state, ls_pc, l, ex_it;
  double rel_gap, dual_gap;
  double alpha, alpha_final, lo, hi;
  i128 Dlo, Dhi;
  Plan plan;
  i128 sums[NSUM];
  double objective;
  // parent-array ring: AON j writes slot min(j, ring - 1)
  int ring, tree_slot;
  // residual loop (Alg. 4) and day loop (Alg. 1)
  int res_j, res_slot, res_skip, res_continue;
  double w_cur;
  int day_i, day_N, day_continue;
  int gap_on;  // measure the duality gap (needs the iteration's link times)
};

// --------------------------------------------------------------------------
// launchers (qdta_kernels.cu)
// --------------------------------------------------------------------------
struct GraphDev {
  int V, L, LB, beta;
  double alpha, quantum_s;
  const int *tail, *head, *c0;
  const double *cap;
  const int *out_off, *in_off;    // [V+1]
  const int *out_link, *in_link;  // [L] link ids grouped by tail / head, ascending
  int num_sms;
  // locality order for the global-memory SSSP (nullable): internal node ids
  // in cell order; per direction the adjacency of each internal node as link
  // ids and neighbours' internal ids
  const int *node_int;             // [V] external -> internal
  const int *node_ext;             // [V] internal -> external
  const int *perm_off[2];          // [V + 1]
  const int *perm_link[2];         // [L]
  const int *perm_nb[2];           // [L]
  int max_deg[2];                  // largest degree per direction
  // rank-keyed four-slot adjacency (degree <= 4): per link, its rank among the
  // candidate parent links of the node it relaxes (out-links of the tail for
  // TO_ROOT, in-links of the head for FROM_ROOT, by link id); per internal
  // node, the link of each rank (-1 past the degree)
  const int *rank_tgt[2];          // [L]
  const int *rank_link[2];         // [4 V]
  int skip_parent;                 // every link has its reverse, lists share one order
  // launch choices of the global-memory SSSP (set at create, changed by
  // qdta_autotune): four-slot adjacency when max_deg <= 4, relaxation mode
  // (0 returning atomic, 1 read then returning atomic, 2 read then
  // non-returning atomic), shared-memory carveout percentage, launch shape
  // of the shared-memory-queue kernel (0: 512 threads, two mark bitmaps;
  // 1: 256 threads, one bitmap; 2: 512 threads, one bitmap)
  int tune_adj, tune_relax, tune_carve, tune_shape;  // tune_adj: 0 compressed, 1 four-slot, 2 rank-keyed, 3 rank-keyed 32-bit
  int tune_out;  // output pass of the queue kernel: 1 internal node order, 0 external order
  int tune_dyn;  // queue kernels: roots after the first wave from an atomic counter (1) or round-robin (0)
  // rounds each root node took in its last queue-kernel batch ([V], zeroed
  // at create; nullable): the dynamic fetch hands out the longest first
  int *root_rounds;
};

// root scheduling of the queue kernels: fetch (nullable) hands out root
// positions after the first wave; order (nullable) maps a position to the
// root's row (longest first); hint (nullable) receives each root node's rounds
struct RootSched {
  int *fetch;
  const int *order;
  int *hint;
};

// Cell partition for the shared-memory cell SSSP (graphs above the
// whole-state-in-shared-memory limit).  Internal node ids are cell-major;
// per relaxation direction d (0 = TO_ROOT pulls over out-links, 1 =
// FROM_ROOT pulls over in-links) entries are grouped by internal node and
// carry a code: >= 0 local index of the neighbour in the same cell,
// < 0 -(k+1) with k the neighbour's slot in the cell's external list.
constexpr int CELL_MAX_NODES = 256;
constexpr int CELL_MAX_EXT = 128;
constexpr int CELL_MAX_LREV = 1024;  // internal reversed links per cell
constexpr int CELL_WARPS = 4;

struct CellDev {
  int n_cells;
  const int *cell_off;   // [n_cells + 1] internal node ranges
  const int *node_int;   // [V] external -> internal
  const int *node_cell;  // [V] internal -> cell
  const int *ent_off[2];   // [V + 1] internal node -> entry range
  const int *ent_link[2];  // [L] link id of each entry
  const int *ent_code[2];  // [L] neighbour code
  const int *ext_off[2];   // [n_cells + 1]
  const int *ext_node[2];  // internal ids of external neighbours
  const int *dep_off[2];   // [n_cells + 1]
  const int *dep_cell[2];  // cells that read this cell's keys
  // internal links reversed: for node w, the cell nodes u that pull through w
  const int *lrev_off[2];   // [V + 1]
  const int *lrev_link[2];  // link id
  const int *lrev_src[2];   // local index of u
  const unsigned char *node_flags[2];  // bit 0: has external entries, bit 1: read by another cell
  // external readers: for node w, the nodes u of other cells that pull through w
  const int *xrev_off[2];   // [V + 1]
  const int *xrev_link[2];  // link id
  const int *xrev_node[2];  // internal id of u
};

struct SsspWork {
  unsigned long long *state;  // [slots][V]
  int *stamp;                 // [slots][V]
  int *queue;                 // [slots][2][V]
  int4 *adj;                  // [L] packed (link, neighbour, q, 0) of the chosen direction
  uint2 *lrev;                // cell kernel: packed internal reversed links (u << 24 | link, q)
  unsigned long long *prio;   // cell kernel: [slots][cells] wake priorities
  int4 *xrev;                 // cell kernel: packed external readers (link, reader, q, 0)
  int *fb_skip;               // 32-bit-key batches: 1 unless the 64-bit redo must run
  int *order;                 // [R_cap] root order of the dynamic fetch (nullable)
  int slots;
};

// skip_dev (nullable): when *skip_dev != 0 the launch does nothing
void launch_pack_adj(const GraphDev &g, int direction, const int *q, int4 *adj, cudaStream_t s,
                     const int *skip_dev = nullptr);
void launch_pack_perm_adj(const GraphDev &g, int direction, const int *q, int4 *adj, cudaStream_t s,
                          const int *skip_dev = nullptr);
void launch_pack_cell_adj(const GraphDev &g, const CellDev &c, int direction, const int *q, int4 *adj,
                          uint2 *lrev_adj, long long n_lrev, int4 *xrev_adj, long long n_xrev, cudaStream_t s,
                          const int *skip_dev = nullptr);
void launch_sssp_cell(const GraphDev &g, const CellDev &c, int direction, const int4 *adj, const uint2 *lrev_adj,
                      const int4 *xrev_adj,
                      long long delta, const int *roots, int R_host, const int *R_dev, int grid,
                      unsigned long long *state, int *flag, int *queue, unsigned long long *prio, int *parent,
                      const int *parent_slot_dev, long long slot_stride, long long *dist,
                      unsigned *status, cudaStream_t s, const int *skip_dev,
                      unsigned long long *roots_counter);
int sssp_cell_blocks_per_sm();
void launch_sssp(const GraphDev &g, int direction, const int4 *adj, const int *roots,
                 int R_host, const int *R_dev, int grid, bool use_smem, const SsspWork &w,
                 int *parent, const int *parent_slot_dev, long long slot_stride, long long *dist,
                 unsigned *status, cudaStream_t s, const int *skip_dev = nullptr,
                 unsigned long long *roots_counter = nullptr);
int sssp_max_smem_nodes();
int sssp_group_size();  // roots per CTA of the global-memory kernel
// parent rows by root index: row r of src goes to row root_slot[r] of the
// parent slot (*slot_dev, or 0), skipped when root_slot[r] < 0
void launch_gather_rows(const int *src, int rows, int V, const int *root_slot, int *parent, const int *slot_dev,
                        long long slot_stride, cudaStream_t s);
// scenario metrics of N intervals' link flows; acc [N*C*16] zeroed by the caller
void launch_metrics(const GraphDev &g, const double *flows, int N, double dt_h, const double *length_m,
                    const int *link_class, int C, double congested_voc, unsigned long long *acc, double *out,
                    unsigned *status, cudaStream_t s);
bool sssp_uses_smq(const GraphDev &g);   // global-memory launch keeps queues and marks in shared memory
int sssp_smq_shape_count();  // launch shapes of the shared-memory-queue kernel
bool sssp_smq_shape_fits(int V, int shape);
int sssp_smq_ctas_per_sm(const GraphDev &g, int direction);
bool sssp_uses_perm(const GraphDev &g);  // global-memory launch reads the locality-ordered adjacency
bool sssp_uses_ell(const GraphDev &g, int direction);
int sssp_adj(const GraphDev &g, int direction);  // adjacency layout the queue kernel uses (0, 1, 2)
void launch_pack_ell8(const GraphDev &g, int direction, const int *q, int2 *ell, cudaStream_t s,
                      const int *skip_dev = nullptr);
const char *sssp_kernel_name(const GraphDev &g, int direction, bool use_smem);  // ... in the four-slot layout
void launch_pack_ell(const GraphDev &g, int direction, const int *q, int4 *ell, cudaStream_t s,
                     const int *skip_dev = nullptr);
long long launch_count();
// which: 0 = fw_continue, 1 = need_sweep, 2 = res_continue
void launch_set_cond(const Ctl *ctl, int which, unsigned long long cond, cudaStream_t s);
int sssp_blocks_per_sm(bool use_smem, int V);

// Residual trips on a link (QDTA_TRUNC_CARRY) merge per (root, link) in an
// open-addressed table: key root * L + link (~0 when empty), the amount, and
// the exact sum of amount x covered fraction as two 64-bit words: the sum of
// the terms' low 32 bits, then the sum of their parts above 2^32 (sum =
// word1 * 2^32 + word0); the merged item carries the floor of the mean.
// mask == 0: no table.
struct CarryAcc {
  unsigned long long *key = nullptr;   // [mask + 1]
  unsigned long long *amt = nullptr;   // [mask + 1]
  unsigned long long *tsum = nullptr;  // [2 * (mask + 1)]
  unsigned long long mask = 0;
  unsigned long long seg = 1;           // slots per root segment, (mask + 1) / roots
};

void launch_pack_head_q(const GraphDev &g, const int *q, int2 *head_q, cudaStream_t s);
// carry, carry_link [n] (nullable): an item with carry_link >= 0 is on that
// link having covered the fraction carry / 2^32 of it; it finishes the link,
// then follows its tree
void launch_load(const GraphDev &g, const int2 *head_q, const int *parent, const int *parent_slot_dev,
                 long long slot_stride, const int *root_slot, const int *roots, long long n_items_host,
                 const long long *n_items_dev, const int *root_idx, const int *src,
                 const long long *amount, long long dt_q, unsigned long long *flow_fx, int *stop_out,
                 unsigned *status, cudaStream_t s, const long long *carry = nullptr,
                 const int *carry_link = nullptr);
// trunc 1 (carry): a trip still on a link at the end of the interval goes
// to the carried table `ca` with the fraction covered; trips stopping at a node
// go to `dense`
void launch_residual(const GraphDev &g, const int2 *head_q_fin, const int *parent,
                     const int *parent_slot_dev, long long slot_stride, const int *root_slot,
                     const int *roots, const long long *n_items_dev, long long n_items_cap,
                     const int *root_idx, const int *src, const long long *amount,
                     const double *weight_dev, long long dt_q, unsigned long long *h_fx,
                     unsigned long long *dense, unsigned *status, cudaStream_t s,
                     const long long *carry = nullptr, const int *carry_link = nullptr, int trunc = 0,
                     CarryAcc ca = CarryAcc{});

// marginal = 1: the system optimum's marginal costs instead of link times
void launch_bpr(const GraphDev &g, const double *flow, double dt_h, double *cost_s, int *cost_q,
                unsigned *status, cudaStream_t s, int marginal = 0);
void launch_link_const(const GraphDev &g, double dt_h, LinkConst *kc, cudaStream_t s);
// ST_BADARG unless every item with carry_link >= 0 names a link whose tail
// is its src and carries a fraction in [0, 2^32) (carry nullable)
void launch_check_carry(const GraphDev &g, long long n, const int *src, const long long *carry,
                        const int *carry_link, unsigned *status, cudaStream_t s);
// replace the graph's capacities by `cap` (device) when every value is finite
// and > 0; otherwise set ST_BADARG and leave them unchanged
void launch_set_capacity(const GraphDev &g, const double *cap, unsigned *status, cudaStream_t s);
void launch_flow_from_fx(int L, const unsigned long long *fx, double *f, cudaStream_t s);
void launch_sweep(const GraphDev &g, const LinkConst *kc, const double *f, const long long *g_fx,
                  const int *q, Ctl *ctl, i128 *partials, unsigned *counter, int grid,
                  unsigned *status, cudaStream_t s, int so = 0);
int sweep_grid(const GraphDev &g);
void launch_update(const GraphDev &g, Ctl *ctl, double *f, const long long *g_fx, cudaStream_t s);
void launch_objective(const GraphDev &g, const LinkConst *kc, const double *f, Ctl *ctl,
                      i128 *partials, unsigned *counter, int grid, unsigned *status, cudaStream_t s, int so = 0);

void launch_ctl_init(Ctl *ctl, int step, int stop, int max_iter, int ls_max, double tol, double dx,
                     double t1, double t2, int ring, long long n_items_host,
                     const long long *n_items_dev, int gap_on, cudaStream_t s);
void launch_tape0(const GraphDev &g, const int *q, const double *f, int *tape_q, double *tape_alpha,
                  double *tape_f, cudaStream_t s);
void launch_res_begin(Ctl *ctl, unsigned long long cond, int use_cond, cudaStream_t s);
void launch_res_prep(Ctl *ctl, const double *w, const int *tape_q, int L, int *q_work, cudaStream_t s);
void launch_res_next(Ctl *ctl, unsigned long long cond, int use_cond, cudaStream_t s);
void launch_store_interval(const GraphDev &g, const Ctl *ctl, const unsigned long long *h_fx,
                           double *flow_out_rows, void *stats_rows, const long long *n_items_dev,
                           cudaStream_t s);
void launch_day_next(Ctl *ctl, unsigned long long cond, int use_cond, cudaStream_t s);
struct OrigTable {
  const int *root_idx; const int *src; const long long *amount; long long n;
  const long long *carry; const int *carry_link;  // nullable: items on a link
};
void launch_scatter_orig(const GraphDev &g, const Ctl *ctl, const OrigTable *tab, long long max_n,
                         unsigned long long *dense, cudaStream_t s, CarryAcc ca = CarryAcc{},
                         unsigned *status = nullptr);
void launch_ctl_begin(Ctl *ctl, unsigned long long cond_fw, int use_cond, cudaStream_t s);
void launch_ctl_step(Ctl *ctl, unsigned long long cond_ls, int use_cond, cudaStream_t s);
void launch_ctl_end(Ctl *ctl, unsigned long long cond_fw, int use_cond, cudaStream_t s);
void launch_tape_record(const GraphDev &g, const Ctl *ctl, const int *q, const double *f,
                        int *tape_q, double *tape_alpha, double *tape_f, int cap, cudaStream_t s);

// items on a link (carry_link >= 0) go to the carried table `ca` (which must exist then)
void launch_scatter_items(const GraphDev &g, long long n, const int *root_idx, const int *src,
                          const long long *amount, unsigned long long *dense, cudaStream_t s,
                          const long long *carry = nullptr, const int *carry_link = nullptr,
                          CarryAcc ca = CarryAcc{}, unsigned *status = nullptr);
// dense (root, node) accumulator -> items in (root, node) order, then (when
// ca.mask is set) the carried table's entries appended in slot order with
// their mean covered fractions and links (src = the link's tail); carry_out and
// link_out (nullable) receive each item's covered fraction and link (0 and -1
// for the first part).  Both sources are cleared; the item count never
// exceeds cap (ST_CAPACITY when entries were dropped).  blk_count / blk_off
// must hold max(R * V, ca.mask + 1) / 4096 + 1 entries.
void launch_compact(const GraphDev &g, int R, unsigned long long *dense, int *blk_count,
                    long long *blk_off, long long cap, int *root_idx, int *src, long long *amount,
                    long long *n_out_dev, unsigned *status, cudaStream_t s, long long *carry_out = nullptr,
                    int *link_out = nullptr, CarryAcc ca = CarryAcc{});
void launch_active_roots(int R, const long long *n_items_dev, long long cap_items,
                         const int *root_idx, const int *zone_nodes, int *flag, int *active_roots,
                         int *root_slot, int *n_active_dev, cudaStream_t s);
void launch_path_weights(const Ctl *ctl, const double *tape_alpha, double *w, cudaStream_t s);
void launch_fill_i32(int *p, long long n, int v, cudaStream_t s);
void launch_fx_to_flow(int L, const unsigned long long *fx, double *out, cudaStream_t s);
void launch_weight_select(const double *w, int j, double *dst, cudaStream_t s);

// adjoint
void launch_adj_reduce(const GraphDev &g, const LinkConst *kc, const double *lam, const double *fprev,
                       const long long *g_fx, double alpha, int implicit, double *partials, double *out2,
                       int grid, cudaStream_t s);
void launch_adj_update(const GraphDev &g, const LinkConst *kc, const double *lam, const double *fprev,
                       const long long *g_fx, double alpha, int implicit, const double *muH,
                       double *gbar, double *lam_prev, double *dcap, cudaStream_t s);
void launch_gather(const GraphDev &g, const int2 *head_q, const int *parent, const int *roots,
                   long long n_items, const int *root_idx, const int *src, long long dt_q,
                   const double *gbar, double *dd, unsigned *status, cudaStream_t s,
                   const long long *carry = nullptr, const int *carry_link = nullptr);

}  // namespace qdta
