/*
 * qdta_oracle.c -- plain, slow, obviously correct CPU oracle for the
 * quasi-dynamic traffic assignment (QDTA) hot path of Chan et al.,
 * "Quasi-Dynamic Traffic Assignment using High Performance Computing"
 * (arXiv 2104.12911).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code with
 * the CUDA library and includes none of its headers.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (contraction off so
 * that every a*b+c rounds twice, as in the CUDA path compiled with -fmad=false).
 *
 * Conventions (all readings of the paper are listed at the end of the file):
 *   - link costs are int32 counts of a time quantum (0.01 s); distances int64;
 *   - trip amounts and AON link flows are int64 fixed point, 2^-32 trips;
 *   - every sum over links is the exact integer sum of the per-link terms,
 *     each rounded (to nearest, ties to even) to 2^-32 fixed point, kept in
 *     a 128-bit integer; it is converted to double once, at the end;
 *   - x^n is the left-to-right product x*x*...*x.
 *
 * Parity status: every function below is pinned by the -m "not gpu" tests
 * (brute force, closed forms, the paper's worked example, invariants, or
 * finite differences), except the residual-demand merge order, which has no
 * independent pin beyond conservation (its multiset result is unique).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_ENONFINITE (-5)
#define OR_EUNREACH (-6)
#define OR_NOTCONV 1

#define DIR_TO_ROOT 0
#define DIR_FROM_ROOT 1

#define STEP_MSA 0
#define STEP_PAPER_QN3 1
#define STEP_SWEEP8 2
#define STEP_EXACT 3

#define STOP_NONE 0
#define STOP_PAPER_OBJ 1
#define STOP_REL_GAP 2

#define DIST_INF INT64_MAX

typedef struct {
  int32_t n_nodes, n_links;
  const int32_t *tail, *head, *fftime_q;
  const double *capacity;
  double alpha;
  int32_t beta;
  double quantum_s;
} or_graph;

typedef struct {
  int32_t n_roots;
  const int32_t *roots;
  int64_t n_items;
  const int32_t *root_idx, *src;
  const int64_t *amount_fx;
  /* Trips carried on a link (R17; both nullable): carry_link[k] >= 0 puts
   * item k on that link (src is its tail) having covered the fraction
   * carry_frac[k] / 2^32 of it, 0 <= carry_frac < 2^32; -1 (or NULL) starts
   * the item at src. */
  const int64_t *carry_frac;
  const int32_t *carry_link;
} or_od;

typedef struct {
  int32_t step, stop, max_iter, ls_max;
  double tol, ls_dx, ls_t1, ls_t2;
  int32_t objective;  /* OBJ_UE (Beckmann, user equilibrium) or OBJ_SO (total cost, system optimum) */
  int32_t truncation; /* TRUNC_NODE (R1) or TRUNC_CARRY (R17) */
} or_params;

#define OBJ_UE 0
#define OBJ_SO 1

#define TRUNC_NODE 0
#define TRUNC_CARRY 1

typedef struct {
  int32_t iterations;   /* accepted FW steps after the initial AON */
  int32_t aon_calls;    /* shortest-path batches run (including the initial one) */
  int32_t ls_passes;    /* link sweeps spent in line searches */
  int32_t converged;
  double rel_gap;       /* last value of the stop-rule measure (NaN if none) */
  double objective;     /* Beckmann objective of the returned flows, quantum*trips */
  double dual_gap;      /* last relative duality gap (sum c f - sum c g) / sum c f */
} or_stats;

/* ------------------------------------------------------------------------ */
/* Fixed point: v -> round_to_nearest_even(v * 2^32) as a 128-bit integer.  */
/* ------------------------------------------------------------------------ */

static i128 fx_of(double v, int *bad) {
  if (!isfinite(v)) { *bad = 1; return 0; }
  if (v == 0.0) return 0;
  int e;
  double m = frexp(fabs(v), &e);            /* |v| = m * 2^e, m in [0.5, 1) */
  int64_t mi = (int64_t)ldexp(m, 53);        /* exact 53-bit integer          */
  int sh = e - 53 + 32;                      /* |v| * 2^32 = mi * 2^sh       */
  i128 r;
  if (sh >= 0) {
    if (sh > 47) { *bad = 1; return 0; }     /* |term| >= 2^68: refuse          */
    r = (i128)mi << sh;
  } else {
    int s = -sh;
    if (s > 60) {
      r = 0;
    } else {
      int64_t q = mi >> s;
      int64_t rem = mi - (q << s);
      int64_t half = (int64_t)1 << (s - 1);
      if (rem > half || (rem == half && (q & 1))) q += 1;
      r = q;
    }
  }
  return v < 0 ? -r : r;
}

/* int128 -> nearest double (ties to even), then exact scaling by 2^-32. */
static double fx_to_double(i128 s) { return (double)s * 0x1p-32; }

/* exported for the pins of the fixed-point format */
void or_to_fx(double v, int64_t *hi, uint64_t *lo, int32_t *bad) {
  int b = 0;
  i128 r = fx_of(v, &b);
  *hi = (int64_t)(r >> 64);
  *lo = (uint64_t)r;
  *bad = b;
}

double or_fx_to_double(int64_t hi, uint64_t lo) {
  i128 r = ((i128)hi << 64) | (i128)lo;
  return fx_to_double(r);
}

/* ------------------------------------------------------------------------ */
/* BPR link cost (Eq. 1) and the Beckmann integral (Eq. 6).                 */
/* ------------------------------------------------------------------------ */

static double pow_n(double x, int n) {
  double p = x;
  for (int i = 1; i < n; i++) p = p * x;
  return p;
}

/* Per link, with cp = C_a * dt_h (capacity over the interval):
 *   inv = 1 / cp,  x = t * inv  (t trips in the interval, so t / dt_h is an
 *   hourly rate: Eq. 1 read with the worked example's hourly demand);
 *   c_a(t)  = c0 * (1 + alpha * x^beta)                       (Eq. 1, quanta)
 *   B_a(t)  = c0 * (t + kb * x^(beta+1)),  kb = alpha cp / (beta+1)
 *           = integral_0^t c_a(s) ds                            (Eq. 6)
 * Each line is one rounded operation in the order written. */
static double inv_cap(const or_graph *g, int a, double dt_h) {
  double cp = g->capacity[a] * dt_h;
  return 1.0 / cp;
}

static double link_cost(const or_graph *g, int a, double t, double dt_h) {
  double x = t * inv_cap(g, a, dt_h);
  double p = pow_n(x, g->beta);
  double w = g->alpha * p;
  double u = 1.0 + w;
  return (double)g->fftime_q[a] * u;
}

/* d c_a / d t = c0 alpha beta x^(beta-1) / cp */
static double link_cost_dt(const or_graph *g, int a, double t, double dt_h) {
  double inv = inv_cap(g, a, dt_h);
  double x = t * inv;
  double p = g->beta > 1 ? pow_n(x, g->beta - 1) : 1.0;
  double w = (double)g->fftime_q[a] * g->alpha;
  w = w * (double)g->beta;
  w = w * p;
  return w * inv;
}

/* d c_a / d C_a  (capacity in veh/h) = -c0 alpha beta x^beta / C */
static double link_cost_dcap(const or_graph *g, int a, double t, double dt_h) {
  double x = t * inv_cap(g, a, dt_h);
  double p = pow_n(x, g->beta);
  return -(double)g->fftime_q[a] * g->alpha * (double)g->beta * p / g->capacity[a];
}

static double beckmann(const or_graph *g, int a, double t, double dt_h) {
  double cp = g->capacity[a] * dt_h;
  double kb = g->alpha * cp;
  kb = kb / (double)(g->beta + 1);
  double x = t * inv_cap(g, a, dt_h);
  double p = pow_n(x, g->beta + 1);
  double w = kb * p;
  double u = t + w;
  return (double)g->fftime_q[a] * u;
}

/* System optimum (the alternative objective of Sections 3 and 8): the total
 * cost Z_a(t) = t * c_a(t) replaces the Beckmann integral, and its derivative
 * m_a(t) = c_a(t) + t * c_a'(t) = c0 * (1 + alpha (beta+1) x^beta), the
 * marginal cost, replaces c_a in routing and in the slope of the line search. */
static double link_total(const or_graph *g, int a, double t, double dt_h) {
  return t * link_cost(g, a, t, dt_h);
}

static double link_marginal(const or_graph *g, int a, double t, double dt_h) {
  double x = t * inv_cap(g, a, dt_h);
  double p = pow_n(x, g->beta);
  double k = g->alpha * (double)(g->beta + 1);
  double w = k * p;
  double u = 1.0 + w;
  return (double)g->fftime_q[a] * u;
}

/* d m_a / d t = c0 alpha beta (beta+1) x^(beta-1) / cp */
static double link_marginal_dt(const or_graph *g, int a, double t, double dt_h) {
  double inv = inv_cap(g, a, dt_h);
  double x = t * inv;
  double p = g->beta > 1 ? pow_n(x, g->beta - 1) : 1.0;
  double w = (double)g->fftime_q[a] * g->alpha;
  w = w * (double)g->beta;
  w = w * (double)(g->beta + 1);
  w = w * p;
  return w * inv;
}

/* objective term, slope cost and slope-cost derivative of link a */
static double obj_term(const or_graph *g, int a, double t, double dt_h, int obj) {
  return obj == OBJ_SO ? link_total(g, a, t, dt_h) : beckmann(g, a, t, dt_h);
}
static double obj_cost(const or_graph *g, int a, double t, double dt_h, int obj) {
  return obj == OBJ_SO ? link_marginal(g, a, t, dt_h) : link_cost(g, a, t, dt_h);
}
static double obj_cost_dt(const or_graph *g, int a, double t, double dt_h, int obj) {
  return obj == OBJ_SO ? link_marginal_dt(g, a, t, dt_h) : link_cost_dt(g, a, t, dt_h);
}

/* nearest integer quantum count, ties up, clamped to [1, 2^31-1] */
static int32_t quantize(double c, int *bad) {
  if (isnan(c)) { *bad = 1; return INT32_MAX; }
  double r = floor(c + 0.5);
  if (r < 1.0) return 1;
  if (r > 2147483647.0) return INT32_MAX;
  return (int32_t)r;
}

int32_t or_bpr(const or_graph *g, const double *flow, double dt_s, double *cost_s,
               int32_t *cost_q) {
  double dt_h = dt_s / 3600.0;
  int bad = 0;
  for (int a = 0; a < g->n_links; a++) {
    if (!isfinite(flow[a])) bad = 1;
    double c = link_cost(g, a, flow[a], dt_h);
    if (cost_s) cost_s[a] = c * g->quantum_s;
    cost_q[a] = quantize(c, &bad);
  }
  return bad ? OR_ENONFINITE : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Shortest paths: textbook binary-heap Dijkstra + parent post-pass.        */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t d; int32_t v; } hitem;

typedef struct { hitem *a; int64_t n, cap; } heap;

static int heap_push(heap *h, int64_t d, int32_t v) {
  if (h->n == h->cap) {
    int64_t nc = h->cap ? 2 * h->cap : 1024;
    hitem *na = (hitem *)realloc(h->a, (size_t)nc * sizeof(hitem));
    if (!na) return -1;
    h->a = na; h->cap = nc;
  }
  int64_t i = h->n++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h->a[p].d <= d) break;
    h->a[i] = h->a[p];
    i = p;
  }
  h->a[i].d = d; h->a[i].v = v;
  return 0;
}

static hitem heap_pop(heap *h) {
  hitem top = h->a[0];
  hitem last = h->a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    int64_t md = last.d;
    if (l < h->n && h->a[l].d < md) { m = l; md = h->a[l].d; }
    if (r < h->n && h->a[r].d < md) { m = r; }
    if (m == i) break;
    h->a[i] = h->a[m];
    i = m;
  }
  if (h->n > 0) h->a[i] = last;
  return top;
}

typedef struct {
  int32_t *out_off, *out_link; /* forward adjacency: links leaving v */
  int32_t *in_off, *in_link;   /* reverse adjacency: links entering v */
} adjacency;

static int build_adj(const or_graph *g, adjacency *adj) {
  int V = g->n_nodes, L = g->n_links;
  adj->out_off = (int32_t *)calloc((size_t)V + 1, 4);
  adj->in_off = (int32_t *)calloc((size_t)V + 1, 4);
  adj->out_link = (int32_t *)malloc((size_t)(L ? L : 1) * 4);
  adj->in_link = (int32_t *)malloc((size_t)(L ? L : 1) * 4);
  if (!adj->out_off || !adj->in_off || !adj->out_link || !adj->in_link) return -1;
  for (int e = 0; e < L; e++) { adj->out_off[g->tail[e] + 1]++; adj->in_off[g->head[e] + 1]++; }
  for (int v = 0; v < V; v++) { adj->out_off[v + 1] += adj->out_off[v]; adj->in_off[v + 1] += adj->in_off[v]; }
  int32_t *po = (int32_t *)malloc((size_t)V * 4 + 4), *pi = (int32_t *)malloc((size_t)V * 4 + 4);
  if (!po || !pi) return -1;
  memcpy(po, adj->out_off, (size_t)V * 4);
  memcpy(pi, adj->in_off, (size_t)V * 4);
  for (int e = 0; e < L; e++) {            /* ascending e: lists are id-sorted */
    adj->out_link[po[g->tail[e]]++] = e;
    adj->in_link[pi[g->head[e]]++] = e;
  }
  free(po); free(pi);
  return 0;
}

static void free_adj(adjacency *adj) {
  free(adj->out_off); free(adj->out_link); free(adj->in_off); free(adj->in_link);
}

/* One root.  TO_ROOT: dist[v] = shortest v -> root; parent[v] = smallest id
 * among out-links e of v with dist[head e] + q[e] == dist[v].
 * FROM_ROOT: dist[v] = shortest root -> v; parent[v] = smallest id among
 * in-links e of v with dist[tail e] + q[e] == dist[v].  parent = -1 at the
 * root and at unreachable nodes (dist = INT64_MAX there). */
static int dijkstra_one(const or_graph *g, const adjacency *adj, const int32_t *q, int32_t root,
                        int32_t dir, int32_t *parent, int64_t *dist, heap *h) {
  int V = g->n_nodes;
  for (int v = 0; v < V; v++) { dist[v] = DIST_INF; parent[v] = -1; }
  h->n = 0;
  dist[root] = 0;
  if (heap_push(h, 0, root)) return -1;
  while (h->n > 0) {
    hitem it = heap_pop(h);
    if (it.d != dist[it.v]) continue;      /* stale entry */
    int32_t w = it.v;
    if (dir == DIR_TO_ROOT) {
      for (int k = adj->in_off[w]; k < adj->in_off[w + 1]; k++) {
        int e = adj->in_link[k];
        int32_t v = g->tail[e];
        int64_t nd = it.d + q[e];
        if (nd < dist[v]) { dist[v] = nd; if (heap_push(h, nd, v)) return -1; }
      }
    } else {
      for (int k = adj->out_off[w]; k < adj->out_off[w + 1]; k++) {
        int e = adj->out_link[k];
        int32_t v = g->head[e];
        int64_t nd = it.d + q[e];
        if (nd < dist[v]) { dist[v] = nd; if (heap_push(h, nd, v)) return -1; }
      }
    }
  }
  /* parent post-pass: independent of the order in which nodes were settled */
  for (int v = 0; v < V; v++) {
    if (v == root || dist[v] == DIST_INF) continue;
    if (dir == DIR_TO_ROOT) {
      for (int k = adj->out_off[v]; k < adj->out_off[v + 1]; k++) {
        int e = adj->out_link[k];
        int64_t dh = dist[g->head[e]];
        if (dh != DIST_INF && dh + q[e] == dist[v]) { parent[v] = e; break; }
      }
    } else {
      for (int k = adj->in_off[v]; k < adj->in_off[v + 1]; k++) {
        int e = adj->in_link[k];
        int64_t dt = dist[g->tail[e]];
        if (dt != DIST_INF && dt + q[e] == dist[v]) { parent[v] = e; break; }
      }
    }
  }
  return 0;
}

int32_t or_sssp(const or_graph *g, const int32_t *q, const int32_t *roots, int32_t R,
                int32_t dir, int32_t *parent, int64_t *dist) {
  adjacency adj;
  if (build_adj(g, &adj)) return OR_ENOMEM;
  int64_t V = g->n_nodes;
  int64_t *d = dist ? NULL : (int64_t *)malloc((size_t)V * 8);
  heap h = {0};
  int rc = OR_OK;
  for (int r = 0; r < R && rc == OR_OK; r++) {
    if (dijkstra_one(g, &adj, q, roots[r], dir, parent + r * V, dist ? dist + r * V : d, &h))
      rc = OR_ENOMEM;
  }
  free(h.a); free(d); free_adj(&adj);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* All-or-nothing loading with route truncation (Alg. 3, Eq. 2, Eq. 5).     */
/* ------------------------------------------------------------------------ */

/* Walk item p -> z along the destination tree and load the links it
 * traverses before dt_q: a link is loaded iff the elapsed time on reaching
 * its tail is < dt_q.
 *  TRUNC_NODE (R1): the walk stops at the first node whose elapsed time is
 *    >= dt_q (the stop node s), or at z.
 *  TRUNC_CARRY (R17, the alternative of Section 3.4): a link that would end
 *    after dt_q holds the trip at the end of the interval; the walk stops on
 *    that link, *link_out = the link, *carry_out = the fraction of it covered,
 *    floor((dt_q - elapsed(tail)) 2^32 / q) (the returned stop node is its
 *    tail).  A link ending exactly at dt_q is completed.
 * An item carried on a link (carry_link >= 0, p its tail, carry the fraction
 * covered) first finishes that link: it covered round(q carry / 2^32) of the
 * link's q quanta and reaches the head after the rest; if the rest exceeds
 * dt_q it is still on the link, having covered carry + floor(dt_q 2^32 / q).
 * From the head it follows the tree.  A link is loaded in the interval the
 * trip enters it (its tail reached before dt_q), so a carried link is not
 * loaded again and both rules load the same links.  Returns the stop node,
 * or -1 if z is unreachable from p. */
/* R17's position on a link: the fraction covered in units of 2^-32.  The
 * quanta a fraction f of a link of q quanta stands for, rounded to nearest
 * (halves up); the fraction that t < q quanta of such a link cover, floor. */
static int64_t carried_quanta(int64_t q, int64_t f) {
  return (int64_t)(((uint64_t)q * (uint64_t)f + (1ull << 31)) >> 32);
}
static int64_t frac_of(int64_t t, int64_t q) {
  return (int64_t)(((uint64_t)t << 32) / (uint64_t)q);
}

static int32_t walk_load(const or_graph *g, const int32_t *walk_q, const int32_t *par,
                         int32_t p, int32_t z, int64_t dt_q, int64_t carry, int32_t carry_link, int trunc,
                         int64_t amount, int64_t *flow_fx, int64_t *carry_out, int32_t *link_out) {
  int32_t u = p;
  int64_t elapsed = 0;
  *carry_out = 0;
  *link_out = -1;
  if (carry_link >= 0) {
    const int64_t q = walk_q[carry_link];
    const int64_t rest = q - carried_quanta(q, carry);
    if (rest > dt_q) {  /* still on the link at the end of this interval */
      *carry_out = carry + frac_of(dt_q, q);
      *link_out = carry_link;
      return u;
    }
    elapsed = rest;
    u = g->head[carry_link];
  }
  while (u != z) {
    if (elapsed >= dt_q) return u;
    int32_t e = par[u];
    if (e < 0) return -1;
    if (flow_fx) flow_fx[e] += amount;
    if (trunc == TRUNC_CARRY && elapsed + walk_q[e] > dt_q) {
      *carry_out = frac_of(dt_q - elapsed, walk_q[e]);
      *link_out = e;
      return u;
    }
    elapsed += walk_q[e];
    u = g->head[e];
  }
  return u;
}

/* parent: [n_roots * V] destination-rooted trees built with tree_q.
 * walk_q: link times used for the elapsed-time truncation (tree_q for an
 * AON; the final costs for the residual of Alg. 4).  Items carried on a link
 * (od->carry_link) finish it first.  stop_out, carry_out, link_out
 * (nullable): per-item stop node, covered fraction and carrying link (-1 when
 * the trip waits at the node or arrived) under truncation mode `trunc`. */
static void item_carry(const or_od *od, int64_t k, int64_t *c, int32_t *l) {
  *l = od->carry_link ? od->carry_link[k] : -1;
  *c = (*l >= 0 && od->carry_frac) ? od->carry_frac[k] : 0;
}

int32_t or_load(const or_graph *g, const int32_t *walk_q, const int32_t *parent,
                const or_od *od, int64_t dt_q, int32_t trunc, int64_t *flow_fx, int32_t *stop_out,
                int64_t *carry_out, int32_t *link_out) {
  int64_t V = g->n_nodes;
  int rc = OR_OK;
  for (int64_t k = 0; k < od->n_items; k++) {
    int32_t r = od->root_idx[k];
    int64_t c0, c = 0;
    int32_t l0, l = -1;
    item_carry(od, k, &c0, &l0);
    int32_t s = walk_load(g, walk_q, parent + r * V, od->src[k], od->roots[r], dt_q, c0, l0, trunc,
                          od->amount_fx[k], flow_fx, &c, &l);
    if (s < 0) rc = OR_EUNREACH;
    if (stop_out) stop_out[k] = s;
    if (carry_out) carry_out[k] = c;
    if (link_out) link_out[k] = l;
  }
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Link sweeps of the line search (Alg. 9, Eq. 7-9).                        */
/* ------------------------------------------------------------------------ */

/* t_a = f_a + alpha * (g_a - f_a), evaluated exactly as the flow update. */
static double step_flow(double f, double gg, double alpha) {
  double d = gg - f;
  double s = alpha * d;
  return f + s;
}

/* phi(alpha) = sum_a fx(B_a(t_a(alpha)))  (Eq. 6 along the search line, Eq. 8);
 * Z_a instead of B_a for the system optimum */
static i128 phi_sum(const or_graph *g, const double *f, const double *gd, double alpha,
                    double dt_h, int obj, int *bad) {
  i128 s = 0;
  for (int a = 0; a < g->n_links; a++) s += fx_of(obj_term(g, a, step_flow(f[a], gd[a], alpha), dt_h, obj), bad);
  return s;
}

/* phi'(alpha) = sum_a fx((g_a - f_a) * c_a(t_a(alpha)))  (exact derivative) */
static i128 dphi_sum(const or_graph *g, const double *f, const double *gd, double alpha,
                     double dt_h, int obj, int *bad) {
  i128 s = 0;
  for (int a = 0; a < g->n_links; a++) {
    double d = gd[a] - f[a];
    s += fx_of(d * obj_cost(g, a, step_flow(f[a], gd[a], alpha), dt_h, obj), bad);
  }
  return s;
}

/* phi''(alpha) = sum_a fx((g_a - f_a)^2 * c_a'(t_a)) */
static i128 ddphi_sum(const or_graph *g, const double *f, const double *gd, double alpha,
                      double dt_h, int obj, int *bad) {
  i128 s = 0;
  for (int a = 0; a < g->n_links; a++) {
    double d = gd[a] - f[a];
    double dd = d * d;
    s += fx_of(dd * obj_cost_dt(g, a, step_flow(f[a], gd[a], alpha), dt_h, obj), bad);
  }
  return s;
}

/* Alg. 8 (quasi-Newton, finite differences of Eq. 9 from Alg. 9's three
 * evaluations).  j = completed FW steps before this search. */
static double ls_paper_qn3(const or_graph *g, const double *f, const double *gd, double dt_h,
                           int j, const or_params *p, int *passes, int *bad) {
  double alpha = 2.0 / (2.0 + (double)j);
  double dx = p->ls_dx;
  for (int l = 1; l < p->ls_max; l++) {
    i128 ym = phi_sum(g, f, gd, alpha - dx, dt_h, p->objective, bad);
    i128 y0 = phi_sum(g, f, gd, alpha, dt_h, p->objective, bad);
    i128 yp = phi_sum(g, f, gd, alpha + dx, dt_h, p->objective, bad);
    (*passes)++;
    double c0 = fx_to_double(y0);
    double d1 = fx_to_double(yp - ym) / (2.0 * dx);
    double d2 = fx_to_double(ym - 2 * y0 + yp) / (dx * dx);
    if (fabs(d1) < p->ls_t1 * fabs(c0)) return alpha;
    double an;
    if (d2 > 0.0) an = alpha - d1 / d2;
    else an = d1 < 0.0 ? 1.0 : 0.0;
    if (an < 0.0) an = 0.0;
    if (an > 1.0) an = 1.0;
    if (fabs(an - alpha) < p->ls_t2) return an;
    alpha = an;
  }
  return alpha;
}

/* Bracketing search on the exact slope with eight evaluations per sweep. */
static double ls_sweep8(const or_graph *g, const double *f, const double *gd, double dt_h,
                        const or_params *p, int *passes, int *bad) {
  i128 D[8];
  double a[8];
  for (int m = 0; m < 8; m++) { a[m] = (double)m / 7.0; D[m] = dphi_sum(g, f, gd, a[m], dt_h, p->objective, bad); }
  (*passes)++;
  if (D[7] <= 0) return 1.0;
  if (D[0] >= 0) return 0.0;
  int ms = 1;
  while (D[ms] < 0) ms++;
  double lo = a[ms - 1], hi = a[ms];
  i128 Dlo = D[ms - 1], Dhi = D[ms];
  while (hi - lo >= p->ls_t2 && *passes < p->ls_max) {
    double step = (hi - lo) / 9.0;
    for (int m = 0; m < 8; m++) { a[m] = lo + step * (double)(m + 1); D[m] = dphi_sum(g, f, gd, a[m], dt_h, p->objective, bad); }
    (*passes)++;
    int mf = 0;
    while (mf < 8 && D[mf] < 0) mf++;
    if (mf == 8) { lo = a[7]; Dlo = D[7]; }
    else {
      hi = a[mf]; Dhi = D[mf];
      if (mf > 0) { lo = a[mf - 1]; Dlo = D[mf - 1]; }
    }
  }
  double dlo = fx_to_double(Dlo), dhi = fx_to_double(Dhi);
  double alpha = lo + (hi - lo) * (-dlo / (dhi - dlo));
  if (alpha < lo) alpha = lo;
  if (alpha > hi) alpha = hi;
  return alpha;
}

/* Newton on the exact slope to |step| < 1e-14 inside a maintained bracket;
 * used by the adjoint so that phi'(alpha*) = 0 holds to rounding. */
static double ls_exact(const or_graph *g, const double *f, const double *gd, double dt_h,
                       int obj, int *passes, int *bad) {
  i128 D0 = dphi_sum(g, f, gd, 0.0, dt_h, obj, bad);
  i128 D1 = dphi_sum(g, f, gd, 1.0, dt_h, obj, bad);
  *passes += 2;
  if (D1 <= 0) return 1.0;
  if (D0 >= 0) return 0.0;
  double lo = 0.0, hi = 1.0, alpha = 0.5;
  for (int it = 0; it < 200; it++) {
    i128 D = dphi_sum(g, f, gd, alpha, dt_h, obj, bad);
    double H = fx_to_double(ddphi_sum(g, f, gd, alpha, dt_h, obj, bad));
    (*passes)++;
    if (D == 0) return alpha;
    if (D < 0) lo = alpha; else hi = alpha;
    double an = (H > 0.0) ? alpha - fx_to_double(D) / H : 0.5 * (lo + hi);
    if (!(an > lo && an < hi)) an = 0.5 * (lo + hi);
    if (fabs(an - alpha) < 1e-14 || hi - lo < 1e-15) return an;
    alpha = an;
  }
  return alpha;
}

static double choose_step(const or_graph *g, const double *f, const double *gd, double dt_h, int k,
                          const or_params *p, int *passes, int *bad) {
  switch (p->step) {
    case STEP_MSA: return 1.0 / ((double)k + 1.0);
    case STEP_PAPER_QN3: return ls_paper_qn3(g, f, gd, dt_h, k - 1, p, passes, bad);
    case STEP_SWEEP8: return ls_sweep8(g, f, gd, dt_h, p, passes, bad);
    default: return ls_exact(g, f, gd, dt_h, p->objective, passes, bad);
  }
}

/* exported line search for the pins: f, g_fx over all links */
int32_t or_line_search(const or_graph *g, const double *f, const int64_t *g_fx, double dt_s,
                       int32_t fw_iter, const or_params *p, double *alpha_out, int32_t *passes_out) {
  int L = g->n_links, bad = 0, passes = 0;
  double *gd = (double *)malloc((size_t)L * 8 + 8);
  if (!gd) return OR_ENOMEM;
  for (int a = 0; a < L; a++) gd[a] = (double)g_fx[a] * 0x1p-32;
  *alpha_out = choose_step(g, f, gd, dt_s / 3600.0, fw_iter, p, &passes, &bad);
  *passes_out = passes;
  free(gd);
  return bad ? OR_ENONFINITE : OR_OK;
}

/* exported objective / slope evaluation for the pins */
double or_objective(const or_graph *g, const double *f, double dt_s) {
  int bad = 0;
  i128 s = 0;
  for (int a = 0; a < g->n_links; a++) s += fx_of(beckmann(g, a, f[a], dt_s / 3600.0), &bad);
  return fx_to_double(s);
}

double or_slope(const or_graph *g, const double *f, const int64_t *g_fx, double dt_s, double alpha) {
  int L = g->n_links, bad = 0;
  double *gd = (double *)malloc((size_t)L * 8 + 8);
  for (int a = 0; a < L; a++) gd[a] = (double)g_fx[a] * 0x1p-32;
  double r = fx_to_double(dphi_sum(g, f, gd, alpha, dt_s / 3600.0, OBJ_UE, &bad));
  free(gd);
  return r;
}


/* ------------------------------------------------------------------------ */
/* Scenario metrics of assigned intervals (Section 7.1: VMT, average volume */
/* over capacity, vehicle hours of delay by functional class, over links    */
/* with positive flow; the congested subset has volume over capacity >= a   */
/* threshold, 1.0 in the paper).  Per interval i and class k, into          */
/* out[(i * n_classes + k) * 8 + m]:                                         */
/*   m 0: links with flow > 0                                               */
/*   m 1: VMT, veh-km        = sum f * len / 1000                           */
/*   m 2: average VOC        = sum x / count, x = f / (C dt_h)              */
/*   m 3: VHD, veh-h         = sum f * (c(f) - c0) * quantum_s / 3600       */
/*   m 4: congested links (x >= threshold)                                  */
/*   m 5: congested length, km;  m 6: congested VMT;  m 7: congested VOC    */
/* f = flows[i * L + a] (trips in the interval); c(f) per Eq. 1.  Links     */
/* whose class is outside [0, n_classes) are not counted.  Every sum is the */
/* exact sum of per-link terms rounded to 2^-32 (R6).                       */
/* ------------------------------------------------------------------------ */
int or_interval_metrics(const or_graph *g, const double *flows, int32_t N, double dt_s,
                        const double *length_m, const int32_t *link_class, int32_t n_classes,
                        double congested_voc, double quantum_s, double *out) {
  if (N < 0 || n_classes < 1 || n_classes > 16 || !(dt_s > 0.0) || !(quantum_s > 0.0)) return OR_EINVAL;
  const int L = g->n_links;
  const double dt_h = dt_s / 3600.0;
  const double hours_per_quantum = quantum_s / 3600.0;
  int bad = 0;
  for (int32_t i = 0; i < N; i++) {
    for (int k = 0; k < n_classes; k++) {
      i128 vmt = 0, voc = 0, vhd = 0, clen = 0, cvmt = 0, cvoc = 0;
      int64_t n = 0, cn = 0;
      for (int a = 0; a < L; a++) {
        const double f = flows[(int64_t)i * L + a];
        if (!isfinite(f)) { bad = 1; continue; }
        if (!(f > 0.0) || link_class[a] != k) continue;
        const double x = f * inv_cap(g, a, dt_h);
        const double d = link_cost(g, a, f, dt_h) - (double)g->fftime_q[a];
        const double fl = f * length_m[a];
        n += 1;
        vmt += fx_of(fl, &bad);
        voc += fx_of(x, &bad);
        vhd += fx_of(f * d, &bad);
        if (x >= congested_voc) {
          cn += 1;
          clen += fx_of(length_m[a], &bad);
          cvmt += fx_of(fl, &bad);
          cvoc += fx_of(x, &bad);
        }
      }
      double *o = out + ((int64_t)i * n_classes + k) * 8;
      o[0] = (double)n;
      o[1] = fx_to_double(vmt) * 1e-3;
      o[2] = n ? fx_to_double(voc) / (double)n : 0.0;
      o[3] = fx_to_double(vhd) * hours_per_quantum;
      o[4] = (double)cn;
      o[5] = fx_to_double(clen) * 1e-3;
      o[6] = fx_to_double(cvmt) * 1e-3;
      o[7] = cn ? fx_to_double(cvoc) / (double)cn : 0.0;
    }
  }
  return bad ? OR_ENONFINITE : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Frank-Wolfe per interval (Alg. 2 / Alg. 6).                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t K;          /* accepted steps */
  int32_t cap;        /* capacity in iterations (K <= cap - 1) */
  int32_t *q;         /* [cap][L] link times of each AON on the path (q_0 = free flow) */
  double *alpha;      /* [cap]  alpha_0 = 1 */
  double *f;          /* [cap][L] iterate after step j (f_0 = g_0) */
} or_tape;

static int64_t dt_quanta(const or_graph *g, double dt_s) {
  if (!(dt_s < 1e300)) return INT64_MAX;    /* infinite interval: no truncation */
  return (int64_t)floor(dt_s / g->quantum_s + 0.5);
}

/* one AON: trees from the routing costs q, loading with truncation under the
 * travel times qt (the same array for the user equilibrium) */
static int aon(const or_graph *g, const adjacency *adj, const int32_t *q, const int32_t *qt, const or_od *od,
               int64_t dt_q, int32_t *parent, int64_t *dist, const uint8_t *root_used,
               int64_t *g_fx, heap *h) {
  int64_t V = g->n_nodes;
  for (int r = 0; r < od->n_roots; r++) {
    if (!root_used[r]) continue;
    if (dijkstra_one(g, adj, q, od->roots[r], DIR_TO_ROOT, parent + r * V, dist, h)) return OR_ENOMEM;
  }
  memset(g_fx, 0, (size_t)g->n_links * 8);
  /* the loaded links do not depend on the truncation mode */
  return or_load(g, qt, parent, od, dt_q, TRUNC_NODE, g_fx, NULL, NULL, NULL);
}

/* routing costs q and travel times qt at flows f: q = qt = quant(c(f)) for the
 * user equilibrium, q = quant(m(f)) (marginal cost) for the system optimum */
static int route_costs(const or_graph *g, const double *f, double dt_s, int obj, int32_t *q, int32_t *qt) {
  int rc = or_bpr(g, f, dt_s, NULL, qt);
  if (obj != OBJ_SO) {
    memcpy(q, qt, (size_t)g->n_links * 4);
    return rc;
  }
  int bad = 0;
  const double dt_h = dt_s / 3600.0;
  for (int a = 0; a < g->n_links; a++) q[a] = quantize(link_marginal(g, a, f[a], dt_h), &bad);
  return bad ? OR_ENONFINITE : rc;
}

static int assign_core(const or_graph *g, const or_od *od, double dt_s, const or_params *p,
                       double *f_out, or_stats *st, or_tape *tape) {
  int L = g->n_links;
  int64_t V = g->n_nodes;
  double dt_h = dt_s / 3600.0;
  int64_t dt_q = dt_quanta(g, dt_s);
  int rc = OR_OK, bad = 0;
  adjacency adj;
  if (build_adj(g, &adj)) return OR_ENOMEM;
  int32_t *q = (int32_t *)malloc((size_t)L * 4 + 4);
  int32_t *qt = (int32_t *)malloc((size_t)L * 4 + 4);
  int32_t *parent = (int32_t *)malloc((size_t)(od->n_roots ? od->n_roots : 1) * V * 4);
  int64_t *dist = (int64_t *)malloc((size_t)V * 8);
  int64_t *g_fx = (int64_t *)malloc((size_t)L * 8 + 8);
  double *gd = (double *)malloc((size_t)L * 8 + 8);
  double *fn = (double *)malloc((size_t)L * 8 + 8);
  uint8_t *used = (uint8_t *)calloc((size_t)od->n_roots + 1, 1);
  heap h = {0};
  if (!q || !qt || !parent || !dist || !g_fx || !gd || !fn || !used) { rc = OR_ENOMEM; goto done; }
  for (int64_t k = 0; k < od->n_items; k++) used[od->root_idx[k]] = 1;
  memset(st, 0, sizeof(*st));
  st->rel_gap = NAN;
  st->dual_gap = NAN;

  /* initial AON at free flow: q = BPR(0) */
  for (int a = 0; a < L; a++) f_out[a] = 0.0;
  if (od->n_items == 0) {          /* no demand: zero flows, converged at once */
    st->converged = 1;
    st->rel_gap = 0.0;
    st->dual_gap = 0.0;
    if (tape) { tape->K = 0; tape->alpha[0] = 1.0; memset(tape->f, 0, (size_t)L * 8);
                or_bpr(g, f_out, dt_s, NULL, tape->q); }
    goto done;
  }
  if (route_costs(g, f_out, dt_s, p->objective, q, qt)) { rc = OR_ENONFINITE; goto done; }
  rc = aon(g, &adj, q, qt, od, dt_q, parent, dist, used, g_fx, &h);
  st->aon_calls = 1;
  if (rc) goto done;
  for (int a = 0; a < L; a++) f_out[a] = (double)g_fx[a] * 0x1p-32;
  if (tape) {
    tape->K = 0;
    memcpy(tape->q, q, (size_t)L * 4);
    tape->alpha[0] = 1.0;
    memcpy(tape->f, f_out, (size_t)L * 8);
  }

  for (int k = 1;; k++) {
    if (k > p->max_iter) { if (p->stop != STOP_NONE) rc = OR_NOTCONV; break; }
    if (route_costs(g, f_out, dt_s, p->objective, q, qt)) { rc = OR_ENONFINITE; break; }
    rc = aon(g, &adj, q, qt, od, dt_q, parent, dist, used, g_fx, &h);
    st->aon_calls++;
    if (rc) break;
    for (int a = 0; a < L; a++) gd[a] = (double)g_fx[a] * 0x1p-32;
    {
      /* relative duality gap (sum q f - sum q g) / sum q f with q the costs
       * at f, measured every iteration; the REL_GAP rule stops on it */
      i128 A = 0, B = 0;
      for (int a = 0; a < L; a++) {
        A += fx_of((double)q[a] * f_out[a], &bad);
        B += (i128)q[a] * (i128)g_fx[a];
      }
      st->dual_gap = fx_to_double(A - B) / fx_to_double(A);
      if (p->stop == STOP_REL_GAP) {
        /* The gap certifies convergence only when it is not negative.  With
         * truncated loading (Eq. 2) the all-or-nothing loading g need not
         * minimise sum c g, so the gap can fall below zero without f being
         * near an equilibrium; such a value does not stop the iteration.
         * -1e-12 absorbs the rounding of the per-link products c f at an
         * exact all-or-nothing equilibrium (gap 0 up to a few ulps). */
        st->rel_gap = st->dual_gap;
        if (st->rel_gap <= p->tol && st->rel_gap >= -1e-12) { st->converged = 1; break; }
      }
    }
    int passes = 0;
    double alpha = choose_step(g, f_out, gd, dt_h, k, p, &passes, &bad);
    st->ls_passes += passes;
    for (int a = 0; a < L; a++) fn[a] = step_flow(f_out[a], gd[a], alpha);
    if (p->stop == STOP_PAPER_OBJ) {
      i128 c1 = 0, c2 = 0;
      for (int a = 0; a < L; a++) {
        c1 += fx_of(obj_term(g, a, f_out[a], dt_h, p->objective), &bad);
        c2 += fx_of(obj_term(g, a, fn[a], dt_h, p->objective), &bad);
      }
      double rel = fabs(fx_to_double(c1 - c2)) / fx_to_double(c1);
      st->rel_gap = rel;
      if (rel < p->tol) { st->converged = 1; break; }   /* keep the pre-step iterate */
    }
    memcpy(f_out, fn, (size_t)L * 8);
    st->iterations = k;
    if (tape) {
      if (k >= tape->cap) { rc = OR_ENOMEM; break; }
      tape->K = k;
      memcpy(tape->q + (int64_t)k * L, q, (size_t)L * 4);
      tape->alpha[k] = alpha;
      memcpy(tape->f + (int64_t)k * L, f_out, (size_t)L * 8);
    }
  }
  if (bad && rc >= 0) rc = OR_ENONFINITE;
  {
    i128 obj = 0;
    for (int a = 0; a < L; a++) obj += fx_of(obj_term(g, a, f_out[a], dt_h, p->objective), &bad);
    st->objective = fx_to_double(obj);
  }
done:
  free(q); free(qt); free(parent); free(dist); free(g_fx); free(gd); free(fn); free(used); free(h.a);
  free_adj(&adj);
  return rc;
}

/* Exported: one interval.  tape_q [(cap) * L], tape_alpha [cap], tape_f
 * [(cap) * L] are optional (all NULL or all set); *tape_K receives K. */
int32_t or_assign_interval(const or_graph *g, const or_od *od, double dt_s, const or_params *p,
                           double *f_out, or_stats *st, int32_t tape_cap, int32_t *tape_q,
                           double *tape_alpha, double *tape_f, int32_t *tape_K) {
  if (tape_q) {
    or_tape t = {0, tape_cap, tape_q, tape_alpha, tape_f};
    int rc = assign_core(g, od, dt_s, p, f_out, st, &t);
    *tape_K = t.K;
    return rc;
  }
  return assign_core(g, od, dt_s, p, f_out, st, NULL);
}

/* ------------------------------------------------------------------------ */
/* Residual demand (Alg. 4).                                                */
/* ------------------------------------------------------------------------ */

/* path weights of h^STA = sum_j w_j AON_j: w_j = alpha_j * prod_{m>j} (1 - alpha_m) */
static void path_weights(const double *alpha, int K, double *w) {
  double P = 1.0;
  for (int j = K; j >= 0; j--) {
    double a = (j == 0) ? 1.0 : alpha[j];
    w[j] = a * P;
    P = P * (1.0 - a);
  }
}

static int64_t scale_amount(int64_t amount_fx, double w) {
  double v = (double)amount_fx * w;
  return (int64_t)nearbyint(v);
}

/* Re-truncate every path of every accepted AON with the final costs.
 * h_fx[L] receives the truncated link flows h(i); residual entries
 * (stop node, root index, amount, covered fraction) are written up to
 * res_cap, *res_n gets the number produced (before any merge).  res_carry,
 * res_link (nullable) receive the covered fraction and carrying link of each
 * entry (0 and
 * -1 for a trip waiting at its stop node). */
int32_t or_residual(const or_graph *g, const or_od *od, double dt_s, int32_t K,
                    const int32_t *tape_q, const double *tape_alpha, const double *f_final,
                    int32_t trunc, int64_t *h_fx, int64_t res_cap, int32_t *res_stop, int32_t *res_root,
                    int64_t *res_amount, int64_t *res_carry, int32_t *res_link, int64_t *res_n) {
  int L = g->n_links;
  int64_t V = g->n_nodes;
  int64_t dt_q = dt_quanta(g, dt_s);
  adjacency adj;
  if (build_adj(g, &adj)) return OR_ENOMEM;
  int32_t *qfin = (int32_t *)malloc((size_t)L * 4 + 4);
  int32_t *parent = (int32_t *)malloc((size_t)(od->n_roots ? od->n_roots : 1) * V * 4);
  int64_t *dist = (int64_t *)malloc((size_t)V * 8);
  double *w = (double *)malloc(((size_t)K + 1) * 8);
  uint8_t *used = (uint8_t *)calloc((size_t)od->n_roots + 1, 1);
  heap h = {0};
  int rc = OR_OK;
  if (!qfin || !parent || !dist || !w || !used) { rc = OR_ENOMEM; goto done; }
  rc = or_bpr(g, f_final, dt_s, NULL, qfin);
  if (rc) goto done;
  path_weights(tape_alpha, K, w);
  for (int64_t k = 0; k < od->n_items; k++) used[od->root_idx[k]] = 1;
  memset(h_fx, 0, (size_t)L * 8);
  *res_n = 0;
  for (int j = 0; j <= K && rc == OR_OK; j++) {
    const int32_t *qj = tape_q + (int64_t)j * L;
    for (int r = 0; r < od->n_roots; r++) {
      if (!used[r]) continue;
      if (dijkstra_one(g, &adj, qj, od->roots[r], DIR_TO_ROOT, parent + r * V, dist, &h)) { rc = OR_ENOMEM; break; }
    }
    for (int64_t k = 0; k < od->n_items && rc == OR_OK; k++) {
      int64_t amt = scale_amount(od->amount_fx[k], w[j]);
      if (amt == 0) continue;
      int32_t r = od->root_idx[k];
      int64_t c0, c = 0;
      int32_t l0, l = -1;
      item_carry(od, k, &c0, &l0);
      int32_t s = walk_load(g, qfin, parent + r * V, od->src[k], od->roots[r], dt_q, c0, l0, trunc, amt, h_fx,
                            &c, &l);
      if (s < 0) { rc = OR_EUNREACH; break; }
      if (s != od->roots[r] || l >= 0) {
        if (*res_n < res_cap) {
          res_stop[*res_n] = s; res_root[*res_n] = r; res_amount[*res_n] = amt;
          if (res_carry) res_carry[*res_n] = c;
          if (res_link) res_link[*res_n] = l;
        }
        (*res_n)++;
      }
    }
  }
done:
  free(qfin); free(parent); free(dist); free(w); free(used); free(h.a); free_adj(&adj);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Full day (Alg. 1): d(i) = d_o(i) + d_r(i); STA; residual.                */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t root, src; int64_t amt, carry; int32_t link; } item3;

static int cmp_item3(const void *a, const void *b) {
  const item3 *x = (const item3 *)a, *y = (const item3 *)b;
  if (x->root != y->root) return x->root < y->root ? -1 : 1;
  if (x->link != y->link) return x->link < y->link ? -1 : 1;
  if (x->src != y->src) return x->src < y->src ? -1 : 1;
  return 0;
}

/* merge an item list as the paper keeps residual demand d_{s,q}: trips
 * waiting at a node (link -1) by (root, node), summing amounts; trips on a
 * link (R17) by (root, link), with the amount-weighted mean covered
 * fraction floor(sum amt * carry / sum amt) in exact 128-bit integers;
 * returns the count */
static int64_t merge_items(item3 *buf, int64_t n) {
  qsort(buf, (size_t)n, sizeof(item3), cmp_item3);
  int64_t m = 0;
  i128 tsum = 0;
  for (int64_t k = 0; k < n; k++) {
    if (m > 0 && buf[m - 1].root == buf[k].root && buf[m - 1].link == buf[k].link && buf[m - 1].src == buf[k].src) {
      buf[m - 1].amt += buf[k].amt;
    } else {
      if (m > 0 && buf[m - 1].link >= 0) buf[m - 1].carry = buf[m - 1].amt > 0 ? (int64_t)(tsum / buf[m - 1].amt) : 0;
      buf[m++] = buf[k];
      tsum = 0;
    }
    if (buf[k].link >= 0) tsum += (i128)buf[k].amt * buf[k].carry;
  }
  if (m > 0 && buf[m - 1].link >= 0) buf[m - 1].carry = buf[m - 1].amt > 0 ? (int64_t)(tsum / buf[m - 1].amt) : 0;
  return m;
}

/* Exported: N intervals over the zone list `zones` (the roots of every
 * interval).  Interval i's original items are [item_off[i], item_off[i+1])
 * of (root_idx, src, amount_fx).  flows_out [N * L] receives h(i) (trips);
 * stats [N]; n_items_out [N] the merged item count of each interval;
 * resid_out_n receives the count of residual items left after the last
 * interval (merged, sorted by root, link, src); the first res_cap of them
 * go to res_root/src/amt/carry/link when res_root is not NULL. */
int32_t or_run_day(const or_graph *g, int32_t n_zones, const int32_t *zones, int32_t N,
                   const int64_t *item_off, const int32_t *root_idx, const int32_t *src,
                   const int64_t *amount_fx, double dt_s, const or_params *p,
                   double *flows_out, or_stats *stats, int64_t *n_items_out,
                   int64_t *resid_out_n, int64_t res_cap, int32_t *res_root, int32_t *res_src,
                   int64_t *res_amt, int64_t *res_carry, int32_t *res_link) {
  int L = g->n_links;
  int rc = OR_OK;
  int cap = p->max_iter + 2;
  int64_t rn = 0, rcap = 0;
  item3 *resid = NULL;
  int32_t *tq = (int32_t *)malloc((size_t)cap * L * 4);
  double *ta = (double *)malloc((size_t)cap * 8);
  double *tf = (double *)malloc((size_t)cap * L * 8);
  double *f = (double *)malloc((size_t)L * 8 + 8);
  int64_t *hfx = (int64_t *)malloc((size_t)L * 8 + 8);
  if (!tq || !ta || !tf || !f || !hfx) { rc = OR_ENOMEM; goto done; }
  for (int i = 0; i < N && rc >= 0; i++) {
    int64_t n0 = item_off[i + 1] - item_off[i];
    item3 *buf = (item3 *)malloc((size_t)(n0 + rn + 1) * sizeof(item3));
    if (!buf) { rc = OR_ENOMEM; break; }
    for (int64_t k = 0; k < n0; k++) {
      buf[k].root = root_idx[item_off[i] + k]; buf[k].src = src[item_off[i] + k];
      buf[k].amt = amount_fx[item_off[i] + k];
      buf[k].carry = 0;
      buf[k].link = -1;
    }
    for (int64_t k = 0; k < rn; k++) buf[n0 + k] = resid[k];
    int64_t n = merge_items(buf, n0 + rn);
    int32_t *ri = (int32_t *)malloc((size_t)(n + 1) * 4), *si = (int32_t *)malloc((size_t)(n + 1) * 4);
    int64_t *ai = (int64_t *)malloc((size_t)(n + 1) * 8), *ci = (int64_t *)malloc((size_t)(n + 1) * 8);
    int32_t *li = (int32_t *)malloc((size_t)(n + 1) * 4);
    for (int64_t k = 0; k < n; k++) {
      ri[k] = buf[k].root; si[k] = buf[k].src; ai[k] = buf[k].amt; ci[k] = buf[k].carry; li[k] = buf[k].link;
    }
    free(buf);
    n_items_out[i] = n;
    or_od od = {n_zones, zones, n, ri, si, ai, ci, li};
    int32_t K = 0;
    int r1 = or_assign_interval(g, &od, dt_s, p, f, &stats[i], cap, tq, ta, tf, &K);
    if (r1 < 0) { rc = r1; free(ri); free(si); free(ai); free(ci); free(li); break; }
    if (r1 > 0) rc = r1;
    /* residual: at most one triple per item and accepted AON */
    int64_t need = n * ((int64_t)K + 1);
    if (need > rcap) {
      free(resid); rcap = need; resid = (item3 *)malloc((size_t)(rcap + 1) * sizeof(item3));
    }
    int32_t *rs = (int32_t *)malloc((size_t)(need + 1) * 4), *rr = (int32_t *)malloc((size_t)(need + 1) * 4);
    int64_t *ra = (int64_t *)malloc((size_t)(need + 1) * 8), *rcy = (int64_t *)malloc((size_t)(need + 1) * 8);
    int32_t *rl = (int32_t *)malloc((size_t)(need + 1) * 4);
    int64_t got = 0;
    int r2 = or_residual(g, &od, dt_s, K, tq, ta, f, p->truncation, hfx, need, rs, rr, ra, rcy, rl, &got);
    for (int64_t k = 0; k < got; k++) {
      resid[k].root = rr[k]; resid[k].src = rs[k]; resid[k].amt = ra[k]; resid[k].carry = rcy[k];
      resid[k].link = rl[k];
    }
    rn = merge_items(resid, got);
    for (int a = 0; a < L; a++) flows_out[(int64_t)i * L + a] = (double)hfx[a] * 0x1p-32;
    free(rs); free(rr); free(ra); free(rcy); free(rl); free(ri); free(si); free(ai); free(ci); free(li);
    if (r2 < 0) { rc = r2; break; }
  }
  *resid_out_n = rn;
  for (int64_t k = 0; res_root && k < rn && k < res_cap; k++) {
    res_root[k] = resid[k].root; res_src[k] = resid[k].src; res_amt[k] = resid[k].amt;
    res_carry[k] = resid[k].carry; res_link[k] = resid[k].link;
  }
done:
  free(resid); free(tq); free(ta); free(tf); free(f); free(hfx);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the unrolled FW map with trees and truncation fixed.          */
/* ------------------------------------------------------------------------ */

/* Loss gradient dL/df of the returned iterate f_K is propagated back through
 * f_k = (1 - alpha_k) f_{k-1} + alpha_k g_k, g_k = Delta_k d.  With a line
 * search, alpha_k solves phi'(alpha) = 0 and its derivatives follow from the
 * implicit function theorem; with MSA (or a clipped alpha) they are zero. */
int32_t or_backward(const or_graph *g, const or_od *od, double dt_s, int32_t step_mode,
                    int32_t K, const int32_t *tape_q, const double *tape_alpha,
                    const double *tape_f, const double *dL_df, double *dL_dd, double *dL_dcap) {
  int L = g->n_links;
  int64_t V = g->n_nodes;
  double dt_h = dt_s / 3600.0;
  int64_t dt_q = dt_quanta(g, dt_s);
  adjacency adj;
  if (build_adj(g, &adj)) return OR_ENOMEM;
  int32_t *parent = (int32_t *)malloc((size_t)(od->n_roots ? od->n_roots : 1) * V * 4);
  int64_t *dist = (int64_t *)malloc((size_t)V * 8);
  int64_t *g_fx = (int64_t *)malloc((size_t)L * 8 + 8);
  double *lam = (double *)malloc((size_t)L * 8 + 8);
  double *lam2 = (double *)malloc((size_t)L * 8 + 8);
  double *gbar = (double *)malloc((size_t)L * 8 + 8);
  uint8_t *used = (uint8_t *)calloc((size_t)od->n_roots + 1, 1);
  heap h = {0};
  int rc = OR_OK;
  if (!parent || !dist || !g_fx || !lam || !lam2 || !gbar || !used) { rc = OR_ENOMEM; goto done; }
  for (int64_t k = 0; k < od->n_items; k++) used[od->root_idx[k]] = 1;
  memcpy(lam, dL_df, (size_t)L * 8);
  for (int64_t k = 0; k < od->n_items; k++) dL_dd[k] = 0.0;
  for (int a = 0; a < L; a++) dL_dcap[a] = 0.0;
  for (int k = K; k >= 0 && rc == OR_OK; k--) {
    const int32_t *qk = tape_q + (int64_t)k * L;
    rc = aon(g, &adj, qk, qk, od, dt_q, parent, dist, used, g_fx, &h);  /* recompute tree k and g_k */
    if (rc) break;
    if (k == 0) {
      memcpy(gbar, lam, (size_t)L * 8);
    } else {
      const double *fp = tape_f + (int64_t)(k - 1) * L;
      double alpha = tape_alpha[k];
      double mu = 0.0;
      for (int a = 0; a < L; a++) mu += lam[a] * ((double)g_fx[a] * 0x1p-32 - fp[a]);
      int implicit = (step_mode != STEP_MSA) && alpha > 0.0 && alpha < 1.0;
      double H = 0.0;
      if (implicit) {
        for (int a = 0; a < L; a++) {
          double d = (double)g_fx[a] * 0x1p-32 - fp[a];
          double t = step_flow(fp[a], (double)g_fx[a] * 0x1p-32, alpha);
          H += d * d * link_cost_dt(g, a, t, dt_h);
        }
        if (!(H > 0.0)) implicit = 0;
      }
      for (int a = 0; a < L; a++) {
        double gg = (double)g_fx[a] * 0x1p-32;
        double d = gg - fp[a];
        gbar[a] = alpha * lam[a];
        lam2[a] = (1.0 - alpha) * lam[a];
        if (implicit) {
          double t = step_flow(fp[a], gg, alpha);
          double c = link_cost(g, a, t, dt_h);
          double cp = link_cost_dt(g, a, t, dt_h);
          gbar[a] -= mu * (c + alpha * d * cp) / H;
          lam2[a] -= mu * (-c + (1.0 - alpha) * d * cp) / H;
          dL_dcap[a] -= mu * d * link_cost_dcap(g, a, t, dt_h) / H;
        }
      }
    }
    /* path-sum gather: transpose of the truncated loading on tree k */
    for (int64_t it = 0; it < od->n_items; it++) {
      int32_t r = od->root_idx[it];
      const int32_t *par = parent + r * V;
      int32_t u = od->src[it], z = od->roots[r];
      int64_t elapsed = 0, c0;
      int32_t l0;
      double acc = 0.0;
      item_carry(od, it, &c0, &l0);
      if (l0 >= 0) {  /* the rest of the carried link (not loaded), then on from its head */
        const int64_t rest = (int64_t)qk[l0] - carried_quanta(qk[l0], c0);
        if (rest > dt_q) continue;
        elapsed = rest;
        u = g->head[l0];
      }
      while (u != z && elapsed < dt_q) {
        int32_t e = par[u];
        if (e < 0) { rc = OR_EUNREACH; break; }
        acc += gbar[e];
        elapsed += qk[e];
        u = g->head[e];
      }
      dL_dd[it] += acc;
    }
    if (k > 0) memcpy(lam, lam2, (size_t)L * 8);
  }
done:
  free(parent); free(dist); free(g_fx); free(lam); free(lam2); free(gbar); free(used); free(h.a);
  free_adj(&adj);
  return rc;
}

/* Replay of the forward map with the taped trees (q_0..q_K) held fixed and
 * the items' amounts replaced; steps re-solved by `step_mode`.  Used by the
 * finite-difference checks of the adjoint. */
int32_t or_replay(const or_graph *g, const or_od *od, double dt_s, const or_params *p, int32_t K,
                  const int32_t *tape_q, double *f_out) {
  int L = g->n_links;
  int64_t V = g->n_nodes;
  double dt_h = dt_s / 3600.0;
  int64_t dt_q = dt_quanta(g, dt_s);
  adjacency adj;
  if (build_adj(g, &adj)) return OR_ENOMEM;
  int32_t *parent = (int32_t *)malloc((size_t)(od->n_roots ? od->n_roots : 1) * V * 4);
  int64_t *dist = (int64_t *)malloc((size_t)V * 8);
  int64_t *g_fx = (int64_t *)malloc((size_t)L * 8 + 8);
  double *gd = (double *)malloc((size_t)L * 8 + 8);
  uint8_t *used = (uint8_t *)calloc((size_t)od->n_roots + 1, 1);
  heap h = {0};
  int rc = OR_OK, bad = 0;
  for (int64_t k = 0; k < od->n_items; k++) used[od->root_idx[k]] = 1;
  for (int k = 0; k <= K && rc == OR_OK; k++) {
    rc = aon(g, &adj, tape_q + (int64_t)k * L, tape_q + (int64_t)k * L, od, dt_q, parent, dist, used, g_fx, &h);
    if (rc) break;
    for (int a = 0; a < L; a++) gd[a] = (double)g_fx[a] * 0x1p-32;
    if (k == 0) { memcpy(f_out, gd, (size_t)L * 8); continue; }
    int passes = 0;
    double alpha = choose_step(g, f_out, gd, dt_h, k, p, &passes, &bad);
    for (int a = 0; a < L; a++) f_out[a] = step_flow(f_out[a], gd[a], alpha);
  }
  free(parent); free(dist); free(g_fx); free(gd); free(used); free(h.a); free_adj(&adj);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Customizable contraction hierarchy (Section 5.1 routes with RoutingKit's  */
/* customizable contraction hierarchies; here an alternative route to the    */
/* same exact distances as the Dijkstra above).                              */
/*   Build (metric-independent): nodes are contracted in a given order;      */
/*   contracting v joins every pair of its neighbours of higher rank, so the */
/*   upward neighbours of every node form a clique (the graph becomes        */
/*   chordal).  Each upward edge {x, y}, rank x < rank y, carries two        */
/*   weights: fw = cost x -> y, bw = cost y -> x.                            */
/*   Customization (per metric): fw / bw start at the cheapest original link */
/*   in that direction (infinite if none); then, for v in increasing rank,   */
/*   every lower triangle {v, u, w} with u, w upward neighbours of v lowers  */
/*   the edge {u, w} by the path through v.  After it, every shortest path   */
/*   has an up-down form in the upward graph.                                */
/*   Queries: s -> t is the minimum over meeting nodes m of an upward search */
/*   from s (fw) plus an upward search from t (bw, the path read backwards); */
/*   all v -> z distances take the upward search from z, then one sweep in   */
/*   decreasing rank: D(v) = min(down(v), min over upward u of fw(v,u)+D(u)).*/
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t V, L;
  int32_t *rank;    /* [V] */
  int64_t *up_off;  /* [V + 1] */
  int32_t *up_node; /* [E] upward neighbours of each node, by increasing rank */
  int64_t *fw, *bw; /* [E] */
  int32_t *tail, *head;
  int64_t E;
} or_cch;

typedef struct { int32_t *a; int64_t n, cap; } ivec;

static int ivec_push(ivec *v, int32_t x) {
  if (v->n == v->cap) {
    int64_t c = v->cap ? 2 * v->cap : 8;
    int32_t *p = (int32_t *)realloc(v->a, (size_t)c * 4);
    if (!p) return 1;
    v->a = p;
    v->cap = c;
  }
  v->a[v->n++] = x;
  return 0;
}

static const int32_t *g_rank_for_sort;
static int cmp_by_rank(const void *a, const void *b) {
  int32_t x = g_rank_for_sort[*(const int32_t *)a], y = g_rank_for_sort[*(const int32_t *)b];
  return (x > y) - (x < y);
}

void or_cch_free(or_cch *c) {
  if (!c) return;
  free(c->rank); free(c->up_off); free(c->up_node); free(c->fw); free(c->bw); free(c->tail); free(c->head);
  free(c);
}

/* order [V]: the nodes in contraction order (a permutation of 0..V-1) */
int32_t or_cch_build(const or_graph *g, const int32_t *order, or_cch **out) {
  const int32_t V = g->n_nodes, L = g->n_links;
  *out = NULL;
  or_cch *c = (or_cch *)calloc(1, sizeof(or_cch));
  ivec *up = (ivec *)calloc((size_t)V + 1, sizeof(ivec));
  if (!c || !up) { free(c); free(up); return OR_ENOMEM; }
  c->V = V; c->L = L;
  c->rank = (int32_t *)malloc((size_t)V * 4 + 4);
  c->tail = (int32_t *)malloc((size_t)L * 4 + 4);
  c->head = (int32_t *)malloc((size_t)L * 4 + 4);
  int rc = OR_OK;
  if (!c->rank || !c->tail || !c->head) { rc = OR_ENOMEM; goto fail; }
  for (int32_t v = 0; v < V; v++) c->rank[v] = -1;
  for (int32_t i = 0; i < V; i++) {
    if (order[i] < 0 || order[i] >= V || c->rank[order[i]] >= 0) { rc = OR_EINVAL; goto fail; }
    c->rank[order[i]] = i;
  }
  memcpy(c->tail, g->tail, (size_t)L * 4);
  memcpy(c->head, g->head, (size_t)L * 4);
  /* undirected neighbours, each stored at its lower end */
  for (int32_t a = 0; a < L; a++) {
    int32_t x = g->tail[a], y = g->head[a];
    if (x == y) continue;
    if (c->rank[x] > c->rank[y]) { int32_t t = x; x = y; y = t; }
    if (ivec_push(&up[x], y)) { rc = OR_ENOMEM; goto fail; }
  }
  /* contraction in order: sort and deduplicate v's upward neighbours, then
   * join every pair of them at the lower end of the pair */
  g_rank_for_sort = c->rank;
  for (int32_t i = 0; i < V; i++) {
    const int32_t v = order[i];
    ivec *U = &up[v];
    qsort(U->a, (size_t)U->n, 4, cmp_by_rank);
    int64_t m = 0;
    for (int64_t k = 0; k < U->n; k++)
      if (m == 0 || U->a[m - 1] != U->a[k]) U->a[m++] = U->a[k];
    U->n = m;
    for (int64_t p = 0; p < m; p++)
      for (int64_t q = p + 1; q < m; q++)
        if (ivec_push(&up[U->a[p]], U->a[q])) { rc = OR_ENOMEM; goto fail; }
  }
  c->up_off = (int64_t *)malloc(((size_t)V + 1) * 8);
  if (!c->up_off) { rc = OR_ENOMEM; goto fail; }
  c->up_off[0] = 0;
  for (int32_t v = 0; v < V; v++) c->up_off[v + 1] = c->up_off[v] + up[v].n;
  c->E = c->up_off[V];
  c->up_node = (int32_t *)malloc((size_t)c->E * 4 + 4);
  c->fw = (int64_t *)malloc((size_t)c->E * 8 + 8);
  c->bw = (int64_t *)malloc((size_t)c->E * 8 + 8);
  if (!c->up_node || !c->fw || !c->bw) { rc = OR_ENOMEM; goto fail; }
  for (int32_t v = 0; v < V; v++)
    if (up[v].n) memcpy(c->up_node + c->up_off[v], up[v].a, (size_t)up[v].n * 4);
  for (int32_t v = 0; v <= V; v++) free(up[v].a);
  free(up);
  *out = c;
  return OR_OK;
fail:
  for (int32_t v = 0; v <= V; v++) free(up[v].a);
  free(up);
  or_cch_free(c);
  return rc;
}

int64_t or_cch_edges(const or_cch *c) { return c->E; }

/* index of the upward edge {x, y} (rank x < rank y), or -1 */
static int64_t cch_edge(const or_cch *c, int32_t x, int32_t y) {
  int64_t lo = c->up_off[x], hi = c->up_off[x + 1] - 1;
  const int32_t ry = c->rank[y];
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    int32_t r = c->rank[c->up_node[mid]];
    if (r == ry) return mid;
    if (r < ry) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

static int64_t add_sat(int64_t a, int64_t b) { return (a == DIST_INF || b == DIST_INF) ? DIST_INF : a + b; }

int32_t or_cch_customize(or_cch *c, const int32_t *q) {
  for (int64_t e = 0; e < c->E; e++) c->fw[e] = c->bw[e] = DIST_INF;
  for (int32_t a = 0; a < c->L; a++) {
    int32_t x = c->tail[a], y = c->head[a];
    if (x == y) continue;
    if (q[a] < 1) return OR_EINVAL;
    if (c->rank[x] < c->rank[y]) {
      int64_t e = cch_edge(c, x, y);
      if (q[a] < c->fw[e]) c->fw[e] = q[a];
    } else {
      int64_t e = cch_edge(c, y, x);
      if (q[a] < c->bw[e]) c->bw[e] = q[a];
    }
  }
  /* lower triangles, bottom up: v lowest, then u below w */
  int32_t *by_rank = (int32_t *)malloc((size_t)c->V * 4 + 4);
  if (!by_rank) return OR_ENOMEM;
  for (int32_t v = 0; v < c->V; v++) by_rank[c->rank[v]] = v;
  for (int32_t r = 0; r < c->V; r++) {
    const int32_t v = by_rank[r];
    for (int64_t i = c->up_off[v]; i < c->up_off[v + 1]; i++) {
      for (int64_t j = i + 1; j < c->up_off[v + 1]; j++) {
        const int32_t u = c->up_node[i], w = c->up_node[j];  /* rank u < rank w */
        const int64_t e3 = cch_edge(c, u, w);
        if (e3 < 0) { free(by_rank); return OR_EINVAL; }  /* not chordal: cannot happen */
        int64_t t = add_sat(c->bw[i], c->fw[j]);           /* u -> v -> w */
        if (t < c->fw[e3]) c->fw[e3] = t;
        t = add_sat(c->bw[j], c->fw[i]);                   /* w -> v -> u */
        if (t < c->bw[e3]) c->bw[e3] = t;
      }
    }
  }
  free(by_rank);
  return OR_OK;
}

/* Dijkstra over upward edges from s: dist [V] (DIST_INF where not reached);
 * weights fw (use_bw = 0) or bw (use_bw = 1) */
static int cch_upward(const or_cch *c, int32_t s, int use_bw, int64_t *dist, heap *h) {
  for (int32_t v = 0; v < c->V; v++) dist[v] = DIST_INF;
  h->n = 0;
  dist[s] = 0;
  if (heap_push(h, 0, s)) return 1;
  while (h->n) {
    hitem it = heap_pop(h);
    if (it.d != dist[it.v]) continue;
    for (int64_t e = c->up_off[it.v]; e < c->up_off[it.v + 1]; e++) {
      const int64_t nd = add_sat(it.d, use_bw ? c->bw[e] : c->fw[e]);
      const int32_t u = c->up_node[e];
      if (nd < dist[u]) {
        dist[u] = nd;
        if (heap_push(h, nd, u)) return 1;
      }
    }
  }
  return 0;
}

/* dist [n] receives the shortest time s[k] -> t[k] (DIST_INF if none) */
int32_t or_cch_distance(const or_cch *c, int32_t n, const int32_t *s, const int32_t *t, int64_t *dist) {
  int64_t *df = (int64_t *)malloc((size_t)c->V * 8 + 8), *db = (int64_t *)malloc((size_t)c->V * 8 + 8);
  heap h = {0};
  int rc = OR_OK;
  if (!df || !db) { rc = OR_ENOMEM; goto done; }
  for (int32_t k = 0; k < n; k++) {
    if (cch_upward(c, s[k], 0, df, &h) || cch_upward(c, t[k], 1, db, &h)) { rc = OR_ENOMEM; break; }
    int64_t best = DIST_INF;
    for (int32_t v = 0; v < c->V; v++) {
      const int64_t x = add_sat(df[v], db[v]);
      if (x < best) best = x;
    }
    dist[k] = best;
  }
done:
  free(df); free(db); free(h.a);
  return rc;
}

/* dist [V]: the shortest time v -> z for every node v (DIST_INF if none) */
int32_t or_cch_to_root(const or_cch *c, int32_t z, int64_t *dist) {
  int32_t *by_rank = (int32_t *)malloc((size_t)c->V * 4 + 4);
  heap h = {0};
  int rc = OR_OK;
  if (!by_rank) return OR_ENOMEM;
  if (cch_upward(c, z, 1, dist, &h)) { rc = OR_ENOMEM; goto done; }  /* down-paths m -> z */
  for (int32_t v = 0; v < c->V; v++) by_rank[c->rank[v]] = v;
  for (int32_t r = c->V - 1; r >= 0; r--) {
    const int32_t v = by_rank[r];
    for (int64_t e = c->up_off[v]; e < c->up_off[v + 1]; e++) {
      const int64_t x = add_sat(c->fw[e], dist[c->up_node[e]]);
      if (x < dist[v]) dist[v] = x;
    }
  }
done:
  free(by_rank); free(h.a);
  return rc;
}

/*
 * Readings of the paper taken here (each also listed in the design notes):
 *  R1 Eq. 2's argmin is garbled; the stop node is the first node on the path
 *     whose elapsed time is >= dt (elapsed == dt counts as reached); a link is
 *     loaded iff the elapsed time at its tail is < dt.  The worked example
 *     (Section 6: l23 straddles the boundary, the residual waits at node 3)
 *     agrees.
 *  R2 BPR flows are trips in the interval divided by its length in hours.
 *  R3 Alg. 8 starts from 2/(2+j) with j the completed FW steps (1 at first);
 *     its slope test reads |C'| < T1 |C| (relative), L = 20 loop bound; a
 *     non-positive FD curvature steps to the end point the slope points to.
 *  R4 Alg. 2/6 return the iterate before the step that met the objective test.
 *  R5 Alg. 4 re-truncates the full (untruncated) path of every AON with the
 *     final costs, weighted by the step weights of the convex combination.
 *  R6 sums over links are exact sums of terms rounded to 2^-32.
 *  R14 The system optimum (Section 3 names it beside the user equilibrium the
 *     paper solves; Sections 1 and 8 ask for other objectives) minimises the
 *     total cost sum t c(t): routing uses the quantised marginal cost
 *     m = c + t c', the line search the total cost and its slope, the stop
 *     rules the total cost and the gap in marginal costs, while loading and
 *     truncation keep the travel times c (a trip still ends its interval
 *     after dt of travel).
 *  R16 The relative-gap stop takes -1e-12 <= gap <= tol: under truncation a
 *     negative gap certifies nothing (the truncated AON loading need not
 *     minimise sum c g); -1e-12 absorbs rounding at an exact equilibrium.
 *  R17 Carried truncation (Section 3.4 proposes tracking the distance the
 *     flow got along a link and adding it up across intervals while it
 *     cannot be propagated to the next link): a trip whose next link would
 *     end after dt stays on that link, carrying the fraction of the link it
 *     covered (2^-32 units); in the next interval it first finishes that
 *     link at that interval's link time (reaching the head after the
 *     uncovered rest, or staying on it with the fraction grown by dt / q),
 *     then follows the tree from the head (rerouted there, as every
 *     interval reroutes).  A link longer than dt is thus crossed over
 *     several intervals.  A trip loads a link in the interval it enters it,
 *     as under R1, so every trip loads each link of its route once.
 *     Residual demand keeps the paper's d_{s,q} form: trips at a node merge
 *     per (root, node); trips on a link per (root, link) with the
 *     amount-weighted mean fraction (exact merging would grow the items
 *     about fourfold per interval on short intervals).
 */
