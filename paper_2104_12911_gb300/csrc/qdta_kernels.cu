// qdta_kernels.cu -- sm_103a kernels of the QDTA hot path.
//
//   pack_adj / sssp       batched shortest paths (Alg. 3 / Alg. 7 routing)
//   pack_head_q / load    truncated all-or-nothing loading (Alg. 3, Eq. 2, Eq. 5)
//   residual              re-truncation of every FW path with final costs (Alg. 4)
//   bpr                   link costs (Eq. 1)
//   sweep / objective     fixed-point link sums for the line search (Alg. 9, Eq. 6-9)
//   ctl_*                 single-thread FW / line-search controller (Alg. 2, 6, 8)
//   update / tape         convex flow update f + alpha (g - f)
//   scatter / compact     residual-demand merge d(i+1) = d_o(i+1) + d_r(i+1) (Alg. 1)
//   adj_* / gather        adjoint of the unrolled FW map
#include <algorithm>
#include <atomic>
#include <climits>
#include <string>
#include <type_traits>
#include <vector>
#include <cstdlib>
#include <cstdio>

#include "qdta.h"
#include "qdta_internal.cuh"

namespace qdta {

// Round limit of the Bellman-Ford loops (a watchdog: link times >= 1 bound
// the rounds by V + 1, so hitting it means an error).  QDTA_MAX_ROUNDS lowers
// it so that tests can exercise the timeout path without faulting anything.
static int round_limit(int V) {
  static long long env = [] { const char *e = getenv("QDTA_MAX_ROUNDS"); return e ? atoll(e) : 0ll; }();
  return (env > 0 && env < (long long)V + 1) ? (int)env : V + 1;
}

// kernels launched (or captured) by the launchers below, host-side count
static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
#define COUNT_LAUNCH() g_launches.fetch_add(1)

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ============================================================================
// shortest paths
// ============================================================================

// Adjacency of node w for the relaxation direction:
//   TO_ROOT   -> links entering w, neighbour = their tail (the node that can
//                reach the root through w);
//   FROM_ROOT -> links leaving w, neighbour = their head.
// Each entry is one 16-byte vector: (link id, neighbour, link time, 0).
__global__ void pack_adj_kernel(int L, const int *__restrict__ link_list,
                                const int *__restrict__ nb_of_link, const int *__restrict__ q,
                                int4 *__restrict__ adj, const int *skip_dev) {
  if (skip_dev && *skip_dev) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
    int e = link_list[k];
    adj[k] = make_int4(e, nb_of_link[e], q[e], 0);
  }
}

__global__ void pack_perm_adj_kernel(int L, const int *__restrict__ perm_link, const int *__restrict__ perm_nb,
                                     const int *__restrict__ q, int4 *__restrict__ adj, const int *skip_dev) {
  if (skip_dev && *skip_dev) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
    const int e = perm_link[k];
    adj[k] = make_int4(e, perm_nb[k], q[e], 0);
  }
}

// four fixed slots per node (graphs whose maximum degree is <= 4): slot k of
// node u holds its k-th link, (-1, 0, 0, 0) when absent
__global__ void pack_ell_kernel(int V, const int *__restrict__ perm_off, const int *__restrict__ perm_link,
                                const int *__restrict__ perm_nb, const int *__restrict__ q, int4 *__restrict__ ell,
                                const int *skip_dev) {
  if (skip_dev && *skip_dev) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 4 * V; t += gridDim.x * blockDim.x) {
    const int u = t >> 2, k = t & 3;
    const int a = perm_off[u] + k;
    if (a < perm_off[u + 1]) {
      const int e = perm_link[a];
      ell[t] = make_int4(e, perm_nb[a], q[e], 0);
    } else {
      ell[t] = make_int4(-1, 0, 0, 0);
    }
  }
}

void launch_pack_ell(const GraphDev &g, int direction, const int *q, int4 *ell, cudaStream_t s,
                     const int *skip_dev) {
  COUNT_LAUNCH();
  pack_ell_kernel<<<cdiv(4ll * g.V, 256), 256, 0, s>>>(g.V, g.perm_off[direction], g.perm_link[direction],
                                                       g.perm_nb[direction], q, ell, skip_dev);
}

// eight-byte four-slot entries: ((neighbour << 3) | rank, link time), with
// (-1, 0) for an absent slot
__global__ void pack_ell8_kernel(int V, const int *__restrict__ perm_off, const int *__restrict__ perm_link,
                                 const int *__restrict__ perm_nb, const int *__restrict__ rank_tgt,
                                 const int *__restrict__ q, int2 *__restrict__ ell, const int *skip_dev) {
  if (skip_dev && *skip_dev) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 4 * V; t += gridDim.x * blockDim.x) {
    const int u = t >> 2, k = t & 3;
    const int a = perm_off[u] + k;
    if (a < perm_off[u + 1]) {
      const int e = perm_link[a];
      ell[t] = make_int2((perm_nb[a] << 3) | rank_tgt[e], q[e]);
    } else {
      ell[t] = make_int2(-1, 0);
    }
  }
}

void launch_pack_ell8(const GraphDev &g, int direction, const int *q, int2 *ell, cudaStream_t s,
                      const int *skip_dev) {
  COUNT_LAUNCH();
  pack_ell8_kernel<<<cdiv(4ll * g.V, 256), 256, 0, s>>>(g.V, g.perm_off[direction], g.perm_link[direction],
                                                        g.perm_nb[direction], g.rank_tgt[direction], q, ell,
                                                        skip_dev);
}

void launch_pack_perm_adj(const GraphDev &g, int direction, const int *q, int4 *adj, cudaStream_t s,
                          const int *skip_dev) {
  if (g.L == 0) return;
  COUNT_LAUNCH();
  pack_perm_adj_kernel<<<cdiv(g.L, 256), 256, 0, s>>>(g.L, g.perm_link[direction], g.perm_nb[direction], q, adj,
                                                      skip_dev);
}

void launch_pack_adj(const GraphDev &g, int direction, const int *q, int4 *adj, cudaStream_t s,
                     const int *skip_dev) {
  if (g.L == 0) return;
  const int *list = direction == 0 ? g.in_link : g.out_link;
  const int *nb = direction == 0 ? g.tail : g.head;
  COUNT_LAUNCH();
  pack_adj_kernel<<<cdiv(g.L, 256), 256, 0, s>>>(g.L, list, nb, q, adj, skip_dev);
}

// One CTA per root (persistent over roots).  Queue-based Bellman-Ford:
// every round relaxes the adjacency of the nodes whose distance improved in
// the previous round.  Node state is one 64-bit key (dist << LB) | link, so
// a single atomicMin keeps the smallest distance and, among links giving
// that distance, the smallest link id -- exactly the parent rule, and
// independent of the order in which relaxations arrive.  A per-node round
// stamp keeps each node at most once per round in the next queue.
template <bool SMEM>
__global__ void __launch_bounds__(SSSP_THREADS)
sssp_kernel(int V, int LB, const int *__restrict__ off, const int4 *__restrict__ adj,
            const int *__restrict__ roots, int R_host, const int *R_dev,
            unsigned long long *g_state, int *g_stamp, int *g_queue, int *parent,
            const int *parent_slot_dev, long long slot_stride, long long *dist, unsigned *status,
            const int *skip_dev, unsigned long long *roots_counter, int max_rounds) {
  extern __shared__ unsigned long long smem_u64[];
  __shared__ int s_cnt[3];
  if (skip_dev && *skip_dev) return;
  const int R = R_dev ? *R_dev : R_host;
  if (roots_counter && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(roots_counter, (unsigned long long)R);
  unsigned long long *state;
  int *stamp, *qa, *qb;
  if (SMEM) {
    state = smem_u64;
    stamp = reinterpret_cast<int *>(smem_u64 + V);
    qa = stamp + V;
    qb = qa + V;
  } else {
    size_t b = blockIdx.x;
    state = g_state + b * (size_t)V;
    stamp = g_stamp + b * (size_t)V;
    qa = g_queue + b * 2 * (size_t)V;
    qb = qa + V;
  }
  if (parent_slot_dev) parent += (long long)(*parent_slot_dev) * slot_stride;
  const unsigned long long NOLINK = (1ull << LB) - 1ull;
  const unsigned long long DMAX = (~0ull) >> LB;
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    state[v] = ~0ull;
    stamp[v] = -1;
  }
  int rid = 0;
  __syncthreads();
  for (int r = blockIdx.x; r < R; r += gridDim.x) {
    const int z = roots[r];
    if (threadIdx.x == 0) {
      state[z] = NOLINK;  // distance 0, no parent link
      qa[0] = z;
      s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    }
    __syncthreads();
    int ncur = 1, round = 0;
    int *cur = qa, *nxt = qb;
    unsigned long long my_relax = 0;
    while (ncur > 0) {
      const int c = round % 3;
      if (threadIdx.x == 0) s_cnt[(round + 1) % 3] = 0;
      const int my_rid = rid + round;
      for (int i = threadIdx.x; i < ncur; i += blockDim.x) {
        const int w = cur[i];
        unsigned long long kw;
        if (SMEM) kw = *(volatile unsigned long long *)&state[w];
        else kw = __ldcg(&state[w]);
        const unsigned long long dw = kw >> LB;
        const int kb = off[w], ke = off[w + 1];
        my_relax += (unsigned long long)(ke - kb);
        for (int k = kb; k < ke; ++k) {
          const int4 ent = __ldg(&adj[k]);
          const unsigned long long cand = dw + (unsigned long long)(unsigned)ent.z;
          if (cand >= DMAX) { atomicOr(status, ST_OVERFLOW); continue; }
          const unsigned long long key = (cand << LB) | (unsigned long long)(unsigned)ent.x;
          const unsigned long long old = atomicMin(&state[ent.y], key);
          if ((old >> LB) > cand) {
            if (atomicExch(&stamp[ent.y], my_rid) != my_rid) {
              const int pos = atomicAdd(&s_cnt[c], 1);
              nxt[pos] = ent.y;
            }
          }
        }
      }
      __syncthreads();
      ncur = s_cnt[c];
      int *t = cur; cur = nxt; nxt = t;
      ++round;
      if (round > max_rounds) {  // cannot happen with link times >= 1 unless lowered
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        break;
      }
    }
    rid += round + 1;
    if (roots_counter) {  // work counters: [1] rounds, [2] relaxations
      if (threadIdx.x == 0) atomicAdd(roots_counter + 1, (unsigned long long)round);
      atomicAdd(roots_counter + 2, my_relax);
    }
    __syncthreads();
    int *prow = parent + (long long)r * V;
    long long *drow = dist ? dist + (long long)r * V : nullptr;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      const unsigned long long key = state[v];
      const unsigned long long lk = key & NOLINK;
      prow[v] = lk == NOLINK ? -1 : (int)lk;
      if (drow) drow[v] = key == ~0ull ? LLONG_MAX : (long long)(key >> LB);
      state[v] = ~0ull;
    }
    __syncthreads();
  }
}

// Global-memory variant for graphs whose per-root state does not fit in
// shared memory.  Same queue Bellman-Ford and packed keys as above, laid out
// for memory-level parallelism: four lanes per frontier node (one in-link
// each), NPT frontier nodes per lane group in flight, and an L2 read of the
// target's key before the atomic, so relaxations that cannot improve (most
// of them) cost a load instead of an atomic.
constexpr int SSSP2_NPT = 4;

template <int SSSP2_THREADS>
__global__ void __launch_bounds__(SSSP2_THREADS)
sssp_ilp_kernel(int V, int LB, const int *__restrict__ off, const int4 *__restrict__ adj,
                const int *__restrict__ roots, int R_host, const int *R_dev,
                unsigned long long *g_state, int *g_stamp, int *g_queue, int *parent,
                const int *parent_slot_dev, long long slot_stride, long long *dist, unsigned *status,
                const int *skip_dev, unsigned long long *roots_counter, int max_rounds) {
  __shared__ int s_cnt[3];
  if (skip_dev && *skip_dev) return;
  const int R = R_dev ? *R_dev : R_host;
  if (roots_counter && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(roots_counter, (unsigned long long)R);
  const size_t b = blockIdx.x;
  unsigned long long *state = g_state + b * (size_t)V;
  int *stamp = g_stamp + b * (size_t)V;
  int *qa = g_queue + b * 2 * (size_t)V;
  int *qb = qa + V;
  if (parent_slot_dev) parent += (long long)(*parent_slot_dev) * slot_stride;
  const unsigned long long NOLINK = (1ull << LB) - 1ull;
  const unsigned long long DMAX = (~0ull) >> LB;
  constexpr int NQ = SSSP2_THREADS / 4;
  const int quad = threadIdx.x >> 2, lane4 = threadIdx.x & 3;
  for (int v = threadIdx.x; v < V; v += blockDim.x) {
    state[v] = ~0ull;
    stamp[v] = -1;
  }
  int rid = 0;
  __syncthreads();
  for (int r = blockIdx.x; r < R; r += gridDim.x) {
    const int z = roots[r];
    if (threadIdx.x == 0) {
      state[z] = NOLINK;
      qa[0] = z;
      s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    }
    __syncthreads();
    int ncur = 1, round = 0;
    int *cur = qa, *nxt = qb;
    unsigned long long my_relax = 0;
    while (ncur > 0) {
      const int c = round % 3;
      if (threadIdx.x == 0) s_cnt[(round + 1) % 3] = 0;
      const int my_rid = rid + round;
      for (int base = 0; base < ncur; base += NQ * SSSP2_NPT) {
        int w[SSSP2_NPT], kb[SSSP2_NPT], ke[SSSP2_NPT];
        unsigned long long dw[SSSP2_NPT];
#pragma unroll
        for (int j = 0; j < SSSP2_NPT; ++j) {
          const int i = base + j * NQ + quad;
          w[j] = i < ncur ? __ldcg(&cur[i]) : -1;
        }
#pragma unroll
        for (int j = 0; j < SSSP2_NPT; ++j) {
          kb[j] = 0; ke[j] = 0; dw[j] = 0;
          if (w[j] >= 0) {
            kb[j] = __ldg(&off[w[j]]) + lane4;
            ke[j] = __ldg(&off[w[j] + 1]);
            dw[j] = __ldcg(&state[w[j]]) >> LB;
          }
        }
        bool more = true;
        while (more) {
          int4 ent[SSSP2_NPT];
          unsigned long long tk[SSSP2_NPT];
#pragma unroll
          for (int j = 0; j < SSSP2_NPT; ++j)
            if (kb[j] < ke[j]) ent[j] = __ldg(&adj[kb[j]]);
#pragma unroll
          for (int j = 0; j < SSSP2_NPT; ++j)
            if (kb[j] < ke[j]) tk[j] = __ldcg(&state[ent[j].y]);
#pragma unroll
          for (int j = 0; j < SSSP2_NPT; ++j) {
            if (kb[j] < ke[j]) {
              ++my_relax;
              const unsigned long long cand = dw[j] + (unsigned long long)(unsigned)ent[j].z;
              if (cand >= DMAX) {
                atomicOr(status, ST_OVERFLOW);
              } else {
                const unsigned long long key = (cand << LB) | (unsigned long long)(unsigned)ent[j].x;
                if (key < tk[j]) {
                  const unsigned long long old = atomicMin(&state[ent[j].y], key);
                  if ((old >> LB) > cand && atomicExch(&stamp[ent[j].y], my_rid) != my_rid) {
                    const int pos = atomicAdd(&s_cnt[c], 1);
                    nxt[pos] = ent[j].y;
                  }
                }
              }
            }
          }
          more = false;
#pragma unroll
          for (int j = 0; j < SSSP2_NPT; ++j) {
            kb[j] += 4;
            more |= kb[j] < ke[j];
          }
        }
      }
      __syncthreads();
      ncur = s_cnt[c];
      int *t = cur; cur = nxt; nxt = t;
      ++round;
      if (round > max_rounds) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        break;
      }
    }
    rid += round + 1;
    if (roots_counter) {
      if (threadIdx.x == 0) atomicAdd(roots_counter + 1, (unsigned long long)round);
      atomicAdd(roots_counter + 2, my_relax);
    }
    __syncthreads();
    int *prow = parent + (long long)r * V;
    long long *drow = dist ? dist + (long long)r * V : nullptr;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      const unsigned long long key = __ldcg(&state[v]);
      const unsigned long long lk = key & NOLINK;
      prow[v] = lk == NOLINK ? -1 : (int)lk;
      if (drow) drow[v] = key == ~0ull ? LLONG_MAX : (long long)(key >> LB);
      state[v] = ~0ull;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// cell-partitioned SSSP: state of the active cell in shared memory
// ---------------------------------------------------------------------------
__global__ void pack_cell_adj_kernel(int L, const int *__restrict__ ent_link,
                                     const int *__restrict__ ent_code, const int *__restrict__ q,
                                     int4 *__restrict__ adj, long long n_lrev, const int *__restrict__ lrev_link,
                                     const int *__restrict__ lrev_src, uint2 *__restrict__ lrev_adj,
                                     long long n_xrev, const int *__restrict__ xrev_link,
                                     const int *__restrict__ xrev_node, int4 *__restrict__ xrev_adj,
                                     const int *skip_dev) {
  if (skip_dev && *skip_dev) return;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_xrev;
       k += (long long)gridDim.x * blockDim.x) {
    const int e = xrev_link[k];
    xrev_adj[k] = make_int4(e, xrev_node[k], q[e], 0);
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
    const int e = ent_link[k];
    adj[k] = make_int4(e, ent_code[k], q[e], 0);
  }
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_lrev;
       k += (long long)gridDim.x * blockDim.x) {
    const int e = lrev_link[k];
    lrev_adj[k] = make_uint2(((unsigned)lrev_src[k] << 24) | (unsigned)e, (unsigned)q[e]);
  }
}

void launch_pack_cell_adj(const GraphDev &g, const CellDev &c, int direction, const int *q, int4 *adj,
                          uint2 *lrev_adj, long long n_lrev, int4 *xrev_adj, long long n_xrev, cudaStream_t s,
                          const int *skip_dev) {
  if (g.L == 0) return;
  COUNT_LAUNCH();
  pack_cell_adj_kernel<<<cdiv(g.L, 256), 256, 0, s>>>(g.L, c.ent_link[direction], c.ent_code[direction], q,
                                                      adj, n_lrev, c.lrev_link[direction],
                                                      c.lrev_src[direction], lrev_adj, n_xrev,
                                                      c.xrev_link[direction], c.xrev_node[direction], xrev_adj,
                                                      skip_dev);
}

// per-warp shared-memory layout of the cell kernel
struct CellWarpSmem {
  unsigned long long key[CELL_MAX_NODES];
  unsigned long long ext[CELL_MAX_EXT];
  uint2 lrev[CELL_MAX_LREV];
  unsigned short lroff[CELL_MAX_NODES + 1];  // node -> range in lrev (cell-relative)
  unsigned char nf[CELL_MAX_NODES];          // node flags
  short fq[2][CELL_MAX_NODES];
  unsigned inq[2][CELL_MAX_NODES / 32];
  unsigned chg[CELL_MAX_NODES / 32];
  int fn[2];
};

// One CTA per root (persistent over roots); each warp processes one cell at
// a time.  Cells woken by a neighbour wait in a pending list with the
// smallest distance that woke them; each round processes the pending cells
// within `delta` of the smallest such distance (near/far ordering at cell
// level, so most cells fire once their inputs are nearly final) and defers
// the rest.  Between activations a cell is locally converged, so only nodes
// with links to other cells can have pending improvements: an activation
// loads the cell's keys, its external neighbours' keys and its internal
// reversed links into shared memory, pulls the boundary nodes over all their
// links, then runs a shared-memory push Bellman-Ford (64-bit shared
// atomicMin on the packed key) from every node whose distance improved.
// The minimum over every link with the neighbours' current keys makes the
// fixed point the shortest distance with the smallest tight link id,
// whatever the processing order.
__global__ void __launch_bounds__(CELL_WARPS * 32)
sssp_cell_kernel(int V, int LB, CellDev C, int dir, const int4 *__restrict__ adj,
                 const uint2 *__restrict__ lrev_adj, const int4 *__restrict__ xrev_adj, long long delta, const int *__restrict__ roots,
                 int R_host, const int *R_dev, unsigned long long *g_state, int *g_flag, int *g_queue,
                 unsigned long long *g_prio, int *parent, const int *parent_slot_dev, long long slot_stride,
                 long long *dist, unsigned *status, const int *skip_dev, unsigned long long *roots_counter) {
  extern __shared__ __align__(16) unsigned char cell_smem[];
  __shared__ int s_np, s_ns, s_nn;
  __shared__ unsigned long long s_min;
  if (skip_dev && *skip_dev) return;
  const int R = R_dev ? *R_dev : R_host;
  if (roots_counter && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(roots_counter, (unsigned long long)R);
  const int nc = C.n_cells;
  const size_t b = blockIdx.x;
  unsigned long long *state = g_state + b * (size_t)V;
  int *inpend = g_flag + b * (size_t)nc;
  int *listA = g_queue + b * 3 * (size_t)nc;  // pending
  int *listS = listA + nc;                    // selected this round
  int *listN = listS + nc;                    // pending next round
  unsigned long long *prio = g_prio + b * (size_t)nc;
  if (parent_slot_dev) parent += (long long)(*parent_slot_dev) * slot_stride;
  const unsigned long long NOLINK = (1ull << LB) - 1ull;
  const unsigned long long DMAX = (~0ull) >> LB;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  CellWarpSmem &W = reinterpret_cast<CellWarpSmem *>(cell_smem)[wid];
  const int *__restrict__ cell_off = C.cell_off;
  const int *__restrict__ ent_off = C.ent_off[dir];
  const int *__restrict__ ext_off = C.ext_off[dir];
  const int *__restrict__ ext_node = C.ext_node[dir];
  const int *__restrict__ lrev_off = C.lrev_off[dir];
  const unsigned char *__restrict__ nflag = C.node_flags[dir];
  const int *__restrict__ xrev_off = C.xrev_off[dir];
  const int *__restrict__ node_cell = C.node_cell;
  for (int v = threadIdx.x; v < V; v += blockDim.x) state[v] = ~0ull;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) { inpend[c] = 0; prio[c] = ~0ull; }
  __syncthreads();
  unsigned long long my_relax = 0, my_act = 0;
  for (int r = blockIdx.x; r < R; r += gridDim.x) {
    const int z = C.node_int[roots[r]];
    if (threadIdx.x == 0) {
      state[z] = NOLINK;
      const int cz = C.node_cell[z];
      listA[0] = cz;
      inpend[cz] = 1;
      prio[cz] = 0;
      s_np = 1;
    }
    __syncthreads();
    int round = 0;
    while (s_np > 0) {
      const int np = s_np;
      // selection: threshold = smallest pending priority + delta
      if (threadIdx.x == 0) { s_min = ~0ull; s_ns = 0; s_nn = 0; }
      __syncthreads();
      unsigned long long m = ~0ull;
      for (int i = threadIdx.x; i < np; i += blockDim.x) m = min(m, __ldcg(&prio[__ldcg(&listA[i])]));
      for (int d = 16; d > 0; d >>= 1) m = min(m, __shfl_down_sync(0xffffffffu, m, d));
      if (lane == 0) atomicMin(&s_min, m);
      __syncthreads();
      const unsigned long long thr = s_min > ~0ull - (unsigned long long)delta ? ~0ull : s_min + (unsigned long long)delta;
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int c = __ldcg(&listA[i]);
        if (__ldcg(&prio[c]) <= thr) {
          listS[atomicAdd(&s_ns, 1)] = c;
          inpend[c] = 0;
          prio[c] = ~0ull;
        } else {
          listN[atomicAdd(&s_nn, 1)] = c;
        }
      }
      __syncthreads();
      const int ns = s_ns;
      for (int ci = wid; ci < ns; ci += CELL_WARPS) {
        const int c = __ldcg(&listS[ci]);
        const int lo = cell_off[c], n = cell_off[c + 1] - lo;
        if (lane == 0) ++my_act;
        for (int i = lane; i < n; i += 32) W.key[i] = __ldcg(&state[lo + i]);
        const int eo = ext_off[c], en = ext_off[c + 1] - eo;
        for (int i = lane; i < en; i += 32) W.ext[i] = __ldcg(&state[ext_node[eo + i]]);
        const int r0 = lrev_off[lo], rn = lrev_off[lo + n] - r0;
        for (int i = lane; i < rn; i += 32) W.lrev[i] = __ldg(&lrev_adj[r0 + i]);
        for (int i = lane; i <= n; i += 32) W.lroff[i] = (unsigned short)(lrev_off[lo + i] - r0);
        for (int i = lane; i < n; i += 32) W.nf[i] = nflag[lo + i];
        if (lane < CELL_MAX_NODES / 32) { W.chg[lane] = 0u; W.inq[0][lane] = 0u; }
        if (lane == 0) W.fn[0] = 0;
        __syncwarp();
        // seed: boundary nodes pulled over all their links (+ the root at the start)
        for (int i = lane; i < n; i += 32) {
          const int u = lo + i;
          bool push = round == 0 && u == z;
          if (W.nf[i] & 1) {
            unsigned long long best = W.key[i];
            const int t0 = ent_off[u], t1 = ent_off[u + 1];
            my_relax += (unsigned long long)(t1 - t0);
            for (int t = t0; t < t1; ++t) {
              const int4 ent = __ldg(&adj[t]);
              const unsigned long long wk = ent.y >= 0 ? W.key[ent.y] : W.ext[-ent.y - 1];
              if (wk == ~0ull) continue;
              const unsigned long long cand = (wk >> LB) + (unsigned long long)(unsigned)ent.z;
              if (cand >= DMAX) { atomicOr(status, ST_OVERFLOW); continue; }
              const unsigned long long key = (cand << LB) | (unsigned long long)(unsigned)ent.x;
              if (key < best) best = key;
            }
            const unsigned long long old = atomicMin(&W.key[i], best);
            if (best < old) {
              atomicOr(&W.chg[i >> 5], 1u << (i & 31));
              if ((old >> LB) > (best >> LB)) push = true;
            }
          }
          if (push && !((atomicOr(&W.inq[0][i >> 5], 1u << (i & 31)) >> (i & 31)) & 1u))
            W.fq[0][atomicAdd(&W.fn[0], 1)] = (short)i;
        }
        __syncwarp();
        // local push rounds over the cell's internal reversed links (shared memory)
        int fn = W.fn[0], side = 0, guard = 0;
        while (fn > 0) {
          const int nx = side ^ 1;
          if (lane == 0) W.fn[nx] = 0;
          if (lane < CELL_MAX_NODES / 32) W.inq[nx][lane] = 0u;
          __syncwarp();
          for (int x = lane; x < fn; x += 32) {
            const int wl = W.fq[side][x];
            const unsigned long long dw = W.key[wl] >> LB;
            const int k0 = W.lroff[wl], k1 = W.lroff[wl + 1];
            my_relax += (unsigned long long)(k1 - k0);
            for (int k = k0; k < k1; ++k) {
              const uint2 ent = W.lrev[k];
              const int ul = (int)(ent.x >> 24);
              const unsigned long long cand = dw + (unsigned long long)ent.y;
              if (cand >= DMAX) { atomicOr(status, ST_OVERFLOW); continue; }
              const unsigned long long key = (cand << LB) | (unsigned long long)(ent.x & 0xFFFFFFu);
              const unsigned long long old = atomicMin(&W.key[ul], key);
              if (key < old) {
                atomicOr(&W.chg[ul >> 5], 1u << (ul & 31));
                if ((old >> LB) > cand && !((atomicOr(&W.inq[nx][ul >> 5], 1u << (ul & 31)) >> (ul & 31)) & 1u))
                  W.fq[nx][atomicAdd(&W.fn[nx], 1)] = (short)ul;
              }
            }
          }
          __syncwarp();
          fn = W.fn[nx];
          side = nx;
          if (++guard > CELL_MAX_NODES + 2) {  // a cell converges within n local rounds
            if (lane == 0) atomicOr(status, ST_TIMEOUT);
            break;
          }
        }
        // write back changed keys
        for (int i = lane; i < n; i += 32)
          if ((W.chg[i >> 5] >> (i & 31)) & 1u) state[lo + i] = W.key[i];
        __syncwarp();
        // wake exactly the cells with a node this change improves: reader u of
        // changed node w through link e is woken iff ((d_w + q_e) << LB | e) is
        // below u's current key (keys only decrease, so a skipped wake is never
        // needed later)
        for (int i = lane; i < n; i += 32) {
          if (!((W.chg[i >> 5] >> (i & 31)) & 1u) || !(W.nf[i] & 2)) continue;
          const unsigned long long dw = W.key[i] >> LB;
          const int x0 = xrev_off[lo + i], x1 = xrev_off[lo + i + 1];
          for (int x = x0; x < x1; ++x) {
            const int4 ent = __ldg(&xrev_adj[x]);
            const unsigned long long cand = dw + (unsigned long long)(unsigned)ent.z;
            if (cand >= DMAX) continue;
            const unsigned long long key = (cand << LB) | (unsigned long long)(unsigned)ent.x;
            if (key < __ldcg(&state[ent.y])) {
              const int d = node_cell[ent.y];
              atomicMin(&prio[d], cand);
              if (atomicExch(&inpend[d], 1) == 0) listN[atomicAdd(&s_nn, 1)] = d;
            }
          }
        }
        __syncwarp();
      }
      __syncthreads();
      // next pending list
      const int nn = s_nn;
      for (int i = threadIdx.x; i < nn; i += blockDim.x) listA[i] = __ldcg(&listN[i]);
      if (threadIdx.x == 0) s_np = nn;
      __syncthreads();
      ++round;
      if (round > nc * 64 + 4) {  // a bounded loop: far beyond any observed round count
        if (threadIdx.x == 0) { atomicOr(status, ST_TIMEOUT); s_np = 0; }
        __syncthreads();
        break;
      }
    }
    if (roots_counter) {
      if (threadIdx.x == 0) atomicAdd(roots_counter + 1, (unsigned long long)round);
      atomicAdd(roots_counter + 2, my_relax);
      if (my_act) atomicAdd(roots_counter + 3, my_act);
      my_relax = 0;
      my_act = 0;
    }
    __syncthreads();
    int *prow = parent + (long long)r * V;
    long long *drow = dist ? dist + (long long)r * V : nullptr;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
      const unsigned long long key = __ldcg(&state[C.node_int[v]]);
      const unsigned long long lk = key & NOLINK;
      prow[v] = lk == NOLINK ? -1 : (int)lk;
      if (drow) drow[v] = key == ~0ull ? LLONG_MAX : (long long)(key >> LB);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < V; v += blockDim.x) state[v] = ~0ull;
    __syncthreads();
  }
}

static size_t cell_smem_bytes() { return sizeof(CellWarpSmem) * CELL_WARPS; }

int sssp_cell_blocks_per_sm() {
  int n = 0;
  cudaFuncSetAttribute(sssp_cell_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem_bytes());
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sssp_cell_kernel, CELL_WARPS * 32, cell_smem_bytes());
  return n > 0 ? n : 1;
}

void launch_sssp_cell(const GraphDev &g, const CellDev &c, int direction, const int4 *adj, const uint2 *lrev_adj,
                      const int4 *xrev_adj, long long delta, const int *roots, int R_host, const int *R_dev, int grid,
                      unsigned long long *state, int *flag, int *queue, unsigned long long *prio, int *parent,
                      const int *parent_slot_dev, long long slot_stride, long long *dist,
                      unsigned *status, cudaStream_t s, const int *skip_dev,
                      unsigned long long *roots_counter) {
  if (grid <= 0) return;
  COUNT_LAUNCH();
  cudaFuncSetAttribute(sssp_cell_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem_bytes());
  cudaFuncSetAttribute(sssp_cell_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  sssp_cell_kernel<<<grid, CELL_WARPS * 32, cell_smem_bytes(), s>>>(
      g.V, g.LB, c, direction, adj, lrev_adj, xrev_adj, delta, roots, R_host, R_dev, state, flag, queue, prio, parent,
      parent_slot_dev, slot_stride, dist, status, skip_dev, roots_counter);
}

// Several roots per CTA in lockstep: the frontier holds (root slot, node)
// entries of G roots, so each round's latency (a few dependent L2 trips and
// one barrier) is paid once for G roots.  Per-root state, stamps and keys are
// as in sssp_ilp_kernel; entries carry the slot in their top 4 bits.
template <int THREADS, int G>
__global__ void __launch_bounds__(THREADS)
sssp_group_kernel(int V, int LB, const int *__restrict__ off, const int4 *__restrict__ adj,
                  const int *__restrict__ roots, int R_host, const int *R_dev,
                  unsigned long long *g_state, int *g_stamp, int *g_queue, int *parent,
                  const int *parent_slot_dev, long long slot_stride, long long *dist, unsigned *status,
                  const int *skip_dev, unsigned long long *roots_counter, int max_rounds) {
  __shared__ int s_cnt[3];
  if (skip_dev && *skip_dev) return;
  const int R = R_dev ? *R_dev : R_host;
  if (roots_counter && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(roots_counter, (unsigned long long)R);
  const size_t b = blockIdx.x;
  unsigned long long *state = g_state + b * (size_t)G * V;
  int *stamp = g_stamp + b * (size_t)G * V;
  int *qa = g_queue + b * 2 * (size_t)G * V;
  int *qb = qa + (size_t)G * V;
  if (parent_slot_dev) parent += (long long)(*parent_slot_dev) * slot_stride;
  const unsigned long long NOLINK = (1ull << LB) - 1ull;
  const unsigned long long DMAX = (~0ull) >> LB;
  constexpr int NQ = THREADS / 4;
  const int quad = threadIdx.x >> 2, lane4 = threadIdx.x & 3;
  for (size_t v = threadIdx.x; v < (size_t)G * V; v += blockDim.x) {
    state[v] = ~0ull;
    stamp[v] = -1;
  }
  int rid = 0;
  __syncthreads();
  for (int r0 = blockIdx.x * G; r0 < R; r0 += gridDim.x * G) {
    const int ng = min(G, R - r0);
    if (threadIdx.x < ng) {
      const int z = roots[r0 + threadIdx.x];
      state[(size_t)threadIdx.x * V + z] = NOLINK;
      qa[threadIdx.x] = (threadIdx.x << 28) | z;
    }
    if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    __syncthreads();
    int ncur = ng, round = 0;
    int *cur = qa, *nxt = qb;
    unsigned long long my_relax = 0;
    while (ncur > 0) {
      const int c = round % 3;
      if (threadIdx.x == 0) s_cnt[(round + 1) % 3] = 0;
      const int my_rid = rid + round;
      for (int base = 0; base < ncur; base += NQ * SSSP2_NPT) {
        int w[SSSP2_NPT], kb[SSSP2_NPT], ke[SSSP2_NPT];
        size_t sb[SSSP2_NPT];
        unsigned long long dw[SSSP2_NPT];
#pragma unroll
        for (int j = 0; j < SSSP2_NPT; ++j) {
          const int i = base + j * NQ + quad;
          const int ent = i < ncur ? __ldcg(&cur[i]) : -1;
          w[j] = ent < 0 ? -1 : (ent & 0x0FFFFFFF);
          sb[j] = ent < 0 ? 0 : (size_t)(ent >> 28) * V;
        }
#pragma unroll
        for (int j = 0; j < SSSP2_NPT; ++j) {
          kb[j] = 0; ke[j] = 0; dw[j] = 0;
          if (w[j] >= 0) {
            kb[j] = __ldg(&off[w[j]]) + lane4;
            ke[j] = __ldg(&off[w[j] + 1]);
            dw[j] = __ldcg(&state[sb[j] + w[j]]) >> LB;
          }
        }
        bool more = true;
        while (more) {
          int4 ent[SSSP2_NPT];
          unsigned long long tk[SSSP2_NPT];
#pragma unroll
          for (int j = 0; j < SSSP2_NPT; ++j)
            if (kb[j] < ke[j]) ent[j] = __ldg(&adj[kb[j]]);
#pragma unroll
          for (int j = 0; j < SSSP2_NPT; ++j)
            if (kb[j] < ke[j]) tk[j] = __ldcg(&state[sb[j] + ent[j].y]);
#pragma unroll
          for (int j = 0; j < SSSP2_NPT; ++j) {
            if (kb[j] < ke[j]) {
              ++my_relax;
              const unsigned long long cand = dw[j] + (unsigned long long)(unsigned)ent[j].z;
              if (cand >= DMAX) {
                atomicOr(status, ST_OVERFLOW);
              } else {
                const unsigned long long key = (cand << LB) | (unsigned long long)(unsigned)ent[j].x;
                if (key < tk[j]) {
                  const unsigned long long old = atomicMin(&state[sb[j] + ent[j].y], key);
                  if ((old >> LB) > cand && atomicExch(&stamp[sb[j] + ent[j].y], my_rid) != my_rid) {
                    const int pos = atomicAdd(&s_cnt[c], 1);
                    nxt[pos] = (int)((sb[j] / V) << 28) | ent[j].y;
                  }
                }
              }
            }
          }
          more = false;
#pragma unroll
          for (int j = 0; j < SSSP2_NPT; ++j) {
            kb[j] += 4;
            more |= kb[j] < ke[j];
          }
        }
      }
      __syncthreads();
      ncur = s_cnt[c];
      int *t = cur; cur = nxt; nxt = t;
      ++round;
      if (round > max_rounds) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        break;
      }
    }
    rid += round + 1;
    if (roots_counter) {
      if (threadIdx.x == 0) atomicAdd(roots_counter + 1, (unsigned long long)round * ng);
      atomicAdd(roots_counter + 2, my_relax);
    }
    __syncthreads();
    for (int gi = 0; gi < ng; ++gi) {
      int *prow = parent + (long long)(r0 + gi) * V;
      long long *drow = dist ? dist + (long long)(r0 + gi) * V : nullptr;
      unsigned long long *st = state + (size_t)gi * V;
      for (int v = threadIdx.x; v < V; v += blockDim.x) {
        const unsigned long long key = __ldcg(&st[v]);
        const unsigned long long lk = key & NOLINK;
        prow[v] = lk == NOLINK ? -1 : (int)lk;
        if (drow) drow[v] = key == ~0ull ? LLONG_MAX : (long long)(key >> LB);
        st[v] = ~0ull;
      }
    }
    __syncthreads();
  }
}

int sssp_group_size() {
  static int gsz = [] {
    const char *e = getenv("QDTA_BF_GROUP");
    int g = e ? atoi(e) : 1;
    return (g == 2 || g == 4 || g == 8) ? g : 1;
  }();
  return gsz;
}

// Global-memory keys with the round bookkeeping in shared memory: the
// frontier queues (with a global overflow) and the "already queued" marks.
// This takes the frontier read and the dedupe atomic off the chain of
// dependent L2 trips of every relaxation.  The marks are either
//  - two bitmaps of V bits that alternate with the round parity (the bits of
//    the queue being read are cleared as it is read, so the bitmap is clean
//    again two rounds later), or
//  - ONEBM: one bitmap; a round first clears the marks of the whole queue it
//    is about to read, then passes a barrier, so a mark seen set during the
//    relaxations always means "already in the next queue" (half the shared
//    memory: four 256-thread CTAs per SM, or graphs up to ~580k nodes).
// Launch shapes (threads, bitmaps, queue entries per buffer):
//   0: 512, two, 3072 (two CTAs per SM)   1: 256, one, 2048 (four CTAs per SM)
//   2: 512, one, 3072 (two CTAs per SM, larger graphs)
//   3: 256, one, 768 (five CTAs per SM: at most 51 registers a thread, so
//      only the 32-bit rank-keyed kernel; wider frontiers spill to the
//      global overflow queue)
//   4, 5: as 1, with 5 or 6 frontier nodes per lane group in flight instead
//      of 4 (a pass covers 320 or 384 nodes; 32-bit rank keys only)
//   6, 7: as 1, one lane per frontier node (sssp_lane_kernel below), 1 or 2
//      nodes per lane per pass (32-bit rank keys only; otherwise as 1)
//   8: as 1 with the L2 prefetch of key blocks (32-bit rank keys only)
//   9: 192 threads, one bitmap, 960 entries, five CTAs per SM (32-bit rank
//      keys only: up to 68 registers a thread)
//  10: as 1 with 288 threads (a pass covers 288 frontier nodes; 32-bit rank
//      keys only, 56 registers a thread so that four CTAs fit; other
//      adjacency layouts run shape 1)
struct SmqShape {
  int threads, bitmaps, qcap, ctas, npt;
};
constexpr int kSmqShapes = 11;
static const SmqShape kSmqShape[kSmqShapes] = {{512, 2, 3072, 2, 4}, {256, 1, 2048, 4, 4}, {512, 1, 3072, 2, 4},
                                               {256, 1, 768, 5, 4},  {256, 1, 2048, 4, 5}, {256, 1, 2048, 4, 6},
                                               {256, 1, 2048, 4, 1}, {256, 1, 2048, 4, 2},
                                               {256, 1, 2048, 4, 4}, {192, 1, 960, 5, 4},
                                               {288, 1, 2048, 4, 4}};

// threads of the kernel a shape runs with adjacency layout `adj` (shape 10
// falls back to shape 1 off the 32-bit rank keys)
static int smq_threads(int shape, int adj) {
  return shape == 10 && adj != 3 ? 256 : kSmqShape[shape].threads;
}

// Next destination root position of this CTA: every gridDim-th one, or,
// with a fetch counter, the next one handed out by that counter (dynamic
// balance over the CTAs; the counter is zeroed before each launch and numbers
// the positions after the first wave).  Called by every thread of the CTA.
__device__ __forceinline__ int next_root(int r, int *fetch, int *s_next) {
  if (!fetch) return r + (int)gridDim.x;
  if (threadIdx.x == 0) *s_next = (int)gridDim.x + atomicAdd(fetch, 1);
  __syncthreads();
  const int n = *s_next;
  __syncthreads();  // read by every thread before thread 0 may write the next one
  return n;
}

// RELAX selects how an offer (cand, link) to neighbour y is applied:
//   0  returning atomicMin; y is queued when the returned old distance was larger
//   1  read y's key first, skip when the offer cannot win, else as 0
//   2  read y's key first; when the offer beats it, a non-returning atomicMin
//      and y is queued when the read distance was larger.  The queued set is
//      the same as under 1: whichever offer lowers y's distance in a round read
//      a key at least as large as the value it replaced (keys only decrease),
//      so its thread queues y; later reads see the update because the round
//      ends in a CTA barrier and every state access goes through L2.
//   3  as 2, with warp-aggregated queue appends (one shared-memory atomicAdd
//      per warp and offsets from a ballot instead of one per queued node)
//
// PF (32-bit keys): when an offer first reaches a 1 KB block of a root's keys
// (256 consecutive internal ids, a cell of the locality order), the whole
// block is prefetched into L2, so the rounds that follow find those keys in
// L2 instead of DRAM (a root's 1 MB of keys does not stay in L2 between its
// first touch and its reset).  A small shared bitmap marks the blocks
// prefetched for the current root.
template <int THREADS, int ADJ, int RELAX, bool ONEBM, int MINB = 65536 / (THREADS * 64), int NPT = SSSP2_NPT,
          bool PF = false>
__global__ void __launch_bounds__(THREADS, MINB)
sssp_smq_kernel(int V, int LB_link, const int *__restrict__ off, const int4 *__restrict__ adj,
                const int *__restrict__ roots, int R_host, const int *R_dev,
                unsigned long long *g_state, int *g_queue, int *parent,
                const int *parent_slot_dev, long long slot_stride, long long *dist, unsigned *status,
                const int *skip_dev, unsigned long long *roots_counter, const int *__restrict__ node_int,
                int max_rounds, int qcap, const int *__restrict__ node_ext, int out_mode,
                const int *__restrict__ rank_link, int skip_parent, RootSched sched) {
  extern __shared__ __align__(16) unsigned smq_smem[];
  __shared__ int s_cnt[3];
  __shared__ int s_next;
  if (skip_dev && *skip_dev) return;
  const int R = R_dev ? *R_dev : R_host;
  if (roots_counter && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(roots_counter, (unsigned long long)R);
  const int W = (V + 31) >> 5;
  constexpr int NBM = ONEBM ? 1 : 2;
  constexpr bool AGG = RELAX == 3;
  constexpr int RM = AGG ? 2 : RELAX;
  constexpr bool ELL = ADJ >= 1;
  // ADJ 2, 3: the key's low field is the rank (0..3) of the link among the
  // keyed node's candidate parent links, ordered by link id (so the smallest
  // rank is the smallest link id); rank_link maps it back to the link.
  // ADJ 3 keeps the keys in 32 bits (distances below 2^29): a larger
  // distance sets ST_K32 and the batch is redone with 64-bit keys.
  constexpr bool RANK = ADJ >= 2;
  using Key = typename std::conditional<ADJ == 3, unsigned, unsigned long long>::type;
  // distances and offers in 32 bits with 32-bit keys: distances stay below
  // 2^29 and link times below 2^31, so a distance plus a link time fits
  using Dist = Key;
  constexpr Key KINF = ~Key(0);
  const int LB = RANK ? 3 : LB_link;
  unsigned *bm0 = smq_smem, *bm1 = smq_smem + (NBM - 1) * W;
  int *sq0 = reinterpret_cast<int *>(smq_smem + NBM * W), *sq1 = sq0 + qcap;
  unsigned *pfm = reinterpret_cast<unsigned *>(sq1 + qcap);  // PF: blocks prefetched (V / 8192 + 1 words)
  const int WPF = (V >> 13) + 1;
  const size_t b = blockIdx.x;
  Key *state = reinterpret_cast<Key *>(g_state) + b * (size_t)V;
  int *gq0 = g_queue + b * 2 * (size_t)V, *gq1 = gq0 + V;  // overflow beyond qcap entries
  if (parent_slot_dev) parent += (long long)(*parent_slot_dev) * slot_stride;
  const Key NOLINK = (Key)((1ull << LB) - 1ull);
  const Dist DMAX = (Dist)(KINF >> LB);
  constexpr int NQ = THREADS / 4;
  const int quad = threadIdx.x >> 2, lane4 = threadIdx.x & 3;
  for (int v = threadIdx.x; v < V; v += blockDim.x) state[v] = KINF;
  for (int i = threadIdx.x; i < NBM * W; i += blockDim.x) smq_smem[i] = 0u;
  if (PF)
    for (int i = threadIdx.x; i < WPF; i += blockDim.x) pfm[i] = 0u;
  __syncthreads();
  for (int pos = blockIdx.x; pos < R; pos = next_root(pos, sched.fetch, &s_next)) {
    const int r = sched.order ? sched.order[pos] : pos;
    const int z = node_int ? node_int[roots[r]] : roots[r];
    if (threadIdx.x == 0) {
      state[z] = NOLINK;
      sq0[0] = z;
      s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    }
    __syncthreads();
    int ncur = 1, round = 0;
    int *scur = sq0, *snxt = sq1, *gcur = gq0, *gnxt = gq1;
    unsigned *bcur = bm1, *bnxt = bm0;  // the root's queue entry has no mark
    unsigned my_relax = 0;
    while (ncur > 0) {
      const int c = round % 3;
      if (threadIdx.x == 0) s_cnt[(round + 1) % 3] = 0;
      if (ONEBM) {
        for (int i = threadIdx.x; i < ncur; i += THREADS) {
          const int y = i < qcap ? scur[i] : __ldcg(&gcur[i - qcap]);
          atomicAnd(&bm0[y >> 5], ~(1u << (y & 31)));
        }
        __syncthreads();
      }
      for (int base = 0; base < ncur; base += NQ * NPT) {
        int w[NPT], kb[NPT], ke[NPT];
        Dist dw[NPT];
        unsigned skipj = 0;
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
          const int i = base + j * NQ + quad;
          w[j] = i < ncur ? (i < qcap ? scur[i] : __ldcg(&gcur[i - qcap])) : -1;
        }
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
          kb[j] = 0; ke[j] = 0; dw[j] = 0;
          if (w[j] >= 0) {
            if (!ONEBM && lane4 == 0) atomicAnd(&bcur[w[j] >> 5], ~(1u << (w[j] & 31)));
            if (ELL) {  // slot lane4 of node w: no offset load on the chain
              kb[j] = 4 * w[j] + lane4;
              ke[j] = kb[j] + 1;
            } else {
              kb[j] = __ldg(&off[w[j]]) + lane4;
              ke[j] = __ldg(&off[w[j] + 1]);
            }
            const Key kw = __ldcg(&state[w[j]]);
            dw[j] = (Dist)(kw >> LB);
            // ADJ 2 on graphs where every link has its reverse and both lists
            // of a node share one order: slot lane4 leads back to w's parent
            // when it equals the parent's rank; that offer (dist(w) plus a
            // positive time) cannot beat the parent's key, so it is dropped
            if (RANK && skip_parent && (Key)lane4 == (kw & NOLINK)) skipj |= 1u << j;
          }
        }
        bool more = true;
        while (more) {
          int4 ent[NPT];
          Key tk[NPT];
#pragma unroll
          for (int j = 0; j < NPT; ++j) {
            if (kb[j] < ke[j]) {
              if (RANK) {  // 8-byte entry: ((neighbour << 3) | rank, link time), -1 when absent
                const int2 e2 = __ldg(&reinterpret_cast<const int2 *>(adj)[kb[j]]);
                ent[j] = make_int4(e2.x < 0 ? -1 : (e2.x & 7), e2.x >> 3, e2.y, 0);
              } else {
                ent[j] = __ldg(&adj[kb[j]]);
              }
            }
          }
#pragma unroll
          for (int j = 0; j < NPT; ++j) {
            if (ELL && kb[j] < ke[j] && (ent[j].x < 0 || ((skipj >> j) & 1u))) ke[j] = kb[j];  // absent / skipped
            tk[j] = KINF;
            if (RM > 0 && kb[j] < ke[j]) tk[j] = __ldcg(&state[ent[j].y]);
            if (PF && kb[j] < ke[j]) {
              // first offer into this 1 KB block of keys: prefetch the block
              // (the plain read may race; a repeated prefetch is harmless)
              const int blk = ent[j].y >> 8;
              const unsigned bit = 1u << (blk & 31);
              if (!(pfm[blk >> 5] & bit)) {
                atomicOr(&pfm[blk >> 5], bit);
                const char *base = reinterpret_cast<const char *>(state + ((size_t)blk << 8));
#pragma unroll
                for (int i = 0; i < 8; ++i) asm volatile("prefetch.global.L2 [%0];" ::"l"(base + i * 128));
              }
            }
          }
#pragma unroll
          for (int j = 0; j < NPT; ++j) {
            int pushy = -1;
            if (kb[j] < ke[j]) {
              ++my_relax;
              const Dist cand = dw[j] + (Dist)(unsigned)ent[j].z;
              if (cand >= DMAX) {
                // 64-bit keys: a distance beyond 2^61 is an error.  32-bit
                // keys: the offer is dropped, and a node that had no key yet
                // gets the sentinel KINF - 1 (above every real key).  A node
                // whose shortest distance is below 2^29 receives all its
                // offers below 2^29, so its key, tie rule included, is exact;
                // on the shortest path of a node at or beyond 2^29 the first
                // such node is offered only dropped offers and keeps the
                // sentinel, which the output pass flags for the 64-bit redo.
                // Nodes with no path keep KINF and need no redo.
                if (ADJ != 3) atomicOr(status, ST_OVERFLOW);
                else if (tk[j] == KINF) atomicMin(&state[ent[j].y], (Key)(KINF - 1));
              } else {
                const Key key = (Key)((cand << LB) | (Dist)(unsigned)ent[j].x);
                if (key < tk[j]) {
                  const int y = ent[j].y;
                  Key seen;
                  if (RM == 2) {
                    atomicMin(&state[y], key);  // result unused: no wait on the reply
                    seen = tk[j];
                  } else {
                    seen = atomicMin(&state[y], key);
                  }
                  if ((Dist)(seen >> LB) > cand &&
                      !((atomicOr(&bnxt[y >> 5], 1u << (y & 31)) >> (y & 31)) & 1u)) {
                    if (AGG) {
                      pushy = y;
                    } else {
                      const int pos = atomicAdd(&s_cnt[c], 1);
                      if (pos < qcap) snxt[pos] = y;
                      else gnxt[pos - qcap] = y;
                    }
                  }
                }
              }
            }
            if (AGG) {
              // the lanes executing here append together: one atomicAdd, ballot offsets
              const unsigned act = __activemask();
              const unsigned m = __ballot_sync(act, pushy >= 0);
              if (m) {
                const int lane = threadIdx.x & 31;
                const int leader = __ffs(m) - 1;
                int base = 0;
                if (lane == leader) base = atomicAdd(&s_cnt[c], __popc(m));
                base = __shfl_sync(act, base, leader);
                if (pushy >= 0) {
                  const int pos = base + __popc(m & ((1u << lane) - 1u));
                  if (pos < qcap) snxt[pos] = pushy;
                  else gnxt[pos - qcap] = pushy;
                }
              }
            }
          }
          more = false;
          if (!ELL) {  // four-slot layouts hold every slot of a node: one step
#pragma unroll
            for (int j = 0; j < NPT; ++j) {
              kb[j] += 4;
              more |= kb[j] < ke[j];
            }
          }
        }
      }
      __syncthreads();
      ncur = s_cnt[c];
      int *t = scur; scur = snxt; snxt = t;
      t = gcur; gcur = gnxt; gnxt = t;
      unsigned *tb = bcur; bcur = bnxt; bnxt = tb;
      ++round;
      if (round > max_rounds) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        break;
      }
    }
    if (roots_counter) {
      if (threadIdx.x == 0) atomicAdd(roots_counter + 1, (unsigned long long)round);
      atomicAdd(roots_counter + 2, (unsigned long long)my_relax);
    }
    if (sched.hint && threadIdx.x == 0) sched.hint[roots[r]] = round;
    __syncthreads();
    // an early exit (timeout) can leave marks behind: clear both bitmaps
    if (round > max_rounds)
      for (int i = threadIdx.x; i < NBM * W; i += blockDim.x) smq_smem[i] = 0u;
    // output: parent link (and distance) per external node id, keys reset
    int *prow = parent + (long long)r * V;
    long long *drow = dist ? dist + (long long)r * V : nullptr;
    bool unreached = false;  // 32-bit keys: a node left at the sentinel asks for the 64-bit redo
    if (out_mode != 0 && node_ext) {
      // internal order: coalesced key reads and resets, parent writes through
      // the inverse permutation (runs of consecutive ids inside a cell); on
      // the metro grid 39.5 ms per 2000-root batch against 40.7 ms for the
      // external-order pass below and 43.6 ms for an external-order pass
      // that reset each key right after reading it (scattered 8-byte stores)
      for (int u0 = threadIdx.x; u0 < V; u0 += 4 * THREADS) {
        Key key[4];
        int v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int u = u0 + k * THREADS;
          key[k] = u < V ? __ldcg(&state[u]) : Key(0);
          v[k] = u < V ? __ldg(&node_ext[u]) : -1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (v[k] < 0) continue;
          const int u = u0 + k * THREADS;
          state[u] = KINF;
          if (ADJ == 3 && key[k] == (Key)(KINF - 1)) {  // offered only beyond 2^29
            unreached = true;
            key[k] = KINF;
          }
          const Key lk = key[k] & NOLINK;
          prow[v[k]] = lk == NOLINK ? -1 : RANK ? __ldg(&rank_link[4 * u + (int)lk]) : (int)lk;
          if (drow) drow[v[k]] = key[k] == KINF ? LLONG_MAX : (long long)(key[k] >> LB);
        }
      }
    } else {
      // external order, then a separate coalesced reset
      for (int v = threadIdx.x; v < V; v += blockDim.x) {
        const int u = node_int ? node_int[v] : v;
        Key key = __ldcg(&state[u]);
        if (ADJ == 3 && key == (Key)(KINF - 1)) {  // offered only beyond 2^29
          unreached = true;
          key = KINF;
        }
        const Key lk = key & NOLINK;
        prow[v] = lk == NOLINK ? -1 : RANK ? __ldg(&rank_link[4 * u + (int)lk]) : (int)lk;
        if (drow) drow[v] = key == KINF ? LLONG_MAX : (long long)(key >> LB);
      }
      __syncthreads();
      for (int v = threadIdx.x; v < V; v += blockDim.x) state[v] = KINF;
    }
    if (ADJ == 3 && unreached) atomicOr(status, ST_K32);
    if (PF)
      for (int i = threadIdx.x; i < WPF; i += blockDim.x) pfm[i] = 0u;
    __syncthreads();
  }
}

// Lane-per-node variant of the shared-memory-queue kernel for 32-bit rank
// keys on the four-slot adjacency (shapes 6 and 7).  One lane owns NPN
// frontier nodes per pass: it reads a node's key once, its whole 32-byte
// adjacency row in two vector loads, and relaxes the (up to four) slots with
// 32-bit arithmetic (distances stay below 2^29 and link times below 2^31, so
// dist + time fits in 32 bits).  The quad-per-node kernel above repeats the
// queue read, the key read and the bookkeeping on all four lanes of a node
// and carries 64-bit distances; the round structure, marks, queues, tie rule
// (key = (distance << 3) | rank, atomicMin), overflow flag and output pass are
// the same, so the results are the same bits.  Signature as SmqKernel.
template <int THREADS, int NPN>
__global__ void __launch_bounds__(THREADS, 65536 / (THREADS * 64))
sssp_lane_kernel(int V, int /*LB_link*/, const int * /*off*/, const int4 *__restrict__ adj,
                 const int *__restrict__ roots, int R_host, const int *R_dev,
                 unsigned long long *g_state, int *g_queue, int *parent,
                 const int *parent_slot_dev, long long slot_stride, long long *dist, unsigned *status,
                 const int *skip_dev, unsigned long long *roots_counter, const int *__restrict__ node_int,
                 int max_rounds, int qcap, const int *__restrict__ node_ext, int /*out_mode*/,
                 const int *__restrict__ rank_link, int skip_parent, RootSched sched) {
  extern __shared__ __align__(16) unsigned smq_smem[];
  __shared__ int s_cnt[3];
  __shared__ int s_next;
  if (skip_dev && *skip_dev) return;
  const int R = R_dev ? *R_dev : R_host;
  if (roots_counter && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(roots_counter, (unsigned long long)R);
  const int W = (V + 31) >> 5;
  constexpr unsigned KINF = 0xffffffffu, NOLINK = 7u, DMAX = KINF >> 3;
  unsigned *bm = smq_smem;
  int *sq0 = reinterpret_cast<int *>(smq_smem + W), *sq1 = sq0 + qcap;
  const size_t b = blockIdx.x;
  unsigned *state = reinterpret_cast<unsigned *>(g_state) + b * (size_t)V;
  int *gq0 = g_queue + b * 2 * (size_t)V, *gq1 = gq0 + V;
  if (parent_slot_dev) parent += (long long)(*parent_slot_dev) * slot_stride;
  const int4 *rows = adj;  // node u: slots 0, 1 in rows[2u], slots 2, 3 in rows[2u + 1]
  for (int v = threadIdx.x; v < V; v += THREADS) state[v] = KINF;
  for (int i = threadIdx.x; i < W; i += THREADS) bm[i] = 0u;
  __syncthreads();
  for (int pos = blockIdx.x; pos < R; pos = next_root(pos, sched.fetch, &s_next)) {
    const int r = sched.order ? sched.order[pos] : pos;
    const int z = node_int ? node_int[roots[r]] : roots[r];
    if (threadIdx.x == 0) {
      state[z] = NOLINK;
      sq0[0] = z;
      s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
    }
    __syncthreads();
    int ncur = 1, round = 0;
    int *scur = sq0, *snxt = sq1, *gcur = gq0, *gnxt = gq1;
    unsigned my_relax = 0;
    while (ncur > 0) {
      const int c = round % 3;
      if (threadIdx.x == 0) s_cnt[(round + 1) % 3] = 0;
      // one bitmap: clear the marks of the queue about to be read, then a
      // barrier, so a set mark during the relaxations means "in the next queue"
      for (int i = threadIdx.x; i < ncur; i += THREADS) {
        const int y = i < qcap ? scur[i] : __ldcg(&gcur[i - qcap]);
        atomicAnd(&bm[y >> 5], ~(1u << (y & 31)));
      }
      __syncthreads();
      for (int base = 0; base < ncur; base += THREADS * NPN) {
        int w[NPN];
        unsigned dw[NPN], prank[NPN];
        int4 ra[NPN], rb[NPN];
#pragma unroll
        for (int n = 0; n < NPN; ++n) {
          const int i = base + n * THREADS + (int)threadIdx.x;
          w[n] = i < ncur ? (i < qcap ? scur[i] : __ldcg(&gcur[i - qcap])) : -1;
        }
#pragma unroll
        for (int n = 0; n < NPN; ++n) {
          dw[n] = 0u;
          prank[n] = 8u;  // no slot
          ra[n] = make_int4(-1, 0, -1, 0);
          rb[n] = ra[n];
          if (w[n] >= 0) {
            const unsigned kw = __ldcg(&state[w[n]]);
            dw[n] = kw >> 3;
            if (skip_parent) prank[n] = kw & NOLINK;
            ra[n] = __ldg(&rows[2 * w[n]]);
            rb[n] = __ldg(&rows[2 * w[n] + 1]);
          }
        }
        // slot s of node n: x = (neighbour << 3) | rank (-1 absent), t = link time
        int sx[NPN][4];
        unsigned st[NPN][4], tk[NPN][4];
#pragma unroll
        for (int n = 0; n < NPN; ++n) {
          sx[n][0] = ra[n].x; st[n][0] = (unsigned)ra[n].y;
          sx[n][1] = ra[n].z; st[n][1] = (unsigned)ra[n].w;
          sx[n][2] = rb[n].x; st[n][2] = (unsigned)rb[n].y;
          sx[n][3] = rb[n].z; st[n][3] = (unsigned)rb[n].w;
#pragma unroll
          for (int s = 0; s < 4; ++s)
            if (sx[n][s] >= 0 && (unsigned)s == prank[n]) sx[n][s] = -1;  // the way back to the parent
        }
#pragma unroll
        for (int n = 0; n < NPN; ++n)
#pragma unroll
          for (int s = 0; s < 4; ++s) tk[n][s] = sx[n][s] >= 0 ? __ldcg(&state[sx[n][s] >> 3]) : 0u;
#pragma unroll
        for (int n = 0; n < NPN; ++n)
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            if (sx[n][s] < 0) continue;
            ++my_relax;
            const unsigned cand = dw[n] + st[n][s];
            if (cand >= DMAX) {  // dropped; a node without a key gets the sentinel (see the output pass)
              if (tk[n][s] == KINF) atomicMin(&state[sx[n][s] >> 3], KINF - 1u);
              continue;
            }
            const unsigned key = (cand << 3) | (unsigned)(sx[n][s] & 7);
            if (key < tk[n][s]) {
              const int y = sx[n][s] >> 3;
              atomicMin(&state[y], key);  // result unused: no wait on the reply
              const unsigned bit = 1u << (y & 31);
              if ((tk[n][s] >> 3) > cand && !(atomicOr(&bm[y >> 5], bit) & bit)) {
                const int pos = atomicAdd(&s_cnt[c], 1);
                if (pos < qcap) snxt[pos] = y;
                else gnxt[pos - qcap] = y;
              }
            }
          }
      }
      __syncthreads();
      ncur = s_cnt[c];
      int *t = scur; scur = snxt; snxt = t;
      t = gcur; gcur = gnxt; gnxt = t;
      ++round;
      if (round > max_rounds) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        break;
      }
    }
    if (roots_counter) {
      if (threadIdx.x == 0) atomicAdd(roots_counter + 1, (unsigned long long)round);
      atomicAdd(roots_counter + 2, (unsigned long long)my_relax);
    }
    if (sched.hint && threadIdx.x == 0) sched.hint[roots[r]] = round;
    __syncthreads();
    if (round > max_rounds)  // an early exit can leave marks behind
      for (int i = threadIdx.x; i < W; i += THREADS) bm[i] = 0u;
    // output in internal order: coalesced key reads and resets, parents
    // (and distances) written through the inverse permutation.  Offers of
    // 2^29 or more were dropped: nodes whose shortest distance is below 2^29
    // have exact keys, and a node left at the sentinel KINF - 1 (offered
    // only beyond 2^29: distance at or beyond 2^29) sets ST_K32 so the batch
    // is redone with 64-bit keys.
    int *prow = parent + (long long)r * V;
    long long *drow = dist ? dist + (long long)r * V : nullptr;
    bool unreached = false;
    for (int u0 = threadIdx.x; u0 < V; u0 += 4 * THREADS) {
      unsigned key[4];
      int v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int u = u0 + k * THREADS;
        key[k] = u < V ? __ldcg(&state[u]) : 0u;
        v[k] = u < V ? (node_ext ? __ldg(&node_ext[u]) : u) : -1;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (v[k] < 0) continue;
        const int u = u0 + k * THREADS;
        state[u] = KINF;
        if (key[k] == KINF - 1u) {  // offered only beyond 2^29
          unreached = true;
          key[k] = KINF;
        }
        const unsigned lk = key[k] & NOLINK;
        prow[v[k]] = lk == NOLINK ? -1 : __ldg(&rank_link[4 * u + (int)lk]);
        if (drow) drow[v[k]] = key[k] == KINF ? LLONG_MAX : (long long)(key[k] >> 3);
      }
    }
    if (unreached) atomicOr(status, ST_K32);
    __syncthreads();
  }
}

size_t sssp_smq_smem_bytes(int V, int shape) {
  const SmqShape &sh = kSmqShape[shape];
  // marks, two queues, and the prefetch bitmap of shape 8 (V / 8192 + 1 words)
  return (size_t)sh.bitmaps * ((V + 31) / 32) * 4 + (size_t)2 * sh.qcap * 4 + (size_t)((V >> 13) + 1) * 4;
}

// does launch shape `shape` fit its CTAs per SM in the 196 KB carveout step
int sssp_smq_shape_count() { return kSmqShapes; }

bool sssp_smq_shape_fits(int V, int shape) {
  if (shape < 0 || shape >= kSmqShapes) return false;
  return sssp_smq_smem_bytes(V, shape) * kSmqShape[shape].ctas <= 192 * 1024;
}

// the global-memory launch runs the shared-memory-queue kernel (which reads
// the locality-ordered adjacency when the graph has one)
bool sssp_uses_smq(const GraphDev &g) {
  return sssp_group_size() == 1 && sssp_smq_shape_fits(g.V, g.tune_shape) && !getenv("QDTA_BF_NOSMQ");
}

bool sssp_uses_perm(const GraphDev &g) { return g.node_int != nullptr && sssp_uses_smq(g); }
// fixed four-slot adjacency: locality order present, every degree <= 4
bool sssp_uses_ell(const GraphDev &g, int direction) {
  return sssp_uses_perm(g) && g.max_deg[direction] <= 4 && g.tune_adj >= 1;
}
int sssp_adj(const GraphDev &g, int direction) {
  if (!sssp_uses_ell(g, direction)) return 0;
  if (g.tune_adj >= 2 && g.rank_tgt[direction] && g.rank_link[direction] && g.V < (1 << 28)) return g.tune_adj;
  return 1;
}

// name of the kernel launch_sssp runs for this graph, direction and storage
const char *sssp_kernel_name(const GraphDev &g, int direction, bool use_smem) {
  if (use_smem) return "sssp_kernel<true>";
  if (sssp_uses_smq(g)) {
    static const char *adj_name[4] = {"csr", "ell", "rank", "rank32"};
    static const std::vector<std::string> names = [] {
      std::vector<std::string> v;
      for (int sh = 0; sh < kSmqShapes; ++sh)
        for (int e = 0; e < 4; ++e)
          for (int r = 0; r < 4; ++r)
            v.push_back(sh == 8 && e == 3   ? std::string("sssp_smq_kernel<256,rank32,2,true,pf>")
                        : sh == 9 && e == 3 ? std::string("sssp_smq_kernel<192,rank32,2,true,5>")
                        : sh >= 6 && sh <= 7 && e == 3
                            ? "sssp_lane_kernel<" + std::to_string(kSmqShape[sh].threads) + ",npn" +
                                  std::to_string(kSmqShape[sh].npt) + ">"
                            : "sssp_smq_kernel<" + std::to_string(smq_threads(sh, e)) + "," + adj_name[e] + "," +
                                  std::to_string(r) + "," + (kSmqShape[sh].bitmaps == 1 ? "true" : "false") +
                                  (sh == 3 && e == 3 ? ",5" : "") +
                                  (sh >= 4 && sh <= 5 && e == 3 ? ",npt" + std::to_string(kSmqShape[sh].npt) : "") +
                                  ">");
      return v;
    }();
    const int adj = sssp_adj(g, direction);
    int r = g.tune_relax < 0 ? 0 : g.tune_relax > 3 ? 3 : g.tune_relax;
    if (adj >= 2 && r < 2) r = 2;
    if (adj == 3) r = 2;
    return names[(g.tune_shape * 4 + adj) * 4 + r].c_str();
  }
  switch (sssp_group_size()) {
    case 2: return "sssp_group_kernel<512,2>";
    case 4: return "sssp_group_kernel<512,4>";
    case 8: return "sssp_group_kernel<512,8>";
    default: return "sssp_ilp_kernel<512>";
  }
}

int sssp_max_smem_nodes() { return (200 * 1024) / 20; }

static size_t sssp_smem_bytes(int V) { return (size_t)V * 20; }

int sssp_blocks_per_sm(bool use_smem, int V) {
  int n = 0;
  if (use_smem) {
    cudaFuncSetAttribute(sssp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sssp_smem_bytes(V));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sssp_kernel<true>, SSSP_THREADS,
                                                  sssp_smem_bytes(V));
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sssp_ilp_kernel<512>, 512, 0);
  }
  return n > 0 ? n : 1;
}

// after a 32-bit-key batch: run the 64-bit redo only if the batch overflowed
// (and was not skipped); clears the overflow bit, which is not an error
// Longest-first order of the batch's roots for the dynamic fetch: by the
// rounds each root node took in its last batch (hint, 0 when never run),
// descending, ties by position.  One CTA, a bitonic sort of up to
// ORDER_MAX keys in shared memory; larger batches keep their order.
constexpr int ORDER_MAX = 4096;
__global__ void __launch_bounds__(1024)
order_roots_kernel(int R_host, const int *R_dev, const int *__restrict__ roots, const int *__restrict__ hint,
                   int *order, const int *skip_dev) {
  __shared__ unsigned long long key[ORDER_MAX];
  if (skip_dev && *skip_dev) return;
  const int R = R_dev ? *R_dev : R_host;
  if (R > ORDER_MAX) {
    for (int i = threadIdx.x; i < R; i += blockDim.x) order[i] = i;
    return;
  }
  int n = 1;
  while (n < R) n <<= 1;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int h = i < R ? max(hint[roots[i]], 0) : 0;
    key[i] = i < R ? ((unsigned long long)(0x7fffffff - h) << 32) | (unsigned)i : ~0ull;
  }
  __syncthreads();
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = key[i], b = key[ixj];
          if (((i & k) == 0) == (a > b)) {
            key[i] = b;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < R; i += blockDim.x) order[i] = (int)(key[i] & 0xffffffffu);
}

__global__ void k32_redo_flag_kernel(unsigned *status, const int *skip_dev, int *fb_skip,
                                     unsigned long long *redo_counter) {
  const unsigned st = *status;
  const bool skipped = skip_dev && *skip_dev;
  const bool redo = !skipped && (st & ST_K32);
  if (st & ST_K32) atomicAnd(status, ~ST_K32);
  *fb_skip = redo ? 0 : 1;
  if (redo && redo_counter) atomicAdd(redo_counter, 1ull);
}

using SmqKernel = void (*)(int, int, const int *, const int4 *, const int *, int, const int *, unsigned long long *,
                          int *, int *, const int *, long long, long long *, unsigned *, const int *,
                          unsigned long long *, const int *, int, int, const int *, int, const int *, int, RootSched);

template <int THREADS, bool ONEBM>
static SmqKernel smq_kernel_relax(int adj, int relax) {
  if (adj == 3) return sssp_smq_kernel<THREADS, 3, 2, ONEBM>;
  if (adj == 2) return relax == 3 ? sssp_smq_kernel<THREADS, 2, 3, ONEBM> : sssp_smq_kernel<THREADS, 2, 2, ONEBM>;
  if (adj == 1) return relax == 3 ? sssp_smq_kernel<THREADS, 1, 3, ONEBM>
                : relax == 2 ? sssp_smq_kernel<THREADS, 1, 2, ONEBM>
                : relax == 1 ? sssp_smq_kernel<THREADS, 1, 1, ONEBM> : sssp_smq_kernel<THREADS, 1, 0, ONEBM>;
  return relax == 3 ? sssp_smq_kernel<THREADS, 0, 3, ONEBM>
       : relax == 2 ? sssp_smq_kernel<THREADS, 0, 2, ONEBM>
       : relax == 1 ? sssp_smq_kernel<THREADS, 0, 1, ONEBM> : sssp_smq_kernel<THREADS, 0, 0, ONEBM>;
}

static SmqKernel smq_kernel_for(int shape, int adj, int relax) {
  if (shape == 6 && adj == 3) return sssp_lane_kernel<256, 1>;
  if (shape == 7 && adj == 3) return sssp_lane_kernel<256, 2>;
  if (shape == 8 && adj == 3) return sssp_smq_kernel<256, 3, 2, true, 4, 4, true>;
  if (shape == 9 && adj == 3) return sssp_smq_kernel<192, 3, 2, true, 5>;
  if (shape == 10 && adj == 3) return sssp_smq_kernel<288, 3, 2, true, 4>;
  if (shape == 3 && adj == 3) return sssp_smq_kernel<256, 3, 2, true, 5>;
  if (shape == 4 && adj == 3) return sssp_smq_kernel<256, 3, 2, true, 4, 5>;
  if (shape == 5 && adj == 3) return sssp_smq_kernel<256, 3, 2, true, 4, 6>;
  if (shape == 9) return smq_kernel_relax<192, true>(adj, relax);
  if (shape == 1 || shape >= 3) return smq_kernel_relax<256, true>(adj, relax);
  if (shape == 2) return smq_kernel_relax<512, true>(adj, relax);
  return smq_kernel_relax<512, false>(adj, relax);
}

// resident CTAs per SM of the selected shared-memory-queue kernel (occupancy
// under the pinned carveout, at most the shape's design count)
int sssp_smq_ctas_per_sm(const GraphDev &g, int direction) {
  const SmqKernel kern = smq_kernel_for(g.tune_shape, sssp_adj(g, direction), g.tune_relax);
  const size_t smq = sssp_smq_smem_bytes(g.V, g.tune_shape);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, g.tune_carve);
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, smq_threads(g.tune_shape, sssp_adj(g, direction)), smq);
  n = std::min(n, kSmqShape[g.tune_shape].ctas);
  return n > 0 ? n : 1;
}

void launch_sssp(const GraphDev &g, int direction, const int4 *adj, const int *roots, int R_host,
                 const int *R_dev, int grid, bool use_smem, const SsspWork &w, int *parent,
                 const int *parent_slot_dev, long long slot_stride, long long *dist,
                 unsigned *status, cudaStream_t s, const int *skip_dev,
                 unsigned long long *roots_counter) {
  const int *off = direction == 0 ? g.in_off : g.out_off;
  if (grid <= 0) return;
  if (use_smem) {
    size_t sm = sssp_smem_bytes(g.V);
    cudaFuncSetAttribute(sssp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(sssp_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    COUNT_LAUNCH();
    sssp_kernel<true><<<grid, SSSP_THREADS, sm, s>>>(g.V, g.LB, off, adj, roots, R_host, R_dev,
                                                     nullptr, nullptr, nullptr, parent,
                                                     parent_slot_dev, slot_stride, dist, status, skip_dev,
                                                     roots_counter, round_limit(g.V));
  } else {
    // block size of the global-memory variant (QDTA_BF_THREADS: 128, 256, 512 or 1024)
    static int bf_threads = [] {
      const char *e = getenv("QDTA_BF_THREADS");
      int t = e ? atoi(e) : 512;
      return (t == 128 || t == 256 || t == 1024) ? t : 512;
    }();
    auto kern = bf_threads == 1024 ? sssp_ilp_kernel<1024> : bf_threads == 512 ? sssp_ilp_kernel<512>
              : bf_threads == 256 ? sssp_ilp_kernel<256> : sssp_ilp_kernel<128>;
    const int G = sssp_group_size();
    if (sssp_uses_smq(g)) {
      const int adjl = sssp_adj(g, direction);
      // Every shape's CTAs fit their marks and queues in the 196 KB
      // shared-memory step (on the metro grid: two 86.5 KB or four 47.6 KB
      // CTAs); the rest of the unified 256 KB stays L1, which the memory
      // requests in flight want (55 ms per batch at 196 KB vs 84 ms at the
      // 228 KB maximum, measured with two 512-thread CTAs).  Pinning the
      // preference gives stream launches and graph kernel nodes the same
      // configuration.  The percentage is rounded up to a supported size:
      // 85 % of 228 KB asks for 194 KB and gets the 196 KB step (86 % would
      // round up to 228 KB).  QDTA_SMQ_CARVEOUT overrides, in percent.
      const size_t smq = sssp_smq_smem_bytes(g.V, g.tune_shape);
      const bool perm = g.node_int != nullptr;
      // dynamic fetch: roots after the first wave come from an atomic
      // counter (w.fb_skip[1] for the kernel, [2] for the redo), zeroed
      // here; with an order buffer, longest roots of their last batch first
      RootSched sched{g.tune_dyn ? w.fb_skip + 1 : nullptr, nullptr, g.root_rounds};
      if (sched.fetch) {
        cudaMemsetAsync(sched.fetch, 0, 2 * sizeof(int), s);
        if (w.order && g.root_rounds) {
          COUNT_LAUNCH();
          order_roots_kernel<<<1, 1024, 0, s>>>(R_host, R_dev, roots, g.root_rounds, w.order, skip_dev);
          sched.order = w.order;
        }
      }
      auto run = [&](SmqKernel kern, int threads, const int *skip, unsigned long long *counters, RootSched rs) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, g.tune_carve);
        COUNT_LAUNCH();
        kern<<<grid, threads, smq, s>>>(g.V, g.LB, perm ? g.perm_off[direction] : off, adj, roots, R_host, R_dev,
                                        w.state, w.queue, parent, parent_slot_dev, slot_stride, dist, status, skip,
                                        counters, perm ? g.node_int : nullptr, round_limit(g.V),
                                        kSmqShape[g.tune_shape].qcap, perm ? g.node_ext : nullptr, g.tune_out,
                                        g.rank_link[direction], g.skip_parent, rs);
      };
      run(smq_kernel_for(g.tune_shape, adjl, g.tune_relax), smq_threads(g.tune_shape, adjl), skip_dev, roots_counter,
          sched);
      if (adjl == 3) {
        // a distance beyond the 32-bit keys' range: redo the batch with 64-bit
        // keys on the same packed adjacency (decided on the device, so graph
        // replays need no host round trip).  The redo's roots are not counted
        // again; counter [4] counts redone batches.
        COUNT_LAUNCH();
        k32_redo_flag_kernel<<<1, 1, 0, s>>>(status, skip_dev, w.fb_skip,
                                             roots_counter ? roots_counter + 4 : nullptr);
        RootSched redo = sched;
        if (redo.fetch) redo.fetch += 1;
        run(smq_kernel_for(g.tune_shape, 2, 2), smq_threads(g.tune_shape, 2), w.fb_skip, nullptr, redo);
      }
      return;
    }
    if (G == 2) kern = sssp_group_kernel<512, 2>;
    else if (G == 4) kern = sssp_group_kernel<512, 4>;
    else if (G == 8) kern = sssp_group_kernel<512, 8>;
    if (G > 1) bf_threads = 512;
    COUNT_LAUNCH();
    kern<<<grid, bf_threads, 0, s>>>(g.V, g.LB, off, adj, roots, R_host, R_dev,
                                                     w.state, w.stamp, w.queue, parent,
                                                     parent_slot_dev, slot_stride, dist, status,
                                                     skip_dev, roots_counter, round_limit(g.V));
  }
}

// ============================================================================
// all-or-nothing loading with truncation
// ============================================================================

__global__ void pack_head_q_kernel(int L, const int *__restrict__ head, const int *__restrict__ q,
                                   int2 *__restrict__ hq) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x)
    hq[a] = make_int2(head[a], q[a]);
}

void launch_pack_head_q(const GraphDev &g, const int *q, int2 *head_q, cudaStream_t s) {
  if (g.L == 0) return;
  COUNT_LAUNCH();
  pack_head_q_kernel<<<cdiv(g.L, 256), 256, 0, s>>>(g.L, g.head, q, head_q);
}

// Carried truncation (Section 3.4): a position on a link is the fraction f
// of it covered, in units of 2^-32.  On a link of q quanta, f stands for
// round(q f / 2^32) quanta (halves up); t < q quanta cover floor(t 2^32 / q).
__device__ __forceinline__ long long carried_quanta(long long q, long long f) {
  return (long long)(((unsigned long long)q * (unsigned long long)f + (1ull << 31)) >> 32);
}
__device__ __forceinline__ long long frac_of(long long t, long long q) {
  return (long long)(((unsigned long long)t << 32) / (unsigned long long)q);
}

// A trip carried on link cl (carry_link >= 0) having covered the fraction f
// of it reaches the link's head after the uncovered rest, or is still on the
// link at the end of the interval when the rest exceeds dt_q.  Returns false
// in the second case; else sets u and elapsed.  The link itself is not
// loaded again: a trip loads a link in the interval it enters it.
__device__ __forceinline__ bool finish_carried_link(const int2 *__restrict__ head_q, int cl, long long f,
                                                    long long dt_q, int &u, long long &elapsed) {
  const int2 hq = __ldg(&head_q[cl]);
  const long long rest = (long long)hq.y - carried_quanta(hq.y, f);
  if (rest > dt_q) return false;
  elapsed = rest;
  u = hq.x;
  return true;
}

// One thread per item: walk origin -> root along the destination tree.  A
// link is loaded iff the elapsed time at its tail is < dt_q; the walk ends
// at the first node reached at >= dt_q (the stop node) or at the root.  An
// item carried on a link walks on from its head (the link was loaded when
// the trip entered it); one still on it at the end of the interval stops at
// src (the link's tail).
__global__ void load_kernel(int V, const int2 *__restrict__ head_q, const int *__restrict__ parent,
                            const int *parent_slot_dev, long long slot_stride,
                            const int *__restrict__ root_slot, const int *__restrict__ roots,
                            long long n_host, const long long *n_dev, const int *__restrict__ root_idx,
                            const int *__restrict__ src, const long long *__restrict__ amount,
                            long long dt_q, unsigned long long *flow_fx, int *stop_out,
                            unsigned *status, const long long *__restrict__ carry,
                            const int *__restrict__ carry_link) {
  const long long n = n_dev ? *n_dev : n_host;
  if (parent_slot_dev) parent += (long long)(*parent_slot_dev) * slot_stride;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = root_idx[k];
    const int z = roots[r];
    const int *par = parent + (long long)(root_slot ? root_slot[r] : r) * V;
    const unsigned long long amt = (unsigned long long)amount[k];
    int u = src[k];
    long long elapsed = 0;
    const int cl = carry_link ? carry_link[k] : -1;
    if (cl >= 0) {
      if (!finish_carried_link(head_q, cl, carry ? carry[k] : 0, dt_q, u, elapsed)) {
        if (stop_out) stop_out[k] = u;
        continue;
      }
    }
    int steps = 0;
    while (u != z) {
      if (elapsed >= dt_q) break;
      const int e = par[u];
      if (e < 0) { atomicOr(status, ST_UNREACH); break; }
      if (amt) atomicAdd(&flow_fx[e], amt);
      const int2 hq = __ldg(&head_q[e]);
      elapsed += hq.y;
      u = hq.x;
      if (++steps > V) { atomicOr(status, ST_TIMEOUT); break; }
    }
    if (stop_out) stop_out[k] = u;
  }
}

static int link_grid(const GraphDev &g, long long n) {
  long long want = (n + 255) / 256;
  long long cap = (long long)g.num_sms * 16;
  if (want > cap) want = cap;
  return want < 1 ? 1 : (int)want;
}

// capacity update: check every value first, copy only if all are valid
__global__ void cap_check_kernel(int L, const double *__restrict__ cap, unsigned *status) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    const double c = cap[a];
    if (!(c > 0.0) || !isfinite(c)) atomicOr(status, ST_BADARG);
  }
}

__global__ void cap_copy_kernel(int L, const double *__restrict__ src, double *__restrict__ dst,
                                const unsigned *status) {
  if (*status & ST_BADARG) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) dst[a] = src[a];
}

// items carried on a link: the link exists, starts at the item's src, and
// the covered fraction is in [0, 2^32) (ST_BADARG otherwise)
__global__ void check_carry_kernel(int L, long long n, const int *__restrict__ src,
                                   const long long *__restrict__ carry, const int *__restrict__ carry_link,
                                   const int *__restrict__ tail, unsigned *status) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int cl = carry_link[k];
    if (cl < 0) continue;
    if (cl >= L || tail[cl] != src[k] || (carry && (carry[k] < 0 || carry[k] >= (1ll << 32))))
      atomicOr(status, ST_BADARG);
  }
}

void launch_check_carry(const GraphDev &g, long long n, const int *src, const long long *carry,
                        const int *carry_link, unsigned *status, cudaStream_t s) {
  if (n <= 0 || !carry_link) return;
  COUNT_LAUNCH();
  check_carry_kernel<<<link_grid(g, n), 256, 0, s>>>(g.L, n, src, carry, carry_link, g.tail, status);
}

void launch_set_capacity(const GraphDev &g, const double *cap, unsigned *status, cudaStream_t s) {
  if (g.L <= 0) return;
  COUNT_LAUNCH();
  cap_check_kernel<<<link_grid(g, g.L), 256, 0, s>>>(g.L, cap, status);
  COUNT_LAUNCH();
  cap_copy_kernel<<<link_grid(g, g.L), 256, 0, s>>>(g.L, cap, const_cast<double *>(g.cap), status);
}


void launch_load(const GraphDev &g, const int2 *head_q, const int *parent, const int *parent_slot_dev,
                 long long slot_stride, const int *root_slot, const int *roots, long long n_items_host,
                 const long long *n_items_dev, const int *root_idx, const int *src,
                 const long long *amount, long long dt_q, unsigned long long *flow_fx, int *stop_out,
                 unsigned *status, cudaStream_t s, const long long *carry, const int *carry_link) {
  long long n = n_items_dev ? (long long)g.num_sms * 16 * 256 : n_items_host;
  if (n <= 0) return;
  COUNT_LAUNCH();
  load_kernel<<<link_grid(g, n), 256, 0, s>>>(g.V, head_q, parent, parent_slot_dev, slot_stride,
                                              root_slot, roots, n_items_host, n_items_dev, root_idx,
                                              src, amount, dt_q, flow_fx, stop_out, status, carry,
                                              carry_link);
}

// unsigned 128-bit accumulation with two 64-bit atomics: the low word's carry
// goes into the high word, so the pair holds the exact total once every add
// has landed (all terms here are >= 0)
__device__ __forceinline__ void add_u128(unsigned long long *p, u128 v) {
  const unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  const unsigned long long old = atomicAdd(p, lo);
  const unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
  if (hi | carry) atomicAdd(p + 1, hi + carry);
}

constexpr unsigned long long CARRY_KEY_EMPTY = ~0ull;

// one residual trip on a link: its amount and amount x covered fraction join
// the entry of key root * L + link.  Root r's keys start probing in its own
// segment [r seg, (r + 1) seg) of the table, at the link's id scaled to the
// segment, so the compaction's slot order is nearly root-major and link-
// ordered, as the dense part's is root-major and node-ordered (neighbouring
// threads of the later walks then start near each other on the same tree);
// linear probing, a key once claimed stays until the compaction clears the
// table.  A full table sets ST_CAPACITY and drops the trip.
__device__ __forceinline__ void carry_add(const CarryAcc &ca, int r, int L, int link, long long frac,
                                          long long amt, unsigned *status) {
  if (!ca.mask) {
    if (status) atomicOr(status, ST_CAPACITY);
    return;
  }
  const unsigned long long key = (unsigned long long)r * (unsigned long long)L + (unsigned long long)link;
  unsigned long long h =
      ((unsigned long long)r * ca.seg + (unsigned long long)link * ca.seg / (unsigned long long)L) & ca.mask;
  for (unsigned long long probe = 0; probe <= ca.mask; ++probe) {
    unsigned long long cur = __ldcg(&ca.key[h]);
    if (cur == CARRY_KEY_EMPTY) cur = atomicCAS(&ca.key[h], CARRY_KEY_EMPTY, key);
    if (cur == CARRY_KEY_EMPTY || cur == key) {
      // amount x fraction < 2^95 in two non-returning adds: the part above
      // 2^32 (below the amount, so the sums stay below 2^63) and the low 32
      // bits (below 2^64 for fewer than 2^32 entries per key)
      const u128 v = (u128)(unsigned long long)amt * (u128)(unsigned long long)frac;
      atomicAdd(&ca.amt[h], (unsigned long long)amt);
      atomicAdd(&ca.tsum[2 * h], (unsigned long long)(v & 0xffffffffull));
      atomicAdd(&ca.tsum[2 * h + 1], (unsigned long long)(v >> 32));
      return;
    }
    h = (h + 1) & ca.mask;
  }
  if (status) atomicOr(status, ST_CAPACITY);
}

// Alg. 4 for one accepted AON j: the item's path on tree j is re-truncated
// with the final link times (head_q_fin); its share RN(amount * w_j) loads
// h and, if the walk stops before the root, joins the residual demand of the
// next interval: in the dense (root, node) accumulator, or, when the trip is
// still on a link (trunc = 1, or an item carried on a link that it does not
// finish), in the carried table under (root, link) with the fraction of the
// link covered.
__global__ void residual_kernel(int V, int L, const int2 *__restrict__ head_q_fin,
                                const int *__restrict__ parent, const int *parent_slot_dev,
                                long long slot_stride, const int *__restrict__ root_slot,
                                const int *__restrict__ roots, const long long *n_dev,
                                const int *__restrict__ root_idx, const int *__restrict__ src,
                                const long long *__restrict__ amount, const double *weight_dev, long long dt_q,
                                unsigned long long *h_fx, unsigned long long *dense, unsigned *status,
                                const long long *__restrict__ carry, const int *__restrict__ carry_link,
                                int trunc, CarryAcc ca) {
  const long long n = *n_dev;
  const double w = *weight_dev;
  if (parent_slot_dev) parent += (long long)(*parent_slot_dev) * slot_stride;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const long long amt = __double2ll_rn(mul(__ll2double_rn(amount[k]), w));
    if (amt == 0) continue;
    const int r = root_idx[k];
    const int z = roots[r];
    const int *par = parent + (long long)root_slot[r] * V;
    int u = src[k];
    long long elapsed = 0, frac = 0;
    int on_link = -1;  // the link holding the trip at the end of the interval
    const int cl = carry_link ? carry_link[k] : -1;
    if (cl >= 0) {
      const long long c0 = carry ? carry[k] : 0;
      if (!finish_carried_link(head_q_fin, cl, c0, dt_q, u, elapsed)) {
        on_link = cl;
        frac = c0 + frac_of(dt_q, __ldg(&head_q_fin[cl]).y);
      }
    }
    int steps = 0;
    while (on_link < 0 && u != z) {
      if (elapsed >= dt_q) break;
      const int e = par[u];
      if (e < 0) { atomicOr(status, ST_UNREACH); break; }
      atomicAdd(&h_fx[e], (unsigned long long)amt);
      const int2 hq = __ldg(&head_q_fin[e]);
      if (trunc && elapsed + hq.y > dt_q) {  // on this link at the end of the interval
        on_link = e;
        frac = frac_of(dt_q - elapsed, hq.y);
        break;
      }
      elapsed += hq.y;
      u = hq.x;
      if (++steps > V) { atomicOr(status, ST_TIMEOUT); break; }
    }
    if (on_link >= 0) carry_add(ca, r, L, on_link, frac, amt, status);
    else if (u != z) atomicAdd(&dense[(long long)r * V + u], (unsigned long long)amt);
  }
}

void launch_residual(const GraphDev &g, const int2 *head_q_fin, const int *parent,
                     const int *parent_slot_dev, long long slot_stride, const int *root_slot,
                     const int *roots, const long long *n_items_dev, long long n_items_cap,
                     const int *root_idx, const int *src, const long long *amount,
                     const double *weight_dev, long long dt_q, unsigned long long *h_fx,
                     unsigned long long *dense, unsigned *status, cudaStream_t s, const long long *carry,
                     const int *carry_link, int trunc, CarryAcc ca) {
  if (n_items_cap <= 0) return;
  COUNT_LAUNCH();
  residual_kernel<<<link_grid(g, n_items_cap), 256, 0, s>>>(
      g.V, g.L, head_q_fin, parent, parent_slot_dev, slot_stride, root_slot, roots, n_items_dev, root_idx, src,
      amount, weight_dev, dt_q, h_fx, dense, status, carry, carry_link, trunc, ca);
}

// ============================================================================
// link-parallel passes
// ============================================================================

// Eq. 1 link times (marginal = 0), or the system optimum's marginal costs
// c + f c' (marginal = 1), quantised; cost_s (seconds) only for link times
__global__ void bpr_kernel(int L, const int *__restrict__ c0, const double *__restrict__ cap,
                           double alpha, int beta, double dt_h, double quantum_s,
                           const double *__restrict__ flow, double *cost_s, int *cost_q,
                           unsigned *status, int marginal) {
  unsigned bad = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    const double f = flow[a];
    if (!isfinite(f)) bad |= ST_NONFINITE;
    const LinkConst k = link_const(cap[a], dt_h, alpha, beta);
    const double c = marginal ? link_marginal((double)c0[a], k.inv, alpha, beta, f)
                              : link_cost((double)c0[a], k.inv, alpha, beta, f);
    if (cost_s && !marginal) cost_s[a] = mul(c, quantum_s);
    cost_q[a] = quantize(c, &bad);
  }
  if (bad) atomicOr(status, bad);
}

void launch_bpr(const GraphDev &g, const double *flow, double dt_h, double *cost_s, int *cost_q,
                unsigned *status, cudaStream_t s, int marginal) {
  if (g.L == 0) return;
  COUNT_LAUNCH();
  bpr_kernel<<<link_grid(g, g.L), LINK_THREADS, 0, s>>>(g.L, g.c0, g.cap, g.alpha, g.beta, dt_h,
                                                        g.quantum_s, flow, cost_s, cost_q, status, marginal);
}

__global__ void link_const_kernel(int L, const double *__restrict__ cap, double dt_h, double alpha,
                                  int beta, LinkConst *kc) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x)
    kc[a] = link_const(cap[a], dt_h, alpha, beta);
}

void launch_link_const(const GraphDev &g, double dt_h, LinkConst *kc, cudaStream_t s) {
  if (g.L == 0) return;
  COUNT_LAUNCH();
  link_const_kernel<<<link_grid(g, g.L), LINK_THREADS, 0, s>>>(g.L, g.cap, dt_h, g.alpha, g.beta, kc);
}

__global__ void flow_from_fx_kernel(int L, const unsigned long long *fx, double *f) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x)
    f[a] = fx64_to_double((long long)fx[a]);
}

void launch_flow_from_fx(int L, const unsigned long long *fx, double *f, cudaStream_t s) {
  if (L == 0) return;
  COUNT_LAUNCH();
  flow_from_fx_kernel<<<cdiv(L, 256), 256, 0, s>>>(L, fx, f);
}

void launch_fx_to_flow(int L, const unsigned long long *fx, double *out, cudaStream_t s) {
  launch_flow_from_fx(L, fx, out, s);
}

__device__ __forceinline__ i128 shfl_down_i128(i128 v, int d) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((u128)v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, d);
  hi = __shfl_down_sync(0xffffffffu, hi, d);
  return (i128)(((u128)hi << 64) | (u128)lo);
}

// Block-reduce acc[0..NSUM) into partials[blockIdx]; the last block to finish
// adds all block partials (integer sums: any order gives the same value)
// and stores them in out[0..NSUM).
__device__ void reduce_sums(i128 (&acc)[NSUM], i128 *partials, unsigned *counter, i128 *out) {
  __shared__ i128 s_w[LINK_THREADS / 32][NSUM];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NSUM; ++m) {
    i128 v = acc[m];
    for (int d = 16; d > 0; d >>= 1) v += shfl_down_i128(v, d);
    if (lane == 0) s_w[wid][m] = v;
  }
  __syncthreads();
  if (threadIdx.x < NSUM) {
    i128 t = 0;
    for (int w = 0; w < LINK_THREADS / 32; ++w) t += s_w[w][threadIdx.x];
    partials[(size_t)blockIdx.x * NSUM + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (threadIdx.x < NSUM) {
      i128 t = 0;
      for (unsigned b = 0; b < gridDim.x; ++b) {
        const volatile unsigned long long *p =
            reinterpret_cast<const volatile unsigned long long *>(&partials[(size_t)b * NSUM + threadIdx.x]);
        t += (i128)(((u128)p[1] << 64) | (u128)p[0]);
      }
      out[threadIdx.x] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
  }
}

// One pass over the links evaluating the controller's plan: up to eight
// step sizes, each one of phi (Beckmann sum, Eq. 6), phi' (exact slope) or
// phi'' at t = f + alpha (g - f), plus optionally the gap sums
// A = sum fx(q f) and B = sum q g (Alg. 9's three values generalised).
__global__ void __launch_bounds__(LINK_THREADS)
sweep_kernel(int L, const int *__restrict__ c0, const LinkConst *__restrict__ kc,
             const double *__restrict__ f, const long long *__restrict__ g_fx,
             const int *__restrict__ q, double alpha_bpr, int beta, Ctl *ctl, i128 *partials,
             unsigned *counter, unsigned *status, int so) {
  __shared__ Plan plan;
  if (threadIdx.x == 0) plan = ctl->plan;
  __syncthreads();
  i128 acc[NSUM];
#pragma unroll
  for (int m = 0; m < NSUM; ++m) acc[m] = 0;
  unsigned bad = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    const double fa = f[a];
    const long long gfx = g_fx[a];
    const double ga = fx64_to_double(gfx);
    const double c0a = (double)c0[a];
    const LinkConst k = kc[a];
    if (plan.want_gap && q) {
      const int qa = q[a];
      acc[MAX_SLOTS] += fx_of(mul((double)qa, fa), &bad);
      acc[MAX_SLOTS + 1] += (i128)qa * (i128)gfx;
    }
    const double d = sub(ga, fa);
#pragma unroll
    for (int m = 0; m < MAX_SLOTS; ++m) {
      if (m < plan.n) {
        const double t = step_flow(fa, ga, plan.alpha[m]);
        double term;
        // user equilibrium: Beckmann integral (Eq. 6), link time, its slope;
        // system optimum: total cost t c(t), marginal cost, its slope
        if (plan.kind[m] == K_PHI)
          term = so ? mul(t, link_cost(c0a, k.inv, alpha_bpr, beta, t)) : beckmann(c0a, k.inv, k.kb, beta, t);
        else if (plan.kind[m] == K_DPHI)
          term = mul(d, so ? link_marginal(c0a, k.inv, alpha_bpr, beta, t) : link_cost(c0a, k.inv, alpha_bpr, beta, t));
        else
          term = mul(mul(d, d), so ? link_marginal_dt(c0a, k.inv, alpha_bpr, beta, t)
                                   : link_cost_dt(c0a, k.inv, alpha_bpr, beta, t));
        acc[m] += fx_of(term, &bad);
      }
    }
  }
  if (bad) atomicOr(status, bad);
  reduce_sums(acc, partials, counter, ctl->sums);
}

int sweep_grid(const GraphDev &g) {
  long long want = ((long long)g.L + LINK_THREADS - 1) / LINK_THREADS;
  long long cap = (long long)g.num_sms * 4;
  if (want > cap) want = cap;
  return want < 1 ? 1 : (int)want;
}

void launch_sweep(const GraphDev &g, const LinkConst *kc, const double *f, const long long *g_fx,
                  const int *q, Ctl *ctl, i128 *partials, unsigned *counter, int grid,
                  unsigned *status, cudaStream_t s, int so) {
  COUNT_LAUNCH();
  sweep_kernel<<<grid, LINK_THREADS, 0, s>>>(g.L, g.c0, kc, f, g_fx, q, g.alpha, g.beta, ctl,
                                             partials, counter, status, so);
}

__global__ void __launch_bounds__(LINK_THREADS)
objective_kernel(int L, const int *__restrict__ c0, const LinkConst *__restrict__ kc,
                 const double *__restrict__ f, double alpha_bpr, int beta, Ctl *ctl, i128 *partials,
                 unsigned *counter, unsigned *status, int so) {
  __shared__ i128 out[NSUM];
  i128 acc[NSUM];
#pragma unroll
  for (int m = 0; m < NSUM; ++m) acc[m] = 0;
  unsigned bad = 0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    const LinkConst k = kc[a];
    const double term = so ? mul(f[a], link_cost((double)c0[a], k.inv, alpha_bpr, beta, f[a]))
                           : beckmann((double)c0[a], k.inv, k.kb, beta, f[a]);
    acc[0] += fx_of(term, &bad);
  }
  if (bad) atomicOr(status, bad);
  if (threadIdx.x == 0) out[0] = 0;
  reduce_sums(acc, partials, counter, out);
  if (threadIdx.x == 0 && out[0] != 0) ctl->objective = fx_to_double(out[0]);
}

void launch_objective(const GraphDev &g, const LinkConst *kc, const double *f, Ctl *ctl,
                      i128 *partials, unsigned *counter, int grid, unsigned *status, cudaStream_t s, int so) {
  COUNT_LAUNCH();
  objective_kernel<<<grid, LINK_THREADS, 0, s>>>(g.L, g.c0, kc, f, g.alpha, g.beta, ctl, partials, counter,
                                                 status, so);
}

// f <- f + alpha* (g - f) when the controller accepted the step
__global__ void update_kernel(int L, const Ctl *ctl, double *f, const long long *__restrict__ g_fx) {
  if (!ctl->do_update) return;
  const double alpha = ctl->alpha_final;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x)
    f[a] = step_flow(f[a], fx64_to_double(g_fx[a]), alpha);
}

void launch_update(const GraphDev &g, Ctl *ctl, double *f, const long long *g_fx, cudaStream_t s) {
  if (g.L == 0) return;
  COUNT_LAUNCH();
  update_kernel<<<link_grid(g, g.L), LINK_THREADS, 0, s>>>(g.L, ctl, f, g_fx);
}

__global__ void tape_record_kernel(int L, const Ctl *ctl, const int *q, const double *f, int *tape_q,
                                   double *tape_alpha, double *tape_f, int cap) {
  if (!ctl->do_update) return;
  const int k = ctl->k;
  if (k >= cap) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) tape_alpha[k] = ctl->alpha_final;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    tape_q[(long long)k * L + a] = q[a];
    if (tape_f) tape_f[(long long)k * L + a] = f[a];
  }
}

void launch_tape_record(const GraphDev &g, const Ctl *ctl, const int *q, const double *f,
                        int *tape_q, double *tape_alpha, double *tape_f, int cap, cudaStream_t s) {
  COUNT_LAUNCH();
  tape_record_kernel<<<link_grid(g, g.L > 0 ? g.L : 1), 256, 0, s>>>(g.L, ctl, q, f, tape_q,
                                                                     tape_alpha, tape_f, cap);
}

// ============================================================================
// device controller (one thread): Alg. 2 / 6 loop and the step rules
// ============================================================================

__device__ void plan_set(Ctl *c, int n, int kind, const double *alphas, int want_gap) {
  c->plan.n = n;
  c->plan.want_gap = want_gap;
  for (int m = 0; m < MAX_SLOTS; ++m) {
    c->plan.kind[m] = kind;
    c->plan.alpha[m] = m < n ? alphas[m] : 0.0;
  }
}

__device__ void plan_qn(Ctl *c, int want_gap) {
  double a[3] = {sub(c->alpha, c->dx), c->alpha, add(c->alpha, c->dx)};
  plan_set(c, 3, K_PHI, a, want_gap);
}

__device__ void finish_ls(Ctl *c, double alpha) {
  c->alpha_final = alpha;
  c->ls_passes += c->ls_pc;
  if (c->stop == 1) {  // PAPER_OBJ: compare C(f) and C(f_new)
    double a[2] = {0.0, alpha};
    plan_set(c, 2, K_PHI, a, 0);
    c->ls_state = LS_OBJ;
    c->need_sweep = 1;
  } else {
    c->do_update = 1;
    c->need_sweep = 0;
    c->ls_state = LS_IDLE;
  }
}

__device__ void sweep8_next_or_finish(Ctl *c) {
  if (sub(c->hi, c->lo) >= c->t2 && c->ls_pc < c->ls_max) {
    const double step = dvd(sub(c->hi, c->lo), 9.0);
    double a[8];
    for (int m = 0; m < 8; ++m) a[m] = add(c->lo, mul(step, (double)(m + 1)));
    plan_set(c, 8, K_DPHI, a, 0);
    c->ls_state = LS_SW_NEXT;
    c->need_sweep = 1;
  } else {
    const double dlo = fx_to_double(c->Dlo), dhi = fx_to_double(c->Dhi);
    double alpha = add(c->lo, mul(sub(c->hi, c->lo), dvd(-dlo, sub(dhi, dlo))));
    if (alpha < c->lo) alpha = c->lo;
    if (alpha > c->hi) alpha = c->hi;
    finish_ls(c, alpha);
  }
}

__global__ void ctl_init_kernel(Ctl *c, int step, int stop, int max_iter, int ls_max, double tol,
                                double dx, double t1, double t2, int ring, long long n_host,
                                const long long *n_dev, int gap_on) {
  const long long n = n_dev ? *n_dev : n_host;
  c->step = step; c->stop = stop; c->max_iter = max_iter; c->ls_max = ls_max;
  c->tol = tol; c->dx = dx; c->t1 = t1; c->t2 = t2;
  c->k = 1;
  c->fw_continue = max_iter >= 1;
  c->notconv = (max_iter < 1 && stop != 0) ? 1 : 0;
  c->need_sweep = 0; c->do_update = 0; c->converged = 0;
  c->iterations = 0; c->aon_calls = 1; c->ls_passes = 0;
  c->ls_state = LS_IDLE; c->ls_pc = 0; c->l = 0; c->ex_it = 0;
  c->rel_gap = __longlong_as_double(0x7ff8000000000000ll);
  c->dual_gap = c->rel_gap;
  c->alpha = c->alpha_final = 0.0;
  c->objective = 0.0;
  c->plan.n = 0; c->plan.want_gap = 0;
  c->ring = ring;
  c->gap_on = gap_on;
  c->tree_slot = ring > 1 ? 1 : 0;
  if (n <= 0) {  // no demand: zero flows, converged at once
    c->fw_continue = 0; c->notconv = 0; c->converged = 1; c->aon_calls = 0;
    c->rel_gap = 0.0;
    c->dual_gap = 0.0;
  }
}

void launch_ctl_init(Ctl *ctl, int step, int stop, int max_iter, int ls_max, double tol, double dx,
                     double t1, double t2, int ring, long long n_items_host,
                     const long long *n_items_dev, int gap_on, cudaStream_t s) {
  COUNT_LAUNCH();
  ctl_init_kernel<<<1, 1, 0, s>>>(ctl, step, stop, max_iter, ls_max, tol, dx, t1, t2, ring,
                                  n_items_host, n_items_dev, gap_on);
}

// after the all-or-nothing of iteration k: set up the step rule
__global__ void ctl_begin_kernel(Ctl *c, cudaGraphConditionalHandle h_ls, int use_cond) {
  c->aon_calls++;
  c->ls_pc = 0;
  c->do_update = 0;
  c->need_sweep = 0;
  // the duality gap is measured on the first sweep of every iteration of a
  // FW solve (a stand-alone line search has no link times to measure it with)
  const int gap = c->gap_on;
  switch (c->step) {
    case 0:  // MSA
      c->alpha = dvd(1.0, add((double)c->k, 1.0));
      if (gap) { plan_set(c, 0, K_PHI, nullptr, 1); c->ls_state = LS_GAPONLY; c->need_sweep = 1; }
      else finish_ls(c, c->alpha);
      break;
    case 1:  // PAPER_QN3
      c->alpha = dvd(2.0, add(2.0, (double)(c->k - 1)));
      c->l = 1;
      if (c->ls_max > 1) { plan_qn(c, gap); c->ls_state = LS_QN; c->need_sweep = 1; }
      else if (gap) { plan_set(c, 0, K_PHI, nullptr, 1); c->ls_state = LS_GAPONLY; c->need_sweep = 1; }
      else finish_ls(c, c->alpha);
      break;
    case 2: {  // SWEEP8
      double a[8];
      for (int m = 0; m < 8; ++m) a[m] = dvd((double)m, 7.0);
      plan_set(c, 8, K_DPHI, a, gap);
      c->ls_state = LS_SW_FIRST;
      c->need_sweep = 1;
      break;
    }
    default: {  // EXACT
      double a[2] = {0.0, 1.0};
      plan_set(c, 2, K_DPHI, a, gap);
      c->ls_state = LS_EX_END;
      c->need_sweep = 1;
      break;
    }
  }
  if (use_cond) cudaGraphSetConditional(h_ls, c->need_sweep ? 1u : 0u);
}

void launch_ctl_begin(Ctl *ctl, unsigned long long cond_ls, int use_cond, cudaStream_t s) {
  COUNT_LAUNCH();
  ctl_begin_kernel<<<1, 1, 0, s>>>(ctl, (cudaGraphConditionalHandle)cond_ls, use_cond);
}

// after a sweep: consume the sums
__global__ void ctl_step_kernel(Ctl *c, cudaGraphConditionalHandle h_ls, int use_cond) {
  c->need_sweep = 0;
  if (c->plan.want_gap) {
    const i128 A = c->sums[MAX_SLOTS], B = c->sums[MAX_SLOTS + 1];
    c->dual_gap = dvd(fx_to_double(A - B), fx_to_double(A));
    c->plan.want_gap = 0;
    if (c->stop == 2) c->rel_gap = c->dual_gap;
    // a negative gap (truncated loading: g need not minimise sum c g) is no
    // certificate and does not stop; -1e-12 is rounding at an exact
    // all-or-nothing equilibrium
    if (c->stop == 2 && c->rel_gap <= c->tol && c->rel_gap >= -1e-12) {
      c->converged = 1;
      c->fw_continue = 0;
      c->do_update = 0;
      c->ls_state = LS_IDLE;
      if (use_cond) cudaGraphSetConditional(h_ls, 0u);
      return;
    }
  }
  const i128 *S = c->sums;
  switch (c->ls_state) {
    case LS_GAPONLY:
      finish_ls(c, c->alpha);
      break;
    case LS_QN: {
      c->ls_pc++;
      const double c0 = fx_to_double(S[1]);
      const double d1 = dvd(fx_to_double(S[2] - S[0]), mul(2.0, c->dx));
      const double d2 = dvd(fx_to_double(S[0] - 2 * S[1] + S[2]), mul(c->dx, c->dx));
      if (fabs(d1) < mul(c->t1, fabs(c0))) { finish_ls(c, c->alpha); break; }
      double an;
      if (d2 > 0.0) an = sub(c->alpha, dvd(d1, d2));
      else an = d1 < 0.0 ? 1.0 : 0.0;
      if (an < 0.0) an = 0.0;
      if (an > 1.0) an = 1.0;
      if (fabs(sub(an, c->alpha)) < c->t2) { finish_ls(c, an); break; }
      c->alpha = an;
      c->l++;
      if (c->l < c->ls_max) { plan_qn(c, 0); c->need_sweep = 1; }
      else finish_ls(c, c->alpha);
      break;
    }
    case LS_SW_FIRST: {
      c->ls_pc++;
      if (S[7] <= 0) { finish_ls(c, 1.0); break; }
      if (S[0] >= 0) { finish_ls(c, 0.0); break; }
      int ms = 1;
      while (S[ms] < 0) ++ms;
      c->lo = c->plan.alpha[ms - 1]; c->Dlo = S[ms - 1];
      c->hi = c->plan.alpha[ms]; c->Dhi = S[ms];
      sweep8_next_or_finish(c);
      break;
    }
    case LS_SW_NEXT: {
      c->ls_pc++;
      int mf = 0;
      while (mf < 8 && S[mf] < 0) ++mf;
      if (mf == 8) { c->lo = c->plan.alpha[7]; c->Dlo = S[7]; }
      else {
        c->hi = c->plan.alpha[mf]; c->Dhi = S[mf];
        if (mf > 0) { c->lo = c->plan.alpha[mf - 1]; c->Dlo = S[mf - 1]; }
      }
      sweep8_next_or_finish(c);
      break;
    }
    case LS_EX_END: {
      c->ls_pc += 2;
      if (S[1] <= 0) { finish_ls(c, 1.0); break; }
      if (S[0] >= 0) { finish_ls(c, 0.0); break; }
      c->lo = 0.0; c->hi = 1.0; c->alpha = 0.5; c->ex_it = 0;
      double a[2] = {0.5, 0.5};
      plan_set(c, 2, K_DPHI, a, 0);
      c->plan.kind[1] = K_DDPHI;
      c->ls_state = LS_EX_NEWTON;
      c->need_sweep = 1;
      break;
    }
    case LS_EX_NEWTON: {
      c->ls_pc++;
      const i128 D = S[0];
      const double H = fx_to_double(S[1]);
      if (D == 0) { finish_ls(c, c->alpha); break; }
      if (D < 0) c->lo = c->alpha; else c->hi = c->alpha;
      double an = (H > 0.0) ? sub(c->alpha, dvd(fx_to_double(D), H)) : mul(0.5, add(c->lo, c->hi));
      if (!(an > c->lo && an < c->hi)) an = mul(0.5, add(c->lo, c->hi));
      if (fabs(sub(an, c->alpha)) < 1e-14 || sub(c->hi, c->lo) < 1e-15) { finish_ls(c, an); break; }
      c->alpha = an;
      c->ex_it++;
      if (c->ex_it >= 200) { finish_ls(c, c->alpha); break; }
      double a[2] = {an, an};
      plan_set(c, 2, K_DPHI, a, 0);
      c->plan.kind[1] = K_DDPHI;
      c->need_sweep = 1;
      break;
    }
    case LS_OBJ: {
      const double rel = dvd(fabs(fx_to_double(S[0] - S[1])), fx_to_double(S[0]));
      c->rel_gap = rel;
      if (rel < c->tol) { c->converged = 1; c->fw_continue = 0; c->do_update = 0; }
      else c->do_update = 1;
      c->ls_state = LS_IDLE;
      break;
    }
    default:
      break;
  }
  if (use_cond) cudaGraphSetConditional(h_ls, c->need_sweep ? 1u : 0u);
}

void launch_ctl_step(Ctl *ctl, unsigned long long cond_ls, int use_cond, cudaStream_t s) {
  COUNT_LAUNCH();
  ctl_step_kernel<<<1, 1, 0, s>>>(ctl, (cudaGraphConditionalHandle)cond_ls, use_cond);
}

// copy a controller flag into a conditional handle (graph schedules)
__global__ void set_cond_kernel(const Ctl *c, int which, cudaGraphConditionalHandle h) {
  const int v = which == 0 ? c->fw_continue : which == 1 ? c->need_sweep : c->res_continue;
  cudaGraphSetConditional(h, v ? 1u : 0u);
}

void launch_set_cond(const Ctl *ctl, int which, unsigned long long cond, cudaStream_t s) {
  COUNT_LAUNCH();
  set_cond_kernel<<<1, 1, 0, s>>>(ctl, which, (cudaGraphConditionalHandle)cond);
}

// after the update of iteration k
__global__ void ctl_end_kernel(Ctl *c, cudaGraphConditionalHandle h_fw, int use_cond) {
  if (c->do_update) {
    c->iterations = c->k;
    c->k++;
    if (c->k > c->max_iter) {
      c->fw_continue = 0;
      if (c->stop != 0) c->notconv = 1;
    }
  }
  if (c->converged) c->fw_continue = 0;
  c->tree_slot = c->k < c->ring - 1 ? c->k : c->ring - 1;
  if (use_cond) cudaGraphSetConditional(h_fw, c->fw_continue ? 1u : 0u);
}

void launch_ctl_end(Ctl *ctl, unsigned long long cond_fw, int use_cond, cudaStream_t s) {
  COUNT_LAUNCH();
  ctl_end_kernel<<<1, 1, 0, s>>>(ctl, (cudaGraphConditionalHandle)cond_fw, use_cond);
}

// w_j = alpha_j prod_{m > j} (1 - alpha_m), alpha_0 = 1 (Alg. 4 path weights)
__global__ void path_weights_kernel(const Ctl *c, const double *tape_alpha, double *w) {
  const int K = c->iterations;
  double P = 1.0;
  for (int j = K; j >= 0; --j) {
    const double a = j == 0 ? 1.0 : tape_alpha[j];
    w[j] = mul(a, P);
    P = mul(P, sub(1.0, a));
  }
}

void launch_path_weights(const Ctl *ctl, const double *tape_alpha, double *w, cudaStream_t s) {
  COUNT_LAUNCH();
  path_weights_kernel<<<1, 1, 0, s>>>(ctl, tape_alpha, w);
}

__global__ void weight_select_kernel(const double *w, int j, double *dst) { *dst = w[j]; }

void launch_weight_select(const double *w, int j, double *dst, cudaStream_t s) {
  COUNT_LAUNCH();
  weight_select_kernel<<<1, 1, 0, s>>>(w, j, dst);
}

__global__ void fill_i32_kernel(int *p, long long n, int v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

void launch_fill_i32(int *p, long long n, int v, cudaStream_t s) {
  if (n <= 0) return;
  long long b = (n + 255) / 256;
  if (b > 4096) b = 4096;
  COUNT_LAUNCH();
  fill_i32_kernel<<<(int)b, 256, 0, s>>>(p, n, v);
}

// initial AON recorded as step 0 of the tape: q_0, alpha_0 = 1, f_0 = g_0
__global__ void tape0_kernel(int L, const int *q, const double *f, int *tape_q, double *tape_alpha,
                             double *tape_f) {
  if (blockIdx.x == 0 && threadIdx.x == 0) tape_alpha[0] = 1.0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    tape_q[a] = q[a];
    if (tape_f) tape_f[a] = f[a];
  }
}

void launch_tape0(const GraphDev &g, const int *q, const double *f, int *tape_q, double *tape_alpha,
                  double *tape_f, cudaStream_t s) {
  COUNT_LAUNCH();
  tape0_kernel<<<link_grid(g, g.L > 0 ? g.L : 1), 256, 0, s>>>(g.L, q, f, tape_q, tape_alpha, tape_f);
}

// residual loop over the accepted AONs j = 0..K
__global__ void res_begin_kernel(Ctl *c, cudaGraphConditionalHandle h, int use_cond) {
  c->res_j = 0;
  c->res_continue = c->aon_calls > 0;  // an interval without demand has nothing to re-walk
  if (use_cond) cudaGraphSetConditional(h, c->res_continue ? 1u : 0u);
}

void launch_res_begin(Ctl *ctl, unsigned long long cond, int use_cond, cudaStream_t s) {
  COUNT_LAUNCH();
  res_begin_kernel<<<1, 1, 0, s>>>(ctl, (cudaGraphConditionalHandle)cond, use_cond);
}

// tree j is still in ring slot j when j < ring - 1; otherwise it is rebuilt
// into the last slot from the taped link times (copied to q_work here)
__global__ void res_prep_kernel(Ctl *c, const double *w, const int *tape_q, int L, int *q_work) {
  const int j = c->res_j;
  const int stored = j < c->ring - 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->res_slot = stored ? j : c->ring - 1;
    c->res_skip = stored;
    c->w_cur = w[j];
  }
  if (!stored)
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x)
      q_work[a] = tape_q[(long long)j * L + a];
}

void launch_res_prep(Ctl *ctl, const double *w, const int *tape_q, int L, int *q_work, cudaStream_t s) {
  int b = (L + 255) / 256;
  if (b > 2048) b = 2048;
  if (b < 1) b = 1;
  COUNT_LAUNCH();
  res_prep_kernel<<<b, 256, 0, s>>>(ctl, w, tape_q, L, q_work);
}

__global__ void res_next_kernel(Ctl *c, cudaGraphConditionalHandle h, int use_cond) {
  c->res_j++;
  c->res_continue = c->res_j <= c->iterations;
  if (use_cond) cudaGraphSetConditional(h, c->res_continue ? 1u : 0u);
}

void launch_res_next(Ctl *ctl, unsigned long long cond, int use_cond, cudaStream_t s) {
  COUNT_LAUNCH();
  res_next_kernel<<<1, 1, 0, s>>>(ctl, (cudaGraphConditionalHandle)cond, use_cond);
}

// h(i) row and the interval's statistics
__global__ void store_interval_kernel(int L, const Ctl *c, const unsigned long long *h_fx,
                                      double *rows, qdta_stats *stats, const long long *n_items) {
  const int i = c->day_i;
  double *row = rows + (long long)i * L;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x)
    row[a] = fx64_to_double((long long)h_fx[a]);
  if (blockIdx.x == 0 && threadIdx.x == 0 && stats) {
    qdta_stats st;
    st.iterations = c->iterations;
    st.aon_calls = c->aon_calls;
    st.ls_passes = c->ls_passes;
    st.converged = c->converged;
    st.rel_gap = c->rel_gap;
    st.objective = c->objective;
    st.n_items = n_items ? *n_items : 0;
    st.dual_gap = c->dual_gap;
    stats[i] = st;
  }
}

void launch_store_interval(const GraphDev &g, const Ctl *ctl, const unsigned long long *h_fx,
                           double *flow_out_rows, void *stats_rows, const long long *n_items_dev,
                           cudaStream_t s) {
  COUNT_LAUNCH();
  store_interval_kernel<<<link_grid(g, g.L > 0 ? g.L : 1), 256, 0, s>>>(
      g.L, ctl, h_fx, flow_out_rows, (qdta_stats *)stats_rows, n_items_dev);
}

__global__ void day_next_kernel(Ctl *c, cudaGraphConditionalHandle h, int use_cond) {
  c->day_i++;
  c->day_continue = c->day_i < c->day_N;
  if (use_cond) cudaGraphSetConditional(h, c->day_continue ? 1u : 0u);
}

void launch_day_next(Ctl *ctl, unsigned long long cond, int use_cond, cudaStream_t s) {
  COUNT_LAUNCH();
  day_next_kernel<<<1, 1, 0, s>>>(ctl, (cudaGraphConditionalHandle)cond, use_cond);
}

// one demand item into the merge: waiting at src -> the dense (root, node)
// accumulator; on a link -> the carried table
__device__ __forceinline__ void scatter_one(int V, int L, int r, int src, long long a, long long frac, int link,
                                            unsigned long long *dense, const CarryAcc &ca, unsigned *status) {
  if (!a) return;
  if (link >= 0) carry_add(ca, r, L, link, frac, a, status);
  else atomicAdd(&dense[(long long)r * V + src], (unsigned long long)a);
}

// original demand of the current interval into the merge
__global__ void scatter_orig_kernel(int V, int L, const Ctl *c, const OrigTable *tab,
                                    unsigned long long *dense, CarryAcc ca, unsigned *status) {
  const OrigTable t = tab[c->day_i];
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < t.n;
       k += (long long)gridDim.x * blockDim.x) {
    const int link = t.carry_link ? t.carry_link[k] : -1;
    scatter_one(V, L, t.root_idx[k], t.src[k], t.amount[k], link >= 0 && t.carry ? t.carry[k] : 0, link, dense,
                ca, status);
  }
}

void launch_scatter_orig(const GraphDev &g, const Ctl *ctl, const OrigTable *tab, long long max_n,
                         unsigned long long *dense, cudaStream_t s, CarryAcc ca, unsigned *status) {
  COUNT_LAUNCH();
  scatter_orig_kernel<<<link_grid(g, max_n > 0 ? max_n : 1), 256, 0, s>>>(g.V, g.L, ctl, tab, dense, ca,
                                                                          status);
}

// ============================================================================
// residual-demand merge: dense (root, node) accumulator -> sorted items
// ============================================================================

__global__ void scatter_items_kernel(int V, int L, long long n, const int *root_idx, const int *src,
                                     const long long *amount, unsigned long long *dense,
                                     const long long *carry, const int *carry_link, CarryAcc ca,
                                     unsigned *status) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int link = carry_link ? carry_link[k] : -1;
    scatter_one(V, L, root_idx[k], src[k], amount[k], link >= 0 && carry ? carry[k] : 0, link, dense, ca, status);
  }
}

void launch_scatter_items(const GraphDev &g, long long n, const int *root_idx, const int *src,
                          const long long *amount, unsigned long long *dense, cudaStream_t s,
                          const long long *carry, const int *carry_link, CarryAcc ca, unsigned *status) {
  if (n <= 0) return;
  COUNT_LAUNCH();
  scatter_items_kernel<<<link_grid(g, n), 256, 0, s>>>(g.V, g.L, n, root_idx, src, amount, dense, carry,
                                                       carry_link, ca, status);
}

constexpr int COMPACT_TILE = 4096;

__global__ void compact_count_kernel(long long total, const unsigned long long *dense, int *blk_count) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * COMPACT_TILE;
  int c = 0;
  for (int i = threadIdx.x; i < COMPACT_TILE; i += blockDim.x) {
    const long long idx = base + i;
    if (idx < total && dense[idx] != 0ull) ++c;
  }
  atomicAdd(&s, c);
  __syncthreads();
  if (threadIdx.x == 0) blk_count[blockIdx.x] = s;
}

__global__ void compact_scan_kernel(int nblk, const int *blk_count, long long *blk_off, long long cap,
                                    long long *n_out, unsigned *status, int append) {
  // single block, 1024 threads: chunked exclusive scan; with `append` the
  // offsets start at the count already in *n_out
  __shared__ long long s_part[1024];
  __shared__ long long s_base;
  if (threadIdx.x == 0) s_base = append ? *n_out : 0;
  const int per = (nblk + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  long long t = 0;
  for (int i = 0; i < per; ++i) if (b0 + i < nblk) t += blk_count[b0 + i];
  s_part[threadIdx.x] = t;
  __syncthreads();
  for (int d = 1; d < 1024; d <<= 1) {
    long long v = threadIdx.x >= d ? s_part[threadIdx.x - d] : 0;
    __syncthreads();
    s_part[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = s_base + s_part[threadIdx.x] - t;
  for (int i = 0; i < per; ++i) {
    if (b0 + i < nblk) { blk_off[b0 + i] = run; run += blk_count[b0 + i]; }
  }
  __syncthreads();  // every thread has read s_base before *n_out changes
  if (threadIdx.x == 1023) {
    long long total = s_base + s_part[1023];
    if (total > cap) { atomicOr(status, ST_CAPACITY); total = cap; }
    *n_out = total;
  }
}

// ordered write of the nonzero entries of each tile.  Dense part (keys ==
// NULL): entry root * V + node, written root-major, node-minor, covered fraction
// 0 and link -1.  Carried part: slot order of the table; the key gives
// (root, link), src is the link's tail, the covered fraction is
// floor(sum amount x fraction / amount); keys and sums are cleared.
__global__ void compact_write_kernel(long long total, int V, unsigned long long *dense,
                                     const long long *blk_off, long long cap, int *root_idx,
                                     int *src, long long *amount, long long *carry_out,
                                     int *link_out, unsigned long long *keys, unsigned long long *tsum,
                                     int L, const int *__restrict__ tail) {
  __shared__ int s_warp[32];
  const long long base = (long long)blockIdx.x * COMPACT_TILE;
  long long out = blk_off[blockIdx.x];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c0 = 0; c0 < COMPACT_TILE; c0 += blockDim.x) {
    const long long idx = base + c0 + threadIdx.x;
    unsigned long long v = 0ull, key = CARRY_KEY_EMPTY;
    if (idx < total) {
      v = dense[idx];
      if (keys) {
        key = keys[idx];
        keys[idx] = CARRY_KEY_EMPTY;
      }
    }
    const bool nz = v != 0ull;
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) s_warp[wid] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < nw; ++w) { if (w < wid) before += s_warp[w]; all += s_warp[w]; }
    if (nz) {
      const long long pos = out + before + __popc(m & ((1u << lane) - 1u));
      long long frac = 0;
      int r, node, link = -1;
      if (keys) {
        const u128 t = ((u128)tsum[2 * idx + 1] << 32) + (u128)tsum[2 * idx];
        frac = (long long)(t / (u128)v);
        tsum[2 * idx] = 0ull;
        tsum[2 * idx + 1] = 0ull;
        r = (int)(key / (unsigned long long)L);
        link = (int)(key % (unsigned long long)L);
        node = __ldg(&tail[link]);
      } else {
        r = (int)(idx / V);
        node = (int)(idx % V);
      }
      if (pos < cap) {
        root_idx[pos] = r;
        src[pos] = node;
        amount[pos] = (long long)v;
        if (carry_out) carry_out[pos] = frac;
        if (link_out) link_out[pos] = link;
      }
      dense[idx] = 0ull;
    }
    out += all;
    __syncthreads();
  }
}

void launch_compact(const GraphDev &g, int R, unsigned long long *dense, int *blk_count,
                    long long *blk_off, long long cap, int *root_idx, int *src, long long *amount,
                    long long *n_out_dev, unsigned *status, cudaStream_t s, long long *carry_out,
                    int *link_out, CarryAcc ca) {
  for (int part = 0; part < (ca.mask ? 2 : 1); ++part) {
    const long long total = part == 0 ? (long long)R * g.V : (long long)ca.mask + 1;
    const int nblk = cdiv(total > 0 ? total : 1, COMPACT_TILE);
    unsigned long long *src_acc = part == 0 ? dense : ca.amt;
    COUNT_LAUNCH();
    compact_count_kernel<<<nblk, 256, 0, s>>>(total, src_acc, blk_count);
    COUNT_LAUNCH();
    compact_scan_kernel<<<1, 1024, 0, s>>>(nblk, blk_count, blk_off, cap, n_out_dev, status, part);
    COUNT_LAUNCH();
    compact_write_kernel<<<nblk, 256, 0, s>>>(total, g.V, src_acc, blk_off, cap, root_idx, src, amount, carry_out,
                                              link_out, part == 0 ? nullptr : ca.key,
                                              part == 0 ? nullptr : ca.tsum, g.L, g.tail);
  }
}

// roots with at least one item, in root order; root_slot maps a root index
// to its row in the parent arrays (or -1)
// ============================================================================
// scenario metrics (Section 7.1): per interval and class, over links with flow
// ============================================================================


// acc [N][C][16] words: pairs (lo, hi) at 0 VMT (veh-m), 2 VOC, 4 delay (veh
// x quanta), 6 congested length (m), 8 congested VMT, 10 congested VOC; 12
// links with flow, 13 congested links.  blockIdx.y = interval.
__global__ void __launch_bounds__(256)
metrics_kernel(int L, const double *__restrict__ flows, const double *__restrict__ length_m,
               const int *__restrict__ link_class, int C, const int *__restrict__ c0, const double *__restrict__ cap,
               double dt_h, double alpha, int beta, double congested_voc, unsigned long long *acc,
               unsigned *status) {
  __shared__ unsigned long long s[16 * 16];
  const int i = blockIdx.y;
  for (int t = threadIdx.x; t < C * 16; t += blockDim.x) s[t] = 0ull;
  __syncthreads();
  unsigned bad = 0;
  const double *fi = flows + (long long)i * L;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    const double f = fi[a];
    if (!isfinite(f)) { bad |= ST_NONFINITE; continue; }
    const int k = link_class[a];
    if (!(f > 0.0) || k < 0 || k >= C) continue;
    const LinkConst kc = link_const(cap[a], dt_h, alpha, beta);
    const double x = mul(f, kc.inv);
    const double c0a = (double)c0[a];
    const double d = sub(link_cost(c0a, kc.inv, alpha, beta, f), c0a);
    const double fl = mul(f, length_m[a]);
    unsigned long long *sk = s + k * 16;
    add_u128(sk + 0, (u128)fx_of(fl, &bad));
    add_u128(sk + 2, (u128)fx_of(x, &bad));
    add_u128(sk + 4, (u128)fx_of(mul(f, d), &bad));
    atomicAdd(sk + 12, 1ull);
    if (x >= congested_voc) {
      add_u128(sk + 6, (u128)fx_of(length_m[a], &bad));
      add_u128(sk + 8, (u128)fx_of(fl, &bad));
      add_u128(sk + 10, (u128)fx_of(x, &bad));
      atomicAdd(sk + 13, 1ull);
    }
  }
  if (bad) atomicOr(status, bad);
  __syncthreads();
  unsigned long long *g = acc + (long long)i * C * 16;
  for (int t = threadIdx.x; t < C * 16; t += blockDim.x) {
    const int w = t & 15;
    if (w < 12 && (w & 1) == 0) {
      const u128 v = ((u128)s[t + 1] << 64) | s[t];
      if (v) add_u128(g + t, v);
    } else if (w == 12 || w == 13) {
      if (s[t]) atomicAdd(g + t, s[t]);
    }
  }
}

// out [N][C][8]: links, VMT km, mean VOC, VHD h, congested links, congested
// km, congested VMT km, congested mean VOC
__global__ void metrics_finish_kernel(int NC, const unsigned long long *__restrict__ acc, double hours_per_quantum,
                                      double *__restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NC) return;
  const unsigned long long *w = acc + (long long)t * 16;
  auto total = [&](int k) { return fx_to_double((i128)(((u128)w[k + 1] << 64) | w[k])); };
  const unsigned long long n = w[12], cn = w[13];
  double *o = out + (long long)t * 8;
  o[0] = __ull2double_rn(n);
  o[1] = mul(total(0), 1e-3);
  o[2] = n ? dvd(total(2), __ull2double_rn(n)) : 0.0;
  o[3] = mul(total(4), hours_per_quantum);
  o[4] = __ull2double_rn(cn);
  o[5] = mul(total(6), 1e-3);
  o[6] = mul(total(8), 1e-3);
  o[7] = cn ? dvd(total(10), __ull2double_rn(cn)) : 0.0;
}

void launch_metrics(const GraphDev &g, const double *flows, int N, double dt_h, const double *length_m,
                    const int *link_class, int C, double congested_voc, unsigned long long *acc, double *out,
                    unsigned *status, cudaStream_t s) {
  if (N <= 0) return;
  if (g.L > 0) {
    COUNT_LAUNCH();
    const int bx = (int)std::min<long long>(cdiv(g.L, 256), 4ll * g.num_sms);
    metrics_kernel<<<dim3(bx, N), 256, 0, s>>>(g.L, flows, length_m, link_class, C, g.c0, g.cap, dt_h, g.alpha,
                                               g.beta, congested_voc, acc, status);
  }
  COUNT_LAUNCH();
  metrics_finish_kernel<<<cdiv((long long)N * C, 128), 128, 0, s>>>(N * C, acc, g.quantum_s / 3600.0, out);
}

// copy free-flow tree rows into the rows of the active roots (row r ->
// root_slot[r]); int4 copies when rows are 16-byte aligned
__global__ void gather_rows_kernel(const int *__restrict__ src, int V, const int *__restrict__ root_slot,
                                   int *__restrict__ parent, const int *slot_dev, long long slot_stride) {
  const int r = blockIdx.x;
  const int k = root_slot[r];
  if (k < 0) return;
  int *dst = parent + (slot_dev ? (long long)(*slot_dev) * slot_stride : 0ll) + (long long)k * V;
  const int *row = src + (long long)r * V;
  if ((V & 3) == 0 && (reinterpret_cast<size_t>(dst) & 15) == 0 && (reinterpret_cast<size_t>(row) & 15) == 0) {
    const int4 *a = reinterpret_cast<const int4 *>(row);
    int4 *b = reinterpret_cast<int4 *>(dst);
    for (int i = threadIdx.x; i < (V >> 2); i += blockDim.x) b[i] = __ldcs(&a[i]);
  } else {
    for (int i = threadIdx.x; i < V; i += blockDim.x) dst[i] = row[i];
  }
}

void launch_gather_rows(const int *src, int rows, int V, const int *root_slot, int *parent, const int *slot_dev,
                        long long slot_stride, cudaStream_t s) {
  if (rows <= 0 || V <= 0) return;
  COUNT_LAUNCH();
  gather_rows_kernel<<<rows, 256, 0, s>>>(src, V, root_slot, parent, slot_dev, slot_stride);
}

__global__ void active_roots_kernel(int R, const long long *n_dev, long long cap, const int *root_idx,
                                    const int *zone_nodes, int *flag, int *active, int *root_slot,
                                    int *n_active) {
  // single block
  for (int r = threadIdx.x; r < R; r += blockDim.x) flag[r] = 0;
  __syncthreads();
  long long n = *n_dev;
  if (n > cap) n = cap;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) flag[root_idx[k]] = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int r = 0; r < R; ++r) {
      if (flag[r]) { active[c] = zone_nodes[r]; root_slot[r] = c; ++c; }
      else root_slot[r] = -1;
    }
    *n_active = c;
  }
}

void launch_active_roots(int R, const long long *n_items_dev, long long cap_items, const int *root_idx,
                         const int *zone_nodes, int *flag, int *active_roots, int *root_slot,
                         int *n_active_dev, cudaStream_t s) {
  COUNT_LAUNCH();
  active_roots_kernel<<<1, 1024, 0, s>>>(R, n_items_dev, cap_items, root_idx, zone_nodes, flag,
                                         active_roots, root_slot, n_active_dev);
}

// ============================================================================
// adjoint
// ============================================================================

// mu = sum lam (g - f_prev), H = sum (g - f_prev)^2 c'(t)   (double, fixed order)
__global__ void __launch_bounds__(LINK_THREADS)
adj_reduce_kernel(int L, const int *__restrict__ c0, const LinkConst *__restrict__ kc, double alpha_bpr,
                  int beta, const double *lam, const double *fprev, const long long *g_fx,
                  double alpha, int implicit, double *partials, double *out2) {
  __shared__ double s_mu[LINK_THREADS / 32], s_h[LINK_THREADS / 32];
  double mu = 0.0, H = 0.0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    const double gg = fx64_to_double(g_fx[a]);
    const double d = sub(gg, fprev[a]);
    mu = add(mu, mul(lam[a], d));
    if (implicit) {
      const double t = step_flow(fprev[a], gg, alpha);
      H = add(H, mul(mul(d, d), link_cost_dt((double)c0[a], kc[a].inv, alpha_bpr, beta, t)));
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    mu = add(mu, __shfl_down_sync(0xffffffffu, mu, d));
    H = add(H, __shfl_down_sync(0xffffffffu, H, d));
  }
  if ((threadIdx.x & 31) == 0) { s_mu[threadIdx.x >> 5] = mu; s_h[threadIdx.x >> 5] = H; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < LINK_THREADS / 32; ++w) { a = add(a, s_mu[w]); b = add(b, s_h[w]); }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

__global__ void adj_finish_kernel(int nblk, const double *partials, double *out2) {
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nblk; ++i) { a = add(a, partials[2 * i]); b = add(b, partials[2 * i + 1]); }
  out2[0] = a;
  out2[1] = b;
}

void launch_adj_reduce(const GraphDev &g, const LinkConst *kc, const double *lam, const double *fprev,
                       const long long *g_fx, double alpha, int implicit, double *partials, double *out2,
                       int grid, cudaStream_t s) {
  COUNT_LAUNCH();
  adj_reduce_kernel<<<grid, LINK_THREADS, 0, s>>>(g.L, g.c0, kc, g.alpha, g.beta, lam, fprev, g_fx,
                                                  alpha, implicit, partials, out2);
  COUNT_LAUNCH();
  adj_finish_kernel<<<1, 1, 0, s>>>(grid, partials, out2);
}

// g_bar = alpha lam - mu dalpha/dg, lam_prev = (1 - alpha) lam - mu dalpha/df,
// dcap += -mu dalpha/dC, with dalpha/dtheta = -(d phi'/d theta) / H
__global__ void adj_update_kernel(int L, const int *__restrict__ c0, const double *__restrict__ cap,
                                  const LinkConst *__restrict__ kc, double alpha_bpr, int beta,
                                  const double *lam, const double *fprev, const long long *g_fx,
                                  double alpha, int implicit, const double *muH, double *gbar,
                                  double *lam_prev, double *dcap) {
  const double mu = muH[0], H = muH[1];
  const int imp = implicit && H > 0.0;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < L; a += gridDim.x * blockDim.x) {
    const double la = lam[a];
    double gb = mul(alpha, la);
    double lp = mul(sub(1.0, alpha), la);
    if (imp) {
      const double gg = fx64_to_double(g_fx[a]);
      const double fp = fprev[a];
      const double d = sub(gg, fp);
      const double t = step_flow(fp, gg, alpha);
      const double c0a = (double)c0[a];
      const double c = link_cost(c0a, kc[a].inv, alpha_bpr, beta, t);
      const double cp = link_cost_dt(c0a, kc[a].inv, alpha_bpr, beta, t);
      const double r = dvd(mu, H);
      gb = sub(gb, mul(r, add(c, mul(mul(alpha, d), cp))));
      lp = sub(lp, mul(r, add(-c, mul(mul(sub(1.0, alpha), d), cp))));
      // d c / d C = -c0 alpha beta x^beta / C
      const double x = mul(t, kc[a].inv);
      const double dcdC = -dvd(mul(mul(mul(c0a, alpha_bpr), (double)beta), powi(x, beta)), cap[a]);
      dcap[a] = sub(dcap[a], mul(r, mul(d, dcdC)));
    }
    gbar[a] = gb;
    lam_prev[a] = lp;
  }
}

void launch_adj_update(const GraphDev &g, const LinkConst *kc, const double *lam, const double *fprev,
                       const long long *g_fx, double alpha, int implicit, const double *muH,
                       double *gbar, double *lam_prev, double *dcap, cudaStream_t s) {
  if (g.L == 0) return;
  COUNT_LAUNCH();
  adj_update_kernel<<<link_grid(g, g.L), LINK_THREADS, 0, s>>>(g.L, g.c0, g.cap, kc, g.alpha, g.beta,
                                                               lam, fprev, g_fx, alpha, implicit, muH,
                                                               gbar, lam_prev, dcap);
}

// path-sum gather (transpose of the truncated loading): dd[k] += sum of
// gbar over the links item k loads on this tree
__global__ void gather_kernel(int V, const int2 *__restrict__ head_q, const int *__restrict__ parent,
                              const int *__restrict__ roots, long long n, const int *__restrict__ root_idx,
                              const int *__restrict__ src, long long dt_q, const double *__restrict__ gbar,
                              double *dd, unsigned *status, const long long *__restrict__ carry,
                              const int *__restrict__ carry_link) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const int r = root_idx[k];
    const int z = roots[r];
    const int *par = parent + (long long)r * V;
    int u = src[k];
    long long elapsed = 0;
    double acc = 0.0;
    const int cl = carry_link ? carry_link[k] : -1;
    if (cl >= 0 && !finish_carried_link(head_q, cl, carry ? carry[k] : 0, dt_q, u, elapsed))
      continue;  // the rest of the carried link (not loaded), then on from its head
    int steps = 0;
    while (u != z && elapsed < dt_q) {
      const int e = par[u];
      if (e < 0) { atomicOr(status, ST_UNREACH); break; }
      acc = add(acc, gbar[e]);
      const int2 hq = __ldg(&head_q[e]);
      elapsed += hq.y;
      u = hq.x;
      if (++steps > V) { atomicOr(status, ST_TIMEOUT); break; }
    }
    dd[k] = add(dd[k], acc);
  }
}

void launch_gather(const GraphDev &g, const int2 *head_q, const int *parent, const int *roots,
                   long long n_items, const int *root_idx, const int *src, long long dt_q,
                   const double *gbar, double *dd, unsigned *status, cudaStream_t s, const long long *carry,
                   const int *carry_link) {
  if (n_items <= 0) return;
  COUNT_LAUNCH();
  gather_kernel<<<link_grid(g, n_items), 256, 0, s>>>(g.V, head_q, parent, roots, n_items, root_idx,
                                                      src, dt_q, gbar, dd, status, carry, carry_link);
}

}  // namespace qdta
