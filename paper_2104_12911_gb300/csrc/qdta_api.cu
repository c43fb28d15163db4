// qdta_api.cu -- host runtime behind the C ABI of include/qdta.h: graph
// handles, grow-only device workspaces, the plain (host loop) and graph
// (CUDA graph with conditional WHILE nodes) schedules of the interval solve,
// the day driver, the tape and the adjoint driver.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qdta.h"
#include "qdta_internal.cuh"

using namespace qdta;

static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) {                                                           \
      int c_ = (e_ == cudaErrorMemoryAllocation) ? QDTA_ENOMEM : QDTA_ECUDA;           \
      return fail(c_, "%s:%d %s: %s", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
    }                                                                                  \
  } while (0)

#define RC(x)              \
  do {                     \
    int r_ = (x);          \
    if (r_ < 0) return r_; \
  } while (0)

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct ProfEvent {
  int kind;  // 0 sssp, 1 load, 2 sweep
  cudaEvent_t a, b;
  long long roots;
};

struct qdta_graph {
  int device = 0;
  GraphDev d{};
  std::vector<void *> owned;
  unsigned *status = nullptr;
  unsigned *status_h = nullptr;
  void *ctl_h = nullptr;  // pinned mirror of Ctl
  std::map<std::string, Buf> ws;
  bool sssp_smem = false;
  int sssp_bpsm = 1;
  int prof_on = 0;
  qdta_profile prof{};
  unsigned long long *prof_roots = nullptr;  // device counter of roots solved
  std::vector<ProfEvent> pending;
  std::vector<cudaEvent_t> evpool;
  // cell partition (graphs above the shared-memory limit)
  bool has_cells = false;
  CellDev cells{};
  int cell_bpsm = 1;
  long long n_lrev[2] = {0, 0};
  long long n_xrev[2] = {0, 0};
  long long cell_delta = 0;  // near/far width of the cell kernel, in quanta
  int sssp_kind = 0;  // 0 shared-memory BF, 1 cell, 2 global-memory BF
  int bf_bpsm = 0;    // resident CTAs per SM of the global-memory BF (0: as many as fit)
  int bf_lpt = 1;     // dynamic fetch of the queue kernels: longest roots first
  unsigned long long sig = 0;  // graph signature (structure, free-flow times, device) for the tuning cache
};

struct qdta_tape {
  qdta_graph *g = nullptr;
  qdta_od od{};
  double dt_s = 0.0;
  int step = 0;
  int K = 0;
  int *q = nullptr;       // [(K+1) * L]
  double *alpha = nullptr; // [K+1]
  double *f = nullptr;    // [(K+1) * L]
  double *cap = nullptr;  // [L] capacities of the taped solve (the graph's may change later)
};

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Host-side fault injection for tests: QDTA_FAULT=alloc:<n> makes the n-th
// workspace allocation of the process (counting from 1) fail as if the device
// were out of memory.  Nothing is injected on the device.
static bool inject_alloc_fault() {
  static long long target = [] {
    const char *e = getenv("QDTA_FAULT");
    return (e && strncmp(e, "alloc:", 6) == 0) ? atoll(e + 6) : 0ll;
  }();
  static long long seen = 0;
  return target > 0 && ++seen == target;
}

template <class T>
static int ws_get(qdta_graph *g, const std::string &name, size_t count, T **out) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  Buf &b = g->ws[name];
  if (b.bytes < bytes) {
    if (inject_alloc_fault())
      return fail(QDTA_ENOMEM, "device allocation of %zu bytes for '%s' failed (injected)", bytes, name.c_str());
    if (b.p) {
      cudaDeviceSynchronize();
      cudaFree(b.p);
      b.p = nullptr;
      b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(QDTA_ENOMEM, "device allocation of %zu bytes for '%s' failed: %s", bytes,
                  name.c_str(), cudaGetErrorString(e));
    }
    b.bytes = bytes;
  }
  *out = reinterpret_cast<T *>(b.p);
  return QDTA_OK;
}

static int status_reset(qdta_graph *g, cudaStream_t s) {
  CK(cudaMemsetAsync(g->status, 0, sizeof(unsigned), s));
  return QDTA_OK;
}

static int prof_harvest(qdta_graph *g);

// synchronise and translate the device status word
static int status_check(qdta_graph *g, cudaStream_t s) {
  CK(cudaMemcpyAsync(g->status_h, g->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  prof_harvest(g);
  unsigned st = *g->status_h;
  if (st & ST_TIMEOUT) return fail(QDTA_ETIMEOUT, "a bounded device loop reached its limit");
  if (st & ST_NONFINITE)
    return fail(QDTA_ENONFINITE, "non-finite flow/cost or a sum term beyond 2^68");
  if (st & ST_OVERFLOW) return fail(QDTA_EOVERFLOW, "a shortest distance exceeded the packed range");
  if (st & ST_UNREACH) return fail(QDTA_EUNREACH, "a destination is unreachable from an origin");
  if (st & ST_CAPACITY) return fail(QDTA_ENOMEM, "an internal item buffer was too small");
  if (st & ST_BADARG) return fail(QDTA_EINVAL, "a device array argument held an invalid value");
  return QDTA_OK;
}

static cudaEvent_t ev_get(qdta_graph *g) {
  if (!g->evpool.empty()) {
    cudaEvent_t e = g->evpool.back();
    g->evpool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

static void prof_begin(qdta_graph *g, cudaStream_t s, ProfEvent *pe, int kind, long long roots) {
  if (!g->prof_on) return;
  pe->kind = kind;
  pe->roots = roots;
  pe->a = ev_get(g);
  pe->b = ev_get(g);
  cudaEventRecord(pe->a, s);
}

static void prof_end(qdta_graph *g, cudaStream_t s, ProfEvent *pe) {
  if (!g->prof_on) return;
  cudaEventRecord(pe->b, s);
  g->pending.push_back(*pe);
}

static int prof_harvest(qdta_graph *g) {
  for (auto &pe : g->pending) {
    float ms = 0.f;
    cudaEventSynchronize(pe.b);
    cudaEventElapsedTime(&ms, pe.a, pe.b);
    if (pe.kind == 0) { g->prof.sssp_launches++; g->prof.sssp_ms += ms; }
    else if (pe.kind == 1) { g->prof.load_launches++; g->prof.load_ms += ms; }
    else { g->prof.sweep_launches++; g->prof.sweep_ms += ms; }
    g->evpool.push_back(pe.a);
    g->evpool.push_back(pe.b);
  }
  g->pending.clear();
  return QDTA_OK;
}

static int64_t dt_quanta(const qdta_graph *g, double dt_s) {
  if (!(dt_s < 1e300)) return INT64_MAX;
  return (int64_t)std::floor(dt_s / g->d.quantum_s + 0.5);
}

static int check_graph(const qdta_graph *g) {
  if (!g) return fail(QDTA_EINVAL, "graph handle is NULL");
  return QDTA_OK;
}

static int check_params(const qdta_params *p) {
  if (!p) return fail(QDTA_EINVAL, "params is NULL");
  if (p->step < 0 || p->step > 3) return fail(QDTA_EINVAL, "unknown step rule %d", p->step);
  if (p->stop < 0 || p->stop > 2) return fail(QDTA_EINVAL, "unknown stop rule %d", p->stop);
  if (p->max_iter < 0 || p->max_iter > 100000) return fail(QDTA_EINVAL, "max_iter out of range");
  if (p->ls_max < 1 || p->ls_max > 1000) return fail(QDTA_EINVAL, "ls_max out of range");
  if (!(p->ls_dx > 0.0) || !(p->ls_t1 >= 0.0) || !(p->ls_t2 > 0.0) || !(p->tol >= 0.0))
    return fail(QDTA_EINVAL, "line-search tolerances must be positive");
  if (p->schedule != QDTA_SCHEDULE_PLAIN && p->schedule != QDTA_SCHEDULE_GRAPH)
    return fail(QDTA_EINVAL, "unknown schedule");
  if (p->objective != QDTA_OBJ_UE && p->objective != QDTA_OBJ_SO) return fail(QDTA_EINVAL, "unknown objective");
  if (p->truncation != QDTA_TRUNC_NODE && p->truncation != QDTA_TRUNC_CARRY)
    return fail(QDTA_EINVAL, "unknown truncation rule %d", p->truncation);
  return QDTA_OK;
}

// ---------------------------------------------------------------------------
// graph handle
// ---------------------------------------------------------------------------
extern "C" const char *qdta_last_error(void) { return g_err.c_str(); }
extern "C" const char *qdta_version(void) { return "qdta-gb300 0.1 (sm_103a)"; }

extern "C" const char *qdta_sssp_kernel_name(const qdta_graph *g, int32_t direction) {
  if (!g || (direction != QDTA_TO_ROOT && direction != QDTA_FROM_ROOT)) {
    fail(QDTA_EINVAL, "qdta_sssp_kernel_name: null graph or bad direction");
    return "";
  }
  if (g->sssp_kind == 1) return "sssp_cell_kernel";
  return sssp_kernel_name(g->d, direction, g->sssp_smem);
}

template <class T>
static int upload(qdta_graph *g, const T *host, size_t n, T **dev) {
  void *p = nullptr;
  CK(cudaMalloc(&p, (n ? n : 1) * sizeof(T)));
  g->owned.push_back(p);
  if (n) CK(cudaMemcpy(p, host, n * sizeof(T), cudaMemcpyHostToDevice));
  *dev = reinterpret_cast<T *>(p);
  return QDTA_OK;
}

// ---------------------------------------------------------------------------
// cell partition (host, once per graph)
// ---------------------------------------------------------------------------
// Undirected breadth-first distances from `src` (-1 where unreachable).
static void bfs_undirected(int V, const std::vector<int> &off, const std::vector<int> &nbr, int src,
                           std::vector<int> &d) {
  d.assign(V, -1);
  std::vector<int> q;
  q.reserve(V);
  d[src] = 0;
  q.push_back(src);
  for (size_t h = 0; h < q.size(); ++h) {
    int u = q[h];
    for (int k = off[u]; k < off[u + 1]; ++k) {
      int w = nbr[k];
      if (d[w] < 0) { d[w] = d[u] + 1; q.push_back(w); }
    }
  }
}

struct HostCells {
  int n_cells = 0;
  std::vector<int> cell_off, node_int, node_cell;
  std::vector<int> ent_off[2], ent_link[2], ent_code[2], ext_off[2], ext_node[2], dep_off[2], dep_cell[2];
  std::vector<int> lrev_off[2], lrev_link[2], lrev_src[2];
  std::vector<int> xrev_off[2], xrev_link[2], xrev_node[2];
  std::vector<unsigned char> node_flags[2];
};

// Cells are blocks of a 2-D coordinate system read off breadth-first
// distances from three far-apart nodes (a, its farthest node b, and the node
// c farthest from both): p = d_a - d_c, s = d_a + d_c.  On a grid these are
// axis-aligned 16 x 16 blocks; on other graphs they are compact clusters.
// Cells above CELL_MAX_NODES nodes or CELL_MAX_EXT external neighbours (in
// either direction) are split in halves until they fit.
static void build_cells(const qdta_graph_desc *d, HostCells &H) {
  const int V = d->n_nodes, L = d->n_links;
  std::vector<int> uo(V + 1, 0), un(2 * (size_t)L);
  for (int e = 0; e < L; ++e) { uo[d->tail[e] + 1]++; uo[d->head[e] + 1]++; }
  for (int v = 0; v < V; ++v) uo[v + 1] += uo[v];
  {
    std::vector<int> pos(uo.begin(), uo.end() - 1);
    for (int e = 0; e < L; ++e) { un[pos[d->tail[e]]++] = d->head[e]; un[pos[d->head[e]]++] = d->tail[e]; }
  }
  std::vector<int> d0, da, db, dc;
  bfs_undirected(V, uo, un, 0, d0);
  int a = 0;
  for (int v = 0; v < V; ++v) if (d0[v] > d0[a]) a = v;
  bfs_undirected(V, uo, un, a, da);
  int b = a;
  for (int v = 0; v < V; ++v) if (da[v] > da[b]) b = v;
  bfs_undirected(V, uo, un, b, db);
  int c = a, best = -1;
  for (int v = 0; v < V; ++v) {
    int m = std::min(da[v], db[v]);
    if (da[v] >= 0 && m > best) { best = m; c = v; }
  }
  bfs_undirected(V, uo, un, c, dc);
  const int W = 32;  // 16 grid steps in each of p and s
  std::vector<long long> key(V);
  long long pmin = 0, smin = 0;
  bool first = true;
  for (int v = 0; v < V; ++v) {
    if (da[v] < 0 || dc[v] < 0) continue;
    long long p = (long long)da[v] - dc[v], s2 = (long long)da[v] + dc[v];
    if (first || p < pmin) pmin = p;
    if (first || s2 < smin) smin = s2;
    first = false;
  }
  // node order: (cell row, cell column, s, p, id); unreachable nodes last
  std::vector<int> order(V);
  for (int v = 0; v < V; ++v) order[v] = v;
  auto coords = [&](int v, long long &cy, long long &cx, long long &sy, long long &sx) {
    if (da[v] < 0 || dc[v] < 0) { cy = cx = (1ll << 40); sy = sx = v; return; }
    long long p = (long long)da[v] - dc[v] - pmin, s2 = (long long)da[v] + dc[v] - smin;
    cy = s2 / W; cx = p / W; sy = s2; sx = p;
  };
  std::vector<long long> cy(V), cx(V), sy(V), sx(V);
  for (int v = 0; v < V; ++v) coords(v, cy[v], cx[v], sy[v], sx[v]);
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    if (cy[x] != cy[y]) return cy[x] < cy[y];
    if (cx[x] != cx[y]) return cx[x] < cx[y];
    if (sy[x] != sy[y]) return sy[x] < sy[y];
    if (sx[x] != sx[y]) return sx[x] < sx[y];
    return x < y;
  });
  // initial cells: runs of equal (cy, cx)
  std::vector<std::pair<int, int>> cells;  // [begin, end) in `order`
  for (int i = 0; i < V;) {
    int j = i + 1;
    while (j < V && cy[order[j]] == cy[order[i]] && cx[order[j]] == cx[order[i]] &&
           !(cy[order[i]] == (1ll << 40))) ++j;
    if (cy[order[i]] == (1ll << 40)) j = std::min(V, i + CELL_MAX_NODES);
    cells.push_back({i, j});
    i = j;
  }
  // split until every cell satisfies both caps
  std::vector<int> cell_of(V);
  for (int iter = 0; iter < 64; ++iter) {
    for (size_t ci = 0; ci < cells.size(); ++ci)
      for (int i = cells[ci].first; i < cells[ci].second; ++i) cell_of[order[i]] = (int)ci;
    std::vector<std::pair<int, int>> next;
    bool split = false;
    for (size_t ci = 0; ci < cells.size(); ++ci) {
      int b0 = cells[ci].first, b1 = cells[ci].second;
      bool too_big = b1 - b0 > CELL_MAX_NODES;
      if (!too_big) {
        std::vector<int> ext_out;
        int internal = 0;
        for (int i = b0; i < b1; ++i) {
          int v = order[i];
          for (int k = uo[v]; k < uo[v + 1]; ++k) {
            if (cell_of[un[k]] != (int)ci) ext_out.push_back(un[k]);
            else ++internal;
          }
        }
        std::sort(ext_out.begin(), ext_out.end());
        ext_out.erase(std::unique(ext_out.begin(), ext_out.end()), ext_out.end());
        // two incidences per directed internal link; each direction's reversed list holds them once
        too_big = (int)ext_out.size() > CELL_MAX_EXT || internal / 2 > CELL_MAX_LREV;
      }
      if (too_big && b1 - b0 > 1) {
        int m = b0 + (b1 - b0) / 2;
        next.push_back({b0, m});
        next.push_back({m, b1});
        split = true;
      } else {
        next.push_back({b0, b1});
      }
    }
    cells.swap(next);
    if (!split) break;
  }
  const int nc = (int)cells.size();
  H.n_cells = nc;
  H.cell_off.assign(nc + 1, 0);
  H.node_int.assign(V, 0);
  H.node_cell.assign(V, 0);
  std::vector<int> node_ext(V);
  for (int ci = 0; ci < nc; ++ci) {
    H.cell_off[ci + 1] = cells[ci].second;
    for (int i = cells[ci].first; i < cells[ci].second; ++i) {
      node_ext[i] = order[i];
      H.node_int[order[i]] = i;
      H.node_cell[i] = ci;
    }
  }
  // per direction: entries by internal node, external lists, dependents
  std::vector<std::vector<int>> out_links(V), in_links(V);
  for (int e = 0; e < L; ++e) { out_links[d->tail[e]].push_back(e); in_links[d->head[e]].push_back(e); }
  for (int dir = 0; dir < 2; ++dir) {
    H.ent_off[dir].assign(V + 1, 0);
    H.ent_link[dir].clear();
    H.ent_code[dir].clear();
    H.ext_off[dir].assign(nc + 1, 0);
    H.ext_node[dir].clear();
    H.dep_off[dir].assign(nc + 1, 0);
    std::vector<std::vector<int>> deps(nc);
    for (int ci = 0; ci < nc; ++ci) {
      const int lo = H.cell_off[ci], hi = H.cell_off[ci + 1];
      std::vector<int> ext;  // external neighbour internal ids, first-seen order
      for (int u = lo; u < hi; ++u) {
        const int v = node_ext[u];
        const std::vector<int> &ls = dir == 0 ? out_links[v] : in_links[v];
        for (int e : ls) {
          const int w = H.node_int[dir == 0 ? d->head[e] : d->tail[e]];
          H.ent_link[dir].push_back(e);
          if (w >= lo && w < hi) {
            H.ent_code[dir].push_back(w - lo);
          } else {
            int k = (int)(std::find(ext.begin(), ext.end(), w) - ext.begin());
            if (k == (int)ext.size()) ext.push_back(w);
            H.ent_code[dir].push_back(-(k + 1));
            deps[H.node_cell[w]].push_back(ci);  // cell ci reads keys of w's cell
          }
        }
        H.ent_off[dir][u + 1] = (int)H.ent_link[dir].size();
      }
      H.ext_node[dir].insert(H.ext_node[dir].end(), ext.begin(), ext.end());
      H.ext_off[dir][ci + 1] = (int)H.ext_node[dir].size();
    }
    // internal reversed links and node flags
    H.node_flags[dir].assign(V, 0);
    std::vector<int> cnt(V + 1, 0);
    for (int u = 0; u < V; ++u)
      for (int t = H.ent_off[dir][u]; t < H.ent_off[dir][u + 1]; ++t) {
        const int code = H.ent_code[dir][t];
        if (code >= 0) cnt[H.cell_off[H.node_cell[u]] + code + 1]++;
        else H.node_flags[dir][u] |= 1;
      }
    for (int ci = 0; ci < nc; ++ci)
      for (int k = H.ext_off[dir][ci]; k < H.ext_off[dir][ci + 1]; ++k) H.node_flags[dir][H.ext_node[dir][k]] |= 2;
    for (int v = 0; v < V; ++v) cnt[v + 1] += cnt[v];
    H.lrev_off[dir] = cnt;
    H.lrev_link[dir].assign(cnt[V], 0);
    H.lrev_src[dir].assign(cnt[V], 0);
    {
      std::vector<int> pos(cnt.begin(), cnt.end() - 1);
      for (int u = 0; u < V; ++u) {
        const int lo = H.cell_off[H.node_cell[u]];
        for (int t = H.ent_off[dir][u]; t < H.ent_off[dir][u + 1]; ++t) {
          const int code = H.ent_code[dir][t];
          if (code < 0) continue;
          const int w = lo + code;
          H.lrev_link[dir][pos[w]] = H.ent_link[dir][t];
          H.lrev_src[dir][pos[w]] = u - lo;
          pos[w]++;
        }
      }
    }
    // external readers of each node: u in another cell pulling through w
    {
      std::vector<int> xc(V + 1, 0);
      for (int u = 0; u < V; ++u) {
        const int lo = H.cell_off[H.node_cell[u]];
        (void)lo;
        for (int t = H.ent_off[dir][u]; t < H.ent_off[dir][u + 1]; ++t) {
          const int code = H.ent_code[dir][t];
          if (code >= 0) continue;
          const int e = H.ent_link[dir][t];
          const int w = H.node_int[dir == 0 ? d->head[e] : d->tail[e]];
          xc[w + 1]++;
        }
      }
      for (int v = 0; v < V; ++v) xc[v + 1] += xc[v];
      H.xrev_off[dir] = xc;
      H.xrev_link[dir].assign(xc[V], 0);
      H.xrev_node[dir].assign(xc[V], 0);
      std::vector<int> pos(xc.begin(), xc.end() - 1);
      for (int u = 0; u < V; ++u)
        for (int t = H.ent_off[dir][u]; t < H.ent_off[dir][u + 1]; ++t) {
          if (H.ent_code[dir][t] >= 0) continue;
          const int e = H.ent_link[dir][t];
          const int w = H.node_int[dir == 0 ? d->head[e] : d->tail[e]];
          H.xrev_link[dir][pos[w]] = e;
          H.xrev_node[dir][pos[w]] = u;
          pos[w]++;
        }
    }
    H.dep_cell[dir].clear();
    for (int ci = 0; ci < nc; ++ci) {
      std::vector<int> &dl = deps[ci];
      std::sort(dl.begin(), dl.end());
      dl.erase(std::unique(dl.begin(), dl.end()), dl.end());
      H.dep_cell[dir].insert(H.dep_cell[dir].end(), dl.begin(), dl.end());
      H.dep_off[dir][ci + 1] = (int)H.dep_cell[dir].size();
    }
  }
}

extern "C" int qdta_graph_create(const qdta_graph_desc *d, int device, qdta_graph **out) {
  if (!d || !out) return fail(QDTA_EINVAL, "NULL argument");
  *out = nullptr;
  const int V = d->n_nodes, L = d->n_links;
  if (V < 1) return fail(QDTA_EINVAL, "n_nodes must be >= 1");
  if (L < 0 || L >= (1 << 24)) return fail(QDTA_EINVAL, "n_links must be in [0, 2^24)");
  if (L > 0 && (!d->tail || !d->head || !d->fftime_q || !d->capacity_vph))
    return fail(QDTA_EINVAL, "link arrays must not be NULL");
  if (!(d->alpha >= 0.0) || !std::isfinite(d->alpha)) return fail(QDTA_EINVAL, "alpha must be finite, >= 0");
  if (d->beta < 1 || d->beta > 16) return fail(QDTA_EINVAL, "beta must be an integer in [1, 16]");
  if (!(d->quantum_s > 0.0) || !std::isfinite(d->quantum_s)) return fail(QDTA_EINVAL, "quantum_s must be > 0");
  for (int e = 0; e < L; ++e) {
    if (d->tail[e] < 0 || d->tail[e] >= V || d->head[e] < 0 || d->head[e] >= V)
      return fail(QDTA_EINVAL, "link %d has a node id out of range", e);
    if (e > 0 && (d->tail[e] < d->tail[e - 1] ||
                  (d->tail[e] == d->tail[e - 1] && d->head[e] < d->head[e - 1])))
      return fail(QDTA_EINVAL, "links must be sorted by (tail, head); link %d is out of order", e);
    if (d->fftime_q[e] < 1) return fail(QDTA_EINVAL, "link %d: fftime_q must be >= 1", e);
    if (!(d->capacity_vph[e] > 0.0) || !std::isfinite(d->capacity_vph[e]))
      return fail(QDTA_EINVAL, "link %d: capacity must be finite and > 0", e);
  }
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(QDTA_EINVAL, "device %d out of range", device);
  DevGuard guard(device);
  // FNV-1a over the device's name and SM count and the network (nodes, links,
  // tails, heads, free-flow times): the key of the launch-shape tuning cache
  unsigned long long sig = 1469598103934665603ull;
  auto mix = [&](const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) { sig ^= b[i]; sig *= 1099511628211ull; }
  };
  {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
      mix(prop.name, strnlen(prop.name, sizeof prop.name));
      mix(&prop.multiProcessorCount, sizeof prop.multiProcessorCount);
    }
    mix(&V, sizeof V);
    mix(&L, sizeof L);
    if (L > 0) {
      mix(d->tail, (size_t)L * 4);
      mix(d->head, (size_t)L * 4);
      mix(d->fftime_q, (size_t)L * 4);
    }
  }

  std::vector<int> out_off(V + 1, 0), in_off(V + 1, 0), out_link(L), in_link(L);
  for (int e = 0; e < L; ++e) { out_off[d->tail[e] + 1]++; in_off[d->head[e] + 1]++; }
  for (int v = 0; v < V; ++v) { out_off[v + 1] += out_off[v]; in_off[v + 1] += in_off[v]; }
  {
    std::vector<int> po(out_off.begin(), out_off.end() - 1), pi(in_off.begin(), in_off.end() - 1);
    for (int e = 0; e < L; ++e) { out_link[po[d->tail[e]]++] = e; in_link[pi[d->head[e]]++] = e; }
  }
  qdta_graph *g = new qdta_graph();
  g->device = device;
  g->sig = sig;
  GraphDev &gd = g->d;
  gd.V = V;
  gd.L = L;
  int lb = 1;
  while ((1ll << lb) - 1 < (long long)L + 1) ++lb;  // NOLINK = 2^lb - 1 > every link id
  gd.LB = lb;
  gd.beta = d->beta;
  gd.alpha = d->alpha;
  gd.quantum_s = d->quantum_s;
  int rc = QDTA_OK;
  int *tail = nullptr, *head = nullptr, *c0 = nullptr, *oo = nullptr, *io = nullptr, *ol = nullptr, *il = nullptr;
  double *cap = nullptr;
  if ((rc = upload(g, d->tail, L, &tail)) || (rc = upload(g, d->head, L, &head)) ||
      (rc = upload(g, d->fftime_q, L, &c0)) || (rc = upload(g, d->capacity_vph, L, &cap)) ||
      (rc = upload(g, out_off.data(), V + 1, &oo)) || (rc = upload(g, in_off.data(), V + 1, &io)) ||
      (rc = upload(g, out_link.data(), L, &ol)) || (rc = upload(g, in_link.data(), L, &il))) {
    qdta_graph_destroy(g);
    return rc;
  }
  gd.tail = tail; gd.head = head; gd.c0 = c0; gd.cap = cap;
  gd.out_off = oo; gd.in_off = io; gd.out_link = ol; gd.in_link = il;
  cudaDeviceGetAttribute(&gd.num_sms, cudaDevAttrMultiProcessorCount, device);
  void *p = nullptr;
  if (cudaMalloc(&p, 64) != cudaSuccess) { qdta_graph_destroy(g); return fail(QDTA_ENOMEM, "status word"); }
  g->owned.push_back(p);
  g->status = (unsigned *)p;
  p = nullptr;
  if (cudaMalloc(&p, (size_t)V * 4 + 16) != cudaSuccess || cudaMemset(p, 0, (size_t)V * 4 + 16) != cudaSuccess) {
    if (p) cudaFree(p);
    qdta_graph_destroy(g);
    return fail(QDTA_ENOMEM, "per-root round counts");
  }
  g->owned.push_back(p);
  gd.root_rounds = (int *)p;
  if (cudaMallocHost(&g->status_h, 64) != cudaSuccess ||
      cudaMallocHost(&g->ctl_h, sizeof(Ctl)) != cudaSuccess) {
    qdta_graph_destroy(g);
    return fail(QDTA_ENOMEM, "pinned host words");
  }
  g->sssp_smem = V <= sssp_max_smem_nodes();
  g->sssp_bpsm = sssp_blocks_per_sm(g->sssp_smem, V);
  // kernel for graphs above the shared-memory limit: the global-memory
  // Bellman-Ford (measured fastest on the metro grid); QDTA_SSSP=cell selects
  // the cell-partitioned kernel
  g->sssp_kind = g->sssp_smem ? 0 : 2;
  // launch choices (environment overrides for experiments; qdta_autotune
  // replaces them by measurement)
  g->d.tune_adj = getenv("QDTA_NO_ELL") ? 0 : 3;  // 32-bit rank keys where the degrees allow
  if (const char *e = getenv("QDTA_SSSP_ADJ")) g->d.tune_adj = std::min(3, std::max(0, atoi(e)));
  g->d.tune_relax = 2;
  if (const char *e = getenv("QDTA_BF_RELAX")) g->d.tune_relax = std::min(3, std::max(0, atoi(e)));
  g->d.tune_carve = 85;  // rounds to the 196 KB step: 2 CTAs' queues + a 60 KB L1
  if (const char *e = getenv("QDTA_SMQ_CARVEOUT")) g->d.tune_carve = atoi(e);
  if (const char *e = getenv("QDTA_BF_BPSM")) g->bf_bpsm = std::max(1, atoi(e));
  // default shape: four 256-thread CTAs per SM where their marks fit
  // (fastest on the metro grid), else two 512-thread CTAs
  g->d.tune_shape = sssp_smq_shape_fits(V, 1) ? 1 : sssp_smq_shape_fits(V, 0) ? 0 : sssp_smq_shape_fits(V, 2) ? 2 : 0;
  g->d.tune_out = 1;  // internal-order output pass where the graph is renumbered
  if (const char *e = getenv("QDTA_SMQ_OUT")) g->d.tune_out = atoi(e) != 0;
  // queue kernels: roots after the first wave from an atomic counter, the
  // longest of their last batch first (QDTA_BF_DYNAMIC=0: round-robin;
  // QDTA_BF_LPT=0: in batch order)
  g->d.tune_dyn = 1;
  if (const char *e = getenv("QDTA_BF_DYNAMIC")) g->d.tune_dyn = atoi(e) != 0;
  g->bf_lpt = 1;
  if (const char *e = getenv("QDTA_BF_LPT")) g->bf_lpt = atoi(e) != 0;
  if (const char *e = getenv("QDTA_BF_SHAPE")) {
    const int sh = atoi(e);
    if (sssp_smq_shape_fits(V, sh)) g->d.tune_shape = sh;
  }
  if (!g->sssp_smem) {
    const char *env = getenv("QDTA_SSSP");
    if (env && strcmp(env, "cell") == 0) g->sssp_kind = 1;
    HostCells H;
    build_cells(d, H);
    CellDev &C = g->cells;
    C.n_cells = H.n_cells;
    int *p_off, *p_ni, *p_nc;
    if ((rc = upload(g, H.cell_off.data(), H.cell_off.size(), &p_off)) ||
        (rc = upload(g, H.node_int.data(), H.node_int.size(), &p_ni)) ||
        (rc = upload(g, H.node_cell.data(), H.node_cell.size(), &p_nc))) {
      qdta_graph_destroy(g);
      return rc;
    }
    C.cell_off = p_off; C.node_int = p_ni; C.node_cell = p_nc;
    for (int dir = 0; dir < 2; ++dir) {
      int *a1, *a2, *a3, *a4, *a5, *a6, *a7;
      if ((rc = upload(g, H.ent_off[dir].data(), H.ent_off[dir].size(), &a1)) ||
          (rc = upload(g, H.ent_link[dir].data(), H.ent_link[dir].size(), &a2)) ||
          (rc = upload(g, H.ent_code[dir].data(), H.ent_code[dir].size(), &a3)) ||
          (rc = upload(g, H.ext_off[dir].data(), H.ext_off[dir].size(), &a4)) ||
          (rc = upload(g, H.ext_node[dir].data(), H.ext_node[dir].size(), &a5)) ||
          (rc = upload(g, H.dep_off[dir].data(), H.dep_off[dir].size(), &a6)) ||
          (rc = upload(g, H.dep_cell[dir].data(), H.dep_cell[dir].size(), &a7))) {
        qdta_graph_destroy(g);
        return rc;
      }
      C.ent_off[dir] = a1; C.ent_link[dir] = a2; C.ent_code[dir] = a3; C.ext_off[dir] = a4;
      C.ext_node[dir] = a5; C.dep_off[dir] = a6; C.dep_cell[dir] = a7;
      int *b1 = nullptr, *b2 = nullptr, *b3 = nullptr;
      unsigned char *b4 = nullptr;
      if ((rc = upload(g, H.lrev_off[dir].data(), H.lrev_off[dir].size(), &b1)) ||
          (rc = upload(g, H.lrev_link[dir].data(), H.lrev_link[dir].size(), &b2)) ||
          (rc = upload(g, H.lrev_src[dir].data(), H.lrev_src[dir].size(), &b3)) ||
          (rc = upload(g, H.node_flags[dir].data(), H.node_flags[dir].size(), &b4))) {
        qdta_graph_destroy(g);
        return rc;
      }
      C.lrev_off[dir] = b1; C.lrev_link[dir] = b2; C.lrev_src[dir] = b3; C.node_flags[dir] = b4;
      g->n_lrev[dir] = (long long)H.lrev_link[dir].size();
      int *x1, *x2, *x3;
      if ((rc = upload(g, H.xrev_off[dir].data(), H.xrev_off[dir].size(), &x1)) ||
          (rc = upload(g, H.xrev_link[dir].data(), H.xrev_link[dir].size(), &x2)) ||
          (rc = upload(g, H.xrev_node[dir].data(), H.xrev_node[dir].size(), &x3))) {
        qdta_graph_destroy(g);
        return rc;
      }
      C.xrev_off[dir] = x1; C.xrev_link[dir] = x2; C.xrev_node[dir] = x3;
      g->n_xrev[dir] = (long long)H.xrev_link[dir].size();
    }
    g->has_cells = true;
    g->cell_bpsm = sssp_cell_blocks_per_sm();
    // locality order for the global-memory kernel: cell-major internal ids
    // (QDTA_NO_REORDER keeps the external order)
    if (!getenv("QDTA_NO_REORDER")) {
      std::vector<int> node_ext(V);
      for (int v = 0; v < V; ++v) node_ext[H.node_int[v]] = v;
      for (int dir = 0; dir < 2; ++dir) {
        const int *ooff = dir == 0 ? in_off.data() : out_off.data();
        const int *olnk = dir == 0 ? in_link.data() : out_link.data();
        const int *nbof = dir == 0 ? d->tail : d->head;
        std::vector<int> po(V + 1, 0), pl(L), pn(L);
        for (int u = 0; u < V; ++u) {
          const int v = node_ext[u];
          po[u + 1] = po[u] + (ooff[v + 1] - ooff[v]);
          for (int k = ooff[v], t = po[u]; k < ooff[v + 1]; ++k, ++t) {
            pl[t] = olnk[k];
            pn[t] = H.node_int[nbof[olnk[k]]];
          }
        }
        int *q1, *q2, *q3;
        if ((rc = upload(g, po.data(), po.size(), &q1)) || (rc = upload(g, pl.data(), pl.size(), &q2)) ||
            (rc = upload(g, pn.data(), pn.size(), &q3))) {
          qdta_graph_destroy(g);
          return rc;
        }
        gd.perm_off[dir] = q1; gd.perm_link[dir] = q2; gd.perm_nb[dir] = q3;
        int md = 0;
        for (int u = 0; u < V; ++u) md = std::max(md, po[u + 1] - po[u]);
        gd.max_deg[dir] = md;
      }
      gd.node_int = C.node_int;
      int *p_ne = nullptr;
      if ((rc = upload(g, node_ext.data(), node_ext.size(), &p_ne))) {
        qdta_graph_destroy(g);
        return rc;
      }
      gd.node_ext = p_ne;
      // rank-keyed four-slot adjacency: ranks of links among the candidate
      // parent links of the node they relax, and the link of each rank
      if (gd.max_deg[0] <= 4 && gd.max_deg[1] <= 4) {
        std::vector<int> rk_out(L), rk_in(L);
        for (int v = 0; v < V; ++v) {
          for (int k = out_off[v]; k < out_off[v + 1]; ++k) rk_out[out_link[k]] = k - out_off[v];
          for (int k = in_off[v]; k < in_off[v + 1]; ++k) rk_in[in_link[k]] = k - in_off[v];
        }
        std::vector<int> rl0(4 * (size_t)V, -1), rl1(4 * (size_t)V, -1);
        bool sym = true;
        for (int u = 0; u < V; ++u) {
          const int v = node_ext[u];
          const int dout = out_off[v + 1] - out_off[v], din = in_off[v + 1] - in_off[v];
          for (int k = 0; k < dout; ++k) rl0[4 * (size_t)u + k] = out_link[out_off[v] + k];
          for (int k = 0; k < din; ++k) rl1[4 * (size_t)u + k] = in_link[in_off[v] + k];
          // k-th out-neighbour == k-th in-neighbour (both lists ascending by link id)
          if (dout != din) sym = false;
          for (int k = 0; sym && k < dout; ++k)
            if (d->head[out_link[out_off[v] + k]] != d->tail[in_link[in_off[v] + k]]) sym = false;
        }
        int *r0, *r1, *l0, *l1;
        // TO_ROOT relaxes tails over their out-links, FROM_ROOT heads over their in-links
        if ((rc = upload(g, rk_out.data(), rk_out.size(), &r0)) || (rc = upload(g, rk_in.data(), rk_in.size(), &r1)) ||
            (rc = upload(g, rl0.data(), rl0.size(), &l0)) || (rc = upload(g, rl1.data(), rl1.size(), &l1))) {
          qdta_graph_destroy(g);
          return rc;
        }
        gd.rank_tgt[0] = r0; gd.rank_tgt[1] = r1;
        gd.rank_link[0] = l0; gd.rank_link[1] = l1;
        gd.skip_parent = sym && !getenv("QDTA_NO_PARENT_SKIP") ? 1 : 0;
      }
    }
    double mean_q = 0.0;
    for (int e = 0; e < L; ++e) mean_q += d->fftime_q[e];
    mean_q = L ? mean_q / L : 1.0;
    double mult = 16.0;
    if (const char *dm = getenv("QDTA_CELL_DELTA")) mult = atof(dm);
    g->cell_delta = (long long)(mult * mean_q) + 1;
  }
  if (cudaGetLastError() != cudaSuccess) { qdta_graph_destroy(g); return fail(QDTA_ECUDA, "occupancy query failed"); }
  *out = g;
  return QDTA_OK;
}

extern "C" int qdta_graph_set_capacity(qdta_graph *g, const double *capacity_vph, void *stream) {
  RC(check_graph(g));
  if (g->d.L > 0 && !capacity_vph) return fail(QDTA_EINVAL, "capacity_vph is NULL");
  if (g->d.L == 0) return QDTA_OK;
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  RC(status_reset(g, s));
  launch_set_capacity(g->d, capacity_vph, g->status, s);
  int rc = status_check(g, s);
  if (rc == QDTA_EINVAL) return fail(QDTA_EINVAL, "capacities must be finite and > 0 (graph unchanged)");
  return rc;
}

extern "C" int qdta_graph_destroy(qdta_graph *g) {
  if (!g) return QDTA_OK;
  DevGuard guard(g->device);
  cudaDeviceSynchronize();
  for (void *p : g->owned) cudaFree(p);
  for (auto &kv : g->ws) if (kv.second.p) cudaFree(kv.second.p);
  for (auto &pe : g->pending) { cudaEventDestroy(pe.a); cudaEventDestroy(pe.b); }
  for (auto e : g->evpool) cudaEventDestroy(e);
  if (g->status_h) cudaFreeHost(g->status_h);
  if (g->ctl_h) cudaFreeHost(g->ctl_h);
  delete g;
  return QDTA_OK;
}

extern "C" int qdta_profile_enable(qdta_graph *g, int32_t on) {
  RC(check_graph(g));
  DevGuard guard(g->device);
  if (!g->prof_roots) {
    void *p = nullptr;
    CK(cudaMalloc(&p, 64));
    g->owned.push_back(p);
    g->prof_roots = (unsigned long long *)p;
  }
  CK(cudaMemset(g->prof_roots, 0, 64));
  g->prof_on = on ? 1 : 0;
  g->prof = qdta_profile{};
  return QDTA_OK;
}

extern "C" int qdta_profile_read(qdta_graph *g, qdta_profile *out) {
  RC(check_graph(g));
  if (!out) return fail(QDTA_EINVAL, "out is NULL");
  DevGuard guard(g->device);
  CK(cudaDeviceSynchronize());
  prof_harvest(g);
  // device counters: roots, rounds, relaxations, cell activations, redone batches
  unsigned long long cnt[5] = {0, 0, 0, 0, 0};
  if (g->prof_roots) CK(cudaMemcpy(cnt, g->prof_roots, sizeof cnt, cudaMemcpyDeviceToHost));
  g->prof.sssp_roots = (int64_t)cnt[0];
  g->prof.sssp_rounds = (int64_t)cnt[1];
  g->prof.sssp_relaxations = (int64_t)cnt[2];
  g->prof.sssp_cell_activations = (int64_t)cnt[3];
  g->prof.sssp_redo_batches = (int64_t)cnt[4];
  g->prof.kernel_launches = launch_count();
  *out = g->prof;
  return QDTA_OK;
}

// ---------------------------------------------------------------------------
// shortest paths, loading, costs
// ---------------------------------------------------------------------------
static int sssp_grid(const qdta_graph *g, int R) {
  long long bpsm = g->sssp_kind == 1 ? g->cell_bpsm : g->sssp_bpsm;
  if (g->sssp_kind == 2) {
    // resident roots of the global-memory variant: as many CTAs per SM as
    // the launch shape was designed for (occupancy-checked), unless capped
    if (sssp_uses_smq(g->d)) bpsm = sssp_smq_ctas_per_sm(g->d, 0);
    if (g->bf_bpsm > 0 && g->bf_bpsm < bpsm) bpsm = g->bf_bpsm;
  }
  long long cap = bpsm * g->d.num_sms;
  if (g->sssp_kind == 2) R = (R + sssp_group_size() - 1) / sssp_group_size();  // CTAs, G roots each
  long long n = R < cap ? R : cap;
  return n < 1 ? 1 : (int)n;
}

static int sssp_work(qdta_graph *g, int grid, int R_cap, SsspWork *w) {
  const size_t V = g->d.V;
  w->slots = grid;
  RC(ws_get(g, "sssp.adj", std::max((size_t)g->d.L, (size_t)4 * V), &w->adj));
  RC(ws_get(g, "sssp.fb", 4, &w->fb_skip));
  // longest-first order of the dynamic fetch (queue kernels)
  w->order = nullptr;
  if (g->sssp_kind == 2 && !g->sssp_smem && sssp_uses_smq(g->d) && g->d.tune_dyn && g->bf_lpt)
    RC(ws_get(g, "sssp.order", (size_t)std::max(R_cap, 1), &w->order));
  if (g->sssp_kind == 1) {
    RC(ws_get(g, "sssp.lrev", (size_t)std::max(g->n_lrev[0], g->n_lrev[1]), &w->lrev));
    RC(ws_get(g, "sssp.prio", (size_t)grid * g->cells.n_cells, &w->prio));
    RC(ws_get(g, "sssp.xrev", (size_t)std::max(g->n_xrev[0], g->n_xrev[1]), &w->xrev));
    RC(ws_get(g, "sssp.state", (size_t)grid * V, &w->state));
    RC(ws_get(g, "sssp.stamp", (size_t)grid * g->cells.n_cells, &w->stamp));
    RC(ws_get(g, "sssp.queue", (size_t)grid * 3 * g->cells.n_cells, &w->queue));
  } else if (!g->sssp_smem) {
    const size_t G = (size_t)sssp_group_size();
    RC(ws_get(g, "sssp.state", (size_t)grid * G * V, &w->state));
    if (sssp_uses_smq(g->d)) w->stamp = nullptr;  // marks live in shared memory
    else RC(ws_get(g, "sssp.stamp", (size_t)grid * G * V, &w->stamp));
    RC(ws_get(g, "sssp.queue", (size_t)grid * 2 * G * V, &w->queue));
  } else {
    w->state = nullptr; w->stamp = nullptr; w->queue = nullptr;
  }
  return QDTA_OK;
}

// one batch: pack adjacency for q, then SSSP over the roots.  `profile`
// false leaves the launch out of the per-kernel timings (a batch the host
// knows is skipped on the device: its kernels return at once)
static int run_sssp(qdta_graph *g, int direction, const int *q, const int *roots, int R_host,
                    const int *R_dev, int R_cap, int *parent, const int *slot_dev, long long stride,
                    long long *dist, cudaStream_t s, const int *skip_dev = nullptr, bool profile = true) {
  SsspWork w;
  const int grid = sssp_grid(g, R_cap);
  RC(sssp_work(g, grid, R_cap, &w));
  const int prof_saved = g->prof_on;
  if (!profile) g->prof_on = 0;
  ProfEvent pe;
  if (g->sssp_kind == 1) {
    launch_pack_cell_adj(g->d, g->cells, direction, q, w.adj, w.lrev, g->n_lrev[direction], w.xrev,
                         g->n_xrev[direction], s, skip_dev);
    prof_begin(g, s, &pe, 0, R_host);
    launch_sssp_cell(g->d, g->cells, direction, w.adj, w.lrev, w.xrev, g->cell_delta, roots, R_host, R_dev, grid,
                     w.state, w.stamp, w.queue, w.prio,
                     parent, slot_dev, stride, dist, g->status, s, skip_dev,
                     g->prof_on ? g->prof_roots : nullptr);
  } else {
    const int adjl = g->sssp_kind == 2 ? sssp_adj(g->d, direction) : 0;
    if (adjl >= 2) launch_pack_ell8(g->d, direction, q, reinterpret_cast<int2 *>(w.adj), s, skip_dev);
    else if (adjl == 1) launch_pack_ell(g->d, direction, q, w.adj, s, skip_dev);
    else if (g->sssp_kind == 2 && sssp_uses_perm(g->d)) launch_pack_perm_adj(g->d, direction, q, w.adj, s, skip_dev);
    else launch_pack_adj(g->d, direction, q, w.adj, s, skip_dev);
    prof_begin(g, s, &pe, 0, R_host);
    launch_sssp(g->d, direction, w.adj, roots, R_host, R_dev, grid, g->sssp_smem, w, parent, slot_dev,
                stride, dist, g->status, s, skip_dev, g->prof_on ? g->prof_roots : nullptr);
  }
  prof_end(g, s, &pe);
  g->prof_on = prof_saved;
  return QDTA_OK;
}

extern "C" int qdta_sssp_batch(qdta_graph *g, const int32_t *cost_q, const int32_t *roots, int32_t R,
                               int32_t direction, int32_t *parent_link, int64_t *dist, void *stream) {
  RC(check_graph(g));
  if (R < 0) return fail(QDTA_EINVAL, "R must be >= 0");
  if (direction != QDTA_TO_ROOT && direction != QDTA_FROM_ROOT) return fail(QDTA_EINVAL, "bad direction");
  if (R > 0 && (!cost_q || !roots || !parent_link)) return fail(QDTA_EINVAL, "NULL array");
  if (R == 0) return QDTA_OK;
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  RC(status_reset(g, s));
  RC(run_sssp(g, direction, cost_q, roots, R, nullptr, R, parent_link, nullptr, 0,
              (long long *)dist, s));
  return status_check(g, s);
}

// ---------------------------------------------------------------------------
// launch-shape autotuning of the shortest-path batch
// ---------------------------------------------------------------------------
namespace {
struct TuneCfg {
  int kind, adj, relax, bpsm, shape;
};

TuneCfg tune_get(const qdta_graph *g) {
  return {g->sssp_kind, g->d.tune_adj, g->d.tune_relax, g->bf_bpsm, g->d.tune_shape};
}

void tune_set(qdta_graph *g, const TuneCfg &c) {
  g->sssp_kind = c.kind;
  g->d.tune_adj = c.adj;
  g->d.tune_relax = c.relax;
  g->bf_bpsm = c.bpsm;
  g->d.tune_shape = c.shape;
}

// Launch-shape tuning cache, keyed by (graph signature, direction); opt-in
// with QDTA_TUNE_CACHE: "mem" keeps the choices of this process, a file path
// also reads and appends them there (one line per choice: signature,
// direction, the five choice fields, milliseconds, kernel name), so that
// later processes on the same GPU model skip the timing.
struct TuneHit {
  TuneCfg cfg;
  qdta_tune_entry entry;
};
std::mutex g_tune_mu;
std::map<std::pair<unsigned long long, int>, TuneHit> g_tune_cache;

const char *tune_cache_path() {
  const char *e = getenv("QDTA_TUNE_CACHE");
  return (e && *e) ? e : nullptr;
}

bool tune_cache_find(unsigned long long sig, int dir, TuneHit *hit) {
  const char *path = tune_cache_path();
  if (!path) return false;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune_cache.find({sig, dir});
  if (it != g_tune_cache.end()) { *hit = it->second; return true; }
  if (strcmp(path, "mem") == 0) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  while (!found && fgets(line, sizeof line, f)) {
    unsigned long long s2 = 0;
    int d2 = 0, k = 0, a = 0, r = 0, b = 0, sh = 0, ctas = 0;
    float ms = 0.f;
    char name[40] = {0};
    if (sscanf(line, "%llx %d %d %d %d %d %d %d %f %39s", &s2, &d2, &k, &a, &r, &b, &sh, &ctas, &ms, name) == 10 &&
        s2 == sig && d2 == dir && sh >= 0 && sh < sssp_smq_shape_count()) {
      hit->cfg = TuneCfg{k, a, r, b, sh};
      hit->entry = qdta_tune_entry{};
      snprintf(hit->entry.kernel, sizeof hit->entry.kernel, "%s", name);
      hit->entry.ctas_per_sm = ctas;
      hit->entry.valid = 1;
      hit->entry.ms = ms;
      g_tune_cache[{sig, dir}] = *hit;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void tune_cache_store(unsigned long long sig, int dir, const TuneCfg &c, const qdta_tune_entry &e) {
  const char *path = tune_cache_path();
  if (!path) return;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[{sig, dir}] = TuneHit{c, e};
  if (strcmp(path, "mem") == 0) return;
  if (FILE *f = fopen(path, "a")) {
    fprintf(f, "%llx %d %d %d %d %d %d %d %.4f %s\n", sig, dir, c.kind, c.adj, c.relax, c.bpsm, c.shape,
            e.ctas_per_sm, e.ms, e.kernel);
    fclose(f);
  }
}
}  // namespace

extern "C" int qdta_autotune(qdta_graph *g, const int32_t *cost_q, const int32_t *roots, int32_t R,
                             int32_t direction, int32_t reps, int32_t *parent_scratch, qdta_tune_report *out_host,
                             void *stream) {
  RC(check_graph(g));
  if (R <= 0 || reps <= 0) return fail(QDTA_EINVAL, "qdta_autotune: R and reps must be positive");
  if (direction != QDTA_TO_ROOT && direction != QDTA_FROM_ROOT) return fail(QDTA_EINVAL, "bad direction");
  if (!cost_q || !roots || !parent_scratch || !out_host) return fail(QDTA_EINVAL, "NULL argument");
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  {
    TuneHit hit;
    if (tune_cache_find(g->sig, direction, &hit)) {
      tune_set(g, hit.cfg);
      qdta_tune_report rep{};
      rep.n = 1;
      rep.best = 0;
      rep.entry[0] = hit.entry;
      rep.cached = 1;
      *out_host = rep;
      return QDTA_OK;
    }
  }
  const TuneCfg start = tune_get(g);
  std::vector<TuneCfg> cand;
  if (g->sssp_smem) {
    cand.push_back(start);  // whole per-root state in shared memory: one shape
  } else {
    // global-memory Bellman-Ford: launch shape x adjacency layout x relaxation
    // mode (each shape with as many CTAs per SM as it was designed for)
    const bool ell_ok = g->d.max_deg[direction] <= 4 && g->d.node_int != nullptr;
    const bool rank_ok = ell_ok && g->d.rank_tgt[direction] != nullptr;
    bool any_smq = false;
    for (int shape = 0; shape < sssp_smq_shape_count(); ++shape) {
      if (!sssp_smq_shape_fits(g->d.V, shape) || getenv("QDTA_BF_NOSMQ")) continue;
      if (shape == 2 && sssp_smq_shape_fits(g->d.V, 0)) continue;  // same block as shape 0, fewer marks
      any_smq = true;
      if (shape >= 3) {  // five CTAs per SM, 5 / 6 nodes per lane group, lane per node, 288 threads: 32-bit rank keys only
        if (rank_ok) cand.push_back({2, 3, 2, 0, shape});
        continue;
      }
      // relaxation mode 2 only: mode 1 (returning atomic) and mode 3
      // (aggregated appends) measured slower in every shape and layout
      for (int adj = rank_ok ? 3 : ell_ok ? 1 : 0; adj >= 0; --adj) cand.push_back({2, adj, 2, 0, shape});
    }
    if (!any_smq) cand.push_back({2, start.adj, start.relax, start.bpsm, start.shape});  // global queues
    if (g->has_cells) cand.push_back({1, start.adj, start.relax, start.bpsm, start.shape});  // cell-partitioned
  }
  if ((int)cand.size() > QDTA_TUNE_MAX) cand.resize(QDTA_TUNE_MAX);
  qdta_tune_report rep{};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = QDTA_OK, best = -1;
  for (size_t i = 0; i < cand.size() && rc == QDTA_OK; ++i) {
    tune_set(g, cand[i]);
    qdta_tune_entry &en = rep.entry[rep.n++];
    const char *name = g->sssp_kind == 1 ? "sssp_cell_kernel" : sssp_kernel_name(g->d, direction, g->sssp_smem);
    snprintf(en.kernel, sizeof(en.kernel), "%s", name);
    en.ctas_per_sm = (int32_t)((long long)sssp_grid(g, 1 << 30) / std::max(1, g->d.num_sms));
    // one untimed batch (workspace sizing, first-touch), then reps timed
    if ((rc = status_reset(g, s)) ||
        (rc = run_sssp(g, direction, cost_q, roots, R, nullptr, R, parent_scratch, nullptr, 0, nullptr, s)) ||
        (rc = status_check(g, s)))
      break;
    cudaEventRecord(e0, s);
    for (int k = 0; k < reps && rc == QDTA_OK; ++k)
      rc = run_sssp(g, direction, cost_q, roots, R, nullptr, R, parent_scratch, nullptr, 0, nullptr, s);
    cudaEventRecord(e1, s);
    if (rc == QDTA_OK) rc = status_check(g, s);
    if (rc != QDTA_OK) break;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = fail(QDTA_ECUDA, "qdta_autotune: event timing failed");
      break;
    }
    en.ms = ms / reps;
    en.valid = 1;
    if (best < 0 || en.ms < rep.entry[best].ms) best = (int)i;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != QDTA_OK || best < 0) {
    tune_set(g, start);
    return rc != QDTA_OK ? rc : fail(QDTA_ECUDA, "qdta_autotune: no candidate ran");
  }
  // keep the handle's current choice unless another candidate is at least 2 %
  // faster: closer timings are within run-to-run noise
  for (size_t i = 0; i < cand.size() && i < (size_t)rep.n; ++i) {
    const TuneCfg &c = cand[i];
    if (c.kind == start.kind && c.adj == start.adj && c.relax == start.relax && c.bpsm == start.bpsm &&
        c.shape == start.shape && rep.entry[i].valid && rep.entry[best].ms > 0.98f * rep.entry[i].ms)
      best = (int)i;
  }
  tune_set(g, cand[best]);
  rep.best = best;
  tune_cache_store(g->sig, direction, cand[best], rep.entry[best]);
  *out_host = rep;
  return QDTA_OK;
}

extern "C" int qdta_interval_metrics(qdta_graph *g, const double *flows, int32_t N, double dt_s,
                                     const double *length_m, const int32_t *link_class, int32_t n_classes,
                                     double congested_voc, double *out, void *stream) {
  RC(check_graph(g));
  if (N < 0 || N > 65535) return fail(QDTA_EINVAL, "qdta_interval_metrics: N must be in [0, 65535]");
  if (n_classes < 1 || n_classes > QDTA_METRIC_MAX_CLASSES)
    return fail(QDTA_EINVAL, "qdta_interval_metrics: n_classes must be in [1, %d]", QDTA_METRIC_MAX_CLASSES);
  if (!(dt_s > 0.0) || !std::isfinite(congested_voc)) return fail(QDTA_EINVAL, "qdta_interval_metrics: bad dt_s or threshold");
  if (N == 0) return QDTA_OK;
  if (!out || (g->d.L > 0 && (!flows || !length_m || !link_class)))
    return fail(QDTA_EINVAL, "qdta_interval_metrics: NULL array");
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  RC(status_reset(g, s));
  const size_t words = (size_t)N * n_classes * 16;
  unsigned long long *acc;
  RC(ws_get(g, "metrics.acc", words, &acc));
  CK(cudaMemsetAsync(acc, 0, words * 8, s));
  launch_metrics(g->d, flows, N, dt_s / 3600.0, length_m, link_class, n_classes, congested_voc, acc, out, g->status,
                 s);
  return status_check(g, s);
}

static int check_carry_items(qdta_graph *g, const qdta_od *od, cudaStream_t s);

extern "C" int qdta_load_aon(qdta_graph *g, const int32_t *cost_q, const int32_t *parent_link,
                             const qdta_od *od, int64_t dt_q, int64_t *flow_fx, int32_t *stop_node,
                             void *stream) {
  RC(check_graph(g));
  if (!od) return fail(QDTA_EINVAL, "od is NULL");
  if (od->n_items < 0 || od->n_roots < 0) return fail(QDTA_EINVAL, "negative sizes");
  if (od->n_items == 0) return QDTA_OK;
  if (!cost_q || !parent_link || !flow_fx || !od->roots || !od->root_idx || !od->src || !od->amount_fx)
    return fail(QDTA_EINVAL, "NULL array");
  if (dt_q < 0) return fail(QDTA_EINVAL, "dt_q must be >= 0");
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  RC(check_carry_items(g, od, s));
  RC(status_reset(g, s));
  int2 *hq;
  RC(ws_get(g, "load.head_q", (size_t)g->d.L, &hq));
  launch_pack_head_q(g->d, cost_q, hq, s);
  ProfEvent pe;
  prof_begin(g, s, &pe, 1, 0);
  launch_load(g->d, hq, parent_link, nullptr, 0, nullptr, od->roots, od->n_items, nullptr, od->root_idx,
              od->src, (const long long *)od->amount_fx, dt_q, (unsigned long long *)flow_fx,
              stop_node, g->status, s, (const long long *)od->carry_frac, od->carry_link);
  prof_end(g, s, &pe);
  return status_check(g, s);
}

extern "C" int qdta_bpr_costs(qdta_graph *g, const double *flow, double dt_s, double *cost_s,
                              int32_t *cost_q, void *stream) {
  RC(check_graph(g));
  if (g->d.L > 0 && (!flow || !cost_q)) return fail(QDTA_EINVAL, "NULL array");
  if (!(dt_s > 0.0)) return fail(QDTA_EINVAL, "dt_s must be > 0");
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  RC(status_reset(g, s));
  launch_bpr(g->d, flow, dt_s / 3600.0, cost_s, cost_q, g->status, s);
  return status_check(g, s);
}

// ---------------------------------------------------------------------------
// interval solver state shared by the schedules
// ---------------------------------------------------------------------------
struct Solver {
  qdta_graph *g;
  cudaStream_t s;
  const qdta_params *p;
  double dt_h;
  long long dt_q;
  // demand
  const int *roots;        // SSSP roots
  int R_host;              // roots when known on the host
  const int *R_dev;        // or on the device
  int R_cap;               // grid sizing
  const int *root_slot;    // item root -> parent row (NULL: identity)
  const int *item_roots;   // node of each root index (load walks end there)
  long long n_host;
  const long long *n_dev;
  const int *root_idx, *src;
  const long long *amount;
  // per item (nullable): the fraction of its link covered (2^-32 units) and the link carrying the trip (-1: none)
  const long long *carry = nullptr;
  const int *carry_link = nullptr;
  // link state
  int *q;
  unsigned long long *g_fx;
  double *f;
  LinkConst *kc;
  int2 *head_q;
  int *parent;
  long long parent_stride;
  int ring;
  Ctl *ctl;
  i128 *partials;
  unsigned *counter;
  int sgrid;
  int *tape_q;
  double *tape_alpha, *tape_f;
  int tape_cap;
  // free-flow trees of every root index (nullable): the initial AON of an
  // interval runs at q = BPR(0), the same link times every interval, so its
  // trees are gathered from here (rows by root index) instead of recomputed
  const int *ff_parent = nullptr;
  int ff_rows = 0;
  // system optimum: q holds the quantised marginal costs (routing), qt the
  // link times (loading and truncation); for the user equilibrium qt == q
  int *qt = nullptr;
  int so = 0;
};

static int solver_alloc(Solver &S, const std::string &tag, int ring, bool tape_f) {
  qdta_graph *g = S.g;
  const size_t L = g->d.L;
  RC(ws_get(g, tag + ".q", L, &S.q));
  S.so = S.p->objective == QDTA_OBJ_SO;
  if (S.so) RC(ws_get(g, tag + ".qt", L, &S.qt));
  else S.qt = S.q;
  RC(ws_get(g, tag + ".gfx", L, &S.g_fx));
  RC(ws_get(g, tag + ".kc", L, &S.kc));
  RC(ws_get(g, tag + ".hq", L, &S.head_q));
  S.parent_stride = (long long)S.R_cap * g->d.V;
  S.ring = ring;
  RC(ws_get(g, tag + ".parent", (size_t)S.parent_stride * ring, &S.parent));
  RC(ws_get(g, tag + ".ctl", 1, &S.ctl));
  S.sgrid = sweep_grid(g->d);
  RC(ws_get(g, tag + ".partials", (size_t)S.sgrid * NSUM, &S.partials));
  RC(ws_get(g, tag + ".counter", 4, &S.counter));
  S.tape_cap = S.p->max_iter + 1;
  RC(ws_get(g, tag + ".tape_q", (size_t)S.tape_cap * L, &S.tape_q));
  RC(ws_get(g, tag + ".tape_alpha", (size_t)S.tape_cap, &S.tape_alpha));
  S.tape_f = nullptr;
  if (tape_f) RC(ws_get(g, tag + ".tape_f", (size_t)S.tape_cap * L, &S.tape_f));
  CK(cudaMemsetAsync(S.counter, 0, 16, S.s));
  SsspWork w;
  RC(sssp_work(g, sssp_grid(g, S.R_cap), S.R_cap, &w));  // nothing is allocated while capturing
  return QDTA_OK;
}

// AON under the link times in S.q: trees into the parent slot, flows into
// g_fx.  gather_ff: the trees are the free-flow ones, copied from S.ff_parent
static int seg_aon(Solver &S, const int *slot_dev, bool gather_ff = false) {
  qdta_graph *g = S.g;
  if (gather_ff)
    launch_gather_rows(S.ff_parent, S.ff_rows, g->d.V, S.root_slot, S.parent, slot_dev, S.parent_stride, S.s);
  else
    RC(run_sssp(g, QDTA_TO_ROOT, S.q, S.roots, S.R_host, S.R_dev, S.R_cap, S.parent, slot_dev,
                S.parent_stride, nullptr, S.s));
  launch_pack_head_q(g->d, S.qt, S.head_q, S.s);
  CK(cudaMemsetAsync(S.g_fx, 0, (size_t)g->d.L * 8, S.s));
  ProfEvent pe;
  prof_begin(g, S.s, &pe, 1, 0);
  launch_load(g->d, S.head_q, S.parent, slot_dev, S.parent_stride, S.root_slot, S.item_roots, S.n_host,
              S.n_dev, S.root_idx, S.src, S.amount, S.dt_q, S.g_fx, nullptr, g->status, S.s, S.carry,
              S.carry_link);
  prof_end(g, S.s, &pe);
  return QDTA_OK;
}

// ctl init + initial AON at free flow (f = 0 -> q = BPR(0) = c0)
static int seg_init(Solver &S) {
  qdta_graph *g = S.g;
  const qdta_params *p = S.p;
  launch_ctl_init(S.ctl, p->step, p->stop, p->max_iter, p->ls_max, p->tol, p->ls_dx, p->ls_t1, p->ls_t2,
                  S.ring, S.n_host, S.n_dev, 1, S.s);
  launch_link_const(g->d, S.dt_h, S.kc, S.s);
  CK(cudaMemsetAsync(S.f, 0, (size_t)g->d.L * 8, S.s));
  launch_bpr(g->d, S.f, S.dt_h, nullptr, S.q, g->status, S.s, S.so);
  if (S.so) launch_bpr(g->d, S.f, S.dt_h, nullptr, S.qt, g->status, S.s);
  RC(seg_aon(S, nullptr, S.ff_parent != nullptr));
  launch_flow_from_fx(g->d.L, S.g_fx, S.f, S.s);
  launch_tape0(g->d, S.q, S.f, S.tape_q, S.tape_alpha, S.tape_f, S.s);
  return QDTA_OK;
}

static int seg_iter_head(Solver &S, unsigned long long h_ls, int use_cond) {
  qdta_graph *g = S.g;
  launch_bpr(g->d, S.f, S.dt_h, nullptr, S.q, g->status, S.s, S.so);
  if (S.so) launch_bpr(g->d, S.f, S.dt_h, nullptr, S.qt, g->status, S.s);
  RC(seg_aon(S, &S.ctl->tree_slot));
  launch_ctl_begin(S.ctl, h_ls, use_cond, S.s);
  return QDTA_OK;
}

static int seg_ls_body(Solver &S, unsigned long long h_ls, int use_cond) {
  qdta_graph *g = S.g;
  ProfEvent pe;
  prof_begin(g, S.s, &pe, 2, 0);
  launch_sweep(g->d, S.kc, S.f, (const long long *)S.g_fx, S.q, S.ctl, S.partials, S.counter, S.sgrid,
               g->status, S.s, S.so);
  prof_end(g, S.s, &pe);
  launch_ctl_step(S.ctl, h_ls, use_cond, S.s);
  return QDTA_OK;
}

static int seg_iter_tail(Solver &S, unsigned long long h_fw, int use_cond) {
  qdta_graph *g = S.g;
  launch_update(g->d, S.ctl, S.f, (const long long *)S.g_fx, S.s);
  launch_tape_record(g->d, S.ctl, S.q, S.f, S.tape_q, S.tape_alpha, S.tape_f, S.tape_cap, S.s);
  launch_ctl_end(S.ctl, h_fw, use_cond, S.s);
  return QDTA_OK;
}

static int seg_finish(Solver &S) {
  launch_objective(S.g->d, S.kc, S.f, S.ctl, S.partials, S.counter, S.sgrid, S.g->status, S.s, S.so);
  return QDTA_OK;
}

static int read_ctl(Solver &S, Ctl *out) {
  CK(cudaMemcpyAsync(out, S.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, S.s));
  CK(cudaStreamSynchronize(S.s));
  return QDTA_OK;
}

// plain schedule: host loop, one synchronisation per decision
static int fw_plain(Solver &S) {
  Ctl *h = (Ctl *)S.g->ctl_h;
  RC(seg_init(S));
  RC(read_ctl(S, h));
  while (h->fw_continue) {
    RC(seg_iter_head(S, 0, 0));
    RC(read_ctl(S, h));
    while (h->need_sweep) {
      RC(seg_ls_body(S, 0, 0));
      RC(read_ctl(S, h));
    }
    RC(seg_iter_tail(S, 0, 0));
    RC(read_ctl(S, h));
  }
  RC(seg_finish(S));
  return QDTA_OK;
}

// capture `fn` into `graph` (an empty body graph owned by a node)
template <class F>
static int capture_into(cudaGraph_t graph, cudaStream_t cs, F fn) {
  CK(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int rc = fn();
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &out);
  if (rc < 0) return rc;
  CK(e);
  return QDTA_OK;
}

static int add_while(cudaGraph_t graph, const cudaGraphNode_t *deps, size_t ndeps, unsigned dflt,
                     cudaGraphNode_t *node, cudaGraph_t *body, cudaGraphConditionalHandle *h) {
  CK(cudaGraphConditionalHandleCreate(h, graph, dflt, cudaGraphCondAssignDefault));
  // the parameter union has no default constructor: build it in zeroed storage
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof raw);
  cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(raw);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = *h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  CK(cudaGraphAddNode(node, graph, deps, nullptr, ndeps, &np));
  *body = np.conditional.phGraph_out[0];
  return QDTA_OK;
}

template <class F>
static int add_captured_child(cudaGraph_t graph, const cudaGraphNode_t *deps, size_t ndeps,
                              cudaStream_t cs, cudaGraphNode_t *node, F fn) {
  cudaGraph_t child;
  CK(cudaGraphCreate(&child, 0));
  int rc = capture_into(child, cs, fn);
  if (rc < 0) { cudaGraphDestroy(child); return rc; }
  cudaError_t e = cudaGraphAddChildGraphNode(node, graph, deps, ndeps, child);
  cudaGraphDestroy(child);
  CK(e);
  return QDTA_OK;
}

// FW loop body: head -> WHILE(line search) -> tail, as nodes of `body`
static int build_fw_body(Solver &S, cudaGraph_t body, cudaGraphConditionalHandle h_fw, cudaStream_t cs) {
  cudaGraphNode_t n_head, n_ls, n_tail;
  cudaGraph_t ls_body;
  cudaGraphConditionalHandle h_ls;
  RC(add_while(body, nullptr, 0, 0, &n_ls, &ls_body, &h_ls));
  // the LS condition is written by ctl_begin, so the head must precede it
  cudaStream_t saved = S.s;
  S.s = cs;
  int rc = add_captured_child(body, nullptr, 0, cs, &n_head, [&] { return seg_iter_head(S, h_ls, 1); });
  if (rc >= 0) rc = capture_into(ls_body, cs, [&] { return seg_ls_body(S, h_ls, 1); });
  if (rc >= 0) rc = add_captured_child(body, &n_ls, 1, cs, &n_tail, [&] { return seg_iter_tail(S, h_fw, 1); });
  S.s = saved;
  RC(rc);
  CK(cudaGraphAddDependencies(body, &n_head, &n_ls, nullptr, 1));
  return QDTA_OK;
}

static int fw_graph(Solver &S) {
  qdta_graph *g = S.g;
  if (g->prof_on) return fail(QDTA_EINVAL, "profiling needs the plain schedule");
  RC(seg_init(S));
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = QDTA_OK;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphCreate"); break; }
    cudaGraphNode_t n_fw;
    cudaGraph_t fw_body;
    cudaGraphConditionalHandle h_fw;
    if ((rc = add_while(graph, nullptr, 0, 1, &n_fw, &fw_body, &h_fw)) < 0) break;
    if ((rc = build_fw_body(S, fw_body, h_fw, cs)) < 0) break;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e)); break; }
    // run the loop only when there is something to iterate (the WHILE body
    // executes while its condition, default 1, stays non-zero)
    Ctl *h = (Ctl *)g->ctl_h;
    if ((rc = read_ctl(S, h)) < 0) break;
    if (h->fw_continue) {
      e = cudaGraphLaunch(exec, S.s);
      if (e != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e)); break; }
    }
    rc = seg_finish(S);
  } while (0);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamSynchronize(S.s);
  cudaStreamDestroy(cs);
  return rc;
}

static void fill_stats(const Ctl *h, long long n_items, qdta_stats *st) {
  st->iterations = h->iterations;
  st->aon_calls = h->aon_calls;
  st->ls_passes = h->ls_passes;
  st->converged = h->converged;
  st->rel_gap = h->rel_gap;
  st->objective = h->objective;
  st->n_items = n_items;
  st->dual_gap = h->dual_gap;
}

static int check_od(const qdta_graph *g, const qdta_od *od) {
  if (!od) return fail(QDTA_EINVAL, "od is NULL");
  if (od->n_items < 0 || od->n_roots < 0) return fail(QDTA_EINVAL, "negative sizes");
  if (od->n_items > 0 && (!od->roots || !od->root_idx || !od->src || !od->amount_fx || od->n_roots < 1))
    return fail(QDTA_EINVAL, "od arrays must not be NULL");
  (void)g;
  return QDTA_OK;
}

// items carried on a link, checked on the device: the link exists, its
// tail is the item's src, the covered fraction is in [0, 2^32) (QDTA_EINVAL otherwise)
static int check_carry_items(qdta_graph *g, const qdta_od *od, cudaStream_t s) {
  if (!od || !od->carry_link || od->n_items <= 0) return QDTA_OK;
  RC(status_reset(g, s));
  launch_check_carry(g->d, od->n_items, od->src, (const long long *)od->carry_frac, od->carry_link, g->status, s);
  return status_check(g, s);
}

extern "C" int qdta_line_search(qdta_graph *g, const double *flow, const int64_t *aon_fx, double dt_s,
                                int32_t fw_iter, const qdta_params *p, double *alpha_out,
                                int32_t *passes_out, void *stream) {
  RC(check_graph(g));
  RC(check_params(p));
  if (fw_iter < 1) return fail(QDTA_EINVAL, "fw_iter must be >= 1");
  if (!(dt_s > 0.0)) return fail(QDTA_EINVAL, "dt_s must be > 0");
  if (g->d.L > 0 && (!flow || !aon_fx)) return fail(QDTA_EINVAL, "NULL array");
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  RC(status_reset(g, s));
  Solver S{};
  S.g = g; S.s = s; S.p = p; S.dt_h = dt_s / 3600.0;
  Ctl *ctl;
  LinkConst *kc;
  i128 *partials;
  unsigned *counter;
  const int sg = sweep_grid(g->d);
  RC(ws_get(g, "ls.ctl", 1, &ctl));
  RC(ws_get(g, "ls.kc", (size_t)g->d.L, &kc));
  RC(ws_get(g, "ls.partials", (size_t)sg * NSUM, &partials));
  RC(ws_get(g, "ls.counter", 4, &counter));
  CK(cudaMemsetAsync(counter, 0, 16, s));
  // a line search alone: no stop rule, iteration k = fw_iter
  launch_ctl_init(ctl, p->step, QDTA_STOP_NONE, fw_iter, p->ls_max, p->tol, p->ls_dx, p->ls_t1, p->ls_t2,
                  1, 1, nullptr, 0, s);
  CK(cudaMemcpyAsync(&ctl->k, &fw_iter, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  launch_link_const(g->d, S.dt_h, kc, s);
  launch_ctl_begin(ctl, 0, 0, s);
  Ctl *h = (Ctl *)g->ctl_h;
  for (int guard_it = 0; guard_it < 10000; ++guard_it) {
    CK(cudaMemcpyAsync(h, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!h->need_sweep) break;
    launch_sweep(g->d, kc, flow, (const long long *)aon_fx, nullptr, ctl, partials, counter, sg, g->status, s,
                 p->objective == QDTA_OBJ_SO);
    launch_ctl_step(ctl, 0, 0, s);
  }
  RC(status_check(g, s));
  if (alpha_out) *alpha_out = h->alpha_final;
  if (passes_out) *passes_out = h->ls_passes;
  return QDTA_OK;
}

static int assign_core(qdta_graph *g, const qdta_od *od, double dt_s, const qdta_params *p,
                       double *flow_out, qdta_stats *stats, qdta_tape **tape_out, cudaStream_t s,
                       const std::string &tag) {
  Solver S{};
  S.g = g; S.s = s; S.p = p;
  S.dt_h = dt_s / 3600.0;
  S.dt_q = dt_quanta(g, dt_s);
  S.roots = od->roots; S.R_host = od->n_roots; S.R_dev = nullptr; S.R_cap = od->n_roots > 0 ? od->n_roots : 1;
  S.root_slot = nullptr; S.item_roots = od->roots;
  S.n_host = od->n_items; S.n_dev = nullptr;
  S.root_idx = od->root_idx; S.src = od->src; S.amount = (const long long *)od->amount_fx;
  S.carry = (const long long *)od->carry_frac;
  S.carry_link = od->carry_link;
  S.f = flow_out;
  const bool want_tape = p->record_tape && tape_out;
  if (want_tape && p->objective == QDTA_OBJ_SO)
    return fail(QDTA_EINVAL, "the adjoint (record_tape) covers the user equilibrium only");
  RC(solver_alloc(S, tag, 1, want_tape));
  RC(status_reset(g, s));
  if (p->schedule == QDTA_SCHEDULE_GRAPH) RC(fw_graph(S));
  else RC(fw_plain(S));
  RC(status_check(g, s));
  Ctl *h = (Ctl *)g->ctl_h;
  RC(read_ctl(S, h));
  if (stats) fill_stats(h, od->n_items, stats);
  if (want_tape) {
    qdta_tape *t = new qdta_tape();
    t->g = g; t->od = *od; t->dt_s = dt_s; t->step = p->step; t->K = h->iterations;
    const size_t L = g->d.L, K1 = (size_t)t->K + 1;
    bool ok = cudaMalloc(&t->q, K1 * L * 4 + 16) == cudaSuccess &&
              cudaMalloc(&t->alpha, K1 * 8 + 16) == cudaSuccess &&
              cudaMalloc(&t->f, K1 * L * 8 + 16) == cudaSuccess &&
              cudaMalloc(&t->cap, L * 8 + 16) == cudaSuccess;
    if (!ok) { cudaGetLastError(); qdta_tape_destroy(t); return fail(QDTA_ENOMEM, "tape allocation"); }
    CK(cudaMemcpyAsync(t->cap, g->d.cap, L * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(t->q, S.tape_q, K1 * L * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(t->alpha, S.tape_alpha, K1 * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(t->f, S.tape_f, K1 * L * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    *tape_out = t;
  }
  return h->notconv ? QDTA_ENOTCONV : QDTA_OK;
}

extern "C" int qdta_assign_interval(qdta_graph *g, const qdta_od *od, double dt_s, const qdta_params *p,
                                    double *flow_out, qdta_stats *stats, qdta_tape **tape_out,
                                    void *stream) {
  RC(check_graph(g));
  RC(check_params(p));
  RC(check_od(g, od));
  if (!(dt_s > 0.0)) return fail(QDTA_EINVAL, "dt_s must be > 0");
  if (g->d.L > 0 && !flow_out) return fail(QDTA_EINVAL, "flow_out is NULL");
  if (tape_out) *tape_out = nullptr;
  DevGuard guard(g->device);
  RC(check_carry_items(g, od, (cudaStream_t)stream));
  return assign_core(g, od, dt_s, p, flow_out, stats, tape_out, (cudaStream_t)stream, "fw");
}

// ---------------------------------------------------------------------------
// many independent instances
// ---------------------------------------------------------------------------
// All instances' FW loops as parallel branches of one CUDA graph: one launch
// solves every instance, the branches running concurrently on the GPU.
static int assign_batch_graph(const qdta_instance *inst, int n, const qdta_params *p, qdta_stats *stats,
                              cudaStream_t s) {
  std::vector<Solver> S(n);
  for (int i = 0; i < n; ++i) {
    Solver &X = S[i];
    qdta_graph *g = inst[i].graph;
    X.g = g; X.s = s; X.p = p;
    X.dt_h = inst[i].dt_s / 3600.0;
    X.dt_q = dt_quanta(g, inst[i].dt_s);
    const qdta_od *od = &inst[i].od;
    X.roots = od->roots; X.R_host = od->n_roots; X.R_dev = nullptr; X.R_cap = od->n_roots > 0 ? od->n_roots : 1;
    X.root_slot = nullptr; X.item_roots = od->roots;
    X.n_host = od->n_items; X.n_dev = nullptr;
    X.root_idx = od->root_idx; X.src = od->src; X.amount = (const long long *)od->amount_fx;
    X.carry = (const long long *)od->carry_frac;
    X.carry_link = od->carry_link;
    X.f = inst[i].flow_out;
    RC(solver_alloc(X, "batch", 1, false));
    RC(status_reset(g, s));
    RC(seg_init(X));
  }
  std::vector<Ctl> h(n);
  for (int i = 0; i < n; ++i) RC(read_ctl(S[i], &h[i]));
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = QDTA_OK;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphCreate"); break; }
    int branches = 0;
    for (int i = 0; i < n && rc >= 0; ++i) {
      if (!h[i].fw_continue) continue;
      cudaGraphNode_t node;
      cudaGraph_t body;
      cudaGraphConditionalHandle hc;
      if ((rc = add_while(graph, nullptr, 0, 1, &node, &body, &hc)) < 0) break;
      rc = build_fw_body(S[i], body, hc, cs);
      ++branches;
    }
    if (rc < 0) break;
    if (branches > 0) {
      cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
      if (e != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e)); break; }
      e = cudaGraphLaunch(exec, s);
      if (e != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e)); break; }
    }
    for (int i = 0; i < n && rc >= 0; ++i) rc = seg_finish(S[i]);
  } while (0);
  cudaStreamSynchronize(s);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  RC(rc);
  int worst = QDTA_OK;
  for (int i = 0; i < n; ++i) {
    RC(status_check(inst[i].graph, s));
    RC(read_ctl(S[i], &h[i]));
    if (stats) fill_stats(&h[i], inst[i].od.n_items, &stats[i]);
    if (h[i].notconv) worst = QDTA_ENOTCONV;
  }
  return worst;
}

extern "C" int qdta_assign_batch(const qdta_instance *inst, int32_t n_inst, const qdta_params *p,
                                 qdta_stats *stats, void *stream) {
  if (n_inst < 0 || (n_inst > 0 && !inst)) return fail(QDTA_EINVAL, "bad instance array");
  RC(check_params(p));
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < n_inst; ++i) {
    RC(check_graph(inst[i].graph));
    RC(check_od(inst[i].graph, &inst[i].od));
    if (!(inst[i].dt_s > 0.0)) return fail(QDTA_EINVAL, "instance %d: dt_s must be > 0", i);
    if (inst[i].graph->d.L > 0 && !inst[i].flow_out) return fail(QDTA_EINVAL, "instance %d: flow_out is NULL", i);
    if (inst[i].graph->device != inst[0].graph->device) return fail(QDTA_EINVAL, "instances span devices");
    for (int j = 0; j < i; ++j)
      if (inst[j].graph == inst[i].graph)
        return fail(QDTA_EINVAL, "instances %d and %d share a graph handle (one workspace each)", j, i);
  }
  if (n_inst == 0) return QDTA_OK;
  DevGuard guard(inst[0].graph->device);
  for (int i = 0; i < n_inst; ++i) RC(check_carry_items(inst[i].graph, &inst[i].od, s));
  if (p->schedule == QDTA_SCHEDULE_GRAPH && !inst[0].graph->prof_on)
    return assign_batch_graph(inst, n_inst, p, stats, s);
  int worst = QDTA_OK;
  for (int i = 0; i < n_inst; ++i) {
    int rc = assign_core(inst[i].graph, &inst[i].od, inst[i].dt_s, p, inst[i].flow_out,
                         stats ? &stats[i] : nullptr, nullptr, s, "batch");
    if (rc < 0) return rc;
    if (rc > 0) worst = rc;
  }
  return worst;
}

// ---------------------------------------------------------------------------
// a day of intervals (Alg. 1)
// ---------------------------------------------------------------------------
struct Day {
  Solver S;
  int Z;                       // zones (roots of every interval)
  const int *zones;
  unsigned long long *dense;   // [Z * V] residual + original demand accumulator
  int *blk_count;
  long long *blk_off;
  long long cap_items;
  int *it_root, *it_src;
  long long *it_amt;
  long long *it_carry;         // items' covered fractions and links (carried trips in play), else NULL
  int *it_link;
  CarryAcc ca;                 // carried (root, link) table (mask 0: none)
  int trunc;                   // QDTA_TRUNC_*
  long long *n_items_dev;
  int *flag, *active, *root_slot, *n_active;
  int *q_fin, *q_work;
  int2 *hq_fin;
  unsigned long long *h_fx;
  double *w;
  OrigTable *tab;
  long long max_orig;
  qdta_stats *stats_dev;
};

static int day_merge(Day &D) {
  qdta_graph *g = D.S.g;
  cudaStream_t s = D.S.s;
  launch_scatter_orig(g->d, D.S.ctl, D.tab, D.max_orig, D.dense, s, D.ca, g->status);
  launch_compact(g->d, D.Z, D.dense, D.blk_count, D.blk_off, D.cap_items, D.it_root, D.it_src, D.it_amt,
                 D.n_items_dev, g->status, s, D.it_carry, D.it_link, D.ca);
  launch_active_roots(D.Z, D.n_items_dev, D.cap_items, D.it_root, D.zones, D.flag, D.active, D.root_slot,
                      D.n_active, s);
  return QDTA_OK;
}

// Alg. 4 preparation: step weights, final costs, cleared h
static int day_res_head(Day &D) {
  qdta_graph *g = D.S.g;
  cudaStream_t s = D.S.s;
  launch_path_weights(D.S.ctl, D.S.tape_alpha, D.w, s);
  launch_bpr(g->d, D.S.f, D.S.dt_h, nullptr, D.q_fin, g->status, s);
  launch_pack_head_q(g->d, D.q_fin, D.hq_fin, s);
  CK(cudaMemsetAsync(D.h_fx, 0, (size_t)g->d.L * 8, s));
  return QDTA_OK;
}

// one accepted AON j: reuse its stored tree or rebuild it, then re-walk
static int day_res_body(Day &D, unsigned long long h, int use_cond) {
  qdta_graph *g = D.S.g;
  Solver &S = D.S;
  cudaStream_t s = S.s;
  launch_res_prep(S.ctl, D.w, S.tape_q, g->d.L, D.q_work, s);
  // On the plain schedule with profiling on, the host reads whether tree j
  // is still stored, so that skipped batches do not enter the per-batch
  // timings.  The kernels are launched either way (and return at once when
  // skipped), as on the graph schedule.
  bool real_batch = true;
  if (!use_cond && g->prof_on) {
    Ctl *hc = (Ctl *)g->ctl_h;
    RC(read_ctl(S, hc));
    real_batch = !hc->res_skip;
  }
  RC(run_sssp(g, QDTA_TO_ROOT, D.q_work, S.roots, 0, S.R_dev, S.R_cap, S.parent, &S.ctl->res_slot,
              S.parent_stride, nullptr, s, &S.ctl->res_skip, real_batch));
  launch_residual(g->d, D.hq_fin, S.parent, &S.ctl->res_slot, S.parent_stride, D.root_slot, D.zones,
                  D.n_items_dev, D.cap_items, D.it_root, D.it_src, D.it_amt, &S.ctl->w_cur, S.dt_q, D.h_fx,
                  D.dense, g->status, s, D.it_carry, D.it_link, D.trunc, D.ca);
  launch_res_next(S.ctl, h, use_cond, s);
  return QDTA_OK;
}

static int day_store(Day &D, double *flow_out) {
  launch_store_interval(D.S.g->d, D.S.ctl, D.h_fx, flow_out, D.stats_dev, D.n_items_dev, D.S.s);
  return QDTA_OK;
}

static int day_interval_plain(Day &D, double *flow_out) {
  Solver &S = D.S;
  Ctl *h = (Ctl *)S.g->ctl_h;
  RC(day_merge(D));
  RC(fw_plain(S));
  RC(day_res_head(D));
  launch_res_begin(S.ctl, 0, 0, S.s);
  RC(read_ctl(S, h));
  while (h->res_continue) {
    RC(day_res_body(D, 0, 0));
    RC(read_ctl(S, h));
  }
  RC(day_store(D, flow_out));
  launch_day_next(S.ctl, 0, 0, S.s);
  return QDTA_OK;
}

// the whole day as one CUDA graph: WHILE(interval) { merge + initial AON;
// WHILE(FW step) { head; WHILE(line-search sweep) {...}; tail }; residual
// head; WHILE(accepted AON j) { re-walk }; store }
static int day_graph(Day &D, double *flow_out) {
  Solver &S = D.S;
  qdta_graph *g = S.g;
  if (g->prof_on) return fail(QDTA_EINVAL, "profiling needs the plain schedule");
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = S.s;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = QDTA_OK;
  do {
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphCreate"); break; }
    cudaGraphNode_t n_day, n_a, n_fw, n_b, n_res, n_c;
    cudaGraph_t day_body, fw_body, res_body;
    cudaGraphConditionalHandle h_day, h_fw, h_res;
    if ((rc = add_while(graph, nullptr, 0, 1, &n_day, &day_body, &h_day)) < 0) break;
    if ((rc = add_while(day_body, nullptr, 0, 0, &n_fw, &fw_body, &h_fw)) < 0) break;
    if ((rc = add_while(day_body, nullptr, 0, 0, &n_res, &res_body, &h_res)) < 0) break;
    S.s = cs;
    rc = add_captured_child(day_body, nullptr, 0, cs, &n_a, [&]() -> int {
      RC(day_merge(D));
      RC(seg_init(S));
      launch_set_cond(S.ctl, 0, h_fw, cs);
      return QDTA_OK;
    });
    if (rc >= 0) rc = build_fw_body(S, fw_body, h_fw, cs);
    if (rc >= 0)
      rc = add_captured_child(day_body, &n_fw, 1, cs, &n_b, [&]() -> int {
        RC(seg_finish(S));
        RC(day_res_head(D));
        launch_res_begin(S.ctl, h_res, 1, cs);
        return QDTA_OK;
      });
    if (rc >= 0) rc = capture_into(res_body, cs, [&]() -> int { return day_res_body(D, h_res, 1); });
    if (rc >= 0)
      rc = add_captured_child(day_body, &n_res, 1, cs, &n_c, [&]() -> int {
        RC(day_store(D, flow_out));
        launch_day_next(S.ctl, h_day, 1, cs);
        return QDTA_OK;
      });
    S.s = saved;
    if (rc < 0) break;
    cudaError_t e = cudaGraphAddDependencies(day_body, &n_a, &n_fw, nullptr, 1);
    if (e == cudaSuccess) e = cudaGraphAddDependencies(day_body, &n_b, &n_res, nullptr, 1);
    if (e != cudaSuccess) { rc = fail(QDTA_ECUDA, "graph edges: %s", cudaGetErrorString(e)); break; }
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e)); break; }
    e = cudaGraphLaunch(exec, S.s);
    if (e != cudaSuccess) { rc = fail(QDTA_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e)); break; }
  } while (0);
  S.s = saved;
  cudaStreamSynchronize(S.s);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  return rc;
}

extern "C" int qdta_run_day(qdta_graph *g, const qdta_od *d_orig, int32_t N, double dt_s,
                            const qdta_params *p, const qdta_od *resid_in, double *flow_out,
                            qdta_stats *stats, qdta_residual *resid_out, void *stream) {
  RC(check_graph(g));
  RC(check_params(p));
  if (N < 0 || (N > 0 && !d_orig)) return fail(QDTA_EINVAL, "bad interval array");
  if (!(dt_s > 0.0)) return fail(QDTA_EINVAL, "dt_s must be > 0");
  if (N == 0) return QDTA_OK;
  if (g->d.L > 0 && !flow_out) return fail(QDTA_EINVAL, "flow_out is NULL");
  const int Z = d_orig[0].n_roots;
  if (Z < 1 || !d_orig[0].roots) return fail(QDTA_EINVAL, "the zone list (d_orig[0].roots) is empty");
  for (int i = 0; i < N; ++i) {
    RC(check_od(g, &d_orig[i]));
    if (d_orig[i].n_roots != Z) return fail(QDTA_EINVAL, "interval %d: every interval must use the zone list", i);
  }
  if (resid_in) {
    RC(check_od(g, resid_in));
    if (resid_in->n_items > 0 && resid_in->n_roots != Z) return fail(QDTA_EINVAL, "resid_in must use the zone list");
  }
  // trips on links in play: the carried (root, link) table and per-item carries
  bool any_carry = p->truncation == QDTA_TRUNC_CARRY || (resid_in && resid_in->carry_link);
  for (int i = 0; i < N; ++i) any_carry = any_carry || d_orig[i].carry_link != nullptr;
  if (any_carry && resid_out && (!resid_out->carry_frac || !resid_out->carry_link))
    return fail(QDTA_EINVAL, "resid_out->carry_frac and carry_link are needed when trips are carried on links");
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < N; ++i) RC(check_carry_items(g, &d_orig[i], s));
  if (resid_in) RC(check_carry_items(g, resid_in, s));
  const size_t V = g->d.V, L = g->d.L;
  Day D{};
  Solver &S = D.S;
  S.g = g; S.s = s; S.p = p;
  S.dt_h = dt_s / 3600.0;
  S.dt_q = dt_quanta(g, dt_s);
  D.Z = Z;
  D.zones = d_orig[0].roots;
  const long long dense_n = (long long)Z * (long long)V;
  RC(ws_get(g, "day.dense", (size_t)dense_n, &D.dense));
  long long max_orig = resid_in ? resid_in->n_items : 0;
  for (int i = 0; i < N; ++i) max_orig = d_orig[i].n_items > max_orig ? d_orig[i].n_items : max_orig;
  D.max_orig = max_orig;
  D.cap_items = dense_n < (64ll << 20) ? dense_n : (64ll << 20);
  D.trunc = p->truncation;
  D.ca = CarryAcc{};
  D.it_carry = nullptr;
  D.it_link = nullptr;
  long long table_n = 0;
  if (any_carry) {
    // trips on links: an open-addressed (root, link) table of amounts and
    // exact 128-bit sums of amount x covered fraction, at most half full when
    // it holds as many entries as the dense part can; items get room for both
    const long long zl = (long long)Z * (long long)L;
    const long long want = 2 * (D.cap_items < zl ? D.cap_items : zl);
    table_n = 1024;
    while (table_n < want) table_n <<= 1;
    D.ca.mask = (unsigned long long)(table_n - 1);
    D.ca.seg = (unsigned long long)std::max(1ll, table_n / Z);
    RC(ws_get(g, "day.carry_key", (size_t)table_n, &D.ca.key));
    RC(ws_get(g, "day.carry_amt", (size_t)table_n, &D.ca.amt));
    RC(ws_get(g, "day.carry_tsum", (size_t)table_n * 2, &D.ca.tsum));
    CK(cudaMemsetAsync(D.ca.key, 0xff, (size_t)table_n * 8, s));
    CK(cudaMemsetAsync(D.ca.amt, 0, (size_t)table_n * 8, s));
    CK(cudaMemsetAsync(D.ca.tsum, 0, (size_t)table_n * 16, s));
    D.cap_items *= 2;
    RC(ws_get(g, "day.it_carry", (size_t)D.cap_items, &D.it_carry));
    RC(ws_get(g, "day.it_link", (size_t)D.cap_items, &D.it_link));
  }
  const long long scan_n = dense_n > table_n ? dense_n : table_n;
  const int nblk = (int)((scan_n + 4095) / 4096);
  RC(ws_get(g, "day.blk_count", (size_t)nblk, &D.blk_count));
  RC(ws_get(g, "day.blk_off", (size_t)nblk, &D.blk_off));
  RC(ws_get(g, "day.it_root", (size_t)D.cap_items, &D.it_root));
  RC(ws_get(g, "day.it_src", (size_t)D.cap_items, &D.it_src));
  RC(ws_get(g, "day.it_amt", (size_t)D.cap_items, &D.it_amt));
  RC(ws_get(g, "day.n_items", 2, &D.n_items_dev));
  RC(ws_get(g, "day.flag", (size_t)Z, &D.flag));
  RC(ws_get(g, "day.active", (size_t)Z, &D.active));
  RC(ws_get(g, "day.root_slot", (size_t)Z, &D.root_slot));
  RC(ws_get(g, "day.n_active", 4, &D.n_active));
  RC(ws_get(g, "day.q_fin", L, &D.q_fin));
  RC(ws_get(g, "day.q_work", L, &D.q_work));
  RC(ws_get(g, "day.hq_fin", L, &D.hq_fin));
  RC(ws_get(g, "day.h_fx", L, &D.h_fx));
  RC(ws_get(g, "day.w", (size_t)p->max_iter + 2, &D.w));
  RC(ws_get(g, "day.stats", (size_t)N, &D.stats_dev));
  // per-interval original demand table (+ the resumed residual folded into interval 0)
  std::vector<OrigTable> tab(N);
  for (int i = 0; i < N; ++i)
    tab[i] = OrigTable{d_orig[i].root_idx, d_orig[i].src, (const long long *)d_orig[i].amount_fx,
                       d_orig[i].n_items, (const long long *)d_orig[i].carry_frac, d_orig[i].carry_link};
  RC(ws_get(g, "day.tab", (size_t)N, &D.tab));
  CK(cudaMemcpyAsync(D.tab, tab.data(), sizeof(OrigTable) * N, cudaMemcpyHostToDevice, s));
  // solver over the zone list
  S.roots = D.active; S.R_host = 0; S.R_dev = D.n_active; S.R_cap = Z;
  S.root_slot = D.root_slot; S.item_roots = D.zones;
  S.n_host = 0; S.n_dev = D.n_items_dev;
  S.root_idx = D.it_root; S.src = D.it_src; S.amount = D.it_amt;
  S.carry = D.it_carry;
  S.carry_link = D.it_link;
  RC(ws_get(g, "day.f", L, &S.f));
  // parent ring: keep every tree of an interval when memory allows.  The
  // ring this handle already holds counts as available (a later day must
  // not shrink the ring because the previous day's ring is still allocated).
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  {
    auto it = g->ws.find("day.parent");
    if (it != g->ws.end()) free_b += it->second.bytes;
  }
  const double per_slot = (double)Z * V * 4.0;
  // free-flow trees of all zones, once per day (skipped when HBM is short:
  // they cost one ring slot)
  if (!getenv("QDTA_NO_FF_CACHE") && (double)free_b >= 6.0 * per_slot) {
    int *ff = nullptr;
    RC(ws_get(g, "day.ff_parent", (size_t)Z * V, &ff));
    RC(ws_get(g, "day.f", L, &S.f));
    CK(cudaMemsetAsync(S.f, 0, L * 8, s));
    RC(status_reset(g, s));
    launch_bpr(g->d, S.f, S.dt_h, nullptr, D.q_work, g->status, s);
    RC(run_sssp(g, QDTA_TO_ROOT, D.q_work, D.zones, Z, nullptr, Z, ff, nullptr, 0, nullptr, s));
    RC(status_check(g, s));
    S.ff_parent = ff;
    S.ff_rows = Z;
    CK(cudaMemGetInfo(&free_b, &total_b));
    auto it = g->ws.find("day.parent");
    if (it != g->ws.end()) free_b += it->second.bytes;
  }
  long long ring = p->max_iter + 1;
  long long afford = (long long)((double)free_b * 0.8 / per_slot);
  if (ring > afford) ring = afford;
  // QDTA_TREE_RING=n caps the ring (tests: residual trees rebuilt from the tape)
  if (const char *e = getenv("QDTA_TREE_RING")) {
    const long long cap = atoll(e);
    if (cap >= 2 && cap < ring) ring = cap;
  }
  if (ring < 2) ring = 2;
  RC(solver_alloc(S, "day", (int)ring, false));
  RC(status_reset(g, s));
  // dense accumulator starts at zero; the resumed residual goes in first
  CK(cudaMemsetAsync(D.dense, 0, (size_t)dense_n * 8, s));
  if (resid_in && resid_in->n_items > 0)
    launch_scatter_items(g->d, resid_in->n_items, resid_in->root_idx, resid_in->src,
                         (const long long *)resid_in->amount_fx, D.dense, s,
                         (const long long *)resid_in->carry_frac, resid_in->carry_link, D.ca, g->status);
  // day counter lives in the solver's controller
  int dayinit[3] = {0, N, 1};
  CK(cudaMemcpyAsync(&S.ctl->day_i, dayinit, sizeof dayinit, cudaMemcpyHostToDevice, s));
  int rc = QDTA_OK;
  if (p->schedule == QDTA_SCHEDULE_PLAIN) {
    for (int i = 0; i < N && rc >= 0; ++i) rc = day_interval_plain(D, flow_out);
  } else {
    rc = day_graph(D, flow_out);
  }
  RC(rc);
  RC(status_check(g, s));
  std::vector<qdta_stats> st(N);
  CK(cudaMemcpy(st.data(), D.stats_dev, sizeof(qdta_stats) * N, cudaMemcpyDeviceToHost));
  for (int i = 0; i < N; ++i) {
    if (stats) stats[i] = st[i];
  }
  // residual after the last interval
  if (resid_out) {
    launch_compact(g->d, Z, D.dense, D.blk_count, D.blk_off, resid_out->capacity, resid_out->root_idx,
                   resid_out->src, (long long *)resid_out->amount_fx, D.n_items_dev, g->status, s,
                   (long long *)resid_out->carry_frac, resid_out->carry_link, D.ca);
    long long cnt = 0;
    CK(cudaMemcpyAsync(&cnt, D.n_items_dev, 8, cudaMemcpyDeviceToHost, s));
    RC(status_check(g, s));
    resid_out->count = cnt;
  } else {
    CK(cudaMemsetAsync(D.dense, 0, (size_t)dense_n * 8, s));
    if (D.ca.mask) {
      CK(cudaMemsetAsync(D.ca.key, 0xff, (size_t)table_n * 8, s));
      CK(cudaMemsetAsync(D.ca.amt, 0, (size_t)table_n * 8, s));
      CK(cudaMemsetAsync(D.ca.tsum, 0, (size_t)table_n * 16, s));
    }
  }
  return QDTA_OK;
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
extern "C" int qdta_tape_destroy(qdta_tape *t) {
  if (!t) return QDTA_OK;
  if (t->q) cudaFree(t->q);
  if (t->alpha) cudaFree(t->alpha);
  if (t->f) cudaFree(t->f);
  if (t->cap) cudaFree(t->cap);
  delete t;
  return QDTA_OK;
}

extern "C" int qdta_tape_info(const qdta_tape *t, int32_t *K, int64_t *n_items) {
  if (!t) return fail(QDTA_EINVAL, "tape is NULL");
  if (K) *K = t->K;
  if (n_items) *n_items = t->od.n_items;
  return QDTA_OK;
}

extern "C" int qdta_backward(qdta_tape *t, const double *dL_dflow, double *dL_ddemand, double *dL_dcap,
                             void *stream) {
  if (!t || !t->g) return fail(QDTA_EINVAL, "tape is NULL");
  qdta_graph *g = t->g;
  const size_t L = g->d.L;
  const long long n = t->od.n_items;
  if (L > 0 && (!dL_dflow || !dL_dcap)) return fail(QDTA_EINVAL, "NULL gradient array");
  if (n > 0 && !dL_ddemand) return fail(QDTA_EINVAL, "dL_ddemand is NULL");
  DevGuard guard(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  RC(status_reset(g, s));
  const double dt_h = t->dt_s / 3600.0;
  const long long dt_q = dt_quanta(g, t->dt_s);
  const int R = t->od.n_roots > 0 ? t->od.n_roots : 1;
  double *lam, *lam2, *gbar, *red, *muH;
  unsigned long long *gfx;
  LinkConst *kc;
  int2 *hq;
  int *parent;
  const int grid = sweep_grid(g->d);
  RC(ws_get(g, "bw.lam", L, &lam));
  RC(ws_get(g, "bw.lam2", L, &lam2));
  RC(ws_get(g, "bw.gbar", L, &gbar));
  RC(ws_get(g, "bw.red", (size_t)grid * 2, &red));
  RC(ws_get(g, "bw.muH", 2, &muH));
  RC(ws_get(g, "bw.gfx", L, &gfx));
  RC(ws_get(g, "bw.kc", L, &kc));
  RC(ws_get(g, "bw.hq", L, &hq));
  RC(ws_get(g, "bw.parent", (size_t)R * g->d.V, &parent));
  std::vector<double> alpha(t->K + 1);
  CK(cudaMemcpy(alpha.data(), t->alpha, sizeof(double) * (t->K + 1), cudaMemcpyDeviceToHost));
  // per-link constants from the capacities the taped solve used
  GraphDev gd_tape = g->d;
  gd_tape.cap = t->cap;
  launch_link_const(gd_tape, dt_h, kc, s);
  CK(cudaMemcpyAsync(lam, dL_dflow, L * 8, cudaMemcpyDeviceToDevice, s));
  if (n > 0) CK(cudaMemsetAsync(dL_ddemand, 0, (size_t)n * 8, s));
  CK(cudaMemsetAsync(dL_dcap, 0, L * 8, s));
  for (int k = t->K; k >= 0; --k) {
    const int *qk = t->q + (size_t)k * L;
    // recompute tree k from the taped link times, and g_k
    RC(run_sssp(g, QDTA_TO_ROOT, qk, t->od.roots, t->od.n_roots, nullptr, R, parent, nullptr, 0, nullptr, s));
    launch_pack_head_q(g->d, qk, hq, s);
    CK(cudaMemsetAsync(gfx, 0, L * 8, s));
    launch_load(g->d, hq, parent, nullptr, 0, nullptr, t->od.roots, n, nullptr, t->od.root_idx, t->od.src,
                (const long long *)t->od.amount_fx, dt_q, gfx, nullptr, g->status, s,
                (const long long *)t->od.carry_frac, t->od.carry_link);
    const double *gb = lam;
    if (k > 0) {
      const double *fprev = t->f + (size_t)(k - 1) * L;
      const double a = alpha[k];
      const int implicit = t->step != QDTA_STEP_MSA && a > 0.0 && a < 1.0;
      launch_adj_reduce(gd_tape, kc, lam, fprev, (const long long *)gfx, a, implicit, red, muH, grid, s);
      launch_adj_update(gd_tape, kc, lam, fprev, (const long long *)gfx, a, implicit, muH, gbar, lam2, dL_dcap, s);
      gb = gbar;
    }
    launch_gather(g->d, hq, parent, t->od.roots, n, t->od.root_idx, t->od.src, dt_q, gb, dL_ddemand,
                  g->status, s, (const long long *)t->od.carry_frac, t->od.carry_link);
    if (k > 0) std::swap(lam, lam2);
  }
  return status_check(g, s);
}

// ---------------------------------------------------------------------------
// batched shortest paths without device allocation
// ---------------------------------------------------------------------------
// The packed adjacency that qdta_sssp_batch keeps in its grow-only workspace
// lives here in a fixed device array instead; the shared-memory SSSP kernel
// needs no other global scratch.
static __device__ __align__(256) int4 g_noalloc_adj[QDTA_NOALLOC_MAX_LINKS];

static std::mutex g_noalloc_mu;
static int4 *g_noalloc_ptr[256];

// device address of g_noalloc_adj on `dev` (looked up once per device, with
// that device current; host code must not use the symbol itself as a pointer)
static int noalloc_scratch(int dev, int4 **out) {
  if (dev < 0 || dev >= 256) return fail(QDTA_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_adj);
    if (e != cudaSuccess)
      return fail(QDTA_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed: %s",
                  cudaGetErrorString(e));
    g_noalloc_ptr[dev] = reinterpret_cast<int4 *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return QDTA_OK;
}

extern "C" int qdta_sssp_batch_noalloc(qdta_graph *g, const int32_t *cost_q, const int32_t *roots,
                                       int32_t R, int32_t direction, int32_t *parent_link,
                                       int64_t *dist, void *stream) {
  RC(check_graph(g));
  if (R < 0) return fail(QDTA_EINVAL, "R must be >= 0");
  if (direction != QDTA_TO_ROOT && direction != QDTA_FROM_ROOT) return fail(QDTA_EINVAL, "bad direction");
  if (g->d.L > QDTA_NOALLOC_MAX_LINKS)
    return fail(QDTA_EINVAL, "graph has %d links; the no-allocation variant holds at most %d",
                g->d.L, QDTA_NOALLOC_MAX_LINKS);
  if (!g->sssp_smem)
    return fail(QDTA_EINVAL, "graph has %d nodes; the no-allocation variant needs the per-root state "
                "in shared memory (at most %d nodes)", g->d.V, sssp_max_smem_nodes());
  if (R > 0 && (!cost_q || !roots || !parent_link)) return fail(QDTA_EINVAL, "NULL array");
  if (R == 0) return QDTA_OK;
  DevGuard guard(g->device);
  int4 *adj = nullptr;
  RC(noalloc_scratch(g->device, &adj));
  cudaStream_t s = (cudaStream_t)stream;
  RC(status_reset(g, s));
  // every entry [0, L) is rewritten before the kernel reads it
  launch_pack_adj(g->d, direction, cost_q, adj, s);
  SsspWork w{};
  w.adj = adj;
  launch_sssp(g->d, direction, adj, roots, R, nullptr, sssp_grid(g, R), true, w, parent_link, nullptr,
              0, (long long *)dist, g->status, s);
  return status_check(g, s);
}
