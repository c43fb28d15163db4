"""Seeded synthetic road networks and travel demand.

This module only produces *inputs*: a jittered grid road graph with a link
hierarchy, zone nodes, and gravity-model trip tables per 15-minute interval.
It holds none of the assignment arithmetic (no link-cost function, no
shortest paths, no loading) and is the one module that both the CUDA path's
callers and the CPU oracle's tests draw their inputs from.

The paper's own inputs (a commercial Bay Area map and an activity-based trip
table, Section 7.1) are not available; these grids stand in for them at the
paper's scale (about 0.5M nodes, 1M links and 19M trips per day).

Conventions shared by everything downstream:
  * node ids are row-major grid positions (``r * n + c``);
  * directed links are sorted by ``(tail, head)`` and the link id is the
    position in that order;
  * free-flow times are int32 counts of ``quantum_s`` seconds (0.01 s);
  * capacities are float64 vehicles per hour;
  * trip amounts are int64 fixed point with 32 fractional bits.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

FX_ONE = 1 << 32  # one trip in the int64 fixed-point amount format

# link classes: (speed km/h, lanes, vehicles per hour per lane)
LOCAL, ARTERIAL, FREEWAY = 0, 1, 2
CLASS_SPEED_KMH = np.array([40.0, 60.0, 105.0])
CLASS_CAPACITY_VPH = np.array([1 * 800.0, 2 * 900.0, 4 * 2000.0])


@dataclasses.dataclass
class Network:
    """A directed road graph in the library's input layout."""

    n_nodes: int
    tail: np.ndarray       # int32 [L], nondecreasing
    head: np.ndarray       # int32 [L]
    fftime_q: np.ndarray   # int32 [L], free-flow time in quanta (>= 1)
    capacity: np.ndarray   # float64 [L], veh/h
    length_m: np.ndarray   # float64 [L]
    link_class: np.ndarray  # int8 [L]
    x: np.ndarray          # float64 [V] metres
    y: np.ndarray          # float64 [V] metres
    alpha: float = 0.15
    beta: int = 4
    quantum_s: float = 0.01

    @property
    def n_links(self) -> int:
        return int(self.tail.shape[0])


@dataclasses.dataclass
class Demand:
    """Trips of one interval, grouped by destination root.

    ``roots`` are destination nodes; every item ``k`` travels from node
    ``src[k]`` to node ``roots[root_idx[k]]`` with ``amount_fx[k]`` trips in
    32-bit fixed point.  Items are sorted by ``(root_idx, src)`` and unique.
    """

    roots: np.ndarray      # int32 [R]
    root_idx: np.ndarray   # int32 [n]
    src: np.ndarray        # int32 [n]
    amount_fx: np.ndarray  # int64 [n]

    @property
    def n_items(self) -> int:
        return int(self.src.shape[0])

    def total_trips(self) -> float:
        return float(self.amount_fx.sum()) / FX_ONE


def grid_network(n: int, seed: int, *, freeways: bool = False,
                 spacing_m: float = 250.0, jitter_m: float = 50.0,
                 delete_frac: float = 0.05, quantum_s: float = 0.01,
                 alpha: float = 0.15, beta: int = 4) -> Network:
    """n x n jittered grid with local / arterial / freeway links.

    Every undirected grid edge gets a length drawn from U[100, 400] m and
    becomes two directed links.  Rows and columns with index % 8 == 0 are
    arterials; with ``freeways`` those with index % 32 == 0 are freeways.
    ``delete_frac`` of the local undirected edges are removed; a random
    spanning tree is protected first, so the graph stays strongly connected.
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree

    rng = np.random.default_rng(seed)
    ids = np.arange(n * n, dtype=np.int64).reshape(n, n)
    gx = np.arange(n)[None, :] * spacing_m + rng.uniform(-jitter_m, jitter_m, (n, n))
    gy = np.arange(n)[:, None] * spacing_m + rng.uniform(-jitter_m, jitter_m, (n, n))

    # undirected edges: horizontal ones lie on row r, vertical ones on column c
    hu, hv = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    hline = np.repeat(np.arange(n), n - 1)
    vu, vv = ids[:-1, :].ravel(), ids[1:, :].ravel()
    vline = np.tile(np.arange(n), n - 1)
    u = np.concatenate([hu, vu])
    v = np.concatenate([hv, vv])
    line = np.concatenate([hline, vline])
    cls = np.full(u.shape[0], LOCAL, dtype=np.int8)
    cls[line % 8 == 0] = ARTERIAL
    if freeways:
        cls[line % 32 == 0] = FREEWAY
    length = rng.uniform(100.0, 400.0, u.shape[0])

    # protect a random spanning tree, then delete a fraction of local edges
    w = rng.uniform(1.0, 2.0, u.shape[0])
    m = coo_matrix((w, (u, v)), shape=(n * n, n * n)).tocsr()
    t = minimum_spanning_tree(m).tocoo()
    tr, tc = t.row.astype(np.int64), t.col.astype(np.int64)  # int64: the key exceeds 2^31 on large grids
    tree_key = set((np.minimum(tr, tc) * (n * n) + np.maximum(tr, tc)).tolist())
    key = np.minimum(u, v) * (n * n) + np.maximum(u, v)
    in_tree = np.fromiter((k in tree_key for k in key.tolist()), dtype=bool, count=key.shape[0])
    cand = np.flatnonzero((cls == LOCAL) & ~in_tree)
    n_del = int(round(delete_frac * int((cls == LOCAL).sum())))
    n_del = min(n_del, cand.shape[0])
    drop = rng.choice(cand, n_del, replace=False)
    keep = np.ones(u.shape[0], dtype=bool)
    keep[drop] = False
    u, v, cls, length = u[keep], v[keep], cls[keep], length[keep]

    tail = np.concatenate([u, v])
    head = np.concatenate([v, u])
    cls2 = np.concatenate([cls, cls])
    len2 = np.concatenate([length, length])
    order = np.lexsort((head, tail))
    tail, head, cls2, len2 = tail[order], head[order], cls2[order], len2[order]
    speed_ms = CLASS_SPEED_KMH[cls2] / 3.6
    fftime_q = np.rint(len2 / speed_ms / quantum_s).astype(np.int64)
    fftime_q = np.maximum(fftime_q, 1).astype(np.int32)
    return Network(
        n_nodes=n * n,
        tail=tail.astype(np.int32), head=head.astype(np.int32),
        fftime_q=fftime_q, capacity=CLASS_CAPACITY_VPH[cls2].astype(np.float64),
        length_m=len2, link_class=cls2, x=gx.ravel().copy(), y=gy.ravel().copy(),
        alpha=alpha, beta=beta, quantum_s=quantum_s)


def pick_zones(net: Network, n_zones: int, seed: int) -> np.ndarray:
    """Distinct random zone nodes (int32)."""
    rng = np.random.default_rng(seed + 7919)
    return np.sort(rng.choice(net.n_nodes, n_zones, replace=False)).astype(np.int32)


def _zone_distance(net: Network, zones: np.ndarray) -> np.ndarray:
    zx, zy = net.x[zones], net.y[zones]
    return np.hypot(zx[:, None] - zx[None, :], zy[:, None] - zy[None, :])


def _largest_remainder(weights: np.ndarray, total: int) -> np.ndarray:
    share = weights / weights.sum() * total
    base = np.floor(share).astype(np.int64)
    rest = int(total - base.sum())
    if rest > 0:
        frac = share - base
        top = np.argsort(-frac, kind="stable")[:rest]
        base[top] += 1
    return base


def demand_from_matrix(zones: np.ndarray, trips: np.ndarray) -> Demand:
    """Zone-by-zone integer trip matrix (origin row, destination column) to
    destination-grouped items.  Only destinations with trips become roots."""
    o, d = np.nonzero(trips)
    amt = trips[o, d].astype(np.int64)
    dest_used = np.unique(d)
    remap = np.full(zones.shape[0], -1, dtype=np.int64)
    remap[dest_used] = np.arange(dest_used.shape[0])
    root_idx = remap[d]
    src = zones[o].astype(np.int64)
    order = np.lexsort((src, root_idx))
    return Demand(roots=zones[dest_used].astype(np.int32),
                  root_idx=root_idx[order].astype(np.int32),
                  src=src[order].astype(np.int32),
                  amount_fx=(amt[order] * FX_ONE).astype(np.int64))


def gravity_fixed_pairs(net: Network, zones: np.ndarray, total: int,
                        scale_m: float) -> np.ndarray:
    """Every off-diagonal zone pair gets one trip; the rest of ``total`` is
    shared by largest remainder in proportion to exp(-d / scale)."""
    z = zones.shape[0]
    w = np.exp(-_zone_distance(net, zones) / scale_m)
    np.fill_diagonal(w, 0.0)
    off = z * (z - 1)
    if total < off:
        raise ValueError("total trips below the number of zone pairs")
    trips = np.ones((z, z), dtype=np.int64)
    np.fill_diagonal(trips, 0)
    trips += _largest_remainder(w.ravel(), total - off).reshape(z, z)
    np.fill_diagonal(trips, 0)
    return trips


def gravity_weights(net: Network, zones: np.ndarray, seed: int,
                    scale_m: float, mu: float = 4.0, sigma: float = 1.0) -> np.ndarray:
    """P_p * P_q * exp(-d/scale) with lognormal productions (attractions equal
    productions); zero diagonal; normalised to sum 1."""
    rng = np.random.default_rng(seed + 104729)
    prod = rng.lognormal(mu, sigma, zones.shape[0])
    w = prod[:, None] * prod[None, :] * np.exp(-_zone_distance(net, zones) / scale_m)
    np.fill_diagonal(w, 0.0)
    return w / w.sum()


def sample_trips(weights: np.ndarray, n_trips: int, seed: int) -> np.ndarray:
    """Multinomial sample of ``n_trips`` integer trips over a pair-weight matrix."""
    rng = np.random.default_rng(seed)
    cdf = np.cumsum(weights.ravel())
    cdf /= cdf[-1]
    pick = np.searchsorted(cdf, rng.random(n_trips), side="right")
    pick = np.minimum(pick, cdf.shape[0] - 1)
    counts = np.bincount(pick, minlength=cdf.shape[0])
    return counts.reshape(weights.shape).astype(np.int64)


def day_profile(n_intervals: int = 96, interval_h: float = 0.25) -> np.ndarray:
    """Bimodal time-of-day weights: a 1 % floor plus AM (08:00) and PM (17:00)
    Gaussian peaks of 0.75 h standard deviation, at interval midpoints."""
    t = (np.arange(n_intervals) + 0.5) * interval_h
    s = 0.75
    return 0.01 + np.exp(-(t - 8.0) ** 2 / (2 * s * s)) + np.exp(-(t - 17.0) ** 2 / (2 * s * s))


def day_interval_totals(total_trips: int, n_intervals: int = 96) -> np.ndarray:
    return _largest_remainder(day_profile(n_intervals), total_trips)


@dataclasses.dataclass
class Instance:
    name: str
    net: Network
    zones: np.ndarray
    demand: list  # list[Demand], one per interval
    dt_s: float = 900.0


def config_small(seed: int = 0) -> Instance:
    """32x32 grid, 64 zones, 20,000 trips over every zone pair, exp(-d/2 km)."""
    net = grid_network(32, seed)
    zones = pick_zones(net, 64, seed)
    trips = gravity_fixed_pairs(net, zones, 20000, 2000.0)
    return Instance("grid32_z64_t20k", net, zones, [demand_from_matrix(zones, trips)])


def config_metro(seed: int = 1, n: int = 500, n_zones: int = 2000,
                 n_trips: int = 250_000) -> Instance:
    """Metro grid (freeways every 32nd line), lognormal productions, gravity
    exp(-d/10 km), multinomially sampled integer trips."""
    net = grid_network(n, seed, freeways=True)
    zones = pick_zones(net, n_zones, seed)
    w = gravity_weights(net, zones, seed, 10000.0)
    trips = sample_trips(w, n_trips, seed + 1)
    return Instance(f"grid{n}_z{n_zones}_t{n_trips // 1000}k", net, zones,
                    [demand_from_matrix(zones, trips)])


def config_day(seed: int = 2, n: int = 500, n_zones: int = 2000,
               trips_per_day: int = 19_000_000, n_intervals: int = 96,
               scale_m: float = 10000.0) -> Instance:
    """Full day: interval totals from the bimodal profile, per-interval
    multinomial OD samples (seed 2 + i) of one gravity distribution.  Every
    interval's demand uses the full zone list as its roots so that residual
    trips can be merged across intervals by zone index."""
    net = grid_network(n, seed, freeways=(n >= 64))
    zones = pick_zones(net, n_zones, seed)
    w = gravity_weights(net, zones, seed, scale_m)
    totals = day_interval_totals(trips_per_day, n_intervals)
    days = []
    for i in range(n_intervals):
        trips = sample_trips(w, int(totals[i]), 2 + i)
        o, d = np.nonzero(trips)
        src = zones[o].astype(np.int64)
        order = np.lexsort((src, d))
        days.append(Demand(roots=zones.copy(), root_idx=d[order].astype(np.int32),
                           src=src[order].astype(np.int32),
                           amount_fx=(trips[o, d][order].astype(np.int64) * FX_ONE)))
    return Instance(f"day{n_intervals}_grid{n}_z{n_zones}_t{trips_per_day // 1000}k",
                    net, zones, days)


def chain_network(fftime_s, capacity_vph, quantum_s: float = 0.01,
                  alpha: float = 0.15, beta: int = 4) -> Network:
    """A serial chain 0 -> 1 -> ... -> m (one directed link per hop)."""
    m = len(fftime_s)
    tail = np.arange(m, dtype=np.int32)
    head = tail + 1
    ff = np.rint(np.asarray(fftime_s, dtype=np.float64) / quantum_s).astype(np.int32)
    return Network(n_nodes=m + 1, tail=tail, head=head, fftime_q=ff,
                   capacity=np.asarray(capacity_vph, dtype=np.float64),
                   length_m=np.zeros(m), link_class=np.zeros(m, dtype=np.int8),
                   x=np.arange(m + 1, dtype=np.float64), y=np.zeros(m + 1),
                   alpha=alpha, beta=beta, quantum_s=quantum_s)


def random_graph(n_nodes: int, n_extra: int, seed: int, *, max_q: int = 9,
                 equal_costs: bool = False) -> Network:
    """Small random strongly connected digraph (a Hamiltonian cycle plus
    ``n_extra`` random links), used for brute-force checks; small integer
    costs make ties frequent."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n_nodes)
    pairs = {(int(perm[i]), int(perm[(i + 1) % n_nodes])) for i in range(n_nodes)}
    while len(pairs) < n_nodes + n_extra and len(pairs) < n_nodes * (n_nodes - 1):
        a, b = (int(v) for v in rng.integers(0, n_nodes, 2))
        if a != b:
            pairs.add((a, b))
    arr = np.array(sorted(pairs), dtype=np.int32).reshape(-1, 2)
    ll = arr.shape[0]
    q = np.ones(ll, dtype=np.int32) if equal_costs else rng.integers(1, max_q + 1, ll).astype(np.int32)
    return Network(n_nodes=n_nodes, tail=arr[:, 0].copy(), head=arr[:, 1].copy(),
                   fftime_q=q, capacity=rng.uniform(50.0, 500.0, ll),
                   length_m=np.zeros(ll), link_class=np.zeros(ll, dtype=np.int8),
                   x=rng.uniform(0, 1000, n_nodes), y=rng.uniform(0, 1000, n_nodes))


def random_demand(net: Network, n_roots: int, n_items: int, seed: int,
                  max_trips: int = 50, fractional: bool = False) -> Demand:
    """Random destination-grouped items over ``n_roots`` distinct roots."""
    rng = np.random.default_rng(seed)
    roots = np.sort(rng.choice(net.n_nodes, n_roots, replace=False)).astype(np.int32)
    ri = rng.integers(0, n_roots, n_items)
    src = rng.integers(0, net.n_nodes, n_items)
    key = np.unique(ri * net.n_nodes + src)
    ri, src = key // net.n_nodes, key % net.n_nodes
    if fractional:
        amt = rng.integers(1, max_trips * FX_ONE, key.shape[0], dtype=np.int64)
    else:
        amt = rng.integers(1, max_trips + 1, key.shape[0]).astype(np.int64) * FX_ONE
    return Demand(roots=roots, root_idx=ri.astype(np.int32), src=src.astype(np.int32),
                  amount_fx=amt)


def scaled_day(inst_small: Instance, trips_per_day: int, n_intervals: int = 96,
               seed: int = 2) -> Instance:
    """Full day on an existing network and zone set (gravity exp(-d/2 km))."""
    net, zones = inst_small.net, inst_small.zones
    w = np.exp(-_zone_distance(net, zones) / 2000.0)
    np.fill_diagonal(w, 0.0)
    w /= w.sum()
    totals = day_interval_totals(trips_per_day, n_intervals)
    days = []
    for i in range(n_intervals):
        trips = sample_trips(w, int(totals[i]), seed + i)
        o, d = np.nonzero(trips)
        src = zones[o].astype(np.int64)
        order = np.lexsort((src, d))
        days.append(Demand(roots=zones.copy(), root_idx=d[order].astype(np.int32),
                           src=src[order].astype(np.int32),
                           amount_fx=(trips[o, d][order].astype(np.int64) * FX_ONE)))
    return Instance(f"day{n_intervals}_{inst_small.name}_t{trips_per_day}", net, zones, days)


def seconds_to_quanta(seconds: float, quantum_s: float) -> int:
    return int(math.floor(seconds / quantum_s + 0.5))
