"""Pins of the CPU oracle against facts fixed outside it: exact arithmetic,
brute force on tiny graphs, closed forms, the paper's worked example
(Section 6), invariants of loading (Eq. 5) and finite differences.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2104_12911_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------------------
# fixed-point reductions
# ----------------------------------------------------------------------------
def _rne(fr: Fraction) -> int:
    fl = math.floor(fr)
    rem = fr - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        return fl + 1
    return fl


def test_fx_rounding_matches_exact_rational():
    rng = np.random.default_rng(1)
    vals = list(rng.standard_normal(2000) * 10.0 ** rng.integers(-12, 18, 2000))
    vals += [0.5 * 2.0 ** -32, 1.5 * 2.0 ** -32, 2.5 * 2.0 ** -32, -0.5 * 2.0 ** -32, 3.0, -7.25,
             2.0 ** -40, 1e15 + 0.123, -(2.0 ** 60)]
    for v in vals:
        got, bad = oracle.to_fx(v)
        assert bad == 0
        assert got == _rne(Fraction(v) * (1 << 32)), v


def test_fx_to_double_is_correctly_rounded():
    rng = np.random.default_rng(2)
    for _ in range(3000):
        nbits = int(rng.integers(1, 126))
        x = int(rng.integers(0, 1 << 62)) << max(nbits - 62, 0) | int(rng.integers(0, 1 << 30))
        x &= (1 << nbits) - 1
        if rng.random() < 0.5:
            x = -x
        want = float(Fraction(x, 1 << 32))   # Python rounds int/int correctly
        assert oracle.fx_to_double(x) == want
    # ties to even at the 53-bit boundary
    x = ((1 << 53) + 1) << 40
    assert oracle.fx_to_double(x) == float(Fraction(x, 1 << 32))


# ----------------------------------------------------------------------------
# BPR (Eq. 1) and the worked example (Section 6)
# ----------------------------------------------------------------------------
def _bpr_exact(c0, cap, flow, dt_h, a=Fraction(15, 100), b=4):
    x = Fraction(flow) / (Fraction(cap) * Fraction(dt_h))
    return Fraction(c0) * (1 + Fraction(a) * x ** b)


def test_bpr_hand_values_and_quantisation():
    net = synth.chain_network([10.0, 20.0, 0.02, 7.0], [800.0, 1800.0, 100.0, 50.0])
    g = oracle.OracleGraph(net)
    flow = np.array([200.0, 0.0, 3.0, 1e-9])
    q, cost, rc = oracle.bpr(g, flow, 900.0)
    assert rc == 0
    for a in range(4):
        want = _bpr_exact(int(net.fftime_q[a]), net.capacity[a], flow[a], Fraction(1, 4))
        assert abs(cost[a] / 0.01 - float(want)) <= 1e-12 * float(want)
        assert q[a] == max(1, math.floor(want + Fraction(1, 2)))
    # NaN flow is reported
    _, _, rc = oracle.bpr(g, np.array([np.nan, 0, 0, 0.0]), 900.0)
    assert rc == oracle.ENONFINITE


def _worked():
    with open(os.path.join(HERE, "golden", "worked_example.json")) as fh:
        ex = json.load(fh)
    ff = [ex["links"][k][0] * 60.0 for k in ("l12", "l23", "l34", "l45")]
    cap = [float(ex["links"][k][1]) for k in ("l12", "l23", "l34", "l45")]
    return ex, synth.chain_network(ff, cap)


def _od(roots, items):
    roots = np.array(roots, dtype=np.int32)
    ri = np.array([i[0] for i in items], dtype=np.int32)
    src = np.array([i[1] for i in items], dtype=np.int32)
    amt = np.array([int(round(i[2] * (1 << 32))) for i in items], dtype=np.int64)
    return synth.Demand(roots, ri, src, amt)


def test_worked_example_bpr_values():
    ex, net = _worked()
    g = oracle.OracleGraph(net)
    # t1: 175 v/h for 15 min = 43.75 trips on l23; t2: 225 v/h = 56.25 trips on l34
    q, cost, _ = oracle.bpr(g, np.array([0.0, 43.75, 56.25, 0.0]), 900.0)
    l23, l34 = cost[1] / 60.0, cost[2] / 60.0
    assert abs(l23 - 6.389) < 5e-4 and abs(l23 - ex["printed"]["l23_t1_minutes"]) < 0.1
    assert abs(l34 - 12.4027) < 5e-4 and abs(l34 - ex["printed"]["l34_t2_minutes"]) < 0.1


def test_worked_example_qdta_day():
    """QDTA over four 15-minute periods: d14 is truncated at node 3 in t1
    (node 2 reached at ~10.9 min, node 3 at ~17.3 min > 15) and finishes in
    t2 together with d35; l45 carries only d35's trips."""
    ex, net = _worked()
    g = oracle.OracleGraph(net)
    zones = np.array([3, 4], dtype=np.int32)   # paper nodes 4 and 5
    d = [_od(zones, [(0, 0, 175 * 0.25)]), _od(zones, [(1, 2, 50 * 0.25)]),
         _od(zones, []), _od(zones, [])]
    flows, stats, nitems, rn, rc = oracle.run_day(g, zones, d, 900.0,
                                                  oracle.make_params(oracle.STEP_SWEEP8,
                                                                     oracle.STOP_REL_GAP, 50))
    assert rc == 0 and rn == 0
    assert ex["printed"]["residual_node_t1"] == 3
    np.testing.assert_array_equal(flows[0], [43.75, 43.75, 0.0, 0.0])
    np.testing.assert_array_equal(flows[1], [0.0, 0.0, 56.25, 12.5])
    np.testing.assert_array_equal(flows[2], 0.0)
    assert list(nitems) == [1, 2, 0, 0]      # residual 3->4 merged into t2


def test_worked_example_sta():
    """STA over the hour (no truncation): flows 175, 175, 225, 50 trips, i.e.
    43.75/43.75/56.25/12.5 per 15 minutes (printed 44, 44, 57, 13)."""
    ex, net = _worked()
    g = oracle.OracleGraph(net)
    zones = np.array([3, 4], dtype=np.int32)
    od = oracle.OracleOD.of(_od(zones, [(0, 0, 175.0), (1, 2, 50.0)]))
    f, st, rc = oracle.assign_interval(g, od, 3600.0,
                                       oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_REL_GAP, 50))
    assert rc == 0
    np.testing.assert_array_equal(f, [175.0, 175.0, 225.0, 50.0])
    p = ex["printed"]["sta_link_flows_vph"]
    half_up = lambda v: math.floor(v + 0.5)   # the paper prints 12.5 as 13
    assert half_up(f[0] / 4) == p["l12"] and half_up(f[1] / 4) == p["l23"] and half_up(f[3] / 4) == p["l45"]


# ----------------------------------------------------------------------------
# shortest paths against Floyd-Warshall and the smallest-id rule
# ----------------------------------------------------------------------------
def _floyd(net, q):
    V = net.n_nodes
    INF = np.iinfo(np.int64).max // 4
    D = np.full((V, V), INF, dtype=np.int64)
    np.fill_diagonal(D, 0)
    for e in range(net.n_links):
        a, b = net.tail[e], net.head[e]
        D[a, b] = min(D[a, b], int(q[e]))
    for k in range(V):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D, INF


@pytest.mark.parametrize("seed,equal", [(s, s % 3 == 0) for s in range(12)])
def test_sssp_against_floyd_warshall(seed, equal):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(2, 40))
    net = synth.random_graph(V, int(rng.integers(0, 3 * V)), seed, max_q=5, equal_costs=equal)
    g = oracle.OracleGraph(net)
    q = net.fftime_q
    D, INF = _floyd(net, q)
    roots = np.arange(V, dtype=np.int32)
    for direction in (oracle.DIR_TO_ROOT, oracle.DIR_FROM_ROOT):
        parent, dist = oracle.sssp(g, q, roots, direction)
        for r in range(V):
            want = D[:, r] if direction == oracle.DIR_TO_ROOT else D[r, :]
            np.testing.assert_array_equal(dist[r], np.where(want >= INF, oracle.DIST_INF, want))
            for v in range(V):
                if v == r:
                    assert parent[r, v] == -1
                    continue
                # brute force: every link that starts (ends) some shortest path
                if direction == oracle.DIR_TO_ROOT:
                    ok = [e for e in range(net.n_links) if net.tail[e] == v
                          and q[e] + D[net.head[e], r] == D[v, r]]
                else:
                    ok = [e for e in range(net.n_links) if net.head[e] == v
                          and D[r, net.tail[e]] + q[e] == D[r, v]]
                assert parent[r, v] == min(ok)


# ----------------------------------------------------------------------------
# loading: conservation (Eq. 5), the cost identity, the truncation rule (Eq. 2)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("dt_q", [np.iinfo(np.int64).max, 7, 15])
def test_load_invariants(seed, dt_q):
    rng = np.random.default_rng(100 + seed)
    V = int(rng.integers(5, 30))
    net = synth.random_graph(V, 2 * V, seed, max_q=6, equal_costs=(seed == 0))
    g = oracle.OracleGraph(net)
    dem = synth.random_demand(net, min(4, V), 40, seed, fractional=(seed % 2 == 1))
    od = oracle.OracleOD.of(dem)
    q = net.fftime_q
    D, INF = _floyd(net, q)
    parent, dist = oracle.sssp(g, q, dem.roots)
    flow, stop, rc = oracle.load(g, q, parent, od, dt_q)
    assert rc == 0
    big = [int(x) for x in dem.amount_fx]
    # identity: sum_a q_a g_a = sum_items amount * (elapsed at stop node)
    lhs = sum(int(q[e]) * int(flow[e]) for e in range(net.n_links))
    rhs = 0
    for k in range(dem.n_items):
        p, z, s = dem.src[k], dem.roots[dem.root_idx[k]], stop[k]
        rhs += big[k] * int(D[p, z] - D[s, z])
        # truncation: the stop node is reached at >= dt, its predecessor before dt
        el = D[p, z] - D[s, z]
        if s != z:
            assert el >= dt_q
        if dt_q == np.iinfo(np.int64).max:
            assert s == z
    assert lhs == rhs
    # conservation at every node: inflow - outflow = arrivals/stops - departures
    bal = np.zeros(V, dtype=object)
    for e in range(net.n_links):
        bal[net.head[e]] += int(flow[e])
        bal[net.tail[e]] -= int(flow[e])
    want = np.zeros(V, dtype=object)
    for k in range(dem.n_items):
        if stop[k] != dem.src[k]:
            want[stop[k]] += big[k]
            want[dem.src[k]] -= big[k]
    assert list(bal) == list(want)


def test_truncation_stops_at_first_node_reaching_dt():
    # chain 0->1->2->3 with link times 5, 5, 5; dt = 10: node 2 is reached at
    # exactly 10 and counts as reached, so links 0 and 1 are loaded.
    net = synth.chain_network([0.05, 0.05, 0.05], [100.0, 100.0, 100.0])
    g = oracle.OracleGraph(net)
    q = net.fftime_q
    od = oracle.OracleOD(np.array([3], np.int32), np.array([0], np.int32),
                         np.array([0], np.int32), np.array([1 << 32], np.int64))
    parent, _ = oracle.sssp(g, q, od.roots)
    for dt, wflow, wstop in [(10, [1, 1, 0], 2), (11, [1, 1, 1], 3), (15, [1, 1, 1], 3),
                             (1, [1, 0, 0], 1), (0, [0, 0, 0], 0)]:
        flow, stop, rc = oracle.load(g, q, parent, od, dt)
        assert list(flow >> 32) == wflow and stop[0] == wstop


# ----------------------------------------------------------------------------
# Beckmann objective (Eq. 6) and its slope against quadrature
# ----------------------------------------------------------------------------
def test_objective_and_slope_against_quadrature():
    from scipy.integrate import quad
    rng = np.random.default_rng(5)
    net = synth.random_graph(8, 10, 5)
    g = oracle.OracleGraph(net)
    L = net.n_links
    dt_s = 900.0
    f = rng.uniform(0, 300, L)
    gfx = (rng.uniform(0, 300, L) * (1 << 32)).astype(np.int64)
    gd = gfx.astype(np.float64) / (1 << 32)

    def c(a, t):
        return net.fftime_q[a] * (1 + 0.15 * (t / (net.capacity[a] * 0.25)) ** 4)

    want = sum(quad(lambda s, a=a: c(a, s), 0, f[a], epsabs=0, epsrel=1e-13)[0] for a in range(L))
    assert abs(oracle.objective(g, f, dt_s) - want) <= 1e-10 * want
    for alpha in (0.0, 0.3, 1.0):
        t = f + alpha * (gd - f)
        want_slope = sum((gd[a] - f[a]) * c(a, t[a]) for a in range(L))
        scale = sum(abs(gd[a] - f[a]) * c(a, t[a]) for a in range(L))
        assert abs(oracle.slope(g, f, gfx, dt_s, alpha) - want_slope) <= 1e-12 * scale


@pytest.mark.parametrize("mode", [oracle.STEP_PAPER_QN3, oracle.STEP_SWEEP8, oracle.STEP_EXACT])
def test_line_search_against_dense_grid(mode):
    from scipy.integrate import quad
    rng = np.random.default_rng(11)
    net = synth.random_graph(10, 15, 3)
    g = oracle.OracleGraph(net)
    L = net.n_links
    f = rng.uniform(0, 400, L)
    gfx = (rng.uniform(0, 400, L) * (1 << 32)).astype(np.int64)
    gd = gfx / float(1 << 32)

    def C(alpha):
        t = f + alpha * (gd - f)
        return sum(net.fftime_q[a] * (t[a] + 0.15 * net.capacity[a] * 0.25 / 5 *
                                      (t[a] / (net.capacity[a] * 0.25)) ** 5) for a in range(L))

    grid = np.linspace(0, 1, 20001)
    vals = np.array([C(a) for a in grid])
    best = grid[int(np.argmin(vals))]
    alpha, passes, rc = oracle.line_search(g, f, gfx, 900.0, 1,
                                           oracle.make_params(mode, oracle.STOP_NONE, 20))
    assert rc == 0 and 0.0 <= alpha <= 1.0
    assert abs(alpha - best) <= 2e-4
    if mode == oracle.STEP_PAPER_QN3:
        assert passes <= 19
    # convexity of phi along the line
    d = np.diff(vals)
    assert np.all(np.diff(d) >= -1e-6 * np.abs(vals).max())


def test_sweep8_returns_the_exact_step_when_the_slope_is_linear():
    """With BPR beta = 1 the objective (Eq. 6) is quadratic along the FW
    direction, so its slope is linear in alpha and the step has a closed form:
    alpha* = -S0 / S1 with S0 = sum c0 (1 + a f/K)(g - f), S1 = sum c0 a (g - f)^2 / K
    (K = C dt_h).  The 8-point sweep returns the secant zero of the slope
    inside its final bracket, which is alpha* up to the rounding of the
    fixed-point sums; a midpoint return would be off by up to T2 / 2."""
    rng = np.random.default_rng(23)
    net = synth.random_graph(10, 15, 5)
    net.beta = 1
    g = oracle.OracleGraph(net)
    L = net.n_links
    K = [Fraction(float(c)) * Fraction(900, 3600) for c in net.capacity]
    a_bpr = Fraction(net.alpha)
    checked = 0
    for trial in range(6):
        f = rng.uniform(0, 400, L)
        gfx = (rng.uniform(0, 400, L) * (1 << 32)).astype(np.int64)
        d = [Fraction(int(gfx[a]), 1 << 32) - Fraction(float(f[a])) for a in range(L)]
        S0 = sum(int(net.fftime_q[a]) * (1 + a_bpr * Fraction(float(f[a])) / K[a]) * d[a] for a in range(L))
        S1 = sum(int(net.fftime_q[a]) * a_bpr * d[a] * d[a] / K[a] for a in range(L))
        if not (S0 < 0 < S0 + S1):  # interior minimiser only
            continue
        want = float(-S0 / S1)
        alpha, passes, rc = oracle.line_search(g, f, gfx, 900.0, 1,
                                               oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_NONE, 20))
        assert rc == 0 and abs(alpha - want) < 1e-9, (trial, alpha, want)
        assert abs(alpha - want) < 1e-3 * 1e-4  # far inside the T2 = 1e-4 bracket
        checked += 1
    assert checked >= 2


# ----------------------------------------------------------------------------
# equilibrium closed forms (Eq. 4 with strictly increasing costs)
# ----------------------------------------------------------------------------
def _two_links(ff1, ff2, cap1, cap2):
    net = synth.Network(n_nodes=2, tail=np.array([0, 0], np.int32), head=np.array([1, 1], np.int32),
                        fftime_q=np.array([ff1, ff2], np.int32),
                        capacity=np.array([cap1, cap2], np.float64), length_m=np.zeros(2),
                        link_class=np.zeros(2, np.int8), x=np.zeros(2), y=np.zeros(2))
    return net


def _solve(net, demand_trips, mode, dt_s=3600.0, it=400, tol=1e-7):
    g = oracle.OracleGraph(net)
    od = oracle.OracleOD(np.array([1], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                         np.array([int(demand_trips * (1 << 32))], np.int64))
    return oracle.assign_interval(g, od, dt_s, oracle.make_params(mode, oracle.STOP_REL_GAP, it, tol))


@pytest.mark.parametrize("mode", [oracle.STEP_SWEEP8, oracle.STEP_PAPER_QN3, oracle.STEP_EXACT])
def test_two_identical_parallel_links_split_evenly(mode):
    f, st, rc = _solve(_two_links(60000, 60000, 1000.0, 1000.0), 3000.0, mode)
    assert rc >= 0
    assert abs(f[0] - 1500.0) <= 1e-6 * 3000.0 and abs(f.sum() - 3000.0) < 1e-9


def test_dominated_link_gets_nothing():
    # link 2's free-flow time exceeds link 1's cost at full demand
    net = _two_links(60000, 90000, 1000.0, 1000.0)
    c1_full = 60000 * (1 + 0.15 * (1000 / 1000.0) ** 4)
    assert 90000 > c1_full
    for mode in (oracle.STEP_MSA, oracle.STEP_SWEEP8):
        f, st, rc = _solve(net, 1000.0, mode, it=30)
        assert f[1] == 0.0 and f[0] == 1000.0


def test_asymmetric_two_links_equal_cost_root():
    net = _two_links(60000, 72000, 1200.0, 800.0)
    D = 2500.0

    def diff(x):   # c1(x) - c2(D - x) with hourly flows over one hour
        return (60000 * (1 + 0.15 * (x / 1200.0) ** 4)) - (72000 * (1 + 0.15 * ((D - x) / 800.0) ** 4))

    lo, hi = 0.0, D
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if diff(mid) < 0 else (lo, mid)
    x_star = 0.5 * (lo + hi)
    for mode in (oracle.STEP_SWEEP8, oracle.STEP_EXACT, oracle.STEP_PAPER_QN3):
        f, st, rc = _solve(net, D, mode, it=2000, tol=1e-8)
        # quantised link times (0.01 s on ~10-20 min) bound the reachable accuracy
        assert abs(f[0] - x_star) <= 2e-3 * D, (mode, f, x_star)


def test_braess_network_wardrop():
    # 0->1 (variable), 0->2 (long fixed), 1->3 (long fixed), 2->3 (variable), 1->2 bridge
    ff = [60000, 150000, 150000, 60000, 6000]
    cap = [500.0, 1e9, 1e9, 500.0, 1e9]
    tail = np.array([0, 0, 1, 1, 2], np.int32)
    head = np.array([1, 2, 2, 3, 3], np.int32)
    order_ff = {(0, 1): (60000, 500.0), (0, 2): (150000, 1e9), (1, 2): (6000, 1e9),
                (1, 3): (150000, 1e9), (2, 3): (60000, 500.0)}
    fq = np.array([order_ff[(int(a), int(b))][0] for a, b in zip(tail, head)], np.int32)
    cp = np.array([order_ff[(int(a), int(b))][1] for a, b in zip(tail, head)], np.float64)
    net = synth.Network(n_nodes=4, tail=tail, head=head, fftime_q=fq, capacity=cp,
                        length_m=np.zeros(5), link_class=np.zeros(5, np.int8),
                        x=np.zeros(4), y=np.zeros(4))
    g = oracle.OracleGraph(net)
    D = 1000.0
    od = oracle.OracleOD(np.array([3], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                         np.array([int(D * (1 << 32))], np.int64))
    f, st, rc = oracle.assign_interval(g, od, 3600.0,
                                       oracle.make_params(oracle.STEP_EXACT, oracle.STOP_REL_GAP, 5000, 1e-7))
    _, cost, _ = oracle.bpr(g, f, 3600.0)
    link = {(int(a), int(b)): e for e, (a, b) in enumerate(zip(tail, head))}
    paths = [[(0, 1), (1, 3)], [(0, 2), (2, 3)], [(0, 1), (1, 2), (2, 3)]]
    pc = [sum(cost[link[x]] for x in p) for p in paths]
    best = min(pc)
    # flows on each path from link flows (the network is small enough to solve)
    for p, c in zip(paths, pc):
        used = min(f[link[x]] for x in p) > 1e-6 * D
        if used:
            assert c <= best * (1 + 2e-4)
        else:
            assert c >= best * (1 - 2e-4)
    assert abs(f[link[(0, 1)]] + f[link[(0, 2)]] - D) < 1e-6


# ----------------------------------------------------------------------------
# step rules and the residual demand (Alg. 4)
# ----------------------------------------------------------------------------
def test_msa_is_the_running_mean_of_aon_flows(small_instance):
    g = oracle.OracleGraph(small_instance.net)
    od = oracle.OracleOD.of(small_instance.demand[0])
    f, st, rc, tape = oracle.assign_interval(g, od, 900.0,
                                             oracle.make_params(oracle.STEP_MSA, oracle.STOP_NONE, 6),
                                             tape=True)
    L = g.n_links
    K = tape.K.value
    assert K == 6 and st["aon_calls"] == 7
    acc = np.zeros(L)
    for j in range(K + 1):
        q = tape.q[j * L:(j + 1) * L]
        par, _ = oracle.sssp(g, q, od.roots, want_dist=False)
        gfx, _, _ = oracle.load(g, q, par, od, 90000)
        acc += gfx / float(1 << 32)
    np.testing.assert_allclose(f, acc / (K + 1), rtol=1e-12, atol=1e-9)


def test_residual_conserves_trips_and_matches_flows_without_truncation(small_instance):
    g = oracle.OracleGraph(small_instance.net)
    od = oracle.OracleOD.of(small_instance.demand[0])
    p = oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_REL_GAP, 60, 1e-3)
    for dt in (600.0, 1e9):
        f, st, rc, tape = oracle.assign_interval(g, od, dt, p, tape=True)
        h, (rs, rr, ra, _, _), rc2 = oracle.residual(g, od, dt, tape, f)
        assert rc2 == 0
        K = tape.K.value
        total_in = int(od.amount_fx.sum())
        if dt > 1e8:
            assert ra.shape[0] == 0
            np.testing.assert_allclose(h / float(1 << 32), f, rtol=1e-9, atol=1e-6)
        else:
            assert ra.shape[0] > 0
            assert np.all(rs != small_instance.demand[0].roots[rr])
            assert int(ra.sum()) <= total_in + (K + 1) * od.src.shape[0]
            # balance of h at nodes that are neither roots nor origins: what
            # flows in and does not flow out is exactly what stopped there
            V = g.n_nodes
            bal = np.zeros(V, dtype=np.int64)
            np.add.at(bal, small_instance.net.head, h)
            np.add.at(bal, small_instance.net.tail, -h)
            stopped = np.zeros(V, dtype=np.int64)
            np.add.at(stopped, rs, ra)
            free = np.ones(V, dtype=bool)
            free[od.roots] = False
            free[od.src] = False
            np.testing.assert_array_equal(bal[free], stopped[free])


# ----------------------------------------------------------------------------
# adjoint against central finite differences (trees held fixed)
# ----------------------------------------------------------------------------
def _small_grid_case(seed=4):
    net = synth.grid_network(6, seed)
    zones = synth.pick_zones(net, 6, seed)
    trips = synth.gravity_fixed_pairs(net, zones, 900, 800.0)
    dem = synth.demand_from_matrix(zones, trips)
    return net, dem


@pytest.mark.parametrize("mode", [oracle.STEP_EXACT, oracle.STEP_MSA])
def test_adjoint_matches_finite_differences(mode):
    net, dem = _small_grid_case()
    g = oracle.OracleGraph(net)
    od = oracle.OracleOD.of(dem)
    dt = 300.0
    p = oracle.make_params(mode, oracle.STOP_NONE, 8)
    f, st, rc, tape = oracle.assign_interval(g, od, dt, p, tape=True)
    rng = np.random.default_rng(0)
    L = g.n_links
    S = rng.choice(L, max(2, L // 4), replace=False)
    y = f[S] * rng.lognormal(0, 0.3, S.shape[0])

    def loss(ff):
        return float(((ff[S] - y) ** 2).sum())

    dLdf = np.zeros(L)
    dLdf[S] = 2 * (f[S] - y)
    dd, dc, rcb = oracle.backward(g, od, dt, mode, tape, dLdf)
    assert rcb == 0
    for k in rng.choice(dem.n_items, 8, replace=False):
        h = 1e-3 * dem.amount_fx[k]
        vals = []
        for sgn in (1, -1):
            amt = dem.amount_fx.copy()
            amt[k] += int(sgn * h)
            ff, _ = oracle.replay(g, oracle.OracleOD(dem.roots, dem.root_idx, dem.src, amt), dt, p, tape)
            vals.append(loss(ff))
        fd = (vals[0] - vals[1]) / (2 * int(h) / float(1 << 32))
        assert abs(fd - dd[k]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(dd).max()), (k, fd, dd[k])
    if mode == oracle.STEP_MSA:
        assert np.all(dc == 0.0)
    else:
        for a in rng.choice(L, 8, replace=False):
            hc = 1e-3 * net.capacity[a]
            vals = []
            for sgn in (1, -1):
                cap = net.capacity.copy()
                cap[a] += sgn * hc
                g2 = oracle.OracleGraph(net, capacity=cap)
                ff, _ = oracle.replay(g2, od, dt, p, tape)
                vals.append(loss(ff))
            fd = (vals[0] - vals[1]) / (2 * hc)
            assert abs(fd - dc[a]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(dc).max()), (a, fd, dc[a])


# ---------------------------------------------------------------------------
# Scenario metrics (Section 7.1): VMT, average VOC, VHD by class; the congested
# subset has VOC >= 1.0.  Pinned against exact rationals on a hand-sized case.
def test_interval_metrics_against_exact_rationals():
    from fractions import Fraction as Fr
    # four links, 10 s free flow (1000 quanta), 400 veh/h: over 15 min the capacity is
    # 100 trips, so the flows below give volume/capacity 0.5, 1.0, 1.5 and 0 exactly
    net = synth.chain_network([10.0] * 4, [400.0] * 4)
    g = oracle.OracleGraph(net)
    flows = np.array([[50.0, 100.0, 150.0, 0.0]])
    length = np.array([100.0, 200.0, 300.0, 400.0])
    cls = np.array([0, 1, 0, 1], np.int32)
    out, rc = oracle.interval_metrics(g, flows, 900.0, length, cls, 2)
    assert rc == 0
    x = [Fr(1, 2), Fr(1), Fr(3, 2)]
    f = [Fr(50), Fr(100), Fr(150)]
    delay_q = [f[a] * 1000 * Fr(15, 100) * x[a] ** 4 for a in range(3)]  # f * (c - c0), quanta
    to_h = Fr(1, 100) / 3600
    # class 0: links 0 and 2; class 1: link 1 (link 3 carries no flow and is not counted)
    want0 = [2, Fr(50 * 100 + 150 * 300, 1000), (x[0] + x[2]) / 2, (delay_q[0] + delay_q[2]) * to_h,
             1, Fr(300, 1000), Fr(150 * 300, 1000), x[2]]
    want1 = [1, Fr(100 * 200, 1000), x[1], delay_q[1] * to_h, 1, Fr(200, 1000), Fr(100 * 200, 1000), x[1]]
    for got, want in ((out[0, 0], want0), (out[0, 1], want1)):
        for m, w in enumerate(want):
            assert abs(got[m] - float(w)) <= 1e-12 * max(1.0, abs(float(w))), (m, got[m], float(w))


def test_interval_metrics_classes_partition_the_network():
    inst = synth.config_small(0)
    net = inst.net
    g = oracle.OracleGraph(net)
    rng = np.random.default_rng(5)
    flows = rng.uniform(0, 250, (3, g.n_links)) * (rng.random((3, g.n_links)) < 0.8)
    length = rng.uniform(100, 400, g.n_links)
    cls = rng.integers(0, 3, g.n_links).astype(np.int32)
    per, rc1 = oracle.interval_metrics(g, flows, 900.0, length, cls, 3)
    one, rc2 = oracle.interval_metrics(g, flows, 900.0, length, np.zeros(g.n_links, np.int32), 1)
    assert rc1 == 0 and rc2 == 0
    for i in range(3):
        assert per[i, :, 0].sum() == one[i, 0, 0] == np.count_nonzero(flows[i] > 0)
        assert per[i, :, 4].sum() == one[i, 0, 4]
        for m in (1, 3, 5, 6):  # additive quantities
            assert abs(per[i, :, m].sum() - one[i, 0, m]) <= 1e-12 * one[i, 0, m]
        # averages are count-weighted means of the class averages
        for m, c in ((2, 0), (7, 4)):
            assert abs((per[i, :, m] * per[i, :, c]).sum() / one[i, 0, c] - one[i, 0, m]) <= 1e-12
        assert np.all(per[i, :, 6] <= per[i, :, 1]) and np.all(per[i, :, 4] <= per[i, :, 0])
        # a class index outside [0, n_classes) is not counted
    bad = cls.copy()
    bad[:10] = 7
    part, rc3 = oracle.interval_metrics(g, flows, 900.0, length, bad, 3)
    assert rc3 == 0 and part[:, :, 0].sum() == np.count_nonzero(flows[:, 10:] > 0)


# ---------------------------------------------------------------------------
# System-optimal objective (the alternative named in Sections 3 and 8): total
# cost sum f c(f), routing on marginal costs m = c + f c'.
def _solve_so(net, demand_trips, mode, it=2000, tol=1e-8, objective=oracle.OBJ_SO):
    g = oracle.OracleGraph(net)
    od = oracle.OracleOD(np.array([1], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                         np.array([int(demand_trips * (1 << 32))], np.int64))
    return oracle.assign_interval(g, od, 3600.0, oracle.make_params(mode, oracle.STOP_REL_GAP, it, tol,
                                                                    objective=objective))


def test_system_optimum_two_identical_links_split_evenly():
    for mode in (oracle.STEP_SWEEP8, oracle.STEP_EXACT):
        f, st, rc = _solve_so(_two_links(60000, 60000, 1000.0, 1000.0), 3000.0, mode, it=400, tol=1e-7)
        assert rc >= 0 and abs(f[0] - 1500.0) <= 1e-6 * 3000.0


def test_system_optimum_equalises_marginal_costs():
    net = _two_links(60000, 72000, 1200.0, 800.0)
    D = 2500.0

    def root(fn):
        lo, hi = 0.0, D
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if fn(mid) < 0 else (lo, mid)
        return 0.5 * (lo + hi)

    # marginal cost c0 (1 + alpha (beta+1) x^beta) of BPR, hourly flows over one hour
    x_so = root(lambda x: 60000 * (1 + 0.75 * (x / 1200.0) ** 4) - 72000 * (1 + 0.75 * ((D - x) / 800.0) ** 4))
    x_ue = root(lambda x: 60000 * (1 + 0.15 * (x / 1200.0) ** 4) - 72000 * (1 + 0.15 * ((D - x) / 800.0) ** 4))
    assert abs(x_so - x_ue) > 10 * 2e-3 * D  # the two objectives are told apart
    for mode in (oracle.STEP_SWEEP8, oracle.STEP_EXACT, oracle.STEP_PAPER_QN3):
        f, st, rc = _solve_so(net, D, mode)
        assert abs(f[0] - x_so) <= 2e-3 * D, (mode, f, x_so)


def test_system_optimum_total_cost_not_above_equilibrium_braess():
    # Braess network: the equilibrium uses the bridge and costs more in total than the optimum
    tail = np.array([0, 0, 1, 1, 2], np.int32)
    head = np.array([1, 2, 2, 3, 3], np.int32)
    spec = {(0, 1): (60000, 500.0), (0, 2): (150000, 1e9), (1, 2): (6000, 1e9),
            (1, 3): (150000, 1e9), (2, 3): (60000, 500.0)}
    fq = np.array([spec[(int(a), int(b))][0] for a, b in zip(tail, head)], np.int32)
    cp = np.array([spec[(int(a), int(b))][1] for a, b in zip(tail, head)], np.float64)
    net = synth.Network(n_nodes=4, tail=tail, head=head, fftime_q=fq, capacity=cp, length_m=np.zeros(5),
                        link_class=np.zeros(5, np.int8), x=np.zeros(4), y=np.zeros(4))
    g = oracle.OracleGraph(net)
    od = oracle.OracleOD(np.array([3], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                         np.array([int(1000.0 * (1 << 32))], np.int64))

    def total(obj):
        f, st, rc = oracle.assign_interval(g, od, 3600.0, oracle.make_params(
            oracle.STEP_EXACT, oracle.STOP_REL_GAP, 5000, 1e-7, objective=obj))
        assert rc >= 0
        _, cost, _ = oracle.bpr(g, f, 3600.0)
        return float((f * cost).sum()), st

    z_ue, _ = total(oracle.OBJ_UE)
    z_so, st_so = total(oracle.OBJ_SO)
    assert z_so <= z_ue * (1 + 1e-9) and z_so < z_ue * (1 - 1e-3)
    # the optimum's reported objective is its total cost, in quanta x trips (cost above is in seconds)
    assert abs(st_so["objective"] * net.quantum_s - z_so) <= 1e-9 * z_so


def test_system_optimum_equals_equilibrium_for_constant_costs():
    """alpha = 0: marginal cost = cost, total cost and Beckmann integral agree
    operation for operation, so both objectives give the same bits."""
    inst = synth.scaled_day(synth.config_small(0), 40000, n_intervals=2, seed=3)
    net = inst.net
    net0 = synth.Network(n_nodes=net.n_nodes, tail=net.tail, head=net.head, fftime_q=net.fftime_q,
                         capacity=net.capacity, length_m=net.length_m, link_class=net.link_class, x=net.x,
                         y=net.y, alpha=0.0, beta=net.beta, quantum_s=net.quantum_s)
    g = oracle.OracleGraph(net0)
    od = oracle.OracleOD.of(inst.demand[1])
    out = []
    for obj in (oracle.OBJ_UE, oracle.OBJ_SO):
        f, st, rc = oracle.assign_interval(g, od, 900.0, oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_NONE, 5,
                                                                            objective=obj))
        assert rc >= 0
        out.append((f, st["iterations"], st["ls_passes"]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


def test_day_advances_a_trip_one_link_per_interval_when_links_outlast_dt():
    """Links of 20 min, intervals of 15 min: under reading R1 the trip is
    loaded on one link per interval (the link it is on when the interval
    starts) and waits at that link's head: no stall at the origin."""
    net = synth.chain_network([1200.0, 1200.0, 1200.0], [1000.0, 1000.0, 1000.0])
    g = oracle.OracleGraph(net)
    zones = np.array([3], np.int32)
    one = synth.Demand(roots=zones, root_idx=np.array([0], np.int32), src=np.array([0], np.int32),
                       amount_fx=np.array([1 << 32], np.int64))
    empty = synth.Demand(roots=zones, root_idx=np.zeros(0, np.int32), src=np.zeros(0, np.int32),
                         amount_fx=np.zeros(0, np.int64))
    f, st, nit, rn, rc = oracle.run_day(g, zones, [one, empty, empty, empty], 900.0,
                                        oracle.make_params(oracle.STEP_MSA, oracle.STOP_NONE, 2))
    assert rc >= 0
    f = np.asarray(f).reshape(4, 3)
    # step-weighted shares are rounded to 2^-32 trips each (R9)
    np.testing.assert_allclose(f, [[1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, 0]], rtol=0, atol=4 * 2.0 ** -32)
    assert list(nit) == [1, 1, 1, 0]


def _frac(x):
    """a fraction of a link in the 2^-32 units of the carried position"""
    return x * 2.0 ** -32


def test_carried_truncation_crosses_a_long_link_over_several_intervals():
    """Section 3.4's alternative to Eq. 2 (reading R17): links of 1000 s on an
    uncongested chain, intervals of 300 s.  A trip leaving node 0 at time 0
    enters link k at 1000 k s, so link k is loaded in exactly the interval
    containing 1000 k s (0, 3 and 6); the trip is in the network until it
    arrives at 3000 s, the end of interval 9.  Under the node rule (R1) the
    same trip advances one link per interval instead."""
    net = synth.chain_network([1000.0, 1000.0, 1000.0], [1e9, 1e9, 1e9])
    g = oracle.OracleGraph(net)
    zones = np.array([3], np.int32)
    one = synth.Demand(roots=zones, root_idx=np.array([0], np.int32), src=np.array([0], np.int32),
                       amount_fx=np.array([1 << 32], np.int64))
    empty = synth.Demand(roots=zones, root_idx=np.zeros(0, np.int32), src=np.zeros(0, np.int32),
                         amount_fx=np.zeros(0, np.int64))
    N = 11
    want = np.zeros((N, 3))
    for k in range(3):
        want[(1000 * k) // 300, k] = 1.0
    f, st, nit, rn, rc = oracle.run_day(g, zones, [one] + [empty] * (N - 1), 300.0,
                                        oracle.make_params(oracle.STEP_MSA, oracle.STOP_NONE, 0,
                                                           truncation=oracle.TRUNC_CARRY))
    assert rc >= 0
    np.testing.assert_array_equal(np.asarray(f).reshape(N, 3), want)
    assert list(nit) == [1] * 10 + [0] and rn == 0
    f, st, nit, rn, rc = oracle.run_day(g, zones, [one] + [empty] * 3, 300.0,
                                        oracle.make_params(oracle.STEP_MSA, oracle.STOP_NONE, 0))
    np.testing.assert_array_equal(np.asarray(f).reshape(4, 3), [[1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, 0]])


def _two_groups(N):
    """chain of 1000 s links, 300 s intervals: 1 trip leaves node 0 in
    interval 0, 3 trips in interval 1"""
    net = synth.chain_network([1000.0, 1000.0, 1000.0], [1e9, 1e9, 1e9])
    zones = np.array([3], np.int32)

    def trips(n):
        return synth.Demand(roots=zones, root_idx=np.array([0], np.int32), src=np.array([0], np.int32),
                            amount_fx=np.array([n << 32], np.int64))
    empty = synth.Demand(roots=zones, root_idx=np.zeros(0, np.int32), src=np.zeros(0, np.int32),
                         amount_fx=np.zeros(0, np.int64))
    return oracle.OracleGraph(net), zones, [trips(1), trips(3)] + [empty] * (N - 2)


def test_carried_trips_merge_with_their_mean_covered_fraction():
    """Reading R17's merge: trips waiting at the same node for the same zone
    are one residual item (the paper's d_{s,q}); trips on a link merge per
    (zone, link) with the amount-weighted mean fraction of the link covered.
    After interval 1 the first trip has covered 0.6 of link 0 and the three
    later ones 0.3, so interval 2 starts one item of 4 trips at
    (0.6 + 3 x 0.3) / 4 = 0.375.  From there, by hand: the group reaches
    node 1 at 25 s into interval 4 (entering link 1 then), node 2 at 125 s
    into interval 7, and arrives 225 s into interval 10.  Each link is loaded
    in the interval the trips enter it."""
    N = 12
    g, zones, days = _two_groups(N)
    f, st, nit, rn, rc = oracle.run_day(g, zones, days, 300.0, oracle.make_params(
        oracle.STEP_MSA, oracle.STOP_NONE, 0, truncation=oracle.TRUNC_CARRY))
    assert rc >= 0
    want = np.zeros((N, 3))
    want[0, 0], want[1, 0], want[4, 1], want[7, 2] = 1, 3, 4, 4
    np.testing.assert_array_equal(np.asarray(f).reshape(N, 3), want)
    assert list(nit) == [1, 2] + [1] * 9 + [0] and rn == 0


def test_day_residual_holds_the_merged_carried_group():
    """The residual a day leaves, for the two trip groups of the test above:
    after intervals 0-1 one item of 4 trips on link 0 having covered 0.375 of
    it; after intervals 0-4 the group is on link 1 (tail node 1), 0.275 along
    it (it reached node 1 at 25 s into interval 4).  Fractions in units of
    2^-32, floored at each step, so within a few units of the exact value."""
    for n_int, (src, link, frac) in ((2, (0, 0, 0.375)), (5, (1, 1, 0.275))):
        g, zones, days = _two_groups(n_int)
        p = oracle.make_params(oracle.STEP_MSA, oracle.STOP_NONE, 0, truncation=oracle.TRUNC_CARRY)
        *_, rn, rc, res = oracle.run_day(g, zones, days, 300.0, p, want_resid=True)
        assert rc >= 0 and rn == 1
        root, s_, amt, f_, l_ = (int(a[0]) for a in res)
        assert (root, s_, amt, l_) == (0, src, 4 << 32, link)
        assert abs(_frac(f_) - frac) < 8 * 2.0 ** -32, _frac(f_)


def test_carried_truncation_stop_node_and_covered_fraction():
    """One walk on the uncongested chain of 1000 s links for a trip already at
    position P seconds from node 0 (on link P // 1000 having covered
    (P mod 1000) / 1000 of it, or at the node when that is 0): after an
    interval of 300 s it is at position P + 300, on link (P + 300) // 1000
    having covered ((P + 300) mod 1000) / 1000 of it, at a node when that is
    0, and has arrived at node 3 when P + 300 >= 3000.  It loads only the
    links it enters."""
    net = synth.chain_network([1000.0, 1000.0, 1000.0], [1e9, 1e9, 1e9])
    g = oracle.OracleGraph(net)
    par, _ = oracle.sssp(g, net.fftime_q, np.array([3], np.int32), want_dist=False)
    for pos in (0, 100, 600, 700, 900, 1000, 1750, 2700, 2850):
        node, along = divmod(pos, 1000)
        od = oracle.OracleOD(np.array([3], np.int32), np.array([0], np.int32), np.array([node], np.int32),
                             np.array([1 << 32], np.int64),
                             carry_frac=np.array([(along << 32) // 1000], np.int64),
                             carry_link=np.array([node if along else -1], np.int32))
        f, stop, carry, link, rc = oracle.load(g, net.fftime_q, par, od, 30000, truncation=oracle.TRUNC_CARRY,
                                               want_carry=True)
        t = pos + 300
        entered = [k for k in range(3) if pos <= 1000 * k < t and (1000 * k > pos or along == 0)]
        assert rc == 0 and list(f >> 32) == [int(k in entered) for k in range(3)], (pos, f >> 32)
        if t >= 3000:
            assert (stop[0], carry[0], link[0]) == (3, 0, -1)
        elif t % 1000 == 0:
            assert (stop[0], carry[0], link[0]) == (t // 1000, 0, -1), pos
        else:
            assert (stop[0], link[0]) == (t // 1000, t // 1000), pos
            assert abs(_frac(carry[0]) - (t % 1000) / 1000) < 4 * 2.0 ** -32, (pos, _frac(carry[0]))


def test_carried_position_is_a_fraction_of_the_link():
    """Section 3.4 tracks the distance covered on a link: a trip that covered
    0.3 of a link whose time then doubles has 0.7 x 2000 s = 1400 s left, not
    the 1700 s a carried time would leave.  Chain of one 1000 s link, link
    time 2000 s in the next interval (given directly as the walk's link
    times), interval of 1000 s: 0.3 + 1000 / 2000 = 0.8 covered; with 1500 s
    it arrives at 1400 s."""
    net = synth.chain_network([1000.0], [1e9])
    g = oracle.OracleGraph(net)
    q2 = np.array([200000], np.int32)
    par, _ = oracle.sssp(g, q2, np.array([1], np.int32), want_dist=False)
    od = oracle.OracleOD(np.array([1], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                         np.array([1 << 32], np.int64), carry_frac=np.array([(3 << 32) // 10], np.int64),
                         carry_link=np.array([0], np.int32))
    f, stop, carry, link, rc = oracle.load(g, q2, par, od, 100000, truncation=oracle.TRUNC_CARRY, want_carry=True)
    assert rc == 0 and int(f[0]) == 0 and (stop[0], link[0]) == (0, 0)
    assert abs(_frac(carry[0]) - 0.8) < 4 * 2.0 ** -32
    f, stop, carry, link, rc = oracle.load(g, q2, par, od, 150000, truncation=oracle.TRUNC_CARRY, want_carry=True)
    assert rc == 0 and (stop[0], carry[0], link[0]) == (1, 0, -1)
    for dt_q in (139999, 140000):  # the rest is exactly 140000 quanta
        _, stop, _, link, _ = oracle.load(g, q2, par, od, dt_q, truncation=oracle.TRUNC_CARRY, want_carry=True)
        assert (stop[0], link[0]) == ((0, 0) if dt_q < 140000 else (1, -1))


def test_carried_trip_finishes_its_link_before_rerouting():
    """A trip carried on link 0->2 of the diamond (routes 0->1->3 and
    0->2->3) stays on it although the tree from node 0 leads through node 1:
    it covers the rest of 0->2, then follows the tree from node 2, loading
    only 2->3 (0->2 was loaded when it was entered).  The same trip waiting
    at node 0 instead takes 0->1."""
    net = _diamond([200, 340, 1000, 400], [1e9, 1e9, 1e9, 1e9])  # links 0->1, 0->2, 1->3, 2->3
    g = oracle.OracleGraph(net)
    q = np.array([20000, 90000, 20000, 20000], np.int32)  # 0->1->3 is shorter than 0->2->3
    par, _ = oracle.sssp(g, q, np.array([3], np.int32), want_dist=False)
    assert par[0][0] == 0  # the tree leaves node 0 by link 0->1
    on = oracle.OracleOD(np.array([3], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                         np.array([1 << 32], np.int64), carry_frac=np.array([(2 << 32) // 3], np.int64),
                         carry_link=np.array([1], np.int32))
    f, stop, carry, link, rc = oracle.load(g, q, par, on, 90000, truncation=oracle.TRUNC_CARRY, want_carry=True)
    # 1/3 of 900 s left on 0->2 (node 2 at 300 s), then 200 s on 2->3: arrived at 500 s
    assert rc == 0 and list(f >> 32) == [0, 0, 0, 1] and (stop[0], carry[0], link[0]) == (3, 0, -1)
    at = oracle.OracleOD(np.array([3], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                         np.array([1 << 32], np.int64))
    f, stop, rc = oracle.load(g, q, par, at, 90000, truncation=oracle.TRUNC_CARRY)
    assert list(f >> 32) == [1, 0, 1, 0] and stop[0] == 3


def test_carried_truncation_loads_the_links_of_the_node_rule():
    """Both truncation rules load a link iff the elapsed time at its tail is
    below dt; they differ only in where the residual trip waits.  So the
    first interval of a day (no carried trips yet) has the same h(0) under
    both, while later intervals differ."""
    inst = synth.scaled_day(synth.config_small(0), 60000, n_intervals=4, seed=5)
    g = oracle.OracleGraph(inst.net)
    out = []
    for trunc in (oracle.TRUNC_NODE, oracle.TRUNC_CARRY):
        f, st, nit, rn, rc = oracle.run_day(g, inst.zones, list(inst.demand), 150.0,
                                            oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_PAPER_OBJ, 30,
                                                               truncation=trunc))
        assert rc >= 0
        out.append((np.asarray(f), nit))
    np.testing.assert_array_equal(out[0][0][0], out[1][0][0])
    assert out[0][1][0] == out[1][1][0]
    assert not np.array_equal(out[0][0][1:], out[1][0][1:]) and out[1][1][1] > out[0][1][1]


# ----------------------------------------------------------------------------
# the relative-gap stop rule under truncation
# ----------------------------------------------------------------------------
def _diamond(ff_s, cap):
    """0 -> 1 -> 3 and 0 -> 2 -> 3 (links 0->1, 0->2, 1->3, 2->3)."""
    return synth.Network(n_nodes=4, tail=np.array([0, 0, 1, 2], np.int32), head=np.array([1, 2, 3, 3], np.int32),
                         fftime_q=np.rint(np.array(ff_s, np.float64) / 0.01).astype(np.int32),
                         capacity=np.array(cap, np.float64), length_m=np.zeros(4), link_class=np.zeros(4, np.int8),
                         x=np.arange(4.0), y=np.zeros(4))


def _diamond_od(trips):
    return oracle.OracleOD(np.array([3], np.int32), np.array([0], np.int32), np.array([0], np.int32),
                           np.array([trips << 32], np.int64))


def test_rel_gap_stop_ignores_a_negative_gap():
    """With Δt = 300 s, route B (0->2 340 s, 2->3 400 s) is shortest at free
    flow and its trips stop at node 2 (Eq. 2), loading only 0->2.  Congested
    by 100 trips at 632.6 veh/h, 0->2 costs c02 ≈ 1000 s, so route A (0->1
    200 s, 1->3 1000 s) becomes shortest and its trips arrive, loading 1200 s.
    The gap (c02·100 - 1200·100) / (c02·100) is then negative: the truncated
    all-or-nothing loading does not minimise sum c g.  Moving towards it raises
    the objective, so every step is 0 and the gap stays; the relative-gap rule
    must not report convergence on it."""
    net = _diamond([200, 340, 1000, 400], [5000, 632.6, 5000, 5000])
    og = oracle.OracleGraph(net)
    # c02 in quanta by Eq. 1, exact: 34000 (1 + 0.15 x^4), x = 100 / (632.6 · 300/3600)
    x = Fraction(100) / (Fraction(6326, 10) * Fraction(300, 3600))
    c02 = Fraction(34000) * (1 + Fraction(15, 100) * x ** 4)
    q02 = math.floor(c02 + Fraction(1, 2))
    want_gap = float(Fraction(q02 * 100 - 120000 * 100, q02 * 100))
    assert want_gap < -0.19
    f, st, rc = oracle.assign_interval(og, _diamond_od(100), 300.0,
                                       oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_REL_GAP, 12))
    assert abs(st["dual_gap"] - want_gap) < 1e-15
    assert st["converged"] == 0 and rc == oracle.NOTCONV and st["iterations"] == 12
    np.testing.assert_array_equal(f, [0.0, 100.0, 0.0, 0.0])
    # the paper's objective-change rule stops at once (the step is 0)
    f, st, rc = oracle.assign_interval(og, _diamond_od(100), 300.0,
                                       oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_PAPER_OBJ, 12))
    assert st["converged"] == 1 and rc == oracle.OK


def test_rel_gap_stop_accepts_zero_and_rounding_level_gaps():
    """Less congestion (700 veh/h): route B stays shortest, g = f and the gap
    is exactly 0, which stops at the first check.  On a two-route split whose
    first links tie in cost, the gap of an equilibrium comes out a few ulps
    below zero from the rounding of the products c f; it still stops."""
    og = oracle.OracleGraph(_diamond([200, 340, 1000, 400], [5000, 700.0, 5000, 5000]))
    f, st, rc = oracle.assign_interval(og, _diamond_od(100), 300.0,
                                       oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_REL_GAP, 12))
    assert st["dual_gap"] == 0.0 and st["converged"] == 1 and st["iterations"] == 0
    og = oracle.OracleGraph(_diamond([301, 340, 1000, 10], [400, 200, 400, 400]))
    f, st, rc = oracle.assign_interval(og, _diamond_od(150), 300.0,
                                       oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_REL_GAP, 30))
    assert -1e-15 < st["dual_gap"] <= 0.0 and st["converged"] == 1 and rc == oracle.OK
    assert abs(f.sum() - 150.0) < 1e-9 and f[2] == f[3] == 0.0


@pytest.mark.parametrize("steps", [(oracle.STEP_MSA, 0, oracle.OBJ_UE), (oracle.STEP_MSA, 5, oracle.OBJ_UE),
                                   (oracle.STEP_SWEEP8, 5, oracle.OBJ_UE), (oracle.STEP_SWEEP8, 5, oracle.OBJ_SO)])
@pytest.mark.parametrize("trunc", [oracle.TRUNC_NODE, oracle.TRUNC_CARRY])
def test_day_conserves_trips_on_a_congested_chain(trunc, steps):
    """Every trip of a single-destination chain loads the chain's last link
    exactly once, in the interval it enters it, under both truncation rules
    (a link is loaded when entered).  With one AON per interval (no FW steps,
    so no step weights and no rounding) the day therefore conserves trips
    exactly: the trips of all intervals = the last link's loads summed over the
    intervals + the residual left that has not entered the last link (trips
    waiting at a node, or carried on an earlier link).  The chain is congested
    (link times change with the interval's flows), so carried positions are
    scaled by changing link times on the way.  With K FW steps the residual
    pass splits each item over the K + 1 accepted AONs by their step weights,
    rounding each share to the nearest fixed-point unit, so the balance holds
    to within half a unit per share, for the system optimum too (routing on
    marginal costs, loading on travel times)."""
    net = synth.chain_network([400.0, 250.0, 700.0, 150.0], [900.0, 300.0, 1200.0, 500.0])
    g = oracle.OracleGraph(net)
    zones = np.array([4], np.int32)
    rng = np.random.default_rng(11)
    N = 10
    days = []
    for i in range(N):
        src = np.array([0, 1, 2], np.int32)
        amt = (rng.integers(0, 40, 3).astype(np.int64) << 32) + rng.integers(0, 1 << 32, 3)
        days.append(synth.Demand(roots=zones, root_idx=np.zeros(3, np.int32), src=src, amount_fx=amt))
    step, K, objective = steps
    p = oracle.make_params(step, oracle.STOP_NONE, K, objective=objective, truncation=trunc)
    f, st, nit, rn, rc, res = oracle.run_day(g, zones, days, 300.0, p, want_resid=True)
    assert rc >= 0
    flows_fx = np.rint(np.asarray(f).reshape(N, 4) * 2.0 ** 32).astype(np.int64)
    total = sum(int(d.amount_fx.sum()) for d in days)
    root_idx, src, amt, carry, link = res
    waiting = int(sum(a for a, l in zip(amt, link) if l != 3))
    shares = sum(int(n) for n in nit) * (K + 1)  # items x accepted AONs, an upper bound on the roundings
    assert abs(total - (int(flows_fx[:, 3].sum()) + waiting)) <= shares // 2 + 1
    assert int(flows_fx[:, 3].sum()) > 0 and waiting > 0  # trips both arrive and remain
    if trunc == oracle.TRUNC_CARRY:
        assert (link >= 0).any()  # some trips end the day on a link


@pytest.mark.parametrize("trunc", [oracle.TRUNC_NODE, oracle.TRUNC_CARRY])
def test_day_conserves_trips_per_destination_on_a_grid(trunc):
    """The chain test above on a small grid: every trip goes from one of five
    zones to a sixth, z, and loads exactly one link into z, on its last step
    (a trip that reaches z stops there).  With one AON per interval the trips
    of all intervals therefore equal the loads of z's in-links summed over the
    intervals plus the residual that has not entered an in-link of z.  One-
    minute intervals make trips cross several of them."""
    net = synth.grid_network(8, 3)
    g = oracle.OracleGraph(net)
    zones = synth.pick_zones(net, 6, 3)
    sink = int(zones[0])
    rng = np.random.default_rng(5)
    N = 8
    days = []
    for i in range(N):
        others = np.array([z for z in zones if z != sink], np.int32)
        amt = (rng.integers(0, 30, others.shape[0]).astype(np.int64) << 32) + rng.integers(0, 1 << 32, others.shape[0])
        days.append(synth.Demand(roots=zones.astype(np.int32), root_idx=np.zeros(others.shape[0], np.int32),
                                 src=others, amount_fx=amt))
    p = oracle.make_params(oracle.STEP_MSA, oracle.STOP_NONE, 0, truncation=trunc)
    f, st, nit, rn, rc, res = oracle.run_day(g, zones.astype(np.int32), days, 60.0, p, want_resid=True)
    assert rc >= 0
    flows_fx = np.rint(np.asarray(f).reshape(N, -1) * 2.0 ** 32).astype(np.int64)
    into = np.flatnonzero(np.asarray(net.head) == sink)
    arrived = int(flows_fx[:, into].sum())
    root_idx, src, amt, carry, link = res
    head = np.asarray(net.head)
    left = int(sum(a for a, l in zip(amt, link) if l < 0 or head[l] != sink))
    total = sum(int(d.amount_fx.sum()) for d in days)
    assert total == arrived + left
    assert arrived > 0 and left > 0


# ----------------------------------------------------------------------------
# customizable contraction hierarchy (the routing alternative of Section 5.1)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cch_distances_equal_dijkstra_on_random_graphs_with_ties(seed):
    """Any contraction order gives exact shortest times: all-pairs P2P
    queries and every one-to-all sweep against Dijkstra (itself pinned to
    Floyd-Warshall above), for two orders and two metrics (the hierarchy is
    built once and customized per metric), with many equal-cost ties.  Two
    extra nodes hang off the strongly connected graph by one link each, one
    leaving it (nothing reaches that node) and one entering it (that node
    reaches nothing): their pairs must stay infinite."""
    base = synth.random_graph(60, 120, seed, max_q=3)
    V0 = base.n_nodes
    tail = np.concatenate([base.tail, [V0, 5]]).astype(np.int32)  # links V0 -> 3 and 5 -> V0 + 1
    head = np.concatenate([base.head, [3, V0 + 1]]).astype(np.int32)
    order_l = np.lexsort((head, tail))
    net = synth.Network(n_nodes=V0 + 2, tail=tail[order_l], head=head[order_l],
                        fftime_q=np.concatenate([base.fftime_q, [2, 1]]).astype(np.int32)[order_l],
                        capacity=np.concatenate([base.capacity, [100.0, 100.0]])[order_l],
                        length_m=np.zeros(tail.shape[0]), link_class=np.zeros(tail.shape[0], np.int8),
                        x=np.zeros(V0 + 2), y=np.zeros(V0 + 2))
    g = oracle.OracleGraph(net)
    rng = np.random.default_rng(seed)
    V = net.n_nodes
    roots = np.arange(V, dtype=np.int32)
    for order in (rng.permutation(V), np.argsort(np.bincount(net.tail, minlength=V), kind="stable")):
        c = oracle.CCH(g, order)
        for q in (net.fftime_q, rng.integers(1, 4, net.tail.shape[0])):
            q = np.asarray(q, np.int32)
            c.customize(q)
            _, d = oracle.sssp(g, q, roots)  # d[z][v] = time v -> z
            assert (d[V0] == np.iinfo(np.int64).max).sum() == V - 1  # only V0 itself reaches V0
            assert (d[:, V0 + 1] == np.iinfo(np.int64).max).sum() == V - 1  # V0 + 1 reaches only itself
            s, t = np.meshgrid(np.arange(V, dtype=np.int32), roots)
            np.testing.assert_array_equal(c.distance(s.ravel(), t.ravel()).reshape(V, V), d)
            for z in range(V):
                np.testing.assert_array_equal(c.to_root(z), d[z])


def test_cch_one_to_all_on_a_grid_with_a_nested_dissection_order():
    """The 32 x 32 grid with a coordinate nested-dissection order and
    congested link times: every node's time to 12 roots, against Dijkstra.
    The destination trees then follow from those times by the tie rule
    (each node's parent is the smallest link id among its out-links that
    begin a shortest path), and equal Dijkstra's trees: a hierarchy can
    stand in for Bellman-Ford without changing a loaded flow."""
    net = synth.grid_network(32, 4)
    g = oracle.OracleGraph(net)
    c = oracle.CCH(g, oracle.nested_dissection_order(net.x, net.y, net.tail, net.head))
    rng = np.random.default_rng(4)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.tail.shape[0])).astype(np.int32)
    c.customize(q)
    roots = rng.choice(net.n_nodes, 12, replace=False).astype(np.int32)
    par, d = oracle.sssp(g, q, roots)
    tail, head = np.asarray(net.tail), np.asarray(net.head)
    for i, z in enumerate(roots):
        dz = c.to_root(z)
        np.testing.assert_array_equal(dz, d[i])
        tight = dz[head] + q.astype(np.int64) == dz[tail]
        tree = np.full(net.n_nodes, -1, np.int64)
        for a in np.flatnonzero(tight)[::-1]:  # descending, so the smallest id is written last
            if tail[a] != z:
                tree[tail[a]] = a
        np.testing.assert_array_equal(tree, par[i])


def test_cch_rejects_an_order_that_is_not_a_permutation():
    net = synth.grid_network(4, 1)
    g = oracle.OracleGraph(net)
    bad = np.zeros(net.n_nodes, np.int32)
    with pytest.raises(RuntimeError):
        oracle.CCH(g, bad)
