"""CUDA path (through the C ABI) against the CPU oracle on identical inputs.

Integer work (costs, distances, parents, loaded flows, stop nodes, merged
residual items) must be bit-exact; the FW iteration is bit-exact too because
every link sum is an exact fixed-point sum and every FP64 operation is
rounded in the same order on both sides.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2104_12911_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2104_12911_gb300 import qdta as Q  # noqa: E402

DEV = torch.device("cuda", 0)


def T(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(DEV)


@pytest.fixture(scope="module")
def small():
    inst = synth.config_small(0)
    return inst, Q.Graph(inst.net), oracle.OracleGraph(inst.net)


@pytest.fixture(scope="module")
def mid():
    # 110 x 110 grid: 12,100 nodes, above the shared-memory SSSP limit
    net = synth.grid_network(110, 5, freeways=True)
    zones = synth.pick_zones(net, 96, 5)
    trips = synth.sample_trips(synth.gravity_weights(net, zones, 5, 4000.0), 30000, 6)
    dem = synth.demand_from_matrix(zones, trips)
    return net, dem, Q.Graph(net), oracle.OracleGraph(net)


# ---------------------------------------------------------------------------
def test_bpr_bit_exact(small):
    inst, g, og = small
    rng = np.random.default_rng(0)
    L = og.n_links
    f = rng.uniform(0, 900, L) * (rng.random(L) < 0.8)
    f[:5] = [0.0, 1e-300, 1e6, 3.5, 800.0]
    for dt in (900.0, 300.0, 3600.0):
        q_o, c_o, rc = oracle.bpr(og, f, dt)
        q_g, c_g = Q.qdta_bpr_costs(g, T(f, np.float64), dt, want_cost_s=True)
        np.testing.assert_array_equal(q_g.cpu().numpy(), q_o)
        np.testing.assert_array_equal(c_g.cpu().numpy(), c_o)


def test_bpr_nonfinite_is_reported(small):
    inst, g, og = small
    f = np.zeros(og.n_links)
    f[3] = np.nan
    with pytest.raises(Q.QdtaError) as e:
        Q.qdta_bpr_costs(g, T(f, np.float64), 900.0)
    assert e.value.code == Q.QDTA_ENONFINITE


@pytest.mark.parametrize("direction", [Q.QDTA_TO_ROOT, Q.QDTA_FROM_ROOT])
def test_sssp_small_all_zones(small, direction):
    inst, g, og = small
    rng = np.random.default_rng(1)
    for trial in range(3):
        q = inst.net.fftime_q if trial == 0 else rng.integers(1, 5000, og.n_links).astype(np.int32)
        roots = inst.zones
        p_o, d_o = oracle.sssp(og, q, roots, direction)
        p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), direction, want_dist=True)
        np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
        np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


@pytest.mark.parametrize("seed", range(8))
def test_sssp_random_graphs_with_ties(seed):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(2, 300))
    net = synth.random_graph(V, int(rng.integers(0, 4 * V)), seed, max_q=3, equal_costs=(seed % 2 == 0))
    g, og = Q.Graph(net), oracle.OracleGraph(net)
    roots = np.arange(V, dtype=np.int32) if V < 64 else rng.choice(V, 64, replace=False).astype(np.int32)
    for direction in (Q.QDTA_TO_ROOT, Q.QDTA_FROM_ROOT):
        p_o, d_o = oracle.sssp(og, net.fftime_q, roots, direction)
        p_g, d_g = Q.qdta_sssp_batch(g, T(net.fftime_q, np.int32), T(roots, np.int32), direction, True)
        np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
        np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


def test_sssp_unreachable_nodes():
    # 0 -> 1 -> 2, node 3 isolated: unreachable rows keep -1 / INF
    net = synth.Network(n_nodes=4, tail=np.array([0, 1], np.int32), head=np.array([1, 2], np.int32),
                        fftime_q=np.array([5, 7], np.int32), capacity=np.ones(2) * 100,
                        length_m=np.zeros(2), link_class=np.zeros(2, np.int8), x=np.zeros(4), y=np.zeros(4))
    g, og = Q.Graph(net), oracle.OracleGraph(net)
    roots = np.array([2, 3, 0], np.int32)
    p_o, d_o = oracle.sssp(og, net.fftime_q, roots)
    p_g, d_g = Q.qdta_sssp_batch(g, T(net.fftime_q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, True)
    np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
    np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


LARGE_VARIANTS = {
    "default": ({}, "sssp_smq_kernel<256,rank32,2,true>"),
    "rank32_without_parent_skip": ({"QDTA_NO_PARENT_SKIP": "1"}, "sssp_smq_kernel<256,rank32,2,true>"),
    "rank64": ({"QDTA_SSSP_ADJ": "2"}, "sssp_smq_kernel<256,rank,2,true>"),
    "rank64_without_parent_skip": ({"QDTA_SSSP_ADJ": "2", "QDTA_NO_PARENT_SKIP": "1"},
                                   "sssp_smq_kernel<256,rank,2,true>"),
    "rank32_512": ({"QDTA_BF_SHAPE": "0"}, "sssp_smq_kernel<512,rank32,2,false>"),
    "rank32_five_ctas": ({"QDTA_BF_SHAPE": "3"}, "sssp_smq_kernel<256,rank32,2,true,5>"),
    "five_cta_shape_ell16": ({"QDTA_BF_SHAPE": "3", "QDTA_SSSP_ADJ": "1"}, "sssp_smq_kernel<256,ell,2,true>"),
    "rank32_npt5": ({"QDTA_BF_SHAPE": "4"}, "sssp_smq_kernel<256,rank32,2,true,npt5>"),
    "rank32_npt6": ({"QDTA_BF_SHAPE": "5"}, "sssp_smq_kernel<256,rank32,2,true,npt6>"),
    "ell16": ({"QDTA_SSSP_ADJ": "1"}, "sssp_smq_kernel<256,ell,2,true>"),
    "csr": ({"QDTA_NO_ELL": "1"}, "sssp_smq_kernel<256,csr,2,true>"),
    "no_reorder": ({"QDTA_NO_REORDER": "1"}, "sssp_smq_kernel<256,csr,2,true>"),
    "returning_atomic": ({"QDTA_BF_RELAX": "1", "QDTA_SSSP_ADJ": "1"}, "sssp_smq_kernel<256,ell,1,true>"),
    "atomic_only": ({"QDTA_BF_RELAX": "0", "QDTA_SSSP_ADJ": "1"}, "sssp_smq_kernel<256,ell,0,true>"),
    "two_bitmaps_512_rank64": ({"QDTA_BF_SHAPE": "0", "QDTA_SSSP_ADJ": "2"}, "sssp_smq_kernel<512,rank,2,false>"),
    "two_bitmaps_512_csr_returning": ({"QDTA_BF_SHAPE": "0", "QDTA_NO_ELL": "1", "QDTA_BF_RELAX": "1"},
                                      "sssp_smq_kernel<512,csr,1,false>"),
    "one_bitmap_512": ({"QDTA_BF_SHAPE": "2"}, "sssp_smq_kernel<512,rank32,2,true>"),
    "one_cta_per_sm": ({"QDTA_BF_BPSM": "1"}, "sssp_smq_kernel<256,rank32,2,true>"),
    "aggregated_appends": ({"QDTA_BF_RELAX": "3", "QDTA_SSSP_ADJ": "2"}, "sssp_smq_kernel<256,rank,3,true>"),
    "aggregated_appends_csr_512": ({"QDTA_BF_RELAX": "3", "QDTA_NO_ELL": "1", "QDTA_BF_SHAPE": "0"},
                                   "sssp_smq_kernel<512,csr,3,false>"),
    "output_external_order": ({"QDTA_SMQ_OUT": "0"}, "sssp_smq_kernel<256,rank32,2,true>"),
    "output_external_order_ell_512": ({"QDTA_SMQ_OUT": "0", "QDTA_BF_SHAPE": "0", "QDTA_SSSP_ADJ": "1"},
                                      "sssp_smq_kernel<512,ell,2,false>"),
    "lane_npn1": ({"QDTA_BF_SHAPE": "6"}, "sssp_lane_kernel<256,npn1>"),
    "lane_npn2": ({"QDTA_BF_SHAPE": "7"}, "sssp_lane_kernel<256,npn2>"),
    "lane_npn1_without_parent_skip": ({"QDTA_BF_SHAPE": "6", "QDTA_NO_PARENT_SKIP": "1"},
                                      "sssp_lane_kernel<256,npn1>"),
    "lane_npn2_external_order_flag": ({"QDTA_BF_SHAPE": "7", "QDTA_SMQ_OUT": "0"}, "sssp_lane_kernel<256,npn2>"),
    "lane_shape_ell16": ({"QDTA_BF_SHAPE": "6", "QDTA_SSSP_ADJ": "1"}, "sssp_smq_kernel<256,ell,2,true>"),
    "rank32_prefetch": ({"QDTA_BF_SHAPE": "8"}, "sssp_smq_kernel<256,rank32,2,true,pf>"),
    "rank32_192x5": ({"QDTA_BF_SHAPE": "9"}, "sssp_smq_kernel<192,rank32,2,true,5>"),
    "shape_192x5_ell16": ({"QDTA_BF_SHAPE": "9", "QDTA_SSSP_ADJ": "1"}, "sssp_smq_kernel<192,ell,2,true>"),
    "rank32_288x4": ({"QDTA_BF_SHAPE": "10"}, "sssp_smq_kernel<288,rank32,2,true>"),
    "shape_288x4_rank64": ({"QDTA_BF_SHAPE": "10", "QDTA_SSSP_ADJ": "2"}, "sssp_smq_kernel<256,rank,2,true>"),
    "shape_192x5_csr_returning": ({"QDTA_BF_SHAPE": "9", "QDTA_NO_ELL": "1", "QDTA_BF_RELAX": "1"},
                                  "sssp_smq_kernel<192,csr,1,true>"),
    "global_queues": ({"QDTA_BF_NOSMQ": "1", "QDTA_NO_REORDER": "1"}, "sssp_ilp_kernel<512>"),
    "cell": ({"QDTA_SSSP": "cell"}, "sssp_cell_kernel"),
}


@pytest.mark.parametrize("variant", list(LARGE_VARIANTS))
@pytest.mark.parametrize("direction", [Q.QDTA_TO_ROOT, Q.QDTA_FROM_ROOT])
def test_sssp_large_graph_variants(mid, variant, direction, monkeypatch):
    """Graphs above the shared-memory limit: every kernel variant, both
    directions, bit-exact against Dijkstra."""
    net, dem, _, og = mid
    env, kernel = LARGE_VARIANTS[variant]
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    g = Q.Graph(net)
    assert Q.qdta_sssp_kernel_name(g, direction) == kernel
    rng = np.random.default_rng(2)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.n_links)).astype(np.int32)
    roots = rng.choice(net.n_nodes, 40, replace=False).astype(np.int32)
    p_o, d_o = oracle.sssp(og, q, roots, direction)
    p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), direction, True)
    np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
    np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


@pytest.mark.parametrize("shape,kernel", [("1", "sssp_smq_kernel<256,rank32,2,true>"),
                                          ("6", "sssp_lane_kernel<256,npn1>"), ("7", "sssp_lane_kernel<256,npn2>")])
def test_sssp_rank_keys_on_a_graph_with_one_way_links(shape, kernel, monkeypatch):
    """Degree <= 4 but 3 % of links lose their reverse: the rank-keyed
    adjacency runs without the parent-slot skip; bit-exact both ways."""
    monkeypatch.setenv("QDTA_BF_SHAPE", shape)
    base = synth.grid_network(110, 9, freeways=True)
    rng = np.random.default_rng(9)
    keep = rng.random(base.n_links) >= 0.03
    net = synth.Network(n_nodes=base.n_nodes, tail=base.tail[keep].copy(), head=base.head[keep].copy(),
                        fftime_q=base.fftime_q[keep].copy(), capacity=base.capacity[keep].copy(),
                        length_m=base.length_m[keep].copy(), link_class=base.link_class[keep].copy(),
                        x=base.x, y=base.y)
    g, og = Q.Graph(net), oracle.OracleGraph(net)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.n_links)).astype(np.int32)
    roots = rng.choice(net.n_nodes, 40, replace=False).astype(np.int32)
    for direction in (Q.QDTA_TO_ROOT, Q.QDTA_FROM_ROOT):
        assert Q.qdta_sssp_kernel_name(g, direction) == kernel
        p_o, d_o = oracle.sssp(og, q, roots, direction)
        p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), direction, True)
        np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
        np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


@pytest.mark.parametrize("adj,shape", [("2", "1"), ("3", "1"), ("3", "6"), ("3", "7"), ("3", "8"), ("3", "9"),
                                       ("2", "9")])
def test_sssp_long_distances_redo_with_64_bit_keys(mid, adj, shape, monkeypatch):
    """Link times of 5e6..1e7 quanta push distances past 2^29: the 32-bit-key
    batch flags it and the 64-bit redo gives the oracle's bits."""
    net, dem, _, og = mid
    monkeypatch.setenv("QDTA_SSSP_ADJ", adj)
    monkeypatch.setenv("QDTA_BF_SHAPE", shape)
    g = Q.Graph(net)
    rng = np.random.default_rng(21)
    q = rng.integers(5_000_000, 10_000_000, net.n_links).astype(np.int32)
    roots = rng.choice(net.n_nodes, 24, replace=False).astype(np.int32)
    for direction in (Q.QDTA_TO_ROOT, Q.QDTA_FROM_ROOT):
        p_o, d_o = oracle.sssp(og, q, roots, direction)
        assert d_o[d_o < np.iinfo(np.int64).max].max() >= 1 << 29
        p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), direction, True)
        np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
        np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


@pytest.mark.parametrize("shape", ["1", "6", "7", "8", "9", "10"])
def test_sssp_redo_touches_only_the_roots_that_overflowed(mid, shape, monkeypatch):
    """Links entering three nodes cost 2^30: destination trees rooted there
    pass 2^29 (so the batch is redone with 64-bit keys), the other roots'
    trees stay below it; all rows bit-exact."""
    net, dem, _, og = mid
    monkeypatch.setenv("QDTA_BF_SHAPE", shape)
    g = Q.Graph(net)
    rng = np.random.default_rng(31)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.n_links)).astype(np.int64)
    bad = rng.choice(net.n_nodes, 3, replace=False)
    q[np.isin(net.head, bad)] = 1 << 30
    q = q.astype(np.int32)
    others = np.setdiff1d(rng.choice(net.n_nodes, 24, replace=False), bad)
    roots = np.concatenate([others[:10], bad, others[10:]]).astype(np.int32)
    p_o, d_o = oracle.sssp(og, q, roots, Q.QDTA_TO_ROOT)
    big = np.array([d[d < np.iinfo(np.int64).max].max() >= 1 << 29 for d in d_o])
    assert big.sum() == 3 and set(roots[big]) == set(bad)
    p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, True)
    np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
    np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


@pytest.mark.parametrize("shape", ["1", "6", "8", "9", "10"])
def test_sssp_32_bit_keys_redo_only_on_distances_beyond_2_29(mid, shape, monkeypatch):
    """An isolated node (no path to or from anything) stays unreached and
    must not trigger the 64-bit redo; a node whose distance passes 2^29 must.
    Bit-exact against Dijkstra either way."""
    net, dem, _, og = mid
    monkeypatch.setenv("QDTA_BF_SHAPE", shape)
    V = net.n_nodes
    iso = synth.Network(n_nodes=V + 1, tail=net.tail, head=net.head, fftime_q=net.fftime_q, capacity=net.capacity,
                        length_m=net.length_m, link_class=net.link_class, x=np.append(net.x, 0.0),
                        y=np.append(net.y, 0.0))
    g, og2 = Q.Graph(iso), oracle.OracleGraph(iso)
    rng = np.random.default_rng(8)
    roots = rng.choice(V, 24, replace=False).astype(np.int32)
    for scale, want_redo in ((1, False), (60_000, True)):
        q = np.minimum(net.fftime_q.astype(np.int64) * scale, 2**31 - 1).astype(np.int32)
        Q.qdta_profile_enable(g, True)
        p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, True)
        prof = Q.qdta_profile_read(g)
        p_o, d_o = oracle.sssp(og2, q, roots)
        np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
        np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)
        assert (prof["sssp_redo_batches"] > 0) == want_redo, (scale, prof["sssp_redo_batches"])
        assert (d_o[:, V] == np.iinfo(np.int64).max).all()


@pytest.mark.parametrize("shape", ["1", "6", "10"])
@pytest.mark.parametrize("schedule", ["round_robin", "fetch", "fetch_longest_first"])
def test_sssp_dynamic_root_fetch_covers_every_root(mid, shape, schedule, monkeypatch):
    """More roots than resident CTAs: handed out round-robin, by an atomic
    counter after the first wave, or by the counter in longest-first order
    (the rounds each root took in the previous batch, so the second batch
    runs in a different order from the first); every row bit-exact, in both
    directions, in both batches."""
    net, dem, _, og = mid
    monkeypatch.setenv("QDTA_BF_DYNAMIC", "0" if schedule == "round_robin" else "1")
    monkeypatch.setenv("QDTA_BF_LPT", "1" if schedule == "fetch_longest_first" else "0")
    monkeypatch.setenv("QDTA_BF_SHAPE", shape)
    g = Q.Graph(net)
    rng = np.random.default_rng(13)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.n_links)).astype(np.int32)
    roots = rng.choice(net.n_nodes, 1500, replace=False).astype(np.int32)
    for direction in (Q.QDTA_TO_ROOT, Q.QDTA_FROM_ROOT):
        p_o, d_o = oracle.sssp(og, q, roots, direction)
        for _ in range(2):
            p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), direction, True)
            np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
            np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


def test_sssp_batch_beyond_the_sort_limit_keeps_batch_order(mid, monkeypatch):
    """More than 4,096 roots: the longest-first sort leaves the batch in its
    own order (the fetch still hands the roots out); two batches, every row
    bit-exact against the oracle."""
    net, dem, _, og = mid
    monkeypatch.setenv("QDTA_BF_DYNAMIC", "1")
    monkeypatch.setenv("QDTA_BF_LPT", "1")
    g = Q.Graph(net)
    rng = np.random.default_rng(17)
    q = (net.fftime_q * rng.uniform(1.0, 2.0, net.n_links)).astype(np.int32)
    roots = rng.choice(net.n_nodes, 4100, replace=False).astype(np.int32)
    p_o, d_o = oracle.sssp(og, q, roots, Q.QDTA_TO_ROOT)
    for _ in range(2):
        p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, True)
        np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
        np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


def test_sssp_large_irregular_graph_with_ties():
    """Above the shared-memory limit with degrees above 4 (so the compressed
    adjacency, not the four-slot one) and many equal-cost ties: bit-exact
    distances and smallest-link-id parents in both directions."""
    net = synth.random_graph(12000, 36000, 11, max_q=3)
    g, og = Q.Graph(net), oracle.OracleGraph(net)
    rng = np.random.default_rng(12)
    roots = rng.choice(net.n_nodes, 48, replace=False).astype(np.int32)
    for direction in (Q.QDTA_TO_ROOT, Q.QDTA_FROM_ROOT):
        assert Q.qdta_sssp_kernel_name(g, direction) == "sssp_smq_kernel<256,csr,2,true>"
        p_o, d_o = oracle.sssp(og, net.fftime_q, roots, direction)
        p_g, d_g = Q.qdta_sssp_batch(g, T(net.fftime_q, np.int32), T(roots, np.int32), direction, True)
        np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
        np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


def test_sssp_graph_beyond_the_two_bitmap_limit():
    """A 600 x 600 grid (360k nodes): two mark bitmaps per CTA no longer fit
    twice in shared memory, so the one-bitmap 512-thread shape runs."""
    net = synth.grid_network(600, 7, freeways=True)
    g, og = Q.Graph(net), oracle.OracleGraph(net)
    rng = np.random.default_rng(8)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.n_links)).astype(np.int32)
    roots = rng.choice(net.n_nodes, 6, replace=False).astype(np.int32)
    for direction in (Q.QDTA_TO_ROOT, Q.QDTA_FROM_ROOT):
        assert Q.qdta_sssp_kernel_name(g, direction) == "sssp_smq_kernel<512,rank32,2,true>"
        p_o, d_o = oracle.sssp(og, q, roots, direction)
        p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), direction, True)
        np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
        np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


def test_autotune_keeps_the_fastest_shape_and_stays_bit_exact(mid):
    net, dem, _, og = mid
    g = Q.Graph(net)
    rng = np.random.default_rng(4)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.n_links)).astype(np.int32)
    roots = rng.choice(net.n_nodes, 64, replace=False).astype(np.int32)
    rep = Q.qdta_autotune(g, T(q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, reps=1)
    kernels = {c["kernel"] for c in rep["candidates"]}
    # launch shapes {512 x 2 CTAs, 256 x 4 CTAs} x adjacency {32-bit rank keys, rank keys, four-slot,
    # compressed} in relaxation mode 2; the 32-bit kernel also with five CTAs per SM (256 and 192
    # threads), with 5 or 6 frontier nodes per lane group, lane per node (1 or 2 nodes per lane),
    # with the L2 prefetch of key blocks and with 288 threads; the cell kernel
    want = {f"sssp_smq_kernel<{t},{e},2,{b}>" for t, b in (("512", "false"), ("256", "true"))
            for e in ("rank32", "rank", "ell", "csr")} | {"sssp_cell_kernel"}
    want |= {"sssp_smq_kernel<256,rank32,2,true,5>", "sssp_smq_kernel<256,rank32,2,true,npt5>",
             "sssp_smq_kernel<256,rank32,2,true,npt6>", "sssp_lane_kernel<256,npn1>", "sssp_lane_kernel<256,npn2>",
             "sssp_smq_kernel<256,rank32,2,true,pf>", "sssp_smq_kernel<192,rank32,2,true,5>",
             "sssp_smq_kernel<288,rank32,2,true>"}
    assert kernels == want
    assert len(rep["candidates"]) == 17
    ctas = {c["kernel"]: c["ctas_per_sm"] for c in rep["candidates"]}
    assert ctas["sssp_smq_kernel<256,rank32,2,true>"] == 4 and ctas["sssp_smq_kernel<256,rank32,2,true,5>"] == 5
    fastest = min(c["ms"] for c in rep["candidates"])
    default = [c for c in rep["candidates"] if c["kernel"] == "sssp_smq_kernel<256,rank32,2,true>"][0]
    # the default shape is kept unless another is at least 2 % faster
    assert rep["best"]["ms"] == fastest or (rep["best"] == default and default["ms"] * 0.98 <= fastest)
    assert Q.qdta_sssp_kernel_name(g, Q.QDTA_TO_ROOT) == rep["best"]["kernel"]
    p_o, d_o = oracle.sssp(og, q, roots)
    p_g, d_g = Q.qdta_sssp_batch(g, T(q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, True)
    np.testing.assert_array_equal(d_g.cpu().numpy(), d_o)
    np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)


def test_autotune_small_graph_has_one_shape(small):
    inst, g, og = small
    rep = Q.qdta_autotune(g, T(inst.net.fftime_q, np.int32), T(inst.zones, np.int32))
    assert [c["kernel"] for c in rep["candidates"]] == ["sssp_kernel<true>"]


def test_empty_batches(small):
    inst, g, og = small
    p, d = Q.qdta_sssp_batch(g, T(inst.net.fftime_q, np.int32), T(np.zeros(0), np.int32))
    assert p.shape == (0, og.n_nodes)
    od = Q.DeviceOD(T(inst.zones, np.int32), T([], np.int32), T([], np.int32), T([], np.int64))
    flow, _ = Q.qdta_load_aon(g, T(inst.net.fftime_q, np.int32), p, od, 90000)
    assert int(flow.abs().sum()) == 0


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dt_q", [0, 1, 20000, 90000, np.iinfo(np.int64).max])
def test_load_bit_exact(small, dt_q):
    inst, g, og = small
    dem = synth.random_demand(inst.net, 64, 3000, 7, fractional=True)
    rng = np.random.default_rng(3)
    q = (inst.net.fftime_q * rng.uniform(1, 4, og.n_links)).astype(np.int32)
    par_o, _ = oracle.sssp(og, q, dem.roots, want_dist=False)
    f_o, s_o, rc = oracle.load(og, q, par_o, oracle.OracleOD.of(dem), dt_q)
    assert rc == 0
    qd = T(q, np.int32)
    par_g, _ = Q.qdta_sssp_batch(g, qd, T(dem.roots, np.int32))
    f_g, s_g = Q.qdta_load_aon(g, qd, par_g, Q.DeviceOD.of(dem), dt_q, want_stop=True)
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    np.testing.assert_array_equal(s_g.cpu().numpy(), s_o)


def test_load_unreachable_is_reported():
    net = synth.Network(n_nodes=3, tail=np.array([0, 1], np.int32), head=np.array([1, 0], np.int32),
                        fftime_q=np.array([5, 7], np.int32), capacity=np.ones(2) * 100,
                        length_m=np.zeros(2), link_class=np.zeros(2, np.int8), x=np.zeros(3), y=np.zeros(3))
    g = Q.Graph(net)
    roots = T([2], np.int32)
    par, _ = Q.qdta_sssp_batch(g, T(net.fftime_q, np.int32), roots)
    od = Q.DeviceOD(roots, T([0], np.int32), T([0], np.int32), T([1 << 32], np.int64))
    with pytest.raises(Q.QdtaError) as e:
        Q.qdta_load_aon(g, T(net.fftime_q, np.int32), par, od, 100)
    assert e.value.code == Q.QDTA_EUNREACH


# ---------------------------------------------------------------------------
def _fg(small, seed=0):
    inst, g, og = small
    rng = np.random.default_rng(seed)
    od = oracle.OracleOD.of(inst.demand[0])
    f, st, rc = oracle.assign_interval(og, od, 900.0, oracle.make_params(oracle.STEP_MSA, oracle.STOP_NONE, 3))
    q, _, _ = oracle.bpr(og, f, 900.0)
    par, _ = oracle.sssp(og, q, od.roots, want_dist=False)
    gfx, _, _ = oracle.load(og, q, par, od, 90000)
    return f, gfx


@pytest.mark.parametrize("step", ["paper_qn3", "sweep8", "exact", "msa"])
@pytest.mark.parametrize("k", [1, 4])
def test_line_search_bit_exact(small, step, k):
    inst, g, og = small
    f, gfx = _fg(small)
    p = oracle.make_params(Q.STEP[step], oracle.STOP_NONE, 20)
    a_o, n_o, rc = oracle.line_search(og, f, gfx, 900.0, k, p)
    a_g, n_g = Q.qdta_line_search(g, T(f, np.float64), T(gfx, np.int64), 900.0, k,
                                  Q.make_params(step, "none", 20))
    assert a_g == a_o and n_g == n_o


# ---------------------------------------------------------------------------
CASES = [("msa", "none", 20, 1e-4), ("sweep8", "rel_gap", 300, 1e-4), ("paper_qn3", "rel_gap", 300, 1e-4),
         ("exact", "rel_gap", 60, 1e-3), ("sweep8", "paper_obj", 300, 1e-4), ("msa", "rel_gap", 15, 1e-4)]


@pytest.mark.parametrize("schedule", ["plain", "graph"])
@pytest.mark.parametrize("step,stop,it,tol", CASES)
def test_assign_interval_bit_exact(small, schedule, step, stop, it, tol):
    inst, g, og = small
    od = oracle.OracleOD.of(inst.demand[0])
    f_o, st_o, rc_o = oracle.assign_interval(og, od, 900.0,
                                             oracle.make_params(Q.STEP[step], Q.STOP[stop], it, tol))
    f_g, st_g, rc_g, _ = Q.qdta_assign_interval(g, Q.DeviceOD.of(inst.demand[0]), 900.0,
                                                 Q.make_params(step, stop, it, tol, schedule=schedule))
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    for key in ("iterations", "aon_calls", "ls_passes", "converged", "objective"):
        assert st_g[key] == st_o[key], key
    for key in ("rel_gap", "dual_gap"):
        if not np.isnan(st_o[key]):
            assert st_g[key] == st_o[key], key
    assert (rc_g == Q.QDTA_ENOTCONV) == (rc_o == oracle.NOTCONV)


def test_assign_interval_mid_network(mid):
    net, dem, g, og = mid
    od = oracle.OracleOD.of(dem)
    p = (Q.STEP["sweep8"], Q.STOP["rel_gap"], 6, 1e-4)
    f_o, st_o, _ = oracle.assign_interval(og, od, 900.0, oracle.make_params(*p))
    f_g, st_g, _, _ = Q.qdta_assign_interval(g, Q.DeviceOD.of(dem), 900.0,
                                              Q.make_params("sweep8", "rel_gap", 6, 1e-4, schedule="graph"))
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    assert st_g["ls_passes"] == st_o["ls_passes"]


def test_empty_interval(small):
    inst, g, og = small
    od = Q.DeviceOD(T(inst.zones, np.int32), T([], np.int32), T([], np.int32), T([], np.int64))
    for schedule in ("plain", "graph"):
        f, st, rc, _ = Q.qdta_assign_interval(g, od, 900.0, Q.make_params(schedule=schedule))
        assert float(f.abs().sum()) == 0.0 and st["converged"] == 1 and st["aon_calls"] == 0


def _diamond(ff_s, cap):
    """0 -> 1 -> 3 and 0 -> 2 -> 3 (links 0->1, 0->2, 1->3, 2->3)."""
    return synth.Network(n_nodes=4, tail=np.array([0, 0, 1, 2], np.int32), head=np.array([1, 2, 3, 3], np.int32),
                         fftime_q=np.rint(np.array(ff_s, np.float64) / 0.01).astype(np.int32),
                         capacity=np.array(cap, np.float64), length_m=np.zeros(4), link_class=np.zeros(4, np.int8),
                         x=np.arange(4.0), y=np.zeros(4))


@pytest.mark.parametrize("schedule", ["plain", "graph"])
@pytest.mark.parametrize("cap02,trips,ff", [(632.6, 100, [200, 340, 1000, 400]), (700.0, 100, [200, 340, 1000, 400]),
                                            (200.0, 150, [301, 340, 1000, 10])])
def test_rel_gap_stop_with_negative_and_rounding_level_gaps(schedule, cap02, trips, ff):
    """Truncation (Δt = 300 s) makes the gap negative on the first case (no
    convergence, every step 0), exactly 0 on the second and a few ulps below 0
    at an equilibrium on the third (both stop); bit-exact with the oracle."""
    caps = [5000, cap02, 5000, 5000] if ff[3] == 400 else [400, cap02, 400, 400]
    net = _diamond(ff, caps)
    dem = synth.Demand(roots=np.array([3], np.int32), root_idx=np.array([0], np.int32), src=np.array([0], np.int32),
                       amount_fx=np.array([trips << 32], np.int64))
    og = oracle.OracleGraph(net)
    f_o, st_o, rc_o = oracle.assign_interval(og, oracle.OracleOD.of(dem), 300.0,
                                             oracle.make_params(Q.STEP["sweep8"], Q.STOP["rel_gap"], 12))
    f_g, st_g, rc_g, _ = Q.qdta_assign_interval(Q.Graph(net), Q.DeviceOD.of(dem), 300.0,
                                                 Q.make_params("sweep8", "rel_gap", 12, schedule=schedule))
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    for key in ("iterations", "aon_calls", "ls_passes", "converged", "dual_gap", "rel_gap"):
        assert st_g[key] == st_o[key], key
    assert (rc_g == Q.QDTA_ENOTCONV) == (rc_o == oracle.NOTCONV)
    assert st_g["converged"] == (0 if cap02 == 632.6 else 1)


# ---------------------------------------------------------------------------
def _day_case(n_int=6, trips=40000):
    base = synth.config_small(0)
    return synth.scaled_day(base, trips, n_intervals=n_int, seed=11)


@pytest.mark.parametrize("schedule", ["plain", "graph"])
@pytest.mark.parametrize("step,stop,it", [("msa", "none", 8), ("sweep8", "rel_gap", 80)])
def test_run_day_bit_exact(step, stop, it, schedule):
    day = _day_case()
    days = [d for d in day.demand]
    og = oracle.OracleGraph(day.net)
    f_o, st_o, nit_o, rn_o, rc_o = oracle.run_day(og, day.zones, days, 900.0,
                                                  oracle.make_params(Q.STEP[step], Q.STOP[stop], it))
    g = Q.Graph(day.net)
    zones = T(day.zones, np.int32)
    dd = [Q.DeviceOD(zones, T(d.root_idx, np.int32), T(d.src, np.int32), T(d.amount_fx, np.int64)) for d in days]
    f_g, st_g, rc_g, resid = Q.qdta_run_day(g, dd, 900.0, Q.make_params(step, stop, it, schedule=schedule),
                                            resid_capacity=1 << 20)
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    for i in range(len(days)):
        assert st_g[i]["n_items"] == nit_o[i]
        for key in ("iterations", "aon_calls", "ls_passes", "converged"):
            assert st_g[i][key] == st_o[i][key], (i, key)
    assert resid[0].shape[0] == rn_o


@pytest.mark.parametrize("schedule", ["plain", "graph"])
def test_run_day_without_the_free_flow_tree_cache(schedule, monkeypatch):
    """The day reuses the free-flow trees for every interval's initial AON;
    recomputing them instead gives the same bits (and the oracle's)."""
    day = _day_case(n_int=4)
    days = list(day.demand)
    og = oracle.OracleGraph(day.net)
    f_o, st_o, nit_o, rn_o, _ = oracle.run_day(og, day.zones, days, 900.0,
                                               oracle.make_params(Q.STEP["sweep8"], Q.STOP["paper_obj"], 60))
    zones = T(day.zones, np.int32)
    dd = [Q.DeviceOD(zones, T(d.root_idx, np.int32), T(d.src, np.int32), T(d.amount_fx, np.int64)) for d in days]
    out = []
    for off in (False, True):
        if off:
            monkeypatch.setenv("QDTA_NO_FF_CACHE", "1")
        g = Q.Graph(day.net)
        Q.qdta_profile_enable(g, schedule == "plain")
        f_g, st_g, _, _ = Q.qdta_run_day(g, dd, 900.0, Q.make_params("sweep8", "paper_obj", 60, schedule=schedule))
        out.append((f_g.cpu().numpy(), [s["iterations"] for s in st_g],
                    Q.qdta_profile_read(g)["sssp_launches"] if schedule == "plain" else None))
        np.testing.assert_array_equal(out[-1][0], f_o)
    assert out[0][1] == out[1][1] == [s["iterations"] for s in st_o]
    if schedule == "plain":
        # cached: one batch for all zones, then no SSSP for the initial AONs
        assert out[0][2] < out[1][2]


@pytest.mark.parametrize("schedule", ["plain", "graph"])
def test_run_day_worked_example(schedule):
    ff = [600.0, 300.0, 600.0, 600.0]
    net = synth.chain_network(ff, [200.0, 150.0, 200.0, 200.0])
    g = Q.Graph(net)
    zones = T([3, 4], np.int32)
    fx = lambda v: int(round(v * (1 << 32)))
    dd = [Q.DeviceOD(zones, T([0], np.int32), T([0], np.int32), T([fx(43.75)], np.int64)),
          Q.DeviceOD(zones, T([1], np.int32), T([2], np.int32), T([fx(12.5)], np.int64)),
          Q.DeviceOD(zones, T([], np.int32), T([], np.int32), T([], np.int64)),
          Q.DeviceOD(zones, T([], np.int32), T([], np.int32), T([], np.int64))]
    f, st, rc, _ = Q.qdta_run_day(g, dd, 900.0, Q.make_params("sweep8", "rel_gap", 50, schedule=schedule))
    f = f.cpu().numpy()
    np.testing.assert_array_equal(f[0], [43.75, 43.75, 0, 0])
    np.testing.assert_array_equal(f[1], [0, 0, 56.25, 12.5])
    assert [s["n_items"] for s in st] == [1, 2, 0, 0]


# ---------------------------------------------------------------------------
# A day on a graph above the shared-memory limit: the kernels the metro day
# runs (the global-key shortest-path kernel with 32-bit rank keys, the tree
# ring of the residual pass, the free-flow tree cache, the dense merge).
def _mid_day():
    """110 x 110 grid (12,100 nodes) plus a pendant node w hung off a boundary
    node u by two 100 s links; w -> u has a capacity of 4/3 veh/h, so its 10
    trips in intervals 1 and 3 price it at about 1.2e9 quanta (Eq. 1).  Every
    distance from w then exceeds the 32-bit keys' 2^29 range, and those
    intervals' batches after the first are rerun with 64-bit keys.  150
    zones, six intervals of uneven gravity demand; at 40 km/h most trips cross
    several intervals, so residual demand is carried between them."""
    net = synth.grid_network(110, 5, freeways=True)
    V = net.n_nodes
    deg_out = np.bincount(net.tail, minlength=V)
    deg_in = np.bincount(net.head, minlength=V)
    u = int(next(c for c in range(5, 100) if deg_out[c] <= 3 and deg_in[c] <= 3))
    w = V
    tail = np.concatenate([net.tail, [u, w]]).astype(np.int32)
    head = np.concatenate([net.head, [w, u]]).astype(np.int32)
    order = np.lexsort((head, tail))

    def ext(a, extra):
        return np.concatenate([a, extra])[order]
    net2 = synth.Network(n_nodes=V + 1, tail=tail[order], head=head[order],
                         fftime_q=ext(net.fftime_q, np.array([10000, 10000], np.int32)).astype(np.int32),
                         capacity=ext(net.capacity, np.array([800.0, 4.0 / 3.0])),
                         length_m=ext(net.length_m, np.array([1000.0, 1000.0])),
                         link_class=ext(net.link_class, np.array([0, 0], np.int8)),
                         x=np.concatenate([net.x, [net.x[u]]]), y=np.concatenate([net.y, [net.y[u] - 1000.0]]),
                         alpha=net.alpha, beta=net.beta, quantum_s=net.quantum_s)
    zones = synth.pick_zones(net, 150, 5)
    wts = synth.gravity_weights(net, zones, 5, 4000.0)
    days = []
    for i, (t, wt) in enumerate(zip((9000, 40000, 80000, 30000, 8000, 2000), (0, 10, 0, 10, 0, 0))):
        d = synth.demand_from_matrix(zones, synth.sample_trips(wts, t, 40 + i))
        if wt:
            ri = np.concatenate([d.root_idx, [0]])
            src = np.concatenate([d.src, [w]])
            am = np.concatenate([d.amount_fx, [wt << 32]])
            o = np.lexsort((src, ri))
            d = synth.Demand(roots=d.roots, root_idx=ri[o].astype(np.int32), src=src[o].astype(np.int32),
                             amount_fx=am[o].astype(np.int64))
        days.append(d)
    return net2, zones, days


MID_DAY_PARAMS = ("sweep8", "paper_obj", 10)


@pytest.fixture(scope="module")
def mid_day():
    net, zones, days = _mid_day()
    og = oracle.OracleGraph(net)
    ref = oracle.run_day(og, zones, days, 900.0, oracle.make_params(Q.STEP[MID_DAY_PARAMS[0]],
                                                                     Q.STOP[MID_DAY_PARAMS[1]], MID_DAY_PARAMS[2]))
    return net, zones, days, ref


@pytest.mark.parametrize("schedule", ["plain", "graph"])
@pytest.mark.parametrize("variant", ["default", "ring3", "no_ff_cache"])
def test_run_day_large_graph_bit_exact(mid_day, schedule, variant, monkeypatch):
    """Bit-exact h(i) flows, per-interval stats, merged item counts and the
    final residual against the oracle's day, on both schedules; with the tree
    ring capped at 3 slots (the residual pass rebuilds trees 2..K from the
    taped link times) and without the free-flow tree cache."""
    net, zones, days, (f_o, st_o, nit_o, rn_o, rc_o) = mid_day
    if variant == "ring3":
        monkeypatch.setenv("QDTA_TREE_RING", "3")
    if variant == "no_ff_cache":
        monkeypatch.setenv("QDTA_NO_FF_CACHE", "1")
    g = Q.Graph(net)
    assert "rank32" in Q.qdta_sssp_kernel_name(g)  # the metro day's kernel family
    zt = T(zones, np.int32)
    dd = [Q.DeviceOD(zt, T(d.root_idx, np.int32), T(d.src, np.int32), T(d.amount_fx, np.int64)) for d in days]
    Q.qdta_profile_enable(g, schedule == "plain")
    f_g, st_g, rc_g, resid = Q.qdta_run_day(g, dd, 900.0, Q.make_params(*MID_DAY_PARAMS, schedule=schedule),
                                            resid_capacity=1 << 20)
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    for i in range(len(days)):
        assert st_g[i]["n_items"] == nit_o[i]
        for key in ("iterations", "aon_calls", "ls_passes", "converged", "rel_gap", "dual_gap", "objective"):
            if not (isinstance(st_o[i][key], float) and np.isnan(st_o[i][key])):
                assert st_g[i][key] == st_o[i][key], (i, key)
    assert resid[0].shape[0] == rn_o
    assert sum(s["iterations"] for s in st_o) >= 20 and max(nit_o) > max(d.n_items for d in days)
    if schedule == "plain":
        prof = Q.qdta_profile_read(g)
        assert prof["sssp_redo_batches"] > 0  # the 2^29 overflow happened inside the day


@pytest.mark.parametrize("schedule", ["plain", "graph"])
def test_run_day_large_graph_carried_truncation_bit_exact(schedule):
    """The large-graph day of the test above under carried truncation."""
    net, zones, days = _mid_day()
    og = oracle.OracleGraph(net)
    f_o, st_o, nit_o, rn_o, rc_o, res_o = oracle.run_day(og, zones, days, 900.0, oracle.make_params(
        Q.STEP[MID_DAY_PARAMS[0]], Q.STOP[MID_DAY_PARAMS[1]], MID_DAY_PARAMS[2], truncation=oracle.TRUNC_CARRY),
        want_resid=True)
    g = Q.Graph(net)
    zt = T(zones, np.int32)
    dd = [Q.DeviceOD(zt, T(d.root_idx, np.int32), T(d.src, np.int32), T(d.amount_fx, np.int64)) for d in days]
    f_g, st_g, rc_g, resid = Q.qdta_run_day(g, dd, 900.0, Q.make_params(*MID_DAY_PARAMS, schedule=schedule,
                                                                          truncation="carry"),
                                            resid_capacity=1 << 21)
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    assert [s["n_items"] for s in st_g] == list(nit_o)
    assert [s["iterations"] for s in st_g] == [s["iterations"] for s in st_o]
    assert resid[0].shape[0] == rn_o
    assert _sorted_resid([r.cpu().numpy() for r in resid]) == _sorted_resid(res_o)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("carried", [False, True])
@pytest.mark.parametrize("step", ["exact", "msa"])
def test_backward_matches_oracle(step, carried):
    net = synth.grid_network(12, 4)
    zones = synth.pick_zones(net, 10, 4)
    dem = synth.demand_from_matrix(zones, synth.gravity_fixed_pairs(net, zones, 3000, 1500.0))
    og = oracle.OracleGraph(net)
    od = oracle.OracleOD.of(dem)
    dod = Q.DeviceOD.of(dem)
    if carried:  # half of the trips start on a link (the adjoint gathers it first)
        carry, link = _carried_items(net, dem, 3)
        od = oracle.OracleOD(dem.roots, dem.root_idx, dem.src, dem.amount_fx, carry_frac=carry, carry_link=link)
        dod.carry_frac, dod.carry_link = T(carry, np.int64), T(link, np.int32)
    p = oracle.make_params(Q.STEP[step], oracle.STOP_NONE, 10)
    f_o, st_o, rc, tape_o = oracle.assign_interval(og, od, 600.0, p, tape=True)
    g = Q.Graph(net)
    f_g, st_g, rc, tape = Q.qdta_assign_interval(g, dod, 600.0, Q.make_params(step, "none", 10, record_tape=True))
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    rng = np.random.default_rng(0)
    S = rng.choice(og.n_links, og.n_links // 10, replace=False)
    dL = np.zeros(og.n_links)
    dL[S] = 2 * (f_o[S] - f_o[S] * rng.lognormal(0, 0.3, S.shape[0]))
    dd_o, dc_o, _ = oracle.backward(og, od, 600.0, Q.STEP[step], tape_o, dL)
    dd_g, dc_g = Q.qdta_backward(tape, T(dL, np.float64))
    np.testing.assert_allclose(dd_g.cpu().numpy(), dd_o, rtol=1e-9, atol=1e-12 * np.abs(dd_o).max())
    np.testing.assert_allclose(dc_g.cpu().numpy(), dc_o, rtol=1e-9, atol=1e-12 * max(np.abs(dc_o).max(), 1e-300))


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("schedule", ["plain", "graph"])
def test_assign_batch_matches_oracle(schedule):
    """Independent networks of different sizes solved in one call."""
    cases = []
    for n, z, trips, seed in [(12, 8, 2000, 1), (20, 16, 6000, 2), (110, 40, 20000, 3)]:
        net = synth.grid_network(n, seed, freeways=n > 64)
        zones = synth.pick_zones(net, z, seed)
        dem = synth.demand_from_matrix(zones, synth.sample_trips(
            synth.gravity_weights(net, zones, seed, 3000.0), trips, seed))
        cases.append((net, dem))
    params = ("sweep8", "rel_gap", 40, 1e-4)
    items, graphs = [], []
    for net, dem in cases:
        g = Q.Graph(net)
        graphs.append(g)
        items.append((g, Q.DeviceOD.of(dem), 900.0, torch.empty(net.n_links, dtype=torch.float64, device=DEV)))
    stats, rc = Q.qdta_assign_batch(items, Q.make_params(*params, schedule=schedule))
    for (net, dem), it, st in zip(cases, items, stats):
        og = oracle.OracleGraph(net)
        f_o, st_o, _ = oracle.assign_interval(og, oracle.OracleOD.of(dem), 900.0,
                                              oracle.make_params(Q.STEP[params[0]], Q.STOP[params[1]], params[2],
                                                                 params[3]))
        np.testing.assert_array_equal(it[3].cpu().numpy(), f_o)
        assert st["iterations"] == st_o["iterations"] and st["ls_passes"] == st_o["ls_passes"]


def test_autograd_function_matches_oracle_adjoint():
    from paper_2104_12911_gb300 import autograd as AG
    net = synth.grid_network(10, 6)
    zones = synth.pick_zones(net, 8, 6)
    dem = synth.demand_from_matrix(zones, synth.gravity_fixed_pairs(net, zones, 2000, 1200.0))
    od = Q.DeviceOD.of(dem)
    amounts = torch.tensor(dem.amount_fx / float(1 << 32), dtype=torch.float64, device=DEV, requires_grad=True)
    cap = torch.tensor(net.capacity, dtype=torch.float64, device=DEV, requires_grad=True)
    params = Q.make_params("exact", "none", 6)
    f = AG.assign(net, od, amounts, cap, 600.0, params)
    rng = np.random.default_rng(1)
    w = torch.tensor(rng.standard_normal(net.n_links), dtype=torch.float64, device=DEV)
    (f * w).sum().backward()
    og = oracle.OracleGraph(net)
    ood = oracle.OracleOD.of(dem)
    f_o, _, _, tape_o = oracle.assign_interval(og, ood, 600.0, oracle.make_params(oracle.STEP_EXACT,
                                                                                 oracle.STOP_NONE, 6), tape=True)
    np.testing.assert_array_equal(f.detach().cpu().numpy(), f_o)
    dd_o, dc_o, _ = oracle.backward(og, ood, 600.0, oracle.STEP_EXACT, tape_o, w.cpu().numpy())
    np.testing.assert_allclose(amounts.grad.cpu().numpy(), dd_o, rtol=1e-9, atol=1e-12 * np.abs(dd_o).max())
    np.testing.assert_allclose(cap.grad.cpu().numpy(), dc_o, rtol=1e-9, atol=1e-12 * max(np.abs(dc_o).max(), 1e-300))


# ---------------------------------------------------------------------------
# Scenario metrics (Section 7.1) of a day's h(i) rows, bit-exact against the oracle
def test_interval_metrics_of_a_day_match_the_oracle():
    day = _day_case(n_int=4)
    net = day.net
    g = Q.Graph(net)
    zones = T(day.zones, np.int32)
    dd = [Q.DeviceOD(zones, T(d.root_idx, np.int32), T(d.src, np.int32), T(d.amount_fx, np.int64)) for d in day.demand]
    f_g, _, _, _ = Q.qdta_run_day(g, dd, 900.0, Q.make_params("sweep8", "paper_obj", 60, schedule="graph"))
    cls = net.link_class.astype(np.int32)
    n_cls = int(cls.max()) + 1
    got = Q.qdta_interval_metrics(g, f_g, 900.0, T(net.length_m, np.float64), T(cls, np.int32), n_cls)
    want, rc = oracle.interval_metrics(oracle.OracleGraph(net), f_g.cpu().numpy(), 900.0, net.length_m, cls, n_cls)
    assert rc == 0
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    assert want[:, :, 0].sum() > 0


def test_interval_metrics_edge_cases():
    inst = synth.config_small(0)
    net = inst.net
    g = Q.Graph(net)
    og = oracle.OracleGraph(net)
    rng = np.random.default_rng(17)
    L = net.n_links
    flows = rng.uniform(0, 400, (3, L)) * (rng.random((3, L)) < 0.7)
    length = rng.uniform(100, 400, L)
    cls = rng.integers(-1, 6, L).astype(np.int32)  # -1 and 5 fall outside 5 classes
    got = Q.qdta_interval_metrics(g, T(flows, np.float64), 900.0, T(length, np.float64), T(cls, np.int32), 5, 0.8)
    want, rc = oracle.interval_metrics(og, flows, 900.0, length, cls, 5, 0.8)
    assert rc == 0
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    empty = Q.qdta_interval_metrics(g, T(np.zeros((0, L)), np.float64), 900.0, T(length, np.float64),
                                    T(cls, np.int32), 5)
    assert tuple(empty.shape) == (0, 5, 8)
    flows[1, 7] = np.nan
    with pytest.raises(Q.QdtaError) as e:
        Q.qdta_interval_metrics(g, T(flows, np.float64), 900.0, T(length, np.float64), T(cls, np.int32), 5)
    assert e.value.code == Q.QDTA_ENONFINITE


# ---------------------------------------------------------------------------
# System-optimal objective: routing on marginal costs, total-cost line search
@pytest.mark.parametrize("step", ["paper_qn3", "sweep8", "exact"])
def test_line_search_system_optimum_bit_exact(small, step):
    inst, g, og = small
    f, gfx = _fg(small)
    a_o, n_o, rc = oracle.line_search(og, f, gfx, 900.0, 3, oracle.make_params(Q.STEP[step], oracle.STOP_NONE, 20,
                                                                              objective=oracle.OBJ_SO))
    a_g, n_g = Q.qdta_line_search(g, T(f, np.float64), T(gfx, np.int64), 900.0, 3,
                                  Q.make_params(step, "none", 20, objective="so"))
    assert a_g == a_o and n_g == n_o
    a_ue, _, _ = oracle.line_search(og, f, gfx, 900.0, 3, oracle.make_params(Q.STEP[step], oracle.STOP_NONE, 20))
    assert step == "paper_qn3" or a_ue != a_o  # the objectives differ on this case


@pytest.mark.parametrize("schedule", ["plain", "graph"])
@pytest.mark.parametrize("step,stop,it,tol", CASES)
def test_assign_interval_system_optimum_bit_exact(small, schedule, step, stop, it, tol):
    inst, g, og = small
    od = oracle.OracleOD.of(inst.demand[0])
    f_o, st_o, rc_o = oracle.assign_interval(og, od, 900.0, oracle.make_params(Q.STEP[step], Q.STOP[stop], it, tol,
                                                                              objective=oracle.OBJ_SO))
    f_g, st_g, rc_g, _ = Q.qdta_assign_interval(g, Q.DeviceOD.of(inst.demand[0]), 900.0,
                                                 Q.make_params(step, stop, it, tol, schedule=schedule, objective="so"))
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    for key in ("iterations", "aon_calls", "ls_passes", "converged", "objective"):
        assert st_g[key] == st_o[key], key
    for key in ("rel_gap", "dual_gap"):
        if not np.isnan(st_o[key]):
            assert st_g[key] == st_o[key], key


@pytest.mark.parametrize("schedule", ["plain", "graph"])
def test_run_day_system_optimum_bit_exact(schedule):
    day = _day_case(n_int=4)
    days = list(day.demand)
    og = oracle.OracleGraph(day.net)
    f_o, st_o, nit_o, rn_o, _ = oracle.run_day(og, day.zones, days, 900.0, oracle.make_params(
        Q.STEP["sweep8"], Q.STOP["paper_obj"], 60, objective=oracle.OBJ_SO))
    g = Q.Graph(day.net)
    zones = T(day.zones, np.int32)
    dd = [Q.DeviceOD(zones, T(d.root_idx, np.int32), T(d.src, np.int32), T(d.amount_fx, np.int64)) for d in days]
    f_g, st_g, _, resid = Q.qdta_run_day(g, dd, 900.0, Q.make_params("sweep8", "paper_obj", 60, schedule=schedule,
                                                                      objective="so"), resid_capacity=1 << 20)
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    assert [s["iterations"] for s in st_g] == [s["iterations"] for s in st_o]
    assert resid[0].shape[0] == rn_o


def test_system_optimum_rejects_a_tape(small):
    inst, g, og = small
    with pytest.raises(Q.QdtaError) as e:
        Q.qdta_assign_interval(g, Q.DeviceOD.of(inst.demand[0]), 900.0,
                               Q.make_params("exact", "none", 3, record_tape=True, objective="so"))
    assert e.value.code == Q.QDTA_EINVAL


# ---------------------------------------------------------------------------
def test_set_capacity_matches_a_fresh_graph_and_keeps_tapes():
    """qdta_graph_set_capacity on one handle gives the bits of a graph built
    with those capacities; a bad value is rejected and changes nothing; a
    tape recorded before the update differentiates with its own capacities."""
    net = synth.grid_network(12, 4)
    zones = synth.pick_zones(net, 10, 4)
    dem = synth.demand_from_matrix(zones, synth.gravity_fixed_pairs(net, zones, 3000, 1500.0))
    od = Q.DeviceOD.of(dem)
    p = Q.make_params("exact", "none", 6, record_tape=True)
    rng = np.random.default_rng(9)
    cap_b = net.capacity * rng.uniform(0.5, 1.5, net.n_links)
    g = Q.Graph(net)
    f_a, _, _, tape_a = Q.qdta_assign_interval(g, od, 600.0, p)
    dL = T(rng.standard_normal(net.n_links), np.float64)
    dd_ref, dc_ref = Q.qdta_backward(tape_a, dL)
    g.set_capacity(T(cap_b, np.float64))
    dd_a, dc_a = Q.qdta_backward(tape_a, dL)   # the tape keeps the capacities of its solve
    assert torch.equal(dd_a, dd_ref) and torch.equal(dc_a, dc_ref)
    f_b, _, _, tape_b = Q.qdta_assign_interval(g, od, 600.0, p)
    fresh = Q.Graph(dataclasses.replace(net, capacity=cap_b))
    f_c, _, _, tape_c = Q.qdta_assign_interval(fresh, od, 600.0, p)
    assert torch.equal(f_b, f_c) and not torch.equal(f_a, f_b)
    dd_b, dc_b = Q.qdta_backward(tape_b, dL)
    dd_c, dc_c = Q.qdta_backward(tape_c, dL)
    assert torch.equal(dd_b, dd_c) and torch.equal(dc_b, dc_c)
    bad = cap_b.copy()
    bad[7] = 0.0
    with pytest.raises(Q.QdtaError) as e:
        g.set_capacity(T(bad, np.float64))
    assert e.value.code == Q.QDTA_EINVAL
    f_d, _, _, _ = Q.qdta_assign_interval(g, od, 600.0, Q.make_params("exact", "none", 6))
    assert torch.equal(f_d, f_b)   # unchanged by the rejected update
    for t in (tape_a, tape_b, tape_c):
        t.close()


def test_autograd_reuses_one_graph_handle():
    from paper_2104_12911_gb300 import autograd as AG
    net = synth.grid_network(10, 6)
    zones = synth.pick_zones(net, 8, 6)
    dem = synth.demand_from_matrix(zones, synth.gravity_fixed_pairs(net, zones, 2000, 1200.0))
    od = Q.DeviceOD.of(dem)
    amounts = torch.tensor(dem.amount_fx / float(1 << 32), dtype=torch.float64, device=DEV)
    params = Q.make_params("exact", "none", 4)
    handles = set()
    for scale in (1.0, 0.8):
        cap = torch.tensor(net.capacity * scale, dtype=torch.float64, device=DEV, requires_grad=True)
        f = AG.assign(net, od, amounts, cap, 600.0, params)
        f.sum().backward()
        handles.add(id(AG.graph_for(net, 0)))
        og = oracle.OracleGraph(dataclasses.replace(net, capacity=net.capacity * scale))
        f_o, _, _ = oracle.assign_interval(og, oracle.OracleOD.of(dem), 600.0,
                                           oracle.make_params(oracle.STEP_EXACT, oracle.STOP_NONE, 4))
        np.testing.assert_array_equal(f.detach().cpu().numpy(), f_o)
    assert len(handles) == 1


# ---------------------------------------------------------------------------
# Carried partial-link truncation (Section 3.4's alternative to Eq. 2)
def _sorted_resid(r):
    """residual arrays (root index, src, amount, covered fraction, link) as a
    sorted list of tuples: the GPU writes carried entries in table order"""
    root, src, amt, carry, link = (np.asarray(a).astype(np.int64) for a in r)
    return sorted(zip(root.tolist(), link.tolist(), src.tolist(), amt.tolist(), carry.tolist()))


def _carry_day_case():
    # 150 s intervals on the 32 x 32 grid: most trips cross several intervals
    return synth.scaled_day(synth.config_small(0), 60000, n_intervals=5, seed=5)


@pytest.mark.parametrize("schedule", ["plain", "graph"])
@pytest.mark.parametrize("step,stop,it", [("msa", "none", 6), ("sweep8", "paper_obj", 40)])
def test_run_day_carried_truncation_bit_exact(schedule, step, stop, it):
    day = _carry_day_case()
    days = list(day.demand)
    og = oracle.OracleGraph(day.net)
    f_o, st_o, nit_o, rn_o, rc_o, res_o = oracle.run_day(og, day.zones, days, 150.0, oracle.make_params(
        Q.STEP[step], Q.STOP[stop], it, truncation=oracle.TRUNC_CARRY), want_resid=True)
    g = Q.Graph(day.net)
    zones = T(day.zones, np.int32)
    dd = [Q.DeviceOD(zones, T(d.root_idx, np.int32), T(d.src, np.int32), T(d.amount_fx, np.int64)) for d in days]
    f_g, st_g, rc_g, resid = Q.qdta_run_day(g, dd, 150.0, Q.make_params(step, stop, it, schedule=schedule,
                                                                          truncation="carry"),
                                            resid_capacity=1 << 21)
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    for i in range(len(days)):
        assert st_g[i]["n_items"] == nit_o[i], i
        for key in ("iterations", "aon_calls", "ls_passes", "converged"):
            assert st_g[i][key] == st_o[i][key], (i, key)
    assert resid[0].shape[0] == rn_o and int((resid[4] >= 0).sum()) > 0
    # the residual itself: (root, link, src) keys, amounts, mean covered fractions
    assert _sorted_resid([r.cpu().numpy() for r in resid]) == _sorted_resid(
        [res_o[0], res_o[1], res_o[2], res_o[3], res_o[4]])
    # the node rule differs on the same inputs (the carried trips wait elsewhere)
    f_n, _, _, _ = Q.qdta_run_day(g, dd, 150.0, Q.make_params(step, stop, it, schedule=schedule))
    assert not torch.equal(f_n[1:], f_g[1:])


def test_carried_truncation_crosses_a_long_link_on_the_gpu():
    """The uncongested chain of 1000 s links with 300 s intervals: link k is
    loaded in the interval the trip enters it, the one containing 1000 k s."""
    net = synth.chain_network([1000.0, 1000.0, 1000.0], [1e9, 1e9, 1e9])
    g = Q.Graph(net)
    zones = T([3], np.int32)
    N = 11
    one = Q.DeviceOD(zones, T([0], np.int32), T([0], np.int32), T([1 << 32], np.int64))
    empty = Q.DeviceOD(zones, T([], np.int32), T([], np.int32), T([], np.int64))
    want = np.zeros((N, 3))
    for k in range(3):
        want[(1000 * k) // 300, k] = 1.0
    for schedule in ("plain", "graph"):
        f, st, rc, _ = Q.qdta_run_day(g, [one] + [empty] * (N - 1), 300.0,
                                      Q.make_params("msa", "none", 0, schedule=schedule, truncation="carry"))
        np.testing.assert_array_equal(f.cpu().numpy(), want)
        assert [s["n_items"] for s in st] == [1] * 10 + [0]


@pytest.mark.parametrize("schedule", ["plain", "graph"])
def test_carried_day_resumes_from_its_residual(schedule):
    """Run intervals 0-1, take the residual (with its carried links) out,
    resume intervals 2-4 from it: the same h(i) as the oracle's whole day."""
    day = _carry_day_case()
    days = list(day.demand)
    og = oracle.OracleGraph(day.net)
    p_o = oracle.make_params(Q.STEP["sweep8"], Q.STOP["paper_obj"], 40, truncation=oracle.TRUNC_CARRY)
    f_o, st_o, nit_o, rn_o, _ = oracle.run_day(og, day.zones, days, 150.0, p_o)
    g = Q.Graph(day.net)
    zones = T(day.zones, np.int32)
    dd = [Q.DeviceOD(zones, T(d.root_idx, np.int32), T(d.src, np.int32), T(d.amount_fx, np.int64)) for d in days]
    p = Q.make_params("sweep8", "paper_obj", 40, schedule=schedule, truncation="carry")
    f_a, _, _, res = Q.qdta_run_day(g, dd[:2], 150.0, p, resid_capacity=1 << 21)
    rin = Q.DeviceOD(zones, *(r.clone() for r in res))
    f_b, st_b, _, _ = Q.qdta_run_day(g, dd[2:], 150.0, p, resid_in=rin)
    np.testing.assert_array_equal(torch.cat([f_a, f_b]).cpu().numpy(), f_o)
    assert [s["n_items"] for s in st_b] == list(nit_o[2:])


def _carried_items(net, dem, seed):
    """half of the items put on a random out-link of their src, having
    covered a random fraction of it (0 included)"""
    rng = np.random.default_rng(seed)
    out = [[] for _ in range(net.n_nodes)]
    for a, t in enumerate(np.asarray(net.tail)):
        out[int(t)].append(a)
    link = np.full(dem.n_items, -1, dtype=np.int32)
    carry = np.zeros(dem.n_items, dtype=np.int64)
    for k in np.flatnonzero(rng.random(dem.n_items) < 0.5):
        a = out[int(dem.src[k])][rng.integers(len(out[int(dem.src[k])]))]
        link[k] = a
        carry[k] = 0 if rng.random() < 0.1 else rng.integers(0, 1 << 32)
    return carry, link


def test_load_aon_with_carried_trips_matches_the_oracle(small):
    inst, g, og = small
    dem = inst.demand[0]
    rng = np.random.default_rng(4)
    carry, link = _carried_items(inst.net, dem, 4)
    q = (inst.net.fftime_q * rng.uniform(1.0, 2.0, og.n_links)).astype(np.int32)
    par_o, _ = oracle.sssp(og, q, dem.roots, want_dist=False)
    od_o = oracle.OracleOD(dem.roots, dem.root_idx, dem.src, dem.amount_fx, carry_frac=carry, carry_link=link)
    for dt_q in (600, 6000, 30000):
        f_o, s_o, rc = oracle.load(og, q, par_o, od_o, dt_q)
        od_g = Q.DeviceOD(T(dem.roots, np.int32), T(dem.root_idx, np.int32), T(dem.src, np.int32),
                          T(dem.amount_fx, np.int64), T(carry, np.int64), T(link, np.int32))
        f_g, s_g = Q.qdta_load_aon(g, T(q, np.int32), T(par_o, np.int32), od_g, dt_q, want_stop=True)
        np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
        np.testing.assert_array_equal(s_g.cpu().numpy(), s_o)


@pytest.mark.parametrize("schedule", ["plain", "graph"])
def test_interval_with_carried_trips_matches_the_oracle(small, schedule):
    """One interval whose items are partly carried on links (the node rule
    and the carried rule), against the oracle, bit-exact."""
    inst, g, og = small
    dem = inst.demand[0]
    carry, link = _carried_items(inst.net, dem, 9)
    od_o = oracle.OracleOD(dem.roots, dem.root_idx, dem.src, dem.amount_fx, carry_frac=carry, carry_link=link)
    od_g = Q.DeviceOD(T(dem.roots, np.int32), T(dem.root_idx, np.int32), T(dem.src, np.int32),
                      T(dem.amount_fx, np.int64), T(carry, np.int64), T(link, np.int32))
    for trunc in ("node", "carry"):
        f_o, st_o, _ = oracle.assign_interval(og, od_o, 300.0, oracle.make_params(
            Q.STEP["sweep8"], Q.STOP["paper_obj"], 30, truncation=Q.TRUNCATION[trunc]))
        f_g, st_g, _, _ = Q.qdta_assign_interval(g, od_g, 300.0, Q.make_params(
            "sweep8", "paper_obj", 30, schedule=schedule, truncation=trunc))
        np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
        for key in ("iterations", "aon_calls", "ls_passes", "converged"):
            assert st_g[key] == st_o[key], (trunc, key)


def test_carried_items_are_checked(small):
    """A carried link must start at the item's src and exist; the covered
    fraction must lie in [0, 2^32)."""
    inst, g, og = small
    dem = inst.demand[0]
    tail = np.asarray(inst.net.tail)
    link = np.full(dem.n_items, -1, dtype=np.int32)
    link[0] = int(np.flatnonzero(tail != dem.src[0])[0])
    od_g = Q.DeviceOD(T(dem.roots, np.int32), T(dem.root_idx, np.int32), T(dem.src, np.int32),
                      T(dem.amount_fx, np.int64), T(np.zeros(dem.n_items), np.int64), T(link, np.int32))
    with pytest.raises(Q.QdtaError):
        Q.qdta_assign_interval(g, od_g, 300.0, Q.make_params("msa", "none", 2))
    link[0] = og.n_links  # no such link
    od_g.carry_link = T(link, np.int32)
    with pytest.raises(Q.QdtaError):
        Q.qdta_assign_interval(g, od_g, 300.0, Q.make_params("msa", "none", 2))
    link[0] = int(np.flatnonzero(tail == dem.src[0])[0])  # a link from src, but a whole link covered
    od_g.carry_link = T(link, np.int32)
    od_g.carry_frac = T(np.full(dem.n_items, 1 << 32), np.int64)
    with pytest.raises(Q.QdtaError):
        Q.qdta_assign_interval(g, od_g, 300.0, Q.make_params("msa", "none", 2))
    od_g.carry_frac = T(np.full(dem.n_items, (1 << 32) - 1), np.int64)  # the largest valid fraction
    Q.qdta_assign_interval(g, od_g, 300.0, Q.make_params("msa", "none", 2))


# ---------------------------------------------------------------------------
# Full size: the metro grid of the benchmark day (250k nodes, 954k links)
@pytest.fixture(scope="module")
def metro():
    inst = synth.config_day(seed=2)
    return inst, Q.Graph(inst.net), oracle.OracleGraph(inst.net)


def test_metro_batch_sampled_parity(metro):
    """One batch over all 2,000 zones in the launch shape the benchmark picks
    (autotuned on free-flow costs), at congested link times (the BPR costs of
    the busiest interval's all-or-nothing flows): 12 sampled roots' parent and
    distance rows, and the truncated loading of those roots' items, against
    the oracle, bit-exact."""
    inst, g, og = metro
    net = inst.net
    zones = T(inst.zones, np.int32)
    Q.qdta_autotune(g, T(net.fftime_q, np.int32), zones, Q.QDTA_TO_ROOT, reps=1)
    peak = int(np.argmax([d.amount_fx.sum() for d in inst.demand]))
    dem = inst.demand[peak]
    # congested costs: BPR of the free-flow all-or-nothing flows of the busiest interval
    par_ff, _ = Q.qdta_sssp_batch(g, T(net.fftime_q, np.int32), zones)
    g_fx, _ = Q.qdta_load_aon(g, T(net.fftime_q, np.int32), par_ff, Q.DeviceOD.of(dem), 90000)
    del par_ff
    f = g_fx.to(torch.float64) / float(1 << 32)
    q_g, _ = Q.qdta_bpr_costs(g, f, 900.0)
    q = q_g.cpu().numpy()
    q_o, _, _ = oracle.bpr(og, f.cpu().numpy(), 900.0)
    np.testing.assert_array_equal(q, q_o)
    assert q.max() > 10 * net.fftime_q.max()  # congested
    parent, dist = Q.qdta_sssp_batch(g, q_g, zones, Q.QDTA_TO_ROOT, want_dist=True)
    rng = np.random.default_rng(12)
    sample = np.sort(rng.choice(inst.zones.shape[0], 12, replace=False))
    p_o, d_o = oracle.sssp(og, q, inst.zones[sample])
    np.testing.assert_array_equal(dist[T(sample, np.int64)].cpu().numpy(), d_o)
    np.testing.assert_array_equal(parent[T(sample, np.int64)].cpu().numpy(), p_o)
    del dist
    # loading of the sampled roots' items (root indices remapped to the sample)
    remap = -np.ones(inst.zones.shape[0], np.int64)
    remap[sample] = np.arange(sample.shape[0])
    sel = remap[dem.root_idx] >= 0
    ri = remap[dem.root_idx[sel]].astype(np.int32)
    od_o = oracle.OracleOD(inst.zones[sample], ri, dem.src[sel], dem.amount_fx[sel])
    f_o, s_o, rc = oracle.load(og, q, p_o, od_o, 90000)
    od_g = Q.DeviceOD(T(inst.zones[sample], np.int32), T(ri, np.int32), T(dem.src[sel], np.int32),
                      T(dem.amount_fx[sel], np.int64))
    f_g, s_g = Q.qdta_load_aon(g, q_g, parent[T(sample, np.int64)].contiguous(), od_g, 90000, want_stop=True)
    np.testing.assert_array_equal(f_g.cpu().numpy(), f_o)
    np.testing.assert_array_equal(s_g.cpu().numpy(), s_o)
    assert rc == 0 and int(sel.sum()) > 1000


def test_autotune_cache_reuses_the_choice(mid, monkeypatch, tmp_path):
    """QDTA_TUNE_CACHE: a second handle on the same network (and a second
    process reading the cache file) applies the first tuning's choice without
    timing; the trees stay bit-exact."""
    import json
    import os
    import subprocess
    import sys
    net, dem, _, og = mid
    path = tmp_path / "tune_cache.txt"
    monkeypatch.setenv("QDTA_TUNE_CACHE", str(path))
    rng = np.random.default_rng(4)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.n_links)).astype(np.int32)
    roots = rng.choice(net.n_nodes, 64, replace=False).astype(np.int32)
    rep1 = Q.qdta_autotune(Q.Graph(net), T(q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, reps=1)
    assert not rep1["cached"] and len(rep1["candidates"]) > 1
    g2 = Q.Graph(net)
    rep2 = Q.qdta_autotune(g2, T(q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, reps=1)
    assert rep2["cached"] and len(rep2["candidates"]) == 1
    assert rep2["best"]["kernel"] == rep1["best"]["kernel"] == Q.qdta_sssp_kernel_name(g2, Q.QDTA_TO_ROOT)
    assert path.read_text().count("\n") == 1
    p_o, d_o = oracle.sssp(og, q, roots)
    p_g, d_g = Q.qdta_sssp_batch(g2, T(q, np.int32), T(roots, np.int32), Q.QDTA_TO_ROOT, True)
    np.testing.assert_array_equal(p_g.cpu().numpy(), p_o)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    child = ("import json, sys, numpy as np, torch; sys.path.insert(0, %r)\n"
             "from paper_2104_12911_gb300 import qdta as Q, synth\n"
             "net = synth.grid_network(110, 5, freeways=True)\n"
             "q = torch.from_numpy(net.fftime_q).cuda(); r = torch.arange(8, dtype=torch.int32, device='cuda')\n"
             "g = Q.Graph(net); rep = Q.qdta_autotune(g, q, r, Q.QDTA_TO_ROOT, reps=1)\n"
             "print(json.dumps({'cached': rep['cached'], 'kernel': rep['best']['kernel']}))\n") % root
    out = subprocess.run([sys.executable, "-c", child], capture_output=True, text=True, timeout=600,
                         env={**os.environ, "QDTA_TUNE_CACHE": str(path)})
    assert out.returncode == 0, out.stderr[-2000:]
    got = json.loads(out.stdout.strip().splitlines()[-1])
    assert got == {"cached": True, "kernel": rep1["best"]["kernel"]}
