"""Properties of the synthetic road grids that the GPU path's defaults rely
on (CPU only): links sorted by (tail, head) as the C ABI requires, every
degree <= 4 (four-slot adjacency), every link with its reverse (the
parent-slot skip of the rank-keyed kernels), and strong connectivity (the
spanning tree protected from the 5 % deletions)."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

from paper_2104_12911_gb300 import synth


@pytest.mark.parametrize("n,freeways,seed", [(32, False, 5), (64, True, 5), (110, True, 5), (500, True, 2),
                                             (500, True, 1)])
def test_grid_network_properties(n, freeways, seed):
    """(500, seed 2) is the metro grid of the benchmark day; its node ids are
    large enough that the spanning-tree keys need 64 bits."""
    net = synth.grid_network(n, seed, freeways=freeways)
    V, L = net.n_nodes, net.n_links
    assert V == n * n
    key = net.tail.astype(np.int64) * V + net.head
    assert np.all(np.diff(key) > 0), "links must be sorted by (tail, head) with no parallel links"
    assert np.bincount(net.tail, minlength=V).max() <= 4 and np.bincount(net.head, minlength=V).max() <= 4
    assert np.isin(net.head.astype(np.int64) * V + net.tail, key).all(), "every link has its reverse"
    adj = sp.csr_matrix((np.ones(L), (net.tail, net.head)), shape=(V, V))
    ncomp, _ = connected_components(adj, directed=True, connection="strong")
    assert ncomp == 1
    assert np.all(net.fftime_q >= 1) and np.all(net.capacity > 0)
    # 5 % of local undirected edges removed: a full grid has 4 n (n - 1) directed links
    assert 0.9 * 4 * n * (n - 1) <= L < 4 * n * (n - 1)


def test_day_demand_uses_the_zone_list_and_sums_to_the_day_total():
    inst = synth.config_day(seed=2, n=32, n_zones=40, trips_per_day=96_000, n_intervals=96)
    assert len(inst.demand) == 96
    total = sum(int(d.amount_fx.sum()) for d in inst.demand)
    assert total == 96_000 * synth.FX_ONE
    for d in inst.demand:
        assert np.array_equal(d.roots, inst.zones)
        assert np.all(np.diff(d.root_idx) >= 0)  # grouped by destination root
        assert np.all(d.src != inst.zones[d.root_idx])  # no intra-zonal trips
