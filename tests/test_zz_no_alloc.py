"""The shortest-path entry point that allocates no device memory.

It serves callers that cannot call cudaMalloc when they need shortest paths
(for example a process whose device memory is held by another allocator).  Its
results must equal qdta_sssp_batch's, call after call, even though every call
reuses one fixed device scratch array.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2104_12911_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2104_12911_gb300 import qdta as Q  # noqa: E402


def _call(lib, g, q, roots, direction, want_dist):
    R = int(roots.shape[0])
    parent = torch.full((R, g.n_nodes), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((R, g.n_nodes), -7, dtype=torch.int64, device="cuda") if want_dist else None
    rc = lib.qdta_sssp_batch_noalloc(g.h, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(roots.data_ptr()),
                                     R, direction, ctypes.c_void_p(parent.data_ptr()),
                                     ctypes.c_void_p(dist.data_ptr()) if want_dist else None,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == Q.QDTA_OK, lib.qdta_last_error()
    return parent, dist


def test_noalloc_matches_the_allocating_entry_point_on_consecutive_calls():
    lib = Q.lib()
    inst = synth.config_small(0)
    g = Q.Graph(inst.net)
    rng = np.random.default_rng(5)
    cases = [(inst.net.fftime_q, inst.zones, Q.QDTA_TO_ROOT, True),
             ((inst.net.fftime_q * rng.uniform(1, 5, inst.net.n_links)).astype(np.int32),
              rng.choice(inst.net.n_nodes, 40, replace=False).astype(np.int32), Q.QDTA_FROM_ROOT, False)]
    for q, roots, direction, want_dist in cases:   # two calls in a row, different inputs
        qd = torch.from_numpy(np.ascontiguousarray(q, np.int32)).cuda()
        rd = torch.from_numpy(np.ascontiguousarray(roots, np.int32)).cuda()
        p_na, d_na = _call(lib, g, qd, rd, direction, want_dist)
        p_ref, d_ref = Q.qdta_sssp_batch(g, qd, rd, direction, want_dist)
        torch.cuda.synchronize()
        assert torch.equal(p_na, p_ref)
        if want_dist:
            assert torch.equal(d_na, d_ref)


def test_noalloc_rejects_graphs_beyond_its_limit():
    lib = Q.lib()
    net = synth.grid_network(140, 3)       # ~75k links, ~19.6k nodes: beyond both limits
    assert net.n_links > 65536
    g = Q.Graph(net)
    q = torch.from_numpy(net.fftime_q).cuda()
    roots = torch.zeros(1, dtype=torch.int32, device="cuda")
    parent = torch.empty((1, net.n_nodes), dtype=torch.int32, device="cuda")
    rc = lib.qdta_sssp_batch_noalloc(g.h, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(roots.data_ptr()), 1,
                                     Q.QDTA_TO_ROOT, ctypes.c_void_p(parent.data_ptr()), None,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == Q.QDTA_EINVAL
    assert b"at most" in lib.qdta_last_error()
