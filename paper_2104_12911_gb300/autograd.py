"""torch.autograd.Function around one interval solve and its adjoint.

``assign(net, od, amounts, capacity, dt_s, params)`` returns the FW link
flows of the interval (trips, float64) as a differentiable function of the
items' trip amounts and the links' capacities (veh/h).  The forward pass is
qdta_assign_interval with a tape; the backward pass is qdta_backward, which
recomputes the shortest-path trees from the taped int32 link times and
gathers the flow adjoint along them (the transpose of loading), adding the
BPR capacity derivative through the line-search steps.  Trees and truncation
masks are held fixed (they are piecewise constant in the inputs).
"""
from __future__ import annotations

import torch

from . import qdta as Q


def graph_for(net, device: int) -> "Q.Graph":
    """One graph handle per (network, device), kept on the network object and
    reused by every solve; capacities are replaced on the device per call
    (qdta_graph_set_capacity) instead of building a new graph."""
    cache = net.__dict__.setdefault("_qdta_graphs", {})
    if device not in cache:
        cache[device] = Q.Graph(net, device)
    return cache[device]


class QdtaAssign(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amounts, capacity, net, roots, root_idx, src, dt_s, params):
        g = graph_for(net, amounts.device.index or 0)
        g.set_capacity(capacity)
        amount_fx = torch.round(amounts.detach() * float(Q.FX_ONE)).to(torch.int64)
        od = Q.DeviceOD(roots, root_idx, src, amount_fx)
        p = Q.Params.from_buffer_copy(params)
        p.record_tape = 1
        flows, stats, rc, tape = Q.qdta_assign_interval(g, od, dt_s, p)
        ctx.tape = tape
        ctx.graph = g
        ctx.stats = stats
        return flows

    @staticmethod
    def backward(ctx, grad_flows):
        dd, dc = Q.qdta_backward(ctx.tape, grad_flows.contiguous().to(torch.float64))
        ctx.tape.close()
        return dd, dc, None, None, None, None, None, None


def assign(net, od: "Q.DeviceOD", amounts: torch.Tensor, capacity: torch.Tensor, dt_s: float,
           params: "Q.Params"):
    """Differentiable interval solve (see module docstring)."""
    return QdtaAssign.apply(amounts, capacity, net, od.roots, od.root_idx, od.src, float(dt_s), params)
