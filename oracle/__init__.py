"""CPU oracle for the QDTA hot path (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It loads ``qdta_oracle.c`` compiled with gcc
(``-ffp-contract=off``) and wraps it with ctypes; it imports nothing from the
CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qdta_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

FX_ONE = 1 << 32
DIR_TO_ROOT, DIR_FROM_ROOT = 0, 1
STEP_MSA, STEP_PAPER_QN3, STEP_SWEEP8, STEP_EXACT = 0, 1, 2, 3
STOP_NONE, STOP_PAPER_OBJ, STOP_REL_GAP = 0, 1, 2
OK, EINVAL, ENOMEM, ENONFINITE, EUNREACH, NOTCONV = 0, -1, -2, -5, -6, 1
DIST_INF = np.iinfo(np.int64).max


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class Graph(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_links", C.c_int32),
                ("tail", C.c_void_p), ("head", C.c_void_p), ("fftime_q", C.c_void_p),
                ("capacity", C.c_void_p), ("alpha", C.c_double), ("beta", C.c_int32),
                ("quantum_s", C.c_double)]


class OD(C.Structure):
    _fields_ = [("n_roots", C.c_int32), ("roots", C.c_void_p), ("n_items", C.c_int64),
                ("root_idx", C.c_void_p), ("src", C.c_void_p), ("amount_fx", C.c_void_p),
                ("carry_frac", C.c_void_p), ("carry_link", C.c_void_p)]


OBJ_UE, OBJ_SO = 0, 1  # user equilibrium (Beckmann) / system optimum (total cost)
TRUNC_NODE, TRUNC_CARRY = 0, 1  # stop at the first node reached at or after dt / carry the partial link


class Params(C.Structure):
    _fields_ = [("step", C.c_int32), ("stop", C.c_int32), ("max_iter", C.c_int32),
                ("ls_max", C.c_int32), ("tol", C.c_double), ("ls_dx", C.c_double),
                ("ls_t1", C.c_double), ("ls_t2", C.c_double), ("objective", C.c_int32),
                ("truncation", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("aon_calls", C.c_int32), ("ls_passes", C.c_int32),
                ("converged", C.c_int32), ("rel_gap", C.c_double), ("objective", C.c_double),
                ("dual_gap", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            sig = {
                "or_to_fx": (None, [C.c_double, P, P, P]),
                "or_fx_to_double": (C.c_double, [C.c_int64, C.c_uint64]),
                "or_bpr": (C.c_int32, [P, P, C.c_double, P, P]),
                "or_sssp": (C.c_int32, [P, P, P, C.c_int32, C.c_int32, P, P]),
                "or_load": (C.c_int32, [P, P, P, P, C.c_int64, C.c_int32, P, P, P, P]),
                "or_line_search": (C.c_int32, [P, P, P, C.c_double, C.c_int32, P, P, P]),
                "or_objective": (C.c_double, [P, P, C.c_double]),
                "or_slope": (C.c_double, [P, P, P, C.c_double, C.c_double]),
                "or_assign_interval": (C.c_int32, [P, P, C.c_double, P, P, P, C.c_int32, P, P, P, P]),
                "or_residual": (C.c_int32, [P, P, C.c_double, C.c_int32, P, P, P, C.c_int32, P, C.c_int64,
                                            P, P, P, P, P, P]),
                "or_run_day": (C.c_int32, [P, C.c_int32, P, C.c_int32, P, P, P, P, C.c_double, P,
                                           P, P, P, P, C.c_int64, P, P, P, P, P]),
                "or_backward": (C.c_int32, [P, P, C.c_double, C.c_int32, C.c_int32, P, P, P, P,
                                            P, P]),
                "or_replay": (C.c_int32, [P, P, C.c_double, P, C.c_int32, P, P]),
                "or_interval_metrics": (C.c_int32, [P, P, C.c_int32, C.c_double, P, P, C.c_int32,
                                                    C.c_double, C.c_double, P]),
                "or_cch_build": (C.c_int32, [P, P, P]),
                "or_cch_free": (None, [P]),
                "or_cch_edges": (C.c_int64, [P]),
                "or_cch_customize": (C.c_int32, [P, P]),
                "or_cch_distance": (C.c_int32, [P, C.c_int32, P, P, P]),
                "or_cch_to_root": (C.c_int32, [P, C.c_int32, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleGraph:
    """Holds contiguous copies of a network's arrays for the C structs."""

    def __init__(self, net, capacity=None):
        self.tail = np.ascontiguousarray(net.tail, dtype=np.int32)
        self.head = np.ascontiguousarray(net.head, dtype=np.int32)
        self.fftime_q = np.ascontiguousarray(net.fftime_q, dtype=np.int32)
        cap = net.capacity if capacity is None else capacity
        self.capacity = np.ascontiguousarray(cap, dtype=np.float64)
        self.n_nodes = int(net.n_nodes)
        self.n_links = int(self.tail.shape[0])
        self.s = Graph(self.n_nodes, self.n_links, _p(self.tail).value, _p(self.head).value,
                       _p(self.fftime_q).value, _p(self.capacity).value, float(net.alpha),
                       int(net.beta), float(net.quantum_s))
        self.quantum_s = float(net.quantum_s)

    def ref(self):
        return C.byref(self.s)


class OracleOD:
    """Items (root_idx, src, amount_fx) over `roots`.  Optionally, carry_link
    puts an item on a link (src its tail; -1: at src) having covered the
    fraction carry_frac / 2^32 of it."""

    def __init__(self, roots, root_idx, src, amount_fx, carry_frac=None, carry_link=None):
        self.roots = np.ascontiguousarray(roots, dtype=np.int32)
        self.root_idx = np.ascontiguousarray(root_idx, dtype=np.int32)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.amount_fx = np.ascontiguousarray(amount_fx, dtype=np.int64)
        self.carry_frac = None if carry_frac is None else np.ascontiguousarray(carry_frac, dtype=np.int64)
        self.carry_link = None if carry_link is None else np.ascontiguousarray(carry_link, dtype=np.int32)
        self.s = OD(int(self.roots.shape[0]), _p(self.roots).value, int(self.src.shape[0]),
                    _p(self.root_idx).value, _p(self.src).value, _p(self.amount_fx).value,
                    None if self.carry_frac is None else _p(self.carry_frac).value,
                    None if self.carry_link is None else _p(self.carry_link).value)

    @classmethod
    def of(cls, dem):
        return cls(dem.roots, dem.root_idx, dem.src, dem.amount_fx)

    def ref(self):
        return C.byref(self.s)


def make_params(step=STEP_MSA, stop=STOP_NONE, max_iter=20, tol=1e-4, ls_max=20,
                ls_dx=1e-4, ls_t1=1e-4, ls_t2=1e-4, objective=OBJ_UE, truncation=TRUNC_NODE) -> Params:
    return Params(step, stop, max_iter, ls_max, tol, ls_dx, ls_t1, ls_t2, objective, truncation)


# --------------------------------------------------------------------------
def to_fx(v: float):
    hi, lo, bad = C.c_int64(), C.c_uint64(), C.c_int32()
    _load().or_to_fx(float(v), C.byref(hi), C.byref(lo), C.byref(bad))
    return (hi.value << 64) | lo.value, bad.value


def fx_to_double(x: int) -> float:
    x &= (1 << 128) - 1
    hi = x >> 64
    if hi >= 1 << 63:
        hi -= 1 << 64
    return _load().or_fx_to_double(hi, x & ((1 << 64) - 1))


def bpr(g: OracleGraph, flow, dt_s: float):
    flow = np.ascontiguousarray(flow, dtype=np.float64)
    cost = np.empty(g.n_links, dtype=np.float64)
    q = np.empty(g.n_links, dtype=np.int32)
    rc = _load().or_bpr(g.ref(), _p(flow), float(dt_s), _p(cost), _p(q))
    return q, cost, rc


def sssp(g: OracleGraph, q, roots, direction=DIR_TO_ROOT, want_dist=True):
    q = np.ascontiguousarray(q, dtype=np.int32)
    roots = np.ascontiguousarray(roots, dtype=np.int32)
    R, V = roots.shape[0], g.n_nodes
    parent = np.empty(R * V, dtype=np.int32)
    dist = np.empty(R * V, dtype=np.int64) if want_dist else None
    rc = _load().or_sssp(g.ref(), _p(q), _p(roots), R, direction, _p(parent),
                         _p(dist) if want_dist else None)
    if rc:
        raise RuntimeError(f"or_sssp failed: {rc}")
    return parent.reshape(R, V), (dist.reshape(R, V) if want_dist else None)


def load(g: OracleGraph, walk_q, parent, od: OracleOD, dt_q: int, flow_fx=None, truncation=TRUNC_NODE,
         want_carry=False):
    """Returns (flow_fx, stop nodes, rc), or with want_carry (flow_fx, stop
    nodes, covered fractions (2^-32 units), carrying links, rc)."""
    walk_q = np.ascontiguousarray(walk_q, dtype=np.int32)
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    if flow_fx is None:
        flow_fx = np.zeros(g.n_links, dtype=np.int64)
    n = od.src.shape[0]
    stop = np.empty(max(n, 1), dtype=np.int32)
    carry = np.empty(max(n, 1), dtype=np.int64)
    link = np.empty(max(n, 1), dtype=np.int32)
    rc = _load().or_load(g.ref(), _p(walk_q), _p(parent), od.ref(), int(dt_q), int(truncation), _p(flow_fx),
                         _p(stop), _p(carry), _p(link))
    if want_carry:
        return flow_fx, stop[:n], carry[:n], link[:n], rc
    return flow_fx, stop[:n], rc


def line_search(g: OracleGraph, f, g_fx, dt_s, fw_iter, params: Params):
    f = np.ascontiguousarray(f, dtype=np.float64)
    g_fx = np.ascontiguousarray(g_fx, dtype=np.int64)
    a, passes = C.c_double(), C.c_int32()
    rc = _load().or_line_search(g.ref(), _p(f), _p(g_fx), float(dt_s), int(fw_iter),
                                C.byref(params), C.byref(a), C.byref(passes))
    return a.value, passes.value, rc


def objective(g: OracleGraph, f, dt_s):
    f = np.ascontiguousarray(f, dtype=np.float64)
    return _load().or_objective(g.ref(), _p(f), float(dt_s))


def slope(g: OracleGraph, f, g_fx, dt_s, alpha):
    f = np.ascontiguousarray(f, dtype=np.float64)
    g_fx = np.ascontiguousarray(g_fx, dtype=np.int64)
    return _load().or_slope(g.ref(), _p(f), _p(g_fx), float(dt_s), float(alpha))


METRIC_NAMES = ("links", "vmt_km", "voc_mean", "vhd_h", "congested_links", "congested_km",
                "congested_vmt_km", "congested_voc_mean")


def interval_metrics(g: OracleGraph, flows, dt_s, length_m, link_class, n_classes, congested_voc=1.0):
    """Section 7.1 scenario metrics of N assigned intervals: returns
    (array [N, n_classes, 8] in METRIC_NAMES order, rc)."""
    flows = np.ascontiguousarray(np.atleast_2d(flows), dtype=np.float64)
    n = flows.shape[0]
    length_m = np.ascontiguousarray(length_m, dtype=np.float64)
    link_class = np.ascontiguousarray(link_class, dtype=np.int32)
    out = np.zeros((n, n_classes, 8), dtype=np.float64)
    rc = _load().or_interval_metrics(g.ref(), _p(flows), n, float(dt_s), _p(length_m), _p(link_class),
                                     int(n_classes), float(congested_voc), g.quantum_s, _p(out))
    return out, rc


class Tape:
    def __init__(self, cap, L):
        self.cap = cap
        self.q = np.zeros(cap * L, dtype=np.int32)
        self.alpha = np.zeros(cap, dtype=np.float64)
        self.f = np.zeros(cap * L, dtype=np.float64)
        self.K = C.c_int32(0)


def assign_interval(g: OracleGraph, od: OracleOD, dt_s: float, params: Params, tape=False):
    f = np.empty(g.n_links, dtype=np.float64)
    st = Stats()
    lib = _load()
    if tape:
        t = Tape(params.max_iter + 2, g.n_links)
        rc = lib.or_assign_interval(g.ref(), od.ref(), float(dt_s), C.byref(params), _p(f),
                                    C.byref(st), t.cap, _p(t.q), _p(t.alpha), _p(t.f), C.byref(t.K))
        return f, st.as_dict(), rc, t
    rc = lib.or_assign_interval(g.ref(), od.ref(), float(dt_s), C.byref(params), _p(f),
                                C.byref(st), 0, None, None, None, None)
    return f, st.as_dict(), rc


def residual(g: OracleGraph, od: OracleOD, dt_s: float, tape: Tape, f_final, truncation=TRUNC_NODE):
    """Returns (h_fx, (stop nodes, root indices, amounts, covered fractions, carrying links), rc)."""
    K = tape.K.value
    cap = od.src.shape[0] * (K + 1) + 1
    h = np.zeros(g.n_links, dtype=np.int64)
    rs = np.empty(cap, dtype=np.int32)
    rr = np.empty(cap, dtype=np.int32)
    ra = np.empty(cap, dtype=np.int64)
    rcy = np.empty(cap, dtype=np.int64)
    rl = np.empty(cap, dtype=np.int32)
    n = C.c_int64()
    f_final = np.ascontiguousarray(f_final, dtype=np.float64)
    rc = _load().or_residual(g.ref(), od.ref(), float(dt_s), K, _p(tape.q), _p(tape.alpha),
                             _p(f_final), int(truncation), _p(h), cap, _p(rs), _p(rr), _p(ra), _p(rcy), _p(rl),
                             C.byref(n))
    m = n.value
    return h, (rs[:m].copy(), rr[:m].copy(), ra[:m].copy(), rcy[:m].copy(), rl[:m].copy()), rc


def run_day(g: OracleGraph, zones, demands, dt_s: float, params: Params, want_resid=False):
    """Returns (flows [N, L], stats, merged item counts, residual count, rc);
    with want_resid a sixth entry, the residual left after the last interval
    as arrays (root index, src, amount_fx, covered fraction, link), sorted by
    root, link, src."""
    zones = np.ascontiguousarray(zones, dtype=np.int32)
    N = len(demands)
    off = np.zeros(N + 1, dtype=np.int64)
    for i, d in enumerate(demands):
        off[i + 1] = off[i] + d.n_items
    ri = np.ascontiguousarray(np.concatenate([d.root_idx for d in demands]), dtype=np.int32)
    si = np.ascontiguousarray(np.concatenate([d.src for d in demands]), dtype=np.int32)
    ai = np.ascontiguousarray(np.concatenate([d.amount_fx for d in demands]), dtype=np.int64)
    flows = np.zeros(N * g.n_links, dtype=np.float64)
    stats = (Stats * N)()
    nit = np.zeros(N, dtype=np.int64)
    rn = C.c_int64()
    # distinct residual keys: (root, node) and (root, link)
    cap = int(zones.shape[0]) * (g.n_nodes + g.n_links) if want_resid else 0
    rr = np.zeros(cap, dtype=np.int32); rs = np.zeros(cap, dtype=np.int32)
    ra = np.zeros(cap, dtype=np.int64); rcy = np.zeros(cap, dtype=np.int64); rl = np.zeros(cap, dtype=np.int32)
    out = [_p(a) for a in (rr, rs, ra, rcy, rl)] if want_resid else [None] * 5
    rc = _load().or_run_day(g.ref(), zones.shape[0], _p(zones), N, _p(off), _p(ri), _p(si), _p(ai),
                            float(dt_s), C.byref(params), _p(flows), stats, _p(nit), C.byref(rn), cap, *out)
    res = (flows.reshape(N, g.n_links), [s.as_dict() for s in stats], nit, rn.value, rc)
    if want_resid:
        m = min(rn.value, cap)
        res += ((rr[:m], rs[:m], ra[:m], rcy[:m], rl[:m]),)
    return res


def backward(g: OracleGraph, od: OracleOD, dt_s: float, step_mode: int, tape: Tape, dL_df):
    dL_df = np.ascontiguousarray(dL_df, dtype=np.float64)
    dd = np.zeros(od.src.shape[0], dtype=np.float64)
    dc = np.zeros(g.n_links, dtype=np.float64)
    rc = _load().or_backward(g.ref(), od.ref(), float(dt_s), int(step_mode), tape.K.value,
                             _p(tape.q), _p(tape.alpha), _p(tape.f), _p(dL_df), _p(dd), _p(dc))
    return dd, dc, rc


def replay(g: OracleGraph, od: OracleOD, dt_s: float, params: Params, tape: Tape):
    f = np.empty(g.n_links, dtype=np.float64)
    rc = _load().or_replay(g.ref(), od.ref(), float(dt_s), C.byref(params), tape.K.value,
                           _p(tape.q), _p(f))
    return f, rc


def dt_quanta(dt_s: float, quantum_s: float) -> int:
    if not np.isfinite(dt_s):
        return np.iinfo(np.int64).max
    return int(np.floor(dt_s / quantum_s + 0.5))


class CCH:
    """Customizable contraction hierarchy over an OracleGraph: build once for
    a contraction order (a permutation of the nodes), customize per metric,
    then query exact shortest times (equal to Dijkstra's)."""

    def __init__(self, g: OracleGraph, order):
        self.g = g
        self.order = np.ascontiguousarray(order, dtype=np.int32)
        h = C.c_void_p()
        rc = _load().or_cch_build(g.ref(), _p(self.order), C.byref(h))
        if rc:
            raise RuntimeError(f"or_cch_build failed: {rc}")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_cch_free(self.h)
            self.h = None

    @property
    def n_edges(self):
        return int(_load().or_cch_edges(self.h))

    def customize(self, q):
        q = np.ascontiguousarray(q, dtype=np.int32)
        rc = _load().or_cch_customize(self.h, _p(q))
        if rc:
            raise RuntimeError(f"or_cch_customize failed: {rc}")

    def distance(self, s, t):
        s = np.ascontiguousarray(s, dtype=np.int32)
        t = np.ascontiguousarray(t, dtype=np.int32)
        out = np.empty(max(s.shape[0], 1), dtype=np.int64)
        rc = _load().or_cch_distance(self.h, s.shape[0], _p(s), _p(t), _p(out))
        if rc:
            raise RuntimeError(f"or_cch_distance failed: {rc}")
        return out[:s.shape[0]]

    def to_root(self, z):
        out = np.empty(self.g.n_nodes, dtype=np.int64)
        rc = _load().or_cch_to_root(self.h, int(z), _p(out))
        if rc:
            raise RuntimeError(f"or_cch_to_root failed: {rc}")
        return out


def nested_dissection_order(x, y, tail, head, nodes=None, leaf=64):
    """Contraction order from node coordinates by nested dissection: split
    the nodes at the median of the wider coordinate; the nodes of the lower
    side that have a link to the upper side form a vertex separator (no link
    joins the two sides once they are removed).  Each side is ordered first,
    recursively, the separator last.  Any permutation gives the same
    distances; this one keeps the fill small."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    tail = np.asarray(tail)
    head = np.asarray(head)
    if nodes is None:
        nodes = np.arange(x.shape[0], dtype=np.int64)
    if nodes.shape[0] <= leaf:
        return [int(v) for v in nodes]
    xs, ys = x[nodes], y[nodes]
    c = xs if np.ptp(xs) >= np.ptp(ys) else ys
    o = np.argsort(c, kind="stable")
    half = nodes.shape[0] // 2
    lower, upper = nodes[o[:half]], nodes[o[half:]]
    in_upper = np.zeros(x.shape[0], dtype=bool)
    in_upper[upper] = True
    in_lower = np.zeros(x.shape[0], dtype=bool)
    in_lower[lower] = True
    crossing = (in_lower[tail] & in_upper[head]) | (in_upper[tail] & in_lower[head])
    sep = np.zeros(x.shape[0], dtype=bool)
    sep[np.where(in_lower[tail], tail, head)[crossing]] = True
    side = lower[~sep[lower]]
    return (nested_dissection_order(x, y, tail, head, side, leaf)
            + nested_dissection_order(x, y, tail, head, upper, leaf)
            + [int(v) for v in lower[sep[lower]]])
