"""Python binding of libqdta (include/qdta.h) -- argument marshalling only.

Every function here has the name of the C entry point it calls.  Device
arrays are torch CUDA tensors; the CUDA stream is torch's current stream.
All computation happens inside the library's kernels; if the library is not
built this module raises instead of computing anything another way.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading

import numpy as np
import torch

from . import build as _build

QDTA_OK, QDTA_EINVAL, QDTA_ENOMEM, QDTA_ECUDA, QDTA_ETIMEOUT = 0, -1, -2, -3, -4
QDTA_ENONFINITE, QDTA_EUNREACH, QDTA_EOVERFLOW, QDTA_ENOTCONV = -5, -6, -7, 1
QDTA_TO_ROOT, QDTA_FROM_ROOT = 0, 1
STEP = {"msa": 0, "paper_qn3": 1, "sweep8": 2, "exact": 3}
STOP = {"none": 0, "paper_obj": 1, "rel_gap": 2}
OBJECTIVE = {"ue": 0, "so": 1}
TRUNCATION = {"node": 0, "carry": 1}
SCHEDULE = {"plain": 0, "graph": 1}
DIST_INF = np.iinfo(np.int64).max
FX_ONE = 1 << 32


class QdtaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qdta error {code}: {msg}")
        self.code = code


class GraphDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_links", C.c_int32), ("tail", C.c_void_p),
                ("head", C.c_void_p), ("fftime_q", C.c_void_p), ("capacity_vph", C.c_void_p),
                ("alpha", C.c_double), ("beta", C.c_int32), ("quantum_s", C.c_double)]


class OD(C.Structure):
    _fields_ = [("n_roots", C.c_int32), ("roots", C.c_void_p), ("n_items", C.c_int64),
                ("root_idx", C.c_void_p), ("src", C.c_void_p), ("amount_fx", C.c_void_p),
                ("carry_frac", C.c_void_p), ("carry_link", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("step", C.c_int32), ("stop", C.c_int32), ("max_iter", C.c_int32),
                ("ls_max", C.c_int32), ("tol", C.c_double), ("ls_dx", C.c_double),
                ("ls_t1", C.c_double), ("ls_t2", C.c_double), ("schedule", C.c_int32),
                ("record_tape", C.c_int32), ("objective", C.c_int32), ("truncation", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("aon_calls", C.c_int32), ("ls_passes", C.c_int32),
                ("converged", C.c_int32), ("rel_gap", C.c_double), ("objective", C.c_double),
                ("n_items", C.c_int64), ("dual_gap", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Residual(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("root_idx", C.c_void_p), ("src", C.c_void_p),
                ("amount_fx", C.c_void_p), ("count", C.c_int64), ("carry_frac", C.c_void_p),
                ("carry_link", C.c_void_p)]


class Profile(C.Structure):
    _fields_ = [("sssp_launches", C.c_int64), ("sssp_ms", C.c_double), ("sssp_roots", C.c_int64),
                ("load_launches", C.c_int64), ("load_ms", C.c_double),
                ("sweep_launches", C.c_int64), ("sweep_ms", C.c_double),
                ("kernel_launches", C.c_int64), ("sssp_rounds", C.c_int64),
                ("sssp_relaxations", C.c_int64), ("sssp_cell_activations", C.c_int64),
                ("sssp_redo_batches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TUNE_MAX = 24


class TuneEntry(C.Structure):
    _fields_ = [("kernel", C.c_char * 40), ("ctas_per_sm", C.c_int32), ("valid", C.c_int32), ("ms", C.c_float)]


class TuneReport(C.Structure):
    _fields_ = [("n", C.c_int32), ("best", C.c_int32), ("entry", TuneEntry * TUNE_MAX), ("cached", C.c_int32)]

    def as_dict(self):
        rows = [{"kernel": e.kernel.decode(), "ctas_per_sm": e.ctas_per_sm, "ms": e.ms}
                for e in self.entry[:self.n] if e.valid]
        return {"best": rows[self.best] if rows else None, "candidates": rows, "cached": bool(self.cached)}


class Instance(C.Structure):
    _fields_ = [("graph", C.c_void_p), ("od", OD), ("dt_s", C.c_double), ("flow_out", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libqdta.so (building it first if its sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not _build.up_to_date():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libqdta.so is missing; run paper_2104_12911_gb300.build.build()")
            L = C.CDLL(path)
            P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            sig = {
                "qdta_graph_create": [P, C.c_int, P],
                "qdta_graph_destroy": [P],
                "qdta_graph_set_capacity": [P, P, P],
                "qdta_sssp_batch": [P, P, P, I32, I32, P, P, P],
                "qdta_sssp_batch_noalloc": [P, P, P, I32, I32, P, P, P],
                "qdta_load_aon": [P, P, P, P, I64, P, P, P],
                "qdta_bpr_costs": [P, P, D, P, P, P],
                "qdta_line_search": [P, P, P, D, I32, P, P, P, P],
                "qdta_assign_interval": [P, P, D, P, P, P, P, P],
                "qdta_assign_batch": [P, I32, P, P, P],
                "qdta_run_day": [P, P, I32, D, P, P, P, P, P, P],
                "qdta_backward": [P, P, P, P, P],
                "qdta_tape_destroy": [P],
                "qdta_tape_info": [P, P, P],
                "qdta_profile_enable": [P, I32],
                "qdta_profile_read": [P, P],
                "qdta_autotune": [P, P, P, I32, I32, I32, P, P, P],
                "qdta_interval_metrics": [P, P, I32, D, P, P, I32, D, P, P],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.qdta_last_error.restype = C.c_char_p
            L.qdta_last_error.argtypes = []
            L.qdta_version.restype = C.c_char_p
            L.qdta_sssp_kernel_name.restype = C.c_char_p
            L.qdta_sssp_kernel_name.argtypes = [P, I32]
            _lib = L
    return _lib


def _check(rc):
    if rc < 0:
        raise QdtaError(rc, lib().qdta_last_error().decode())
    return rc


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_params(step="sweep8", stop="rel_gap", max_iter=200, tol=1e-4, ls_max=20, ls_dx=1e-4,
                ls_t1=1e-4, ls_t2=1e-4, schedule="plain", record_tape=False, objective="ue",
                truncation="node") -> Params:
    return Params(STEP[step] if isinstance(step, str) else int(step),
                  STOP[stop] if isinstance(stop, str) else int(stop), int(max_iter), int(ls_max),
                  float(tol), float(ls_dx), float(ls_t1), float(ls_t2),
                  SCHEDULE[schedule] if isinstance(schedule, str) else int(schedule),
                  1 if record_tape else 0, OBJECTIVE[objective] if isinstance(objective, str) else int(objective),
                  TRUNCATION[truncation] if isinstance(truncation, str) else int(truncation))


class Graph:
    """Owns a qdta_graph handle for a network (host arrays are copied)."""

    def __init__(self, net, device: int = 0, capacity=None):
        tail = np.ascontiguousarray(net.tail, dtype=np.int32)
        head = np.ascontiguousarray(net.head, dtype=np.int32)
        ff = np.ascontiguousarray(net.fftime_q, dtype=np.int32)
        cap = np.ascontiguousarray(net.capacity if capacity is None else capacity, dtype=np.float64)
        d = GraphDesc(int(net.n_nodes), int(tail.shape[0]), tail.ctypes.data, head.ctypes.data,
                      ff.ctypes.data, cap.ctypes.data, float(net.alpha), int(net.beta),
                      float(net.quantum_s))
        h = C.c_void_p()
        _check(lib().qdta_graph_create(C.byref(d), int(device), C.byref(h)))
        self.h = h
        self.n_nodes = int(net.n_nodes)
        self.n_links = int(tail.shape[0])
        self.device = torch.device("cuda", device)
        self.quantum_s = float(net.quantum_s)

    def set_capacity(self, capacity):
        """qdta_graph_set_capacity: capacity is a float64 CUDA tensor [L] (veh/h)."""
        cap = capacity.detach().to(self.device, torch.float64).contiguous()
        _check(lib().qdta_graph_set_capacity(self.h, _ptr(cap), _stream()))

    def close(self):
        if getattr(self, "h", None):
            lib().qdta_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class DeviceOD:
    roots: torch.Tensor
    root_idx: torch.Tensor
    src: torch.Tensor
    amount_fx: torch.Tensor
    # trips carried on a link (both None, or int64 / int32 per item): the
    # fraction of carry_link covered, in 2^-32 units (-1: the trip waits at src)
    carry_frac: torch.Tensor = None
    carry_link: torch.Tensor = None

    @classmethod
    def of(cls, dem, device="cuda", pin=False):
        def t(a, dt):
            x = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
            return x.to(device)
        return cls(t(dem.roots, np.int32), t(dem.root_idx, np.int32), t(dem.src, np.int32),
                   t(dem.amount_fx, np.int64))

    @property
    def n_items(self):
        return int(self.src.shape[0])

    def struct(self) -> OD:
        return OD(int(self.roots.shape[0]), self.roots.data_ptr(), self.n_items,
                  self.root_idx.data_ptr(), self.src.data_ptr(), self.amount_fx.data_ptr(),
                  self.carry_frac.data_ptr() if self.carry_frac is not None else None,
                  self.carry_link.data_ptr() if self.carry_link is not None else None)


# ---------------------------------------------------------------------------
def qdta_sssp_batch(g: Graph, cost_q, roots, direction=QDTA_TO_ROOT, want_dist=False):
    R = int(roots.shape[0])
    parent = torch.empty((R, g.n_nodes), dtype=torch.int32, device=g.device)
    dist = torch.empty((R, g.n_nodes), dtype=torch.int64, device=g.device) if want_dist else None
    _check(lib().qdta_sssp_batch(g.h, _ptr(cost_q), _ptr(roots), R, int(direction), _ptr(parent),
                                 _ptr(dist), _stream()))
    return parent, dist


def qdta_sssp_batch_noalloc(g: Graph, cost_q, roots, direction=QDTA_TO_ROOT, want_dist=False):
    R = int(roots.shape[0])
    parent = torch.empty((R, g.n_nodes), dtype=torch.int32, device=g.device)
    dist = torch.empty((R, g.n_nodes), dtype=torch.int64, device=g.device) if want_dist else None
    _check(lib().qdta_sssp_batch_noalloc(g.h, _ptr(cost_q), _ptr(roots), R, int(direction), _ptr(parent),
                                         _ptr(dist), _stream()))
    return parent, dist


def qdta_autotune(g: Graph, cost_q, roots, direction=QDTA_TO_ROOT, reps=2):
    """Time every launch shape of the shortest-path batch on (cost_q, roots)
    and keep the fastest in ``g``; returns the report as a dict."""
    R = int(roots.shape[0])
    scratch = torch.empty((R, g.n_nodes), dtype=torch.int32, device=g.device)
    rep = TuneReport()
    _check(lib().qdta_autotune(g.h, _ptr(cost_q), _ptr(roots), R, int(direction), int(reps), _ptr(scratch),
                               C.byref(rep), _stream()))
    return rep.as_dict()


METRIC_NAMES = ("links", "vmt_km", "voc_mean", "vhd_h", "congested_links", "congested_km",
                "congested_vmt_km", "congested_voc_mean")


def qdta_interval_metrics(g: Graph, flows, dt_s, length_m, link_class, n_classes, congested_voc=1.0):
    """Scenario metrics of N intervals' link flows ([N, L] float64 on the
    device): returns [N, n_classes, 8] float64 in METRIC_NAMES order."""
    flows = flows.reshape(-1, g.n_links).contiguous()
    n = int(flows.shape[0])
    out = torch.empty((n, int(n_classes), 8), dtype=torch.float64, device=g.device)
    _check(lib().qdta_interval_metrics(g.h, _ptr(flows), n, float(dt_s), _ptr(length_m.contiguous()),
                                       _ptr(link_class.contiguous()), int(n_classes), float(congested_voc),
                                       _ptr(out), _stream()))
    return out


def qdta_load_aon(g: Graph, cost_q, parent, od: DeviceOD, dt_q: int, flow_fx=None, want_stop=False):
    if flow_fx is None:
        flow_fx = torch.zeros(g.n_links, dtype=torch.int64, device=g.device)
    stop = torch.empty(max(od.n_items, 1), dtype=torch.int32, device=g.device) if want_stop else None
    s = od.struct()
    _check(lib().qdta_load_aon(g.h, _ptr(cost_q), _ptr(parent), C.byref(s), int(dt_q), _ptr(flow_fx),
                               _ptr(stop), _stream()))
    return flow_fx, (stop[:od.n_items] if want_stop else None)


def qdta_bpr_costs(g: Graph, flow, dt_s: float, want_cost_s=False):
    q = torch.empty(g.n_links, dtype=torch.int32, device=g.device)
    cs = torch.empty(g.n_links, dtype=torch.float64, device=g.device) if want_cost_s else None
    _check(lib().qdta_bpr_costs(g.h, _ptr(flow), float(dt_s), _ptr(cs), _ptr(q), _stream()))
    return q, cs


def qdta_line_search(g: Graph, flow, aon_fx, dt_s: float, fw_iter: int, params: Params):
    a = C.c_double()
    n = C.c_int32()
    _check(lib().qdta_line_search(g.h, _ptr(flow), _ptr(aon_fx), float(dt_s), int(fw_iter),
                                  C.byref(params), C.byref(a), C.byref(n), _stream()))
    return a.value, n.value


class Tape:
    def __init__(self, h, od):
        self.h = h
        self.od = od  # keeps the device arrays alive

    def info(self):
        K, n = C.c_int32(), C.c_int64()
        _check(lib().qdta_tape_info(self.h, C.byref(K), C.byref(n)))
        return K.value, n.value

    def close(self):
        if self.h:
            lib().qdta_tape_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qdta_assign_interval(g: Graph, od: DeviceOD, dt_s: float, params: Params, flow_out=None):
    if flow_out is None:
        flow_out = torch.empty(g.n_links, dtype=torch.float64, device=g.device)
    st = Stats()
    s = od.struct()
    th = C.c_void_p()
    rc = _check(lib().qdta_assign_interval(g.h, C.byref(s), float(dt_s), C.byref(params),
                                           _ptr(flow_out), C.byref(st),
                                           C.byref(th) if params.record_tape else None, _stream()))
    tape = Tape(th, od) if params.record_tape and th.value else None
    return flow_out, st.as_dict(), rc, tape


def qdta_assign_batch(items, params: Params):
    """items: list of (Graph, DeviceOD, dt_s, flow_out tensor)."""
    arr = (Instance * len(items))()
    for i, (g, od, dt, fo) in enumerate(items):
        arr[i] = Instance(g.h.value, od.struct(), float(dt), fo.data_ptr())
    st = (Stats * len(items))()
    rc = _check(lib().qdta_assign_batch(arr, len(items), C.byref(params), st, _stream()))
    return [s.as_dict() for s in st], rc


def qdta_run_day(g: Graph, days, dt_s: float, params: Params, resid_in: DeviceOD = None,
                 resid_capacity: int = 0, flow_out=None):
    """days: list of DeviceOD sharing one roots (zone) tensor."""
    N = len(days)
    arr = (OD * N)(*[d.struct() for d in days])
    if flow_out is None:
        flow_out = torch.empty((N, g.n_links), dtype=torch.float64, device=g.device)
    st = (Stats * N)()
    rin = resid_in.struct() if resid_in is not None else None
    rout = None
    bufs = None
    if resid_capacity > 0:
        bufs = (torch.empty(resid_capacity, dtype=torch.int32, device=g.device),
                torch.empty(resid_capacity, dtype=torch.int32, device=g.device),
                torch.empty(resid_capacity, dtype=torch.int64, device=g.device),
                torch.empty(resid_capacity, dtype=torch.int64, device=g.device),
                torch.empty(resid_capacity, dtype=torch.int32, device=g.device))
        rout = Residual(resid_capacity, bufs[0].data_ptr(), bufs[1].data_ptr(), bufs[2].data_ptr(), 0,
                        bufs[3].data_ptr(), bufs[4].data_ptr())
    rc = _check(lib().qdta_run_day(g.h, arr, N, float(dt_s), C.byref(params),
                                   C.byref(rin) if rin is not None else None, _ptr(flow_out), st,
                                   C.byref(rout) if rout is not None else None, _stream()))
    resid = None
    if rout is not None:
        n = rout.count
        # root index, stop node (a carried trip: its link's tail), amount, covered fraction (2^-32 units), link (-1: none)
        resid = tuple(b[:n] for b in bufs)
    return flow_out, [s.as_dict() for s in st], rc, resid


def qdta_backward(tape: Tape, dL_dflow):
    K, n = tape.info()
    dev = dL_dflow.device
    dd = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    dc = torch.empty(dL_dflow.shape[0], dtype=torch.float64, device=dev)
    _check(lib().qdta_backward(tape.h, _ptr(dL_dflow.contiguous()), _ptr(dd), _ptr(dc), _stream()))
    return dd[:n], dc


def qdta_profile_enable(g: Graph, on=True):
    _check(lib().qdta_profile_enable(g.h, 1 if on else 0))


def qdta_profile_read(g: Graph):
    p = Profile()
    _check(lib().qdta_profile_read(g.h, C.byref(p)))
    return p.as_dict()


def version():
    return lib().qdta_version().decode()


def qdta_sssp_kernel_name(g: Graph, direction: int = QDTA_TO_ROOT) -> str:
    """Name of the shortest-path kernel qdta_sssp_batch launches on ``g``."""
    name = lib().qdta_sssp_kernel_name(g.h, direction).decode()
    if not name:
        raise QdtaError(-1, lib().qdta_last_error().decode())
    return name
