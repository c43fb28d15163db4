"""Failure detection without a GPU fault: a watchdog on the shortest-path
rounds and an injected allocation failure must come back as error codes, and
the library must keep working afterwards.  Each case runs in a child process
so that its environment switches stay local to it."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys, numpy as np, torch
    sys.path.insert(0, {root!r})
    from paper_2104_12911_gb300 import synth, qdta as Q
    inst = synth.config_small(0)
    g = Q.Graph(inst.net)
    q = torch.from_numpy(inst.net.fftime_q).cuda()
    roots = torch.from_numpy(inst.zones).cuda()
    codes = []
    for _ in range(2):
        try:
            Q.qdta_sssp_batch(g, q, roots)
            codes.append(0)
        except Q.QdtaError as e:
            codes.append(e.code)
    if {mode!r} == "watchdog":
        # the library keeps working: a 3-node chain needs fewer rounds than the limit
        c = synth.chain_network([1.0, 2.0], [100.0, 100.0])
        gc = Q.Graph(c)
        par, _ = Q.qdta_sssp_batch(gc, torch.from_numpy(c.fftime_q).cuda(),
                                   torch.tensor([2], dtype=torch.int32, device="cuda"))
        print("CODES", codes, "OK", par.cpu().tolist() == [[0, 1, -1]])
    else:
        # the handle must still solve an interval afterwards
        f, st, rc, _ = Q.qdta_assign_interval(g, Q.DeviceOD.of(inst.demand[0]), 900.0,
                                               Q.make_params("msa", "none", 3))
        print("CODES", codes, "OK", bool(torch.isfinite(f).all()), st["iterations"])
""")


def run_child(env_extra, mode):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, mode=mode)], env=env, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("CODES")][-1]
    return line


def test_round_watchdog_reports_timeout():
    # 3 rounds cannot settle a 32 x 32 grid: every batch must report ETIMEOUT
    line = run_child({"QDTA_MAX_ROUNDS": "3"}, "watchdog")
    assert "CODES [-4, -4]" in line
    assert "OK True" in line


def test_injected_allocation_failure_is_reported_and_recovers():
    # the first workspace allocation fails, the next call allocates normally
    line = run_child({"QDTA_FAULT": "alloc:1"}, "alloc")
    assert "CODES [-2, 0]" in line
    assert "OK True 3" in line
