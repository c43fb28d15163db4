"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point declared in include/qdta.h (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "qdta.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qdta_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("qdta_graph_create", "qdta_sssp_batch", "qdta_load_aon", "qdta_bpr_costs",
                 "qdta_line_search", "qdta_assign_interval", "qdta_run_day", "qdta_backward"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2104_12911_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    lib.qdta_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.qdta_version()


def test_library_rejects_bad_graphs_without_touching_a_gpu():
    from paper_2104_12911_gb300 import qdta as Q
    import numpy as np
    lib = Q.lib()
    # unsorted links are rejected before any device call
    tail = np.array([1, 0], np.int32)
    head = np.array([0, 1], np.int32)
    ff = np.array([1, 1], np.int32)
    cap = np.array([1.0, 1.0])
    d = Q.GraphDesc(2, 2, tail.ctypes.data, head.ctypes.data, ff.ctypes.data, cap.ctypes.data, 0.15, 4, 0.01)
    h = ctypes.c_void_p()
    assert lib.qdta_graph_create(ctypes.byref(d), 0, ctypes.byref(h)) == Q.QDTA_EINVAL
    assert b"sorted" in lib.qdta_last_error()
    d.beta = 0
    assert lib.qdta_graph_create(ctypes.byref(d), 0, ctypes.byref(h)) == Q.QDTA_EINVAL


def test_null_handles_are_rejected_without_touching_a_gpu():
    from paper_2104_12911_gb300 import qdta as Q
    lib = Q.lib()
    rep = Q.TuneReport()
    assert lib.qdta_autotune(None, None, None, 4, 0, 1, None, ctypes.byref(rep), None) == Q.QDTA_EINVAL
    assert lib.qdta_sssp_kernel_name(None, 0) == b""
    assert lib.qdta_last_error()
    assert lib.qdta_interval_metrics(None, None, 1, 900.0, None, None, 3, 1.0, None, None) == Q.QDTA_EINVAL


def test_tune_report_layout_matches_the_header():
    """The ctypes mirror of qdta_tune_report has the C struct's size (compiled here with gcc)."""
    import shutil
    import subprocess
    import tempfile
    from paper_2104_12911_gb300 import qdta as Q
    if not shutil.which("gcc"):
        import pytest
        pytest.skip("no gcc")
    src = ('#include <stdio.h>\n#include "qdta.h"\nint main(void){printf("%zu %zu %zu %zu\\n", '
           'sizeof(qdta_tune_entry), sizeof(qdta_tune_report), sizeof(qdta_profile), sizeof(qdta_params)); '
           'return 0;}\n')
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "sz.c")
        exe = os.path.join(d, "sz")
        with open(c, "w") as fh:
            fh.write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert [int(x) for x in out] == [ctypes.sizeof(Q.TuneEntry), ctypes.sizeof(Q.TuneReport),
                                     ctypes.sizeof(Q.Profile), ctypes.sizeof(Q.Params)]


def test_tune_report_as_dict_keeps_valid_rows_and_the_best():
    from paper_2104_12911_gb300 import qdta as Q
    rep = Q.TuneReport()
    rep.n, rep.best = 3, 1
    for i, (name, ms, valid) in enumerate((("a<1>", 5.0, 1), ("b<2>", 3.0, 1), ("c<3>", 0.0, 0))):
        rep.entry[i].kernel = name.encode()
        rep.entry[i].ctas_per_sm = 4
        rep.entry[i].ms = ms
        rep.entry[i].valid = valid
    d = rep.as_dict()
    assert [c["kernel"] for c in d["candidates"]] == ["a<1>", "b<2>"]
    assert d["best"]["kernel"] == "b<2>" and d["best"]["ms"] == 3.0
