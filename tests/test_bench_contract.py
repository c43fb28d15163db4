"""bench.py's reference arm (the CPU oracle on every host core) prints one
JSON line with the keys the benchmark contract asks for.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "day_small", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["unit"] == "s"
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_day_extrapolation_counts_batches_residual_rewalks_and_sweeps():
    """The CPU legs scale a timed per-root and per-sweep cost by the day's
    work: per interval, (shortest-path batches + accepted FW steps + 1
    residual re-walks) x destination roots, plus sweeps (an interval with no
    batch has no residual pass either)."""
    sys.path.insert(0, ROOT)
    import bench
    work = {"aon": [2, 0, 5], "fw": [1, 0, 3], "sweeps": [5, 0, 9]}
    got = bench.day_oracle_seconds(work, [3, 4, 2], 0.5, 0.1)
    want = (2 + 2) * 3 * 0.5 + 5 * 0.1 + (5 + 4) * 2 * 0.5 + 9 * 0.1
    assert abs(got - want) < 1e-12
    w = bench.METRO_DAY_WORK
    assert len(w["aon"]) == len(w["fw"]) == len(w["sweeps"]) == 96
    assert (sum(w["aon"]), sum(w["fw"]), sum(w["sweeps"])) == (3869, 3677, 18701)
