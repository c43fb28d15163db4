#!/usr/bin/env python3
"""Benchmark: full-day quasi-dynamic traffic assignment on one GB300.

One step = one full day (96 x 15-minute intervals, Alg. 1): for every
interval the residual demand is merged, the static user equilibrium is
solved by Frank-Wolfe (batched shortest paths, truncated loading, 8-point
line search) until the paper's Converged test holds (relative objective
change < 1e-4, Section 4; --stop rel_gap stops on the relative duality gap
instead), and the residual demand is re-truncated and carried to the next
interval.  Every interval's duality gap is reported either way.  The timed steps run the graph schedule
(device-side control, CUDA graphs); one extra day runs the plain host launch
loop for the batched-vs-plain comparison and for per-kernel CUDA-event
timings (the SSSP roofline line).

One metro day takes minutes, so the run is bounded by a wall-clock budget
(--budget-s, counted from process start): at most three warm-up days (the
plain profiling day and two graph days), then timed days while another one
still fits the budget, at least one and at most --steps.  The JSON line's
"steps" and "warmup" are the days actually run; "steps_requested" and
"warmup_requested" echo the command line.  A progress line per day goes to
stderr.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

T_START = time.monotonic()
ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Full-day QDTA s @rel-gap 1e-4, batched vs plain on 1 GB300; SSSP GTEPS, %HBM"

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per destination
# root of the SSSP kernels, from one ncu capture each on the 500x500 metro
# grid (one wave of 608 resident roots); the roofline's `traffic` scales them
# by the roots per launch.  Only kernels whose code is unchanged since their
# capture are listed.
SSSP_DRAM_BYTES_PER_ROOT = {
    "sssp_smq_kernel<256,rank32,2,true>": (1.338081e9 + 2.564112e9) / 608,
}


def progress(msg):
    """One line on stderr, stamped with the seconds since process start."""
    print(f"[bench {time.monotonic() - T_START:7.1f} s] {msg}", file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="day_metro",
                    choices=["day_metro", "day_small", "sssp_metro", "batch32", "adjoint_metro", "interval_metro",
                             "sta_vs_qdta", "gap_peak", "floor_small"])
    ap.add_argument("--roots", type=int, default=2000, help="sssp_metro: destination roots per batch")
    ap.add_argument("--intervals", default=None,
                    help="a:b -- run only intervals a..b-1 of the day (profiling captures; not a bench line)")
    ap.add_argument("--max-iter", type=int, default=200)
    ap.add_argument("--stop", default="paper_obj", choices=["paper_obj", "rel_gap"])
    ap.add_argument("--step", default="sweep8", choices=["sweep8", "paper_qn3", "exact", "msa"],
                    help="FW step rule (the paper compares its line search with MSA)")
    ap.add_argument("--objective", default="ue", choices=["ue", "so"],
                    help="user equilibrium (the paper's) or system optimum")
    ap.add_argument("--truncation", default="node", choices=["node", "carry"],
                    help="day workloads: Eq. 2's node rule, or Section 3.4's carried partial links")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default SSSP launch shape")
    ap.add_argument("--budget-s", type=float, default=1350.0,
                    help="day workloads: wall-clock budget of the whole run, from process start; warm-up is "
                         "capped at 3 days and timed days stop when the next one would not fit")
    ap.add_argument("--max-warmup-days", type=int, default=3)
    return ap.parse_args()


def make_workload(name):
    from paper_2104_12911_gb300 import synth
    if name == "day_metro":
        inst = synth.config_day(seed=2)
        cfg = {"workload": "full day, 96 x 15 min, 500x500 jittered grid (250k nodes, "
                           f"{inst.net.n_links} links), 2000 zones, 19M trips/day",
               "grid": 500, "zones": 2000, "trips_per_day": 19_000_000}
    else:
        base = synth.config_small(0)
        inst = synth.scaled_day(base, 400_000, n_intervals=96, seed=2)
        cfg = {"workload": "full day, 96 x 15 min, 32x32 grid (1024 nodes, "
                           f"{inst.net.n_links} links), 64 zones, 400k trips/day",
               "grid": 32, "zones": 64, "trips_per_day": 400_000}
    cfg.update({"intervals": 96, "dt_s": 900.0, "step_rule": "sweep8",
                "stop": "paper Converged rule: relative objective change < 1e-4 (Section 4)",
                "l2": "working set (per-root SSSP state, trees) far above the 129 MB L2"})
    return inst, cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(values, world, device):
    """Element-wise maximum over all ranks (the slowest replica defines the
    job's time); identity for a single process."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_seconds_per_day(ms_max, world):
    """Whole-job seconds per simulated day: `world` replicas each simulate one
    day per step in ms_max milliseconds (the slowest rank)."""
    return ms_max / 1e3 / world


# ---------------------------------------------------------------------------
# root-parallel CPU oracle: the unmodified oracle, one destination root per
# task, in a process pool started with "spawn" (safe after CUDA is live)
_POOL_OG, _POOL_Q = None, None


def _pool_init(net, q):
    global _POOL_OG, _POOL_Q
    import oracle
    _POOL_OG, _POOL_Q = oracle.OracleGraph(net), q


def _pool_root(task):
    import oracle
    root, src, amt, dt_q = task
    od = oracle.OracleOD(np.array([root], np.int32), np.zeros(len(src), np.int32), src, amt)
    par, _ = oracle.sssp(_POOL_OG, _POOL_Q, od.roots, want_dist=False)
    oracle.load(_POOL_OG, _POOL_Q, par, od, dt_q)
    return 1


class OraclePool:
    """Times Dijkstra + loading per destination root on every host core."""

    def __init__(self, net, q):
        import multiprocessing as mp
        self.n = max(1, os.cpu_count() or 1)
        self.pool = mp.get_context("spawn").Pool(self.n, initializer=_pool_init, initargs=(net, q))
        self.pool.map(_pool_root, [], chunksize=1)

    @staticmethod
    def tasks(dem, roots):
        out = []
        for r in roots:
            sel = dem.root_idx == r
            out.append((int(dem.roots[r]), dem.src[sel].copy(), dem.amount_fx[sel].copy(), 90000))
        return out

    def seconds_per_root(self, tasks):
        """Wall seconds per root when `tasks` run on all cores (after one warm task per worker)."""
        self.pool.map(_pool_root, tasks[:self.n], chunksize=1)
        t0 = time.perf_counter()
        self.pool.map(_pool_root, tasks, chunksize=1)
        return (time.perf_counter() - t0) / max(len(tasks), 1)

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(inst, day_stats, budget_s=20.0):
    """Time the CPU oracle on a bounded sample of the same day and scale it
    to the day's work: per-root Dijkstra + walks and per-sweep costs,
    multiplied by the AON / line-search counts of the day."""
    import oracle
    og = oracle.OracleGraph(inst.net)
    V, L = og.n_nodes, og.n_links
    peak = int(np.argmax([d.n_items for d in inst.demand]))
    dem = inst.demand[peak]
    active = np.unique(dem.root_idx)
    t0 = time.perf_counter()
    roots_done = 0
    q = inst.net.fftime_q
    while roots_done < len(active) and time.perf_counter() - t0 < budget_s * 0.7:
        r = int(active[roots_done])
        sel = dem.root_idx == r
        od = oracle.OracleOD(dem.roots[r:r + 1], np.zeros(int(sel.sum()), np.int32), dem.src[sel],
                             dem.amount_fx[sel])
        par, _ = oracle.sssp(og, q, od.roots, want_dist=False)
        oracle.load(og, q, par, od, 90000)
        roots_done += 1
    t_root = (time.perf_counter() - t0) / max(roots_done, 1)
    rng = np.random.default_rng(0)
    f = rng.uniform(0, 50, L)
    gfx = (rng.uniform(0, 50, L) * (1 << 32)).astype(np.int64)
    t1 = time.perf_counter()
    _, passes, _ = oracle.line_search(og, f, gfx, 900.0, 1,
                                      oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_NONE, 20))
    t_pass = (time.perf_counter() - t1) / max(passes, 1)
    n_roots = [len(np.unique(d.root_idx)) for d in inst.demand]
    work = {"aon": [st["aon_calls"] for st in day_stats], "fw": [st["iterations"] for st in day_stats],
            "sweeps": [st["ls_passes"] for st in day_stats]}

    def day_seconds(t_r):
        return day_oracle_seconds(work, n_roots, t_r, t_pass)
    spent = time.perf_counter() - t0
    # the same roots again on every host core (the sweeps stay single-core)
    par = None
    try:
        pool = OraclePool(inst.net, q)
        n_par = min(len(active), max(pool.n * 4, roots_done))
        t_root_par = pool.seconds_per_root(OraclePool.tasks(dem, active[:n_par]))
        pool.close()
        par = {"value": day_seconds(t_root_par), "unit": "s", "cores": pool.n, "sec_per_root": t_root_par,
               "sample": f"{n_par} destination roots of the peak interval, one process per core"}
    except Exception as exc:  # no process pool on this host: report the single-core figure only
        par = {"unavailable": f"{type(exc).__name__}: {exc}"}
    return {"value": day_seconds(t_root), "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"{roots_done} destination roots (Dijkstra + loading) of the peak interval and one "
                       f"8-point sweep over {L} links, {spent:.1f} s of CPU; scaled by "
                       "the day's AON / root / sweep counts (extrapolated)"),
            "sec_per_root": t_root, "sec_per_sweep": t_pass, "all_cores": par}


def day_oracle_seconds(day_work, n_roots, t_root, t_sweep):
    """Seconds the oracle needs for a day whose interval i runs
    day_work["aon"][i] shortest-path batches over n_roots[i] destination roots
    (one Dijkstra + the walks of its items per root) and
    day_work["sweeps"][i] line-search sweeps; the residual pass (Alg. 4)
    re-walks the iterations + 1 accepted AONs of every interval."""
    est = 0.0
    for i, n in enumerate(n_roots):
        aons = day_work["aon"][i] + (day_work["fw"][i] + 1 if day_work["aon"][i] else 0)
        est += aons * n * t_root + day_work["sweeps"][i] * t_sweep
    return est


# Work counts of the default metro day (500x500 grid, 2000 zones, 19M trips,
# sweep8 steps, the paper's stop rule), per interval: shortest-path batches,
# accepted FW steps and line-search sweeps.  The oracle and the CUDA path
# compute the same iterates bit for bit, so these counts are the oracle's too;
# they were recorded from the bench line's "per_interval" entry.  The
# reference arm scales its timed sample by them.
METRO_DAY_WORK = {
    "aon": [2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2, 3, 4, 8, 37, 56, 92, 182, 115, 116,
             120, 116, 94, 67, 44, 62, 77, 69, 55, 50, 54, 51, 48, 45, 2, 2, 43, 34, 33, 14, 24, 35, 21, 2, 2, 2, 2,
             4, 4, 7, 41, 52, 84, 191, 158, 112, 114, 68, 69, 82, 54, 60, 55, 71, 45, 62, 69, 61, 78, 37, 3, 44, 53,
             38, 49, 46, 75, 20, 26, 26, 32, 40, 10, 2],
    "fw": [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 2, 6, 35, 54, 90, 180, 113, 114,
             118, 114, 92, 65, 42, 60, 75, 67, 53, 48, 52, 49, 46, 43, 0, 0, 41, 32, 31, 12, 22, 33, 19, 0, 0, 0, 0,
             2, 2, 5, 39, 50, 82, 189, 156, 110, 112, 66, 67, 80, 52, 58, 53, 69, 43, 60, 67, 59, 76, 35, 1, 42, 51,
             36, 47, 44, 73, 18, 24, 24, 30, 38, 8, 0],
    "sweeps": [1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 5, 1, 1, 5, 1, 1, 5, 1, 6, 15, 35, 180, 275, 455, 905,
             570, 575, 595, 575, 465, 330, 215, 305, 380, 336, 266, 241, 261, 246, 231, 220, 1, 1, 206, 161, 160, 65,
             115, 170, 100, 1, 1, 5, 5, 11, 15, 30, 200, 255, 415, 950, 785, 555, 565, 335, 340, 405, 265, 295, 270,
             350, 216, 305, 340, 296, 385, 180, 6, 211, 256, 181, 236, 225, 370, 95, 125, 125, 155, 195, 45, 5],
}


def reference_arm(args, inst, cfg):
    """CPU oracle on every host core, timed on a bounded sample per step:
    Dijkstra + loading of a few destination roots from four intervals of the
    day (the busiest and intervals 0, 30, 60), one root per task, one process
    per core; a line-search sweep timed once on one core.  The day's seconds
    are those per-root and per-sweep times scaled by the day's work counts."""
    import oracle
    q = inst.net.fftime_q
    og = oracle.OracleGraph(inst.net)
    L = og.n_links
    rng = np.random.default_rng(0)
    f = rng.uniform(0, 50, L)
    gfx = (rng.uniform(0, 50, L) * (1 << 32)).astype(np.int64)
    t1 = time.perf_counter()
    _, passes, _ = oracle.line_search(og, f, gfx, 900.0, 1,
                                      oracle.make_params(oracle.STEP_SWEEP8, oracle.STOP_NONE, 20))
    t_sweep = (time.perf_counter() - t1) / max(passes, 1)
    pool = OraclePool(inst.net, q)
    n_roots = [len(np.unique(d.root_idx)) for d in inst.demand]
    picks = [int(np.argmax([d.n_items for d in inst.demand])), 0, 30, 60]
    tasks = []
    for i in picks:
        dem = inst.demand[i]
        tasks += OraclePool.tasks(dem, np.unique(dem.root_idx)[:4 * pool.n])  # four roots per core
    work = METRO_DAY_WORK if args.workload == "day_metro" else None
    if work is not None and len(work["aon"]) == len(n_roots):
        scaling = "the day's recorded AON / FW-step / sweep counts per interval"
    else:
        work = {"aon": [2] * len(n_roots), "fw": [1] * len(n_roots), "sweeps": [0] * len(n_roots)}
        scaling = "2 AONs + 2 residual re-walks per interval, no sweeps (a lower bound; no recorded counts)"

    def one_step():
        t0 = time.perf_counter()
        t_root = pool.seconds_per_root(tasks)
        return day_oracle_seconds(work, n_roots, t_root, t_sweep), time.perf_counter() - t0

    for _ in range(args.warmup):
        one_step()
    vals, spent = [], []
    for _ in range(args.steps):
        v, s_ = one_step()
        vals.append(v)
        spent.append(s_)
    pool.close()
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": value * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int32+f64",
            "data": "synthetic", "config": cfg,
            "timed_s_per_step": float(np.mean(spent)),
            "cpu_baseline": {"value": value, "unit": "s", "cores": pool.n, "kind": "oracle",
                             "sample": (f"{len(tasks)} destination roots (Dijkstra + loading) from 4 intervals per "
                                        f"step, one process per core on {pool.n} cores ({np.mean(spent):.2f} s "
                                        f"timed per step), and one 8-point sweep over {L} links on one core "
                                        f"({t_sweep:.3f} s); extrapolated to the day by {scaling}")},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sssp_only(args):
    """Batched shortest paths alone on the metro grid (for profiling the
    SSSP kernel): --roots destination zones, congested link times."""
    import torch
    from paper_2104_12911_gb300 import qdta as Q, synth
    net = synth.grid_network(500, 2, freeways=True)
    zones = synth.pick_zones(net, 2000, 2)
    rng = np.random.default_rng(0)
    q = (net.fftime_q * rng.uniform(1.0, 3.0, net.n_links)).astype(np.int32)
    g = Q.Graph(net)
    qd = torch.from_numpy(q).cuda()
    roots = torch.from_numpy(zones[:args.roots].astype(np.int32)).cuda()
    tune = None
    if not args.no_tune:
        tune = Q.qdta_autotune(g, qd, roots, reps=max(args.steps, 1))
        tune = {f'{c["kernel"]}x{c["ctas_per_sm"]}': round(c["ms"], 3) for c in tune["candidates"]}
    for _ in range(args.warmup):
        Q.qdta_sssp_batch(g, qd, roots)
    Q.qdta_profile_enable(g, True)
    for _ in range(args.steps):
        Q.qdta_sssp_batch(g, qd, roots)
    p = Q.qdta_profile_read(g)
    ms = p["sssp_ms"] / max(p["sssp_launches"], 1)
    V, L, R = net.n_nodes, net.n_links, args.roots
    b_alg = R * 12.0 * V + 4.0 * (V + 1) + 8.0 * L
    print(json.dumps({"metric": "SSSP batch (metro grid)", "kernel": Q.qdta_sssp_kernel_name(g),
                      "roots": R, "ms_per_launch": ms,
                      "gteps": R * L / (ms * 1e-3) / 1e9, "alg_gbs": b_alg / (ms * 1e-3) / 1e9,
                      "rounds_per_root": p["sssp_rounds"] / max(p["sssp_roots"], 1),
                      "relax_per_link": p["sssp_relaxations"] / max(p["sssp_roots"], 1) / L,
                      "cell_activations_per_root": p["sssp_cell_activations"] / max(p["sssp_roots"], 1),
                      "redo_batches_64bit": p["sssp_redo_batches"], "batches": p["sssp_launches"],
                      "autotune_ms_per_batch": tune}),
          flush=True)


def batch32(args):
    """Many independent networks, one interval each: 32 grids with n spaced
    geometrically from 64 to 700, zones 100 -> 3,000 and trips 10k -> 400k,
    each with its autotuned shortest-path launch shape, solved as parallel
    branches of one CUDA graph launch vs one network at a time (plain
    launches); --stop rel_gap for the relative-gap target."""
    import torch
    from paper_2104_12911_gb300 import qdta as Q, synth
    k = np.arange(32)
    ns = np.rint(64 * (700 / 64) ** (k / 31)).astype(int)
    zs = np.rint(100 * (3000 / 100) ** (k / 31)).astype(int)
    ts = np.rint(10_000 * (400_000 / 10_000) ** (k / 31)).astype(int)
    items, links = [], 0
    for i in range(32):
        net = synth.grid_network(int(ns[i]), 100 + i, freeways=True)
        zones = synth.pick_zones(net, int(zs[i]), 100 + i)
        dem = synth.demand_from_matrix(zones, synth.sample_trips(
            synth.gravity_weights(net, zones, 100 + i, 10000.0), int(ts[i]), 200 + i))
        g = Q.Graph(net)
        if not args.no_tune:  # each network's shortest-path launch shape, by measurement on its zones
            Q.qdta_autotune(g, torch.from_numpy(net.fftime_q.astype(np.int32)).cuda(),
                            torch.from_numpy(zones.astype(np.int32)).cuda(), reps=1)
        items.append((g, Q.DeviceOD.of(dem), 900.0, torch.empty(net.n_links, dtype=torch.float64, device="cuda")))
        links += net.n_links
    res = {}
    for sched in ("graph", "plain"):
        p = Q.make_params(args.step, args.stop, args.max_iter, 1e-4, schedule=sched)
        for _ in range(args.warmup):
            Q.qdta_assign_batch(items, p)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            stats, rc = Q.qdta_assign_batch(items, p)
        e1.record()
        torch.cuda.synchronize()
        res[sched] = (e0.elapsed_time(e1) / args.steps, stats)
    st = res["graph"][1]
    print(json.dumps({"metric": "32 independent networks, one interval each, seconds", "workload": "batch32",
                      "links_total": links, "one_graph_launch_s": res["graph"][0] / 1e3,
                      "one_at_a_time_s": res["plain"][0] / 1e3,
                      "speedup": res["plain"][0] / res["graph"][0],
                      "fw_iterations": [s["iterations"] for s in st],
                      "converged": int(sum(s["converged"] for s in st)),
                      "stop": args.stop, "max_iter": args.max_iter}), flush=True)


def adjoint_metro(args):
    """Forward solve with a tape, then the adjoint, on the metro grid's peak
    interval (its original demand, 2000 destination zones): the loss is a
    link-count misfit L = sum over a 5 % link sample S of (f_a - y_a)^2 with
    counts y = f * lognormal(0, 0.3) (seed 3) taken from the first solve."""
    import torch
    from paper_2104_12911_gb300 import qdta as Q, synth
    inst = synth.config_day(seed=2)
    peak = int(np.argmax([d.amount_fx.sum() for d in inst.demand]))
    dem = inst.demand[peak]
    net = inst.net
    g = Q.Graph(net)
    dev = torch.device("cuda", 0)
    if not args.no_tune:
        Q.qdta_autotune(g, torch.from_numpy(net.fftime_q.astype(np.int32)).to(dev),
                        torch.from_numpy(inst.zones.astype(np.int32)).to(dev), reps=2)
    od = Q.DeviceOD.of(dem)
    p = Q.make_params(args.step, args.stop, args.max_iter, 1e-4, record_tape=True)
    rng = np.random.default_rng(3)
    S = torch.from_numpy(rng.choice(net.n_links, net.n_links // 20, replace=False)).to(dev)
    noise = torch.from_numpy(rng.lognormal(0.0, 0.3, S.shape[0])).to(dev)
    y = None
    fwd, bwd = [], []
    for it in range(args.warmup + args.steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record()
        f, st, rc, tape = Q.qdta_assign_interval(g, od, 900.0, p)
        e1.record()
        if y is None:
            y = f[S] * noise
        dL = torch.zeros_like(f)
        dL[S] = 2.0 * (f[S] - y)
        dd, dc = Q.qdta_backward(tape, dL)
        e2.record()
        torch.cuda.synchronize()
        tape.close()
        if it >= args.warmup:
            fwd.append(e0.elapsed_time(e1))
            bwd.append(e1.elapsed_time(e2))
    print(json.dumps({"metric": "interval forward (taped) + adjoint, metro peak interval, seconds",
                      "workload": f"500x500 grid, 2000 zones, interval {peak} ({dem.src.shape[0]} OD items, "
                                  f"{dem.amount_fx.sum() / 2**32:.0f} trips)",
                      "forward_s": float(np.mean(fwd)) / 1e3, "backward_s": float(np.mean(bwd)) / 1e3,
                      "fw_iterations": st["iterations"], "aon_calls": st["aon_calls"],
                      "sample_links": int(S.shape[0]), "loss": float(((f[S] - y) ** 2).sum()),
                      "dL_ddemand_absmax": float(dd.abs().max()), "dL_dcap_absmax": float(dc.abs().max()),
                      "sssp_kernel": Q.qdta_sssp_kernel_name(g), "stop": args.stop}), flush=True)


def interval_metro(args):
    """One static interval on the metro grid: 250k gravity trips over 2000
    zones (lognormal productions, exp(-d/10 km)), Frank-Wolfe with the chosen
    step rule to the chosen stop rule (max_iter caps it), on the graph
    schedule; seconds per interval, FW steps, SSSP GTEPS from a plain solve."""
    import torch
    from paper_2104_12911_gb300 import qdta as Q, synth
    inst = synth.config_metro(seed=1)
    net, dem = inst.net, inst.demand[0]
    g = Q.Graph(net)
    dev = torch.device("cuda", 0)
    if not args.no_tune:
        Q.qdta_autotune(g, torch.from_numpy(net.fftime_q.astype(np.int32)).to(dev),
                        torch.from_numpy(inst.zones.astype(np.int32)).to(dev), reps=2)
    od = Q.DeviceOD.of(dem)
    # one plain solve with per-kernel events (GTEPS), then timed graph solves
    Q.qdta_profile_enable(g, True)
    _, st_p, _, _ = Q.qdta_assign_interval(g, od, 900.0, Q.make_params(args.step, args.stop, args.max_iter, 1e-4))
    prof = Q.qdta_profile_read(g)
    Q.qdta_profile_enable(g, False)
    p = Q.make_params(args.step, args.stop, args.max_iter, 1e-4, schedule="graph")
    for _ in range(args.warmup):
        Q.qdta_assign_interval(g, od, 900.0, p)
    times = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        _, st, rc, _ = Q.qdta_assign_interval(g, od, 900.0, p)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    V, L = net.n_nodes, net.n_links
    avg = prof["sssp_ms"] / max(prof["sssp_launches"], 1)
    R_avg = prof["sssp_roots"] / max(prof["sssp_launches"], 1)
    print(json.dumps({"metric": "static interval on the metro grid, seconds", "workload":
                      f"500x500 grid, 2000 zones, 250k trips ({dem.src.shape[0]} OD items), one 15-min interval",
                      "seconds": float(np.mean(times)) / 1e3, "fw_iterations": st["iterations"],
                      "aon_calls": st["aon_calls"], "ls_sweeps": st["ls_passes"], "converged": st["converged"],
                      "stop_measure": st["rel_gap"], "dual_gap": st["dual_gap"], "stop": args.stop,
                      "step": args.step, "max_iter": args.max_iter, "plain_equals_graph":
                      st_p["iterations"] == st["iterations"],
                      "sssp_ms_per_batch": avg, "roots_per_batch": R_avg, "sssp_gteps": R_avg * L / (avg * 1e-3) / 1e9,
                      "sssp_alg_gbs": (R_avg * 12.0 * V + 4.0 * (V + 1) + 8.0 * L) / (avg * 1e-3) / 1e9,
                      "sssp_kernel": Q.qdta_sssp_kernel_name(g)}), flush=True)


def sta_vs_qdta(args):
    """The paper's comparison of a static and a quasi-dynamic morning peak
    (Section 7.1) on the metro day: 07:00-10:00 as one 3-hour static
    assignment (all of its original trips, no truncation inside the period)
    vs twelve 15-minute QDTA intervals with residual demand; scenario metrics
    by link class (over the period for both; the congested subset for the
    07:45-08:00 interval of QDTA and for the static period)."""
    import torch
    from paper_2104_12911_gb300 import qdta as Q, synth
    inst = synth.config_day(seed=2)
    net = inst.net
    dev = torch.device("cuda", 0)
    g = Q.Graph(net)
    if not args.no_tune:
        Q.qdta_autotune(g, torch.from_numpy(net.fftime_q.astype(np.int32)).to(dev),
                        torch.from_numpy(inst.zones.astype(np.int32)).to(dev), reps=2)
    first, n_int = 28, 12  # 07:00-10:00
    days = inst.demand[first:first + n_int]
    zones = torch.from_numpy(inst.zones.astype(np.int32)).to(dev)
    length = torch.from_numpy(net.length_m.astype(np.float64)).to(dev)
    cls = torch.from_numpy(net.link_class.astype(np.int32)).to(dev)
    n_cls = int(net.link_class.max()) + 1
    p = Q.make_params(args.step, args.stop, args.max_iter, 1e-4, schedule="graph", objective=args.objective,
                      truncation=args.truncation)
    # QDTA: twelve intervals with residual demand
    dd = [Q.DeviceOD(zones, *(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                              for a in (d.root_idx, d.src, d.amount_fx))) for d in days]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h, st_q, _, _ = Q.qdta_run_day(g, dd, 900.0, p)
    torch.cuda.synchronize()
    t_qdta = time.perf_counter() - t0
    m_q = Q.qdta_interval_metrics(g, h, 900.0, length, cls, n_cls).cpu().numpy()
    # STA: the period's original trips summed per (root, origin), one 3-hour interval
    ri = np.concatenate([d.root_idx for d in days])
    si = np.concatenate([d.src for d in days])
    am = np.concatenate([d.amount_fx for d in days])
    key = ri.astype(np.int64) * net.n_nodes + si
    uk, inv = np.unique(key, return_inverse=True)
    amount = np.zeros(uk.shape[0], np.int64)
    np.add.at(amount, inv, am)
    sta_od = Q.DeviceOD(zones, torch.from_numpy((uk // net.n_nodes).astype(np.int32)).to(dev),
                        torch.from_numpy((uk % net.n_nodes).astype(np.int32)).to(dev),
                        torch.from_numpy(amount).to(dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f_s, st_s, _, _ = Q.qdta_assign_interval(g, sta_od, 3 * 3600.0, p)
    torch.cuda.synchronize()
    t_sta = time.perf_counter() - t0
    m_s = Q.qdta_interval_metrics(g, f_s, 3 * 3600.0, length, cls, n_cls).cpu().numpy()[0]
    peak = 31 - first  # 07:45-08:00

    def table(rows):
        return {f"class_{k}": {name: round(float(v), 4) for name, v in zip(Q.METRIC_NAMES, rows[k])}
                for k in range(n_cls)}

    qdta_period = m_q.sum(axis=0)  # additive metrics summed over the intervals
    for c in range(n_cls):  # the averages: count-weighted over the intervals
        n = m_q[:, c, 0].sum()
        qdta_period[c, 2] = float((m_q[:, c, 2] * m_q[:, c, 0]).sum() / n) if n else 0.0
        cn = m_q[:, c, 4].sum()
        qdta_period[c, 7] = float((m_q[:, c, 7] * m_q[:, c, 4]).sum() / cn) if cn else 0.0
    print(json.dumps({"metric": "static vs quasi-dynamic morning peak (07:00-10:00), scenario metrics",
                      "workload": "500x500 grid, 2000 zones, metro day intervals 28..39",
                      "sta": {"seconds": t_sta, "fw_iterations": st_s["iterations"], "metrics": table(m_s)},
                      "qdta": {"seconds": t_qdta, "fw_iterations": [s["iterations"] for s in st_q],
                               "metrics_period": table(qdta_period),
                               "metrics_0745_0800": table(m_q[peak]),
                               "items_per_interval": [s["n_items"] for s in st_q]},
                      "step": args.step, "stop": args.stop, "objective": args.objective}), flush=True)


def gap_peak(args):
    """The relative duality gap target on the metro day's busiest hour: the
    day runs under the paper's stop rule up to the hour, and the hour's four
    intervals are then solved from that residual demand with the relative-gap
    stop (tolerance 1e-4, at most --max-iter FW steps each), on the graph
    schedule.  Reports per interval the FW steps, whether 1e-4 was reached,
    the gap at the end and the seconds."""
    import torch
    from paper_2104_12911_gb300 import qdta as Q, synth
    inst = synth.config_day(seed=2)
    net = inst.net
    dev = torch.device("cuda", 0)
    g = Q.Graph(net)
    if not args.no_tune:
        Q.qdta_autotune(g, torch.from_numpy(net.fftime_q.astype(np.int32)).to(dev),
                        torch.from_numpy(inst.zones.astype(np.int32)).to(dev), reps=2)
    totals = [d.amount_fx.sum() for d in inst.demand]
    first = max(0, int(np.argmax(totals)) - 1)
    zones = torch.from_numpy(inst.zones.astype(np.int32)).to(dev)
    dd = [Q.DeviceOD(zones, *(torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                              for a in (d.root_idx, d.src, d.amount_fx))) for d in inst.demand]
    p0 = Q.make_params(args.step, "paper_obj", 200, 1e-4, schedule="graph")
    _, _, _, res = Q.qdta_run_day(g, dd[:first], 900.0, p0, resid_capacity=64 << 20)
    rin = Q.DeviceOD(zones, res[0].clone(), res[1].clone(), res[2].clone())
    p1 = Q.make_params(args.step, "rel_gap", args.max_iter, 1e-4, schedule="graph")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st, rc, _ = Q.qdta_run_day(g, dd[first:first + 4], 900.0, p1, resid_in=rin)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    rows = [{"interval": first + i, "trips_original": round(float(totals[first + i]) / 2**32),
             "items": s["n_items"], "fw_steps": s["iterations"], "converged_1e-4": bool(s["converged"]),
             "dual_gap_end": s["dual_gap"]} for i, s in enumerate(st)]
    print(json.dumps({"metric": "FW steps to relative duality gap 1e-4, metro day's busiest hour",
                      "workload": f"500x500 grid, 2000 zones, 19M trips/day: intervals {first}..{first + 3} "
                                  f"resumed from the residual of intervals 0..{first - 1} (paper's rule)",
                      "stop": "relative duality gap <= 1e-4 (a negative gap does not stop)",
                      "max_iter": args.max_iter, "step": args.step, "seconds_for_the_hour": secs,
                      "intervals": rows, "sssp_kernel": Q.qdta_sssp_kernel_name(g)}), flush=True)


def floor_small(args):
    """How low the relative duality gap goes on the 32 x 32 network (64
    zones, 20k trips, one 15-minute interval) with sweep8 steps, at the 0.01 s
    time quantum and at a 100x finer one: the gap after K FW steps."""
    import torch
    from paper_2104_12911_gb300 import qdta as Q, synth
    inst = synth.config_small(0)
    dem = inst.demand[0]
    out = {}
    for quantum in (0.01, 0.0001):
        net = dataclasses.replace(inst.net, quantum_s=quantum,
                                  fftime_q=np.maximum(1, np.rint(inst.net.fftime_q * (0.01 / quantum))).astype(np.int32))
        g = Q.Graph(net)
        od = Q.DeviceOD.of(dem)
        row = {}
        for K in (10, 20, 40, 80, 160, 320, 640, 1280):
            _, st, _, _ = Q.qdta_assign_interval(g, od, 900.0, Q.make_params(args.step, "none", K, schedule="graph"))
            row[K] = st["dual_gap"]
        _, st, rc, _ = Q.qdta_assign_interval(g, od, 900.0, Q.make_params(args.step, "rel_gap", 5000, 1e-4,
                                                                          schedule="graph"))
        out[f"quantum_{quantum}s"] = {"dual_gap_after_K_steps": row, "steps_to_1e-4": st["iterations"],
                                      "converged": bool(st["converged"])}
    print(json.dumps({"metric": "relative duality gap floor, 32x32 network (config 1 inputs), one interval",
                      "step": args.step, "results": out}), flush=True)


def main():
    args = parse()
    if args.workload == "gap_peak":
        gap_peak(args)
        return
    if args.workload == "floor_small":
        floor_small(args)
        return
    if args.workload == "sssp_metro":
        sssp_only(args)
        return
    if args.workload == "batch32":
        batch32(args)
        return
    if args.workload == "adjoint_metro":
        adjoint_metro(args)
        return
    if args.workload == "interval_metro":
        interval_metro(args)
        return
    if args.workload == "sta_vs_qdta":
        sta_vs_qdta(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        inst, cfg = make_workload(args.workload)
        cfg["parallelism"] = f"cpu oracle, one process per core ({os.cpu_count()} cores)"
        reference_arm(args, inst, cfg)
        return

    import torch
    import torch.distributed as dist
    from paper_2104_12911_gb300 import qdta as Q

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    t_gen = time.perf_counter()
    inst, cfg = make_workload(args.workload)
    if args.intervals:
        a, b = (int(x) for x in args.intervals.split(":"))
        inst.demand = inst.demand[a:b]
        cfg["workload"] += f" -- intervals {a}..{b - 1} only (profiling slice)"
        cfg["intervals"] = b - a
    t_gen = time.perf_counter() - t_gen
    cfg["parallelism"] = f"replicas x{world} (one independent day per GPU)"
    g = Q.Graph(inst.net, local)
    if not args.no_tune:
        # launch shape of the shortest-path batch, chosen by measurement on the
        # day's destination zones at free-flow costs (setup, untimed)
        tune = Q.qdta_autotune(g, torch.from_numpy(inst.net.fftime_q.astype(np.int32)).to(dev),
                               torch.from_numpy(inst.zones.astype(np.int32)).to(dev), reps=2)
        cfg["sssp_launch"] = {"kernel": tune["best"]["kernel"], "ctas_per_sm": tune["best"]["ctas_per_sm"],
                              "autotune_ms_per_batch": {f'{c["kernel"]}x{c["ctas_per_sm"]}': round(c["ms"], 3)
                                                        for c in tune["candidates"]}}
    torch.cuda.empty_cache()

    def upload(dem, pin=False):
        def t(a, dt):
            x = torch.from_numpy(np.ascontiguousarray(a, dtype=dt))
            return x.pin_memory() if pin else x.to(dev)
        return t(dem.root_idx, np.int32), t(dem.src, np.int32), t(dem.amount_fx, np.int64)

    host = [upload(d, pin=True) for d in inst.demand]
    zones_host = torch.from_numpy(inst.zones.astype(np.int32)).pin_memory()
    params_graph = Q.make_params(args.step, args.stop, args.max_iter, 1e-4, schedule="graph", objective=args.objective,
                                 truncation=args.truncation)
    params_plain = Q.make_params(args.step, args.stop, args.max_iter, 1e-4, schedule="plain", objective=args.objective,
                                 truncation=args.truncation)
    cfg["step_rule"] = args.step
    cfg["objective"] = {"ue": "user equilibrium (Beckmann)", "so": "system optimum (total cost)"}[args.objective]
    cfg["truncation"] = {"node": "Eq. 2: first node reached at or after dt",
                         "carry": "Section 3.4: partial links carried across intervals"}[args.truncation]
    flow_out = torch.empty((len(inst.demand), g.n_links), dtype=torch.float64, device=dev)
    flows_host = torch.empty((len(inst.demand), g.n_links), dtype=torch.float64).pin_memory()
    h2d = sum(a.numel() * a.element_size() for h in host for a in h) + zones_host.numel() * 4
    d2h = flows_host.numel() * 8
    stream = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def one_day(params):
        """One step through the public API: inputs from pinned host memory to
        the device, the day, the h(i) flows back.  Returns (e2e ms, day ms)."""
        e0, e1, e2, e3 = ev(), ev(), ev(), ev()
        e0.record(stream)
        zdev = zones_host.to(dev, non_blocking=True)
        dd = [Q.DeviceOD(zdev, *(a.to(dev, non_blocking=True) for a in h)) for h in host]
        e1.record(stream)
        _, st, _, _ = Q.qdta_run_day(g, dd, 900.0, params, flow_out=flow_out)
        e2.record(stream)
        flows_host.copy_(flow_out, non_blocking=True)
        e3.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e3), e1.elapsed_time(e2), st

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def agree(flag):
        """True on every rank only if `flag` holds on every rank (replicas stay
        in step: they run the same number of days)."""
        if world <= 1:
            return bool(flag)
        t = torch.tensor([1.0 if flag else 0.0], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        return bool(t.item() > 0.5)

    # Warm-up: the first day runs the plain schedule (host launch loop) with
    # per-kernel CUDA events: the batched-vs-plain comparison and the SSSP
    # roofline come from it; the other warm-up days run the graph schedule.
    # At most --max-warmup-days days, and no more warm-up once another day
    # plus the first timed day and the CPU leg would not fit the budget.
    reserve_s = 0.0 if (args.no_cpu or rank != 0) else 90.0
    budget = args.budget_s
    progress(f"setup done ({args.workload}, generation {t_gen:.1f} s)")
    plain_ms, prof, plain_launches, stats_plain = None, None, None, None
    day_s = []  # wall seconds of every day run so far
    warm_done = 0
    while warm_done < min(args.warmup, max(args.max_warmup_days, 1)):
        if warm_done >= 1:
            est = max(day_s)
            if not agree(time.monotonic() - T_START + 2 * est + reserve_s < budget):
                break
        t0 = time.monotonic()
        if warm_done == 0 and not args.no_plain:
            Q.qdta_profile_enable(g, True)
            barrier()
            p0 = Q.qdta_profile_read(g)["kernel_launches"]
            _, plain_ms, stats_plain = one_day(params_plain)
            prof = Q.qdta_profile_read(g)
            plain_launches = prof["kernel_launches"] - p0
            Q.qdta_profile_enable(g, False)
            kind = "plain"
        else:
            one_day(params_graph)
            kind = "graph"
        day_s.append(time.monotonic() - t0)
        warm_done += 1
        progress(f"warm-up day {warm_done} ({kind} schedule): {day_s[-1]:.1f} s")
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    e2e_list, day_list, stats = [], [], None
    while len(day_list) < max(args.steps, 1):
        if day_list:
            est = max(day_s[-3:])
            if not agree(time.monotonic() - T_START + est + reserve_s < budget):
                break
        t0 = time.monotonic()
        e2e_ms_i, day_ms_i, stats = one_day(params_graph)
        day_s.append(time.monotonic() - t0)
        e2e_list.append(e2e_ms_i)
        day_list.append(day_ms_i)
        progress(f"timed day {len(day_list)} (graph schedule): {day_ms_i / 1e3:.2f} s on the device, "
                 f"{e2e_ms_i / 1e3:.2f} s end to end")
    barrier()
    clk = clocks.stop()
    ms = float(np.mean(day_list))
    e2e_ms = float(np.mean(e2e_list))
    ms, e2e_ms = max_over_ranks([ms, e2e_ms], world, dev)
    if stats_plain is not None:
        cfg["plain_equals_batched"] = all(a["iterations"] == b["iterations"] and a["n_items"] == b["n_items"]
                                          for a, b in zip(stats, stats_plain))

    V, L = g.n_nodes, g.n_links
    roofline, gteps = None, None
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    if prof and prof["sssp_launches"]:
        avg_ms = prof["sssp_ms"] / prof["sssp_launches"]
        R_avg = prof["sssp_roots"] / prof["sssp_launches"]
        b_alg = R_avg * 12.0 * V + 4.0 * (V + 1) + 8.0 * L
        achieved = b_alg / (avg_ms * 1e-3) / 1e9
        gteps = R_avg * L / (avg_ms * 1e-3) / 1e9
        kname = Q.qdta_sssp_kernel_name(g, Q.QDTA_TO_ROOT)
        per_root = SSSP_DRAM_BYTES_PER_ROOT.get(kname) if args.workload == "day_metro" else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": per_root * R_avg if per_root else None,
                    "traffic_unit": "bytes per launch",
                    "kernel": kname,
                    "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                    "sssp_avg_ms": avg_ms, "roots_per_launch": R_avg, "gteps": gteps,
                    "sssp_share_of_plain_day": prof["sssp_ms"] / plain_ms if plain_ms else None,
                    "load_share_of_plain_day": prof["load_ms"] / plain_ms if plain_ms else None,
                    "sweep_share_of_plain_day": prof["sweep_ms"] / plain_ms if plain_ms else None}

    tot = {k: sum(s[k] for s in stats) for k in ("iterations", "aon_calls", "ls_passes")}
    cfg["fw_iterations_per_day"] = tot["iterations"]
    cfg["aon_per_day"] = tot["aon_calls"]
    cfg["ls_sweeps_per_day"] = tot["ls_passes"]
    cfg["converged_intervals"] = int(sum(s["converged"] for s in stats))
    cfg["max_stop_measure"] = max((s["rel_gap"] for s in stats if s["aon_calls"]), default=0.0)
    gaps = [s["dual_gap"] for s in stats if s["aon_calls"]]
    cfg["duality_gap_max"] = max(gaps, default=0.0)
    cfg["duality_gap_median"] = float(np.median(gaps)) if gaps else 0.0
    cfg["intervals_with_duality_gap_le_1e-4"] = int(sum(1 for x in gaps if -1e-12 <= x <= 1e-4))
    cfg["intervals_with_demand"] = len(gaps)
    cfg["per_interval"] = {"aon": [s["aon_calls"] for s in stats], "fw": [s["iterations"] for s in stats],
                           "sweeps": [s["ls_passes"] for s in stats],
                           "dual_gap": [round(s["dual_gap"], 7) for s in stats],
                           "items": [s["n_items"] for s in stats]}
    cfg["generation_s"] = t_gen

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(inst, stats)

    if rank == 0:
        line = {"metric": METRIC, "value": job_seconds_per_day(ms, world), "unit": "s", "n_gpus": world,
                "steps": len(day_list), "warmup": warm_done, "ms_per_step": ms,
                "steps_requested": args.steps, "warmup_requested": args.warmup,
                "budget_s": args.budget_s,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "int32 costs/int64 flows + f64 line search", "data": "synthetic",
                "config": cfg, "clocks": clk,
                "e2e": {"value": job_seconds_per_day(e2e_ms, world), "unit": "s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(plain_launches * len(day_list)) if plain_launches else None,
                "gpu_launches_note": ("kernels per timed step, counted on the plain schedule of the same day "
                                      "(first warm-up step; the graph schedule replays the identical kernel "
                                      "sequence)"),
                "timing": ("value = CUDA events around qdta_run_day with the day's inputs resident; e2e = the same "
                           "step from pinned-host inputs to pinned-host h(i) flows"),
                "plain_s": plain_ms / 1e3 if plain_ms else None,
                "batched_speedup_vs_plain": (plain_ms / ms) if plain_ms else None,
                "sssp_gteps": gteps, "roofline": roofline, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
