"""The N > 1 host logic of the benchmark on CPU: two gloo ranks run replica
days; the job's time is the slowest rank's, and the reported value is
seconds per simulated day of the whole job."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 100 * (r + 1) ms for the day and 150 * (r + 1) ms end to end
    ms, e2e = bench.max_over_ranks([100.0 * (rank + 1), 150.0 * (rank + 1)], world, "cpu")
    q.put((rank, ms, e2e, bench.job_seconds_per_day(ms, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_count_all_days():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, e2e, value in got:
        assert ms == 200.0 and e2e == 300.0        # slowest rank on every rank
        assert value == pytest.approx(0.1)          # 2 days in 0.2 s -> 0.1 s per day


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    assert bench.job_seconds_per_day(2500.0, 1) == 2.5
