"""The N > 1 path of the benchmark ("replicas only": every rank runs its own
seeded problems, no data-path collective): the timing reduction and the
whole-job rate, on two gloo ranks on the CPU, and the reference arm's
non-zero ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r was slower on the step total, faster on the p99
        tot, p99, e2e = bench.reduce_over_ranks([10.0 + rank, 5.0 - rank, 7.0 + 2 * rank], world)
        out.put((rank, tot, p99, e2e, bench.whole_job_rate(16384, world, tot / 50)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tot, p99, e2e, rate in res:
        assert (tot, p99, e2e) == (11.0, 5.0, 9.0)            # the max of each, on every rank
        assert rate == pytest.approx(16384 * 2 / (11.0 / 50 / 1e3))


def test_reduce_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
    assert bench.whole_job_rate(100, 1, 10.0) == pytest.approx(1e4)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        seed, steps, warmup = 0, 1, 0
    assert bench.run_reference(A(), rank=1, world=2) is None
