"""The N > 1 host path of bench.py (replicas, weak scaling) on world-size-2
gloo process groups: the barrier, the max over ranks of the timed region
and the whole-job throughput, with no GPU."""

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


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        assert bench._dist() == (rank, world, rank)
        bench._barrier(world)
        t = bench._max_over_ranks(times[rank], world)
        out.put((rank, t, bench._job_glups(128 ** 3, 10, world, t)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_cells():
    world, times = 2, [0.25, 0.4]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(out.get(timeout=10) for _ in range(world))
    for rank, t, glups in res:
        assert t == max(times)
        assert glups == pytest.approx(128 ** 3 * 10 * world / max(times) / 1e9, rel=1e-15)


def test_one_rank_is_the_identity():
    import bench
    assert bench._max_over_ranks(0.3, 1) == 0.3
    bench._barrier(1)
    assert bench._job_glups(512 ** 3, 100, 1, 0.5) == pytest.approx(512 ** 3 * 100 / 0.5 / 1e9)
