"""The N > 1 replicas path of bench.py on CPU: two gloo ranks, launched the way
torchrun would (RANK / WORLD_SIZE / LOCAL_RANK / MASTER_* in the environment),
agree on the whole-job rate set by the slowest rank."""
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


def _rank(rank, world, port, seconds, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()  # the barrier that opens the timed region
        value, total = bench.job_rate(seconds[rank], 3, dist, device="cpu")
        out.put((rank, value, total))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_job_rate_is_set_by_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    seconds = [1.5, 2.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, seconds, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(world))
    for rank, value, total in got:
        assert total == max(seconds)
        assert value == pytest.approx(world * 3 / max(seconds))


def test_job_rate_single_process():
    import bench
    assert bench.job_rate(2.0, 4) == (2.0, 2.0)
