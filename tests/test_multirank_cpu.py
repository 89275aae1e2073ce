"""The multi-rank path of bench.py on CPU: two gloo ranks (no GPU).

Under torchrun every rank solves its own instance (independent problems,
no collective on the data path); the timed region ends with a barrier, the
slowest rank's time is taken (all-reduce MAX) and the whole-job value is
world x steps / that time.  These ranks exercise exactly that host logic
with made-up per-rank times."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t_local = 0.5 + 0.25 * rank            # the slower rank decides
        dist.barrier()
        t = bench.rank_max_seconds(t_local, dist, "cpu")
        value = bench.whole_job_value(world, 40, t)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.instance_seed(7, rank))
        out[rank] = (t, value, tuple(seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_distinct_instances():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, value, seeds = res[rank]
        assert t == pytest.approx(0.75)
        assert value == pytest.approx(world * 40 / 0.75)
        assert len(set(seeds)) == world          # every rank its own instance


def test_single_process_path_needs_no_collective():
    import bench
    assert bench.rank_max_seconds(1.25, None, "cpu") == 1.25
    assert bench.whole_job_value(1, 100, 0.5) == 200.0
    assert bench.instance_seed(3, 0) == 3
