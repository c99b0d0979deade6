"""The N > 1 benchmark path on CPU: two gloo ranks, each with its own box
(independent problems, no collective on the data path); the job value uses
the slowest rank's time and the units of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [40.0, 50.0][rank]                 # rank 1 is the slower one
    seed = bench.rank_seed(1, rank)
    v, t = bench.job_value(local_ms, 1000, 10, world, bench.torch_reduce_max("cpu"))
    out[rank] = (seed, v, t)
    tdist.barrier()
    tdist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_all_units():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    (s0, v0, t0), (s1, v1, t1) = out[0], out[1]
    assert (s0, s1) == (1, 2)                      # independent boxes
    assert t0 == t1 == 50.0                        # max over ranks
    assert v0 == v1 == pytest.approx(1000 * 10 * 2 / 0.050)


def test_single_rank_needs_no_process_group():
    import bench
    v, t = bench.job_value(20.0, 100, 5, 1)
    assert t == 20.0 and v == pytest.approx(100 * 5 / 0.020)
