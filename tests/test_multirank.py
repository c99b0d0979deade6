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


def _rank_step(rank, world, port, out):
    """One SDC step per rank on that rank's own seeded box (the oracle stands in
    for the GPU on CPU), no collective but the timing reduction."""
    import time

    import numpy as np

    import bench
    import oracle as O
    from paper_1910_12578_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.rank_seed(1, rank)
    P, U = W.config_box(n=8, nspec=7, seed=seed, T0=0.5)
    o = O.Oracle(P)
    dt = o.cfl_dt(U)
    tdist.barrier()
    t0 = time.perf_counter()
    V, st = o.step(U, dt)
    ms = (time.perf_counter() - t0) * 1e3
    tdist.barrier()
    v, t = bench.job_value(ms, bench.units_per_step(P), 1, world, bench.torch_reduce_max("cpu"))
    out[rank] = (seed, float(np.abs(V).sum()), st.newton_solves, v, t, ms, bench.units_per_step(P))
    tdist.destroy_process_group()


def test_two_ranks_each_step_their_own_box():
    """Each rank's step equals a single-process step of the same seed (nothing
    couples the ranks' data), the boxes differ, and the job value counts both
    ranks' units over the slower rank's time."""
    import numpy as np

    import oracle as O
    from paper_1910_12578_gb300 import workloads as W
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_step, args=(world, port, out), nprocs=world, join=True)
    sums = []
    for rank in range(world):
        seed, s, solves, v, t, ms, units = out[rank]
        P, U = W.config_box(n=8, nspec=7, seed=seed, T0=0.5)
        o = O.Oracle(P)
        V, _ = o.step(U, o.cfl_dt(U))
        assert s == float(np.abs(V).sum())
        assert solves == units
        assert t == max(out[r][5] for r in range(world))
        assert v == pytest.approx(units * world / (t * 1e-3))
        sums.append(s)
    assert sums[0] != sums[1]
