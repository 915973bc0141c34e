"""The multi-GPU path of bench.py on CPU: two gloo ranks, each with its own seeded batch
(weak scaling, no data-path collective); the whole-job value sums every rank's units
and divides by the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    wl = bench.make_workload("batch256", rank, steps=2)
    units = bench.units_per_step(wl)
    ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
    value, ms_max, units_all = bench.weak_scaling_value(units, 3, ms, dist, "cpu")
    out[rank] = (units, value, ms_max, units_all, [sh.N for sh in wl.sheets[:8]])
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (u0, v0, ms0, ua0, n0), (u1, v1, ms1, ua1, n1) = res[0], res[1]
    assert n0 != n1  # each rank carries its own seeded batch
    assert ms0 == ms1 == 150.0
    assert ua0 == ua1 == u0 + u1
    assert v0 == v1 == pytest.approx((u0 + u1) * 3 / 0.150)
