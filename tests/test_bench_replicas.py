"""The multi-GPU form of the benchmark runs independent replicas (one image per
rank, no data-path collective): rank timings are max-reduced and the
aggregate rate counts every rank's pixels.  This checks that host logic with
two gloo ranks on the CPU."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 10 ms per step and (r + 1) * 20 ms for the plain form
        step_ms, plain_ms = bench.max_over_ranks([(rank + 1) * 10.0, (rank + 1) * 20.0], world,
                                                 device="cpu")
        out[rank] = (step_ms, plain_ms, bench.aggregate_rate(2048 * 2048, world, step_ms * 1e-3))
    finally:
        tdist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        step_ms, plain_ms, rate = res[r]
        assert step_ms == 20.0 and plain_ms == 40.0          # the slower rank's times
        assert rate == pytest.approx(2 * 2048 * 2048 / 0.020 / 1e6)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.aggregate_rate(1e6, 1, 0.5) == pytest.approx(2.0)
