"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, one problem per rank)
combine their step times with the max-over-ranks reduction, and the whole-job rate is
the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, _ = bench.dist_env()
        step = bench.max_over_ranks(100.0 + 50.0 * r, w, "cpu")   # rank 1 is slower
        out[r] = (w, step, bench.job_rate(100, w, step))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ws, step, rate = res[r]
        assert ws == 2 and step == 150.0
        assert rate == pytest.approx(2 * 100 / 0.150)


def test_single_rank_needs_no_group():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(100, 1, 2000.0) == pytest.approx(50.0)
