"""The multi-GPU path of the benchmark runs independent replicas (the product
needs no exchange).  Its only cross-rank logic is the throughput aggregation:
whole-job units over the slowest rank's time.  Tested with two gloo ranks on
the CPU (127.0.0.1 rendezvous)."""
import os

import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, sec = bench.replica_throughput(units=1000.0, seconds=1.0 + rank, device="cpu")
    out[rank] = (value, sec)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")  # no fork of this (multi-threaded) process
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # both ranks see the slowest time (2 s) and the whole-job units (2 x 1000)
    assert out[0] == pytest.approx((1000.0, 2.0))
    assert out[1] == pytest.approx((1000.0, 2.0))


def test_replica_throughput_single_process():
    import bench
    assert bench.replica_throughput(500.0, 0.5) == (1000.0, 0.5)
