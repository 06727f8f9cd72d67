"""The N > 1 path of the benchmark is replicas only: each rank runs the whole workload
on its own GPU and only the slowest time and the summed flops are reduced. This checks
that reduction with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, f = bench.aggregate_over_ranks(dist, 100.0 + 50.0 * rank, 1e12 * (rank + 1))
    out[rank] = (t, f)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (150.0, 3e12)     # max time, summed flops
    # whole-job throughput of the two replicas: 3e12 flops in 0.15 s
    t, f = out[0]
    assert abs(f / (t / 1e3) / 1e9 - 20000.0) < 1e-6


def test_single_rank_aggregation_is_identity():
    import bench
    assert bench.aggregate_over_ranks(None, 12.5, 7.0) == (12.5, 7.0)
