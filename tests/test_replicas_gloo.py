"""The N > 1 path of the benchmark runs independent replicas, one per rank,
and reports the whole-job throughput from the slowest rank's time.  Checked
with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = [120.0, 150.0][rank]
    v, ms = bench.replica_mlups(ms_local, n_sites=1_000_000, steps=10, world=world, device="cpu")
    q.put((rank, v, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, v, ms in res:
        assert ms == 150.0
        assert v == pytest.approx(2 * 1_000_000 * 10 / 0.150 / 1e6)
