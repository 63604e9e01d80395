"""Multi-GPU path of bench.py: independent replicas, one image per rank.

The path shards over images with no data-path collective; only the timing is
reduced (maximum over ranks).  Two gloo ranks on the CPU check that each rank
gets its own seeded image and that the job throughput is counted from the
slowest rank.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)                    # rank 1 is the slow one
    units = bench.head_units(bench.N, 250, 70)      # dual updates of one headline step (example counts)
    value, total = bench.replica_value(local_ms, world, 4, units, dist, torch.device("cpu"))
    img = bench.make_input(64, rank)
    out.put((rank, value, total, float(img[:8, :8].sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    want = bench.head_units(bench.N, 250, 70) * 2 * 4 / (200.0 / 1e3) / 1e9
    for rank, value, total, _ in res:
        assert total == 200.0
        assert value == pytest.approx(want, rel=1e-12)
    assert res[0][3] != res[1][3]                   # each rank denoises its own seeded image


def test_single_replica_needs_no_process_group():
    import bench
    units = bench.head_units(bench.N, 250, 70)
    value, total = bench.replica_value(50.0, 1, 2, units)
    assert total == 50.0
    assert value == pytest.approx(units * 2 / 0.05 / 1e9)
