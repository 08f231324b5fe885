"""Host logic of the multi-GPU benchmark path on CPU ranks (gloo, world size 2).

Every rank runs its own copy of the workload (independent vessels: weak
scaling, no data-path collective); ranks only meet at barriers around the timed
region and in the max-over-ranks reduction of the elapsed time.  This test runs
that timing logic on two gloo ranks and checks the aggregate-rate arithmetic.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    bench.barrier(ws)
    elapsed = [0.25, 0.40][rank]  # seconds this rank took for its replica
    worst = bench.max_over_ranks(ws, elapsed)
    sites, steps = 1000, 10
    out[rank] = (worst, ws * sites * steps / worst / 1e6)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    worst, mlups = out[0]
    assert worst == pytest.approx(0.40)
    assert mlups == pytest.approx(2 * 1000 * 10 / 0.40 / 1e6)
