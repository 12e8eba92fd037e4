"""The bench's multi-rank host logic (barrier, max and sum over ranks) on two gloo ranks on CPU.
Rendering itself is replicated per rank (weak scaling), so these reductions are the only
cross-rank steps."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    d = bench.Dist()
    d.init("gloo")
    d.barrier()
    mx = d.max(float(rank + 1) * 10.0)
    sm = d.sum(float(rank + 1))
    out[rank] = (d.world, d.rank, mx, sm)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_dist_max_and_sum_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    assert out[0] == (2, 0, 20.0, 3.0) and out[1] == (2, 1, 20.0, 3.0)


def test_dist_single_process_is_identity():
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    d = bench.Dist()
    assert d.world == 1 and d.max(3.5) == 3.5 and d.sum(2.0) == 2.0
