"""The N > 1 benchmark path on CPU: two gloo ranks run the replica/timing
logic of bench.py (independent seeds, slowest-rank time, summed path-steps)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2301_05780_gb300 import workloads as W
    r, lr, ws = bench.dist_env()
    seed = bench.replica_seed(W.config2().seed, r)
    t, s = bench.reduce_timing(100.0 + 50.0 * rank, 1e9 * (rank + 1))
    dist.barrier()
    out[rank] = (seed, t, s, ws)
    dist.destroy_process_group()


def test_two_rank_replica_timing():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (s0, t0, n0, w0), (s1, t1, n1, w1) = res[0], res[1]
    assert w0 == w1 == 2
    assert s0 != s1                      # independent replicas
    assert t0 == t1 == 150.0             # slowest rank
    assert n0 == n1 == 3e9               # all ranks' path-steps
