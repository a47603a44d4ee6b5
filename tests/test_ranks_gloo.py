"""The N > 1 path of bench.py on CPU: two gloo ranks (the path has no data
exchange; ranks only agree on the step time and the eigenpair count)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    env = bench.dist_env()
    t = bench.reduce_over_ranks(10.0 + rank, "max")      # slowest rank's step time
    g = bench.reduce_over_ranks(3.0 * (rank + 1), "sum")  # eigenpairs of all ranks
    bench.barrier()
    # the reference arm runs on rank 0 only: other ranks return without work
    if rank != 0:
        import argparse
        bench.run_reference(argparse.Namespace(workload="qep_plain_n256", seed=0, warmup=1,
                                               steps=1))
    q.put((rank, env, t, g))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_time_and_count():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, t, g in out:
        assert env == (2, rank, rank)
        assert t == 11.0 and g == 9.0
