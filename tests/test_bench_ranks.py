"""The benchmark's multi-rank bookkeeping, on CPU with two gloo ranks: each replica's time
is reduced to the slowest one (the job ends with it), the job rate counts every rank's ions,
and in the reference arm the ranks other than 0 exit at once without work."""
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


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = [3.0, 5.0][rank]
    ms = bench.slowest_rank_ms(local_ms, ws, torch.device("cpu"))
    rate = bench.job_rate(32768, ws, ms)
    ref = None
    if rank == 1:
        class Args:
            workload = "nacl32k"
            steps = 1
            warmup = 0
        ref = bench.run_reference(Args())
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, rate, ref))


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(ws))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, ms, rate, ref in res:
        assert ms == 5.0, rank
        assert abs(rate - 2 * 32768 / 5e-3 / 1e6) < 1e-9
    assert res[1][3] == 0   # rank 1 of the reference arm did no work
