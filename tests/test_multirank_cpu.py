"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2).

bench.py runs one independent replica per GPU; the only cross-rank steps are
the barrier around the timed region and the max over ranks of the elapsed
time.  These run here on two gloo ranks.
"""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        w, r, local = bench.dist_env()
        ms_local = (10.0, 25.0)[rank]
        bench.barrier(w)
        ms, value = bench.aggregate(ms_local, 100, w, torch.device("cpu"))
        ref = bench.run_reference(_Args()) if rank == 1 else "skipped"
        q.put((rank, w, r, local, ms, value, ref))
    finally:
        dist.destroy_process_group()


class _Args:
    config, seed, steps, warmup = "tiny", 1, 1, 0


def test_two_rank_aggregation_and_reference_arm():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, w, r, local, ms, value, ref = q.get(timeout=120)
        out[rank] = (w, r, local, ms, value, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (w, r, local, ms, value, ref) in out.items():
        assert (w, r, local) == (2, rank, rank)
        assert ms == 25.0                          # the slowest rank's time
        assert value == pytest.approx(2 * 100 / 0.025)   # both ranks' iterations / that time
    assert out[1][5] is None                       # the reference arm runs on rank 0 only
