"""The multi-rank logic of bench.py on CPU: two gloo ranks (one process per
rank, as torchrun starts them), no GPU.  Every rank runs its own replica of
the layer (the path has no exchange step), so the only cross-rank step is the
maximum of the ranks' times, and the reference arm works on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 + r ms: everyone must report the slowest
        got = bench.max_over_ranks(10.0 + rank, dist, "cpu")
        dist.barrier()
        # the reference arm returns at once on ranks other than 0
        class A:
            gpus, steps, warmup = world, 1, 0
        ref_rc = bench.run_reference(A) if rank != 0 else 0
        out.put((rank, got, ref_rc))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert res == [(0, 11.0, 0), (1, 11.0, 0)]
