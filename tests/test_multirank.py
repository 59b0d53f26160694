"""Host logic of the multi-GPU benchmark path (replicas, no data-path collective), run as
two gloo ranks on the CPU: disjoint root shards, max-over-ranks time, N x harmonic mean."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    roots = bench.rank_roots(list(range(100, 100 + 8 * world)), rank, 8)
    ms = [3.0, 5.0][rank]
    hm = [200.0, 100.0][rank]
    out = bench.combine_ranks(ms, hm, dist, torch.device("cpu"))
    q.put((rank, roots, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, (roots, out)) for r, roots, out in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res[0][0] == list(range(100, 108)) and res[1][0] == list(range(108, 116))
    for r in range(world):
        ms, value = res[r][1]
        assert ms == 5.0
        assert abs(value - 2 * (2 / (1 / 200.0 + 1 / 100.0))) < 1e-9
