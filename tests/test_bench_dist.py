"""bench.py's multi-rank path on CPU: gloo, world size 2, 127.0.0.1.

Ranks search their own patterns (weak scaling, no collective on the data
path); timing takes a barrier and the maximum over ranks.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    class A:
        n, kinds, ms, patterns = 1 << 16, "4", "8", 5
    w, r, _ = bench.dist_setup(A)
    bench.barrier(w)
    worst = bench.max_over_ranks(float(rank + 1) * 0.5, w)
    kinds, ms, texts, pats = bench.make_workload(A, r)
    q.put((r, w, worst, pats[(4, 8)]))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 1.0 for o in out)            # max over ranks of 0.5 and 1.0
    assert out[0][3] != out[1][3]                   # each rank has its own patterns
