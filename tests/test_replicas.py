"""The N > 1 path (independent replicas) with world size 2 on gloo (CPU)."""
import os
import socket

import torch.multiprocessing as mp

from paper_2512_21909_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    r, w = replicas.init("gloo")
    replicas.barrier(w)
    mx = replicas.allmax(1.5 + r, w)
    mine = replicas.shard(list(range(7)), r, w)
    replicas.finalize(w)
    q.put((r, w, mx, mine))


def test_two_ranks_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q))
             for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2, 2]
    assert all(o[2] == 2.5 for o in out)          # max over ranks
    assert out[0][3] == [0, 2, 4, 6] and out[1][3] == [1, 3, 5]
    assert sorted(out[0][3] + out[1][3]) == list(range(7))
