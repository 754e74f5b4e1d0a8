"""The multi-GPU path is replicas only: each rank solves its own grids and the
benchmark reduces elapsed time with MAX and work with SUM.  Checked here with
two gloo ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1504_05869_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, l = replicas.env()
        # rank k takes k+1 seconds and does 10 (k+1) site updates
        t, u = replicas.aggregate(float(r + 1), 10.0 * (r + 1))
        dist.barrier()
        q.put((r, w, l, t, u))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    for r in res:
        assert r[3] == 2.0           # slowest rank's time
        assert r[4] == 30.0          # all ranks' work


def test_single_rank_is_identity():
    pytest.importorskip("torch")
    from paper_1504_05869_gb300 import replicas
    assert replicas.aggregate(1.5, 7.0) == (1.5, 7.0)
