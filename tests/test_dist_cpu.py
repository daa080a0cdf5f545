"""The N>1 path of bench.py on CPU: two gloo ranks, each timing its own independent problem (weak
scaling, no data-path collective); the job's throughput is the updates of all ranks over the slowest
rank's time, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist("gloo")
    d.barrier()
    # rank r: (1 + r) seconds for 100 (1 + r) updates
    v, t = bench.aggregate(d, 1.0 + rank, 100.0 * (1 + rank))
    ran = []

    class Args:
        workload, cells, steps, warmup, gpus = "periodic", 64, 1, 0, world

    # non-zero ranks of the reference arm return before any work
    if rank != 0:
        bench.run_reference(Args, d)
        ran.append("reference-returned")
    d.barrier()
    d.close()
    q.put((rank, v, t, ran))


@pytest.mark.timeout(300)
def test_two_gloo_ranks_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=240) for _ in ps)
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    for rank, v, t, ran in out:
        assert t == pytest.approx(2.0)          # slowest rank's time
        assert v == pytest.approx(300.0 / 2.0)  # all ranks' updates / that time
    assert out[0][3] == [] and out[1][3] == ["reference-returned"]


def test_ranks_get_independent_problems():
    # weak scaling: every rank solves its own box, seeded by its rank
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    a = bench.make_problem("periodic", 0, 2, cells=512)
    b = bench.make_problem("periodic", 1, 2, cells=512)
    assert a.mesh.n_cells == b.mesh.n_cells == 512
    assert not np.allclose(a.mesh.volume, b.mesh.volume)
