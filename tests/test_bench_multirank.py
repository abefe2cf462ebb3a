"""Multi-rank path of bench.py on CPU: two gloo ranks, each with its own realisation,
combine work by sum and time by max (no collective touches the solver's data)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank builds its own realisation (seed 2 + rank)
    import workloads as W
    prob = W.quarter_five_spot(32, seed=2 + rank)
    vals = [1000.0 * (rank + 1), 0.5 + rank, 10.0 * (rank + 1), 0.1 * (rank + 1)]
    res = bench.aggregate(vals, dist, device="cpu")
    out.put((rank, res, float(prob.K.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for rank, res, ksum in got:
        assert res == (3000.0, 1.5, 30.0, 0.2)
    assert got[0][2] != got[1][2]        # distinct realisations per rank
