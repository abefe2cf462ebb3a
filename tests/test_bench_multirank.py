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


def _solver_worker(rank, world, port, out):
    """Each rank steps its own realisation (seed 2 + rank) with the FP64 oracle -- the CPU
    stand-in for the per-rank solver -- and combines its node updates and time the way the
    bench does; the ranks exchange only those scalars, never solver data."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    import bench
    import oracle as O
    import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    O.set_threads(1)                  # two ranks on one host: one oracle thread each
    prob = W.quarter_five_spot(24, seed=2 + rank)
    orc = O.Oracle(prob, init_replay=16, check_every=8, max_sub_iters=4000)
    st, k, r = orc.step(2)
    updates = float(np.sum(k + 1) * prob.nx * prob.ny)
    seconds = 0.25 * (rank + 1)
    res = bench.aggregate([updates, seconds, updates, seconds], dist, device="cpu")
    P = orc.fields()["P"]
    # every rank's pressure field, gathered only to check that the realisations differ
    Ps = [torch.zeros(P.size, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(Ps, torch.from_numpy(P.ravel().copy()))
    out.put((rank, res, updates, [float(t.sum()) for t in Ps], int(st)))
    dist.barrier()
    dist.destroy_process_group()
    orc.close()


def test_two_gloo_ranks_with_solver_work():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solver_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = got[0][2] + got[1][2]
    for rank, res, updates, psums, st in got:
        assert st == 0                              # both solves met their tolerance
        assert res[0] == total and res[2] == total  # work summed over the ranks
        assert res[1] == 0.5 and res[3] == 0.5      # time: the slowest rank
        assert updates > 0
    assert got[0][3] == got[1][3]                   # both ranks gathered the same fields
    assert got[0][3][0] != got[0][3][1]             # distinct realisations per rank
