"""The N > 1 path of bench.py on CPU: two gloo ranks at 127.0.0.1. Each rank takes its
round-robin shard of independent problems (no data-path collective), evaluates it
(here with the oracle, on the CPU), and the job time is the maximum over ranks."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench
    from oracle import element as OE
    from synthetic import mesh as M
    from synthetic import workloads as W

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    assert (w, r) == (world, rank)
    problems = [(W.POISSON, 1), (W.MASS, 2), (W.ELASTICITY, 1), (W.POISSON, 2), (W.MASS, 1)]
    mesh = M.unit_cube_tets(2, 0.1, seed=3)
    mine = bench.shard(len(problems), rank, world)
    sums = {}
    for k in mine:
        form, q = problems[k]
        sums[k] = float(np.abs(OE.element_tensors(form, M.gather_cell_vertices(mesh), q)).sum())
    t = bench.max_over_ranks(0.25 + rank, world)  # stand-in per-rank times
    gathered = [None] * world
    dist.all_gather_object(gathered, sums)
    if rank == 0:
        out.put((t, gathered))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_independent_problems_and_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 1.25
    keys = sorted(k for g in gathered for k in g)
    assert keys == [0, 1, 2, 3, 4]  # every problem exactly once across ranks
    assert set(gathered[0]) == {0, 2, 4} and set(gathered[1]) == {1, 3}
