"""The benchmark's multi-GPU host logic on CPU ranks (gloo, world size 2):
each rank takes a disjoint slice of one seeded stream of cells, and the
result combines the ranks' units by sum and their times by max, the only
exchange (after the timed region).  No GPU is used."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, cells, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from synth.workloads import make
    _, T, nH, Av, y0 = make(bench.WORKLOAD, cells=cells * world)
    sl = bench.rank_cells(cells, rank)
    # per-rank "work": a deterministic function of its own cells
    units = int(np.round(T[sl].sum()))
    ms = 100.0 + 25.0 * rank
    tot_units, tot_ms = bench.combine_ranks(units, ms, world, torch.device("cpu"))
    q.put((rank, sl.start, sl.stop, units, tot_units, tot_ms, float(T[sl][0])))
    dist.destroy_process_group()


def test_two_cpu_ranks_combine_by_sum_and_max():
    import torch.multiprocessing as mp
    pytest.importorskip("torch.distributed")
    world, cells = 2, 64
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, cells, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, b0, u0, s0, m0, t0), (r1, a1, b1, u1, s1, m1, t1) = res
    assert (a0, b0, a1, b1) == (0, cells, cells, 2 * cells)     # disjoint, covering
    assert s0 == s1 == u0 + u1                                   # units summed
    assert m0 == m1 == 125.0                                     # slowest rank's time
    from synth.workloads import make
    import bench
    _, T, _, _, _ = make(bench.WORKLOAD, cells=2 * cells)
    assert t0 == float(T[0]) and t1 == float(T[cells])          # slices of one seeded stream
