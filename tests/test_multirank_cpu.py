"""The N > 1 host path of the benchmark on CPU: world size 2 over gloo.

Every rank meshes its own seeded aggregate (independent problems, no
data-path collective), and the whole-job time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2108_07212_gb300 import binding as B
    w = bench.workload_for(rank, None)
    S = B.Simulation(w)                                   # host meshing only
    mine = torch.tensor([float(S.N), float(w.grain_geom[:, :2].sum())], dtype=torch.float64)
    allv = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(allv, mine)
    t = bench.max_over_ranks(dist, [1.0 + rank, 5.0 - rank], "cpu")
    out[rank] = (allv[0].tolist(), allv[1].tolist(), t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_run_independent_aggregates_and_take_the_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        ps = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
        assert all(p.exitcode == 0 for p in ps)
        res = dict(out)
    a0, a1, t0 = res[0]
    _, _, t1 = res[1]
    assert a0 != a1                       # different seeded aggregates per rank
    assert t0 == t1 == [2.0, 5.0]         # element-wise max over ranks on every rank
