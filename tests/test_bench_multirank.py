"""The N > 1 benchmark path on CPU: two gloo ranks (one replica each) report
the whole-job figure -- the units of all ranks over the slowest rank's time --
through the same helper bench.py uses under torchrun."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) * 100 ms for 1000 * (r + 1) units per step, 2 steps
    v, ms = bench.whole_job((rank + 1) * 100.0, 1000 * (rank + 1), 2)
    out[rank] = (v, ms)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = 29500 + os.getpid() % 1000
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    # 3000 units per step over the slowest rank's 200 ms, 2 steps
    for r in range(2):
        v, ms = res[r]
        assert ms == pytest.approx(200.0)
        assert v == pytest.approx(3000 * 2 / 0.2)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    v, ms = bench.whole_job(50.0, 10, 3)
    assert ms == 50.0 and v == pytest.approx(10 * 3 / 0.05)
