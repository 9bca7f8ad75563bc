"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank
gets its own pairs (weak scaling, no data-path collective) and the reported
value is the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ranks = bench.Ranks(world, "cpu")
        pairs, _, _ = bench.workload(2, rank, 8)
        cells = sum(len(a) * len(b) for a, b in pairs)
        t = 1.0 + rank            # the slower rank sets the time
        ranks.barrier()
        total = ranks.sum(cells)
        t_max = ranks.max(t)
        out[rank] = (cells, total, t_max, tuple(pairs[0]))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    cells0, total0, tmax0, first0 = res[0]
    cells1, total1, tmax1, first1 = res[1]
    assert total0 == total1 == cells0 + cells1
    assert tmax0 == tmax1 == 2.0
    assert first0 != first1          # each rank draws its own pairs


def test_single_rank_needs_no_group():
    import bench
    r = bench.Ranks(1, "cpu")
    r.barrier()
    assert r.max(3.5) == 3.5 and r.sum(7) == 7
