"""The multi-GPU benchmark path on CPU ranks (gloo, world size 2): each rank
processes its own box (weak scaling, no collective on the data path); the
only collective is the max over ranks of the step time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [12.0, 20.0][rank]
    value, ms = bench.whole_job_rate(1_000_000, ms_local, world, dist, "cpu")
    out[rank] = (value, ms, bench.make_workload_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_rate():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in (0, 1):
        value, ms, _ = out[r]
        assert ms == 20.0  # the slowest rank sets the job time
        assert value == pytest.approx(2 * 1_000_000 / 0.020)
    assert out[0][2] != out[1][2]  # every rank draws its own box
