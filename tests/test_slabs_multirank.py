"""One box over several ranks (the strict slab segmentation of Sec. 2.1):
ghost exchange, cross-edge L0 merge and group migration reproduce the
single-box result bit for bit.

The exchange protocol is host logic (paper_2110_11408_gb300.slabs); here each
rank's compute is the CPU oracle, so that the protocol is checked on CPU
ranks (gloo, world sizes 2 and 4) and in one process.  The same protocol on
the GPU library is checked in tests/test_stages_gpu.py."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2110_11408_gb300 import slabs, synth

BOX = 1 << 21


class OracleOps:
    def __init__(self, u):
        self.p = O.params(u)

    def density(self, pos, n_query):
        return O.density_at(pos, self.p, np.arange(n_query))

    def fof(self, pos, ids, sigma):
        return O.fof(pos, ids, sigma, self.p)[0]

    def levels(self, pos, ids, sigma, l0):
        l1, l2, halos, _ = O.compaso(pos, ids, sigma, l0, self.p)
        return l1, l2, halos


def box():
    # the tiny recipe at a fifth of the particles: groups cross every slab edge
    return synth.nfw_box(64, 0.5, 20, 20000, seed=61, n_total=60000)


def split(pos, edges):
    return [np.nonzero((pos[:, 0] >= edges[r]) & (pos[:, 0] < edges[r + 1]))[0] for r in range(len(edges) - 1)]


def check(results, parts, pos, ids, u):
    o = O.find_groups(pos, ids, O.params(u))
    for key in ("sigma", "l0", "l1", "l2"):
        got = np.empty_like(o[key])
        for r, idx in enumerate(parts):
            got[idx] = results[r][key]
        if not np.array_equal(got, o[key]):
            bad = np.nonzero(got != o[key])[0]
            raise AssertionError("%s differs at %d of %d particles" % (key, bad.size, got.size))
    rows = np.concatenate([r["halos"] for r in results if r["halos"] is not None])
    rows = rows[np.argsort(rows["nucleus_id"])]
    assert len(rows) == len(o["halos"])
    for f in ("nucleus_id", "N", "R2", "l2max_id", "l2max_N", "l2_top5_N", "n_l2", "l0_id"):
        assert np.array_equal(rows[f], o["halos"][f]), f
    np.testing.assert_allclose(rows["com"], o["halos"]["com"], rtol=1e-12)
    return o


@pytest.mark.parametrize("world", [2, 3, 4])
def test_serial_ranks_reproduce_the_box(world):
    pos, ids, meta = box()
    edges = [BOX * k // world for k in range(world + 1)]
    edges[1] += 12345  # uneven slabs
    parts = split(pos, edges)
    ops = OracleOps(meta["u"])
    p = O.params(meta["u"])
    gens = [slabs.slab_rank(r, world, pos[parts[r]], ids[parts[r]], edges, p, ops) for r in range(world)]
    res = slabs.run_serial(gens)
    o = check(res, parts, pos, ids, meta["u"])
    # groups really cross the edges and move between ranks
    assert sum(r["migrated_in"] for r in res) > 0 and all(r["ghosts"] > 0 for r in res)
    assert o["stats"]["l0_groups"] > 50


def test_slabs_narrower_than_two_ghost_widths_are_refused():
    pos, ids, meta = box()
    p = O.params(meta["u"])
    edges = [0, 1000, BOX]
    g = slabs.slab_rank(0, 2, pos[:10], ids[:10], edges, p, OracleOps(meta["u"]))
    with pytest.raises(ValueError):
        next(g)


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pos, ids, meta = box()
        edges = [BOX * k // world for k in range(world + 1)]
        parts = split(pos, edges)
        p = O.params(meta["u"])
        gen = slabs.slab_rank(rank, world, pos[parts[rank]], ids[parts[rank]], edges, p, OracleOps(meta["u"]))
        res = slabs.run_distributed(gen, dist, rank, world)
        out = [None] * world
        dist.all_gather_object(out, res)
        if rank == 0:
            check(out, parts, pos, ids, meta["u"])
            q.put("ok")
    except Exception as e:  # reported to the parent
        q.put("rank %d: %r" % (rank, e))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_reproduce_the_box(world):
    import multiprocessing as mp
    import socket
    ctx = mp.get_context("spawn")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=600)
    msgs = []
    while not q.empty():
        msgs.append(q.get())
    assert all(pr.exitcode == 0 for pr in procs), msgs
    assert msgs and all(m == "ok" for m in msgs), msgs
