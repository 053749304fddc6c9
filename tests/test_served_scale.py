"""The served stream at full size: the side-512 box (134M particles) as 64
x-slabs through cso_submit / cso_poll under a 40 GB budget, in the
benchmark's launch configuration, checked against the oracle on one slab.

The oracle runs on the particles of that slab alone.  A group whose members
all lie at least b + l_FoF inside the slab in x is the same group in the
whole box (every particle within b of a member, and every particle that can
link to one, is inside), with the same kernel sums, so its L0, L1 and L2
labels must equal the stream's; so must the no-group labels of particles
that far inside."""
import numpy as np
import pytest

import oracle as O
from paper_2110_11408_gb300 import cso, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_side_512_stream_against_the_oracle_on_one_slab():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    box = synth.served512()
    slabs = []
    for k, pos, ids in box.slabs(workers=16, shuffle_seed=box.seed + 99):
        slabs.append((pos, ids, torch.from_numpy(pos).cuda(), torch.from_numpy(ids.view(np.int64)).cuda()))
    p = cso.cso_params_default(box.u)
    bufs, tickets = [], []
    with cso.Context(0, budget_bytes=40 << 30, flags=cso.FLAG_BATCHED | cso.FLAG_SLOTS(2)) as ctx:
        for k, (_, _, dp, di) in enumerate(slabs):
            b = cso.Buffers(dp, di, True, halo_cap=len(dp) // 20 + 64, x_lo=int(box.edges[k]),
                            x_hi=int(box.edges[k + 1]), request_id=512, want=("l0", "l1", "l2", "sigma"))
            bufs.append(b)
            tickets.append(ctx.submit(b, p))
        for t in tickets:
            done, rc = ctx.wait(t)
            assert done and rc == cso.CSO_OK, cso.cso_last_error()
    assert sum(len(s[0]) for s in slabs) == 512 ** 3
    k = int(np.random.default_rng(box.seed).integers(1, 63))
    pos, ids = slabs[k][0], slabs[k][1]
    g = bufs[k].result()
    po = O.params(box.u)
    o = O.find_groups(pos, ids, po)
    margin = int(np.ceil((0.4 + 0.25) * box.u)) + 1
    lo, hi = int(box.edges[k]) + margin, int(box.edges[k + 1]) - margin
    inside = (pos[:, 0] >= lo) & (pos[:, 0] < hi)
    # no-group particles far inside: exact kernel sums, so the same labels
    nog = inside & (o["l0"] == O.NONE)
    assert np.array_equal(g["sigma"][nog], o["sigma"][nog])
    assert (g["l0"][nog] == cso.NO_GROUP).all()
    # groups wholly inside
    dense = o["l0"] != O.NONE
    labs = o["l0"][dense]
    out_of = np.unique(labs[~inside[dense]])
    whole = dense & ~np.isin(o["l0"], out_of)
    assert whole.sum() > 100_000
    for key in ("sigma", "l0", "l1", "l2"):
        a, b = g[key][whole], o[key][whole]
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError("%s differs on %d of %d particles of groups inside slab %d"
                                 % (key, bad.size, a.size, k))
