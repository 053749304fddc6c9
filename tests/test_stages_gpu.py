"""The three steps one at a time through the C ABI (cso_density, cso_fof,
cso_levels) against the oracle's steps on the same inputs, and the slab
decomposition protocol over several ranks with each rank's compute on the
GPU library (the ranks run in lockstep in one process, one after another on
one GPU: no rank's kernels wait on another's)."""
import numpy as np
import pytest

import oracle as O
from paper_2110_11408_gb300 import cso, slabs, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BOX = 1 << 21


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cso.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("case", ["tiny", "patch"])
def test_steps_against_the_oracle(ctx, case):
    if case == "tiny":
        pos, ids, meta = synth.tiny(seed=31)
    else:
        pos, ids, meta = synth.patch(extent=16.0, lo=-8.0, seed=3)
    u = meta["u"]
    p, po = cso.cso_params_default(u), O.params(u)
    o = O.find_groups(pos, ids, po)
    sig = cso.cso_density(ctx.h, pos, len(pos), p)
    assert np.array_equal(sig, o["sigma"])
    # the first n_query only, the rest as neighbours
    nq = len(pos) // 3
    assert np.array_equal(cso.cso_density(ctx.h, pos, nq, p), o["sigma"][:nq])
    l0 = cso.cso_fof(ctx.h, pos, ids, o["sigma"], p)
    assert np.array_equal(l0, o["l0"])
    l1, l2, halos = cso.cso_levels(ctx.h, pos, ids, o["sigma"], o["l0"], p)
    assert np.array_equal(l1, o["l1"]) and np.array_equal(l2, o["l2"])
    for f in ("nucleus_id", "N", "R2", "l2max_id", "l2max_N", "l2_top5_N", "n_l2", "l0_id"):
        assert np.array_equal(halos[f], o["halos"][f]), f
    np.testing.assert_allclose(halos["com"], o["halos"]["com"], rtol=1e-9, atol=1e-9 * BOX)


def test_levels_on_caller_groups_of_another_order(ctx):
    """cso_levels takes any labelling of the same groups (members in any order)."""
    pos, ids, meta = synth.patch(extent=16.0, lo=-8.0, seed=5)
    po = O.params(meta["u"])
    o = O.find_groups(pos, ids, po)
    perm = np.random.default_rng(2).permutation(len(pos))
    l1, l2, halos = cso.cso_levels(ctx.h, pos[perm], ids[perm], o["sigma"][perm], o["l0"][perm],
                                   cso.cso_params_default(meta["u"]))
    assert np.array_equal(l1, o["l1"][perm]) and np.array_equal(l2, o["l2"][perm])


@pytest.mark.parametrize("world", [2, 4])
def test_slab_protocol_on_the_gpu(ctx, world):
    pos, ids, meta = synth.nfw_box(64, 0.5, 20, 20000, seed=61, n_total=60000)
    p = cso.cso_params_default(meta["u"])
    edges = [BOX * k // world for k in range(world + 1)]
    parts = [np.nonzero((pos[:, 0] >= edges[r]) & (pos[:, 0] < edges[r + 1]))[0] for r in range(world)]
    ops = slabs.GpuOps(ctx, p)
    res = slabs.run_serial([slabs.slab_rank(r, world, pos[parts[r]], ids[parts[r]], edges, p, ops)
                            for r in range(world)])
    o = O.find_groups(pos, ids, O.params(meta["u"]))
    for key in ("sigma", "l0", "l1", "l2"):
        got = np.empty_like(o[key])
        for r, idx in enumerate(parts):
            got[idx] = res[r][key]
        assert np.array_equal(got, o[key]), key
    rows = np.concatenate([r["halos"] for r in res if r["halos"] is not None])
    rows = rows[np.argsort(rows["nucleus_id"])]
    assert np.array_equal(rows["nucleus_id"], o["halos"]["nucleus_id"])
    assert np.array_equal(rows["N"], o["halos"]["N"])
    assert sum(r["migrated_in"] for r in res) > 0
