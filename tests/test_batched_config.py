"""The batched workload: pre-formed groups of uneven size (one giant of 2e6
particles, sizes with equal particles per logarithmic interval down to 35),
and its stress variant of 100,000 groups of 35-45 particles.

Both schedules (plain: a 256-thread block per group; batched: warps, 256-
and 1024-thread blocks and 8-CTA clusters by size, largest first) are checked
against the oracle: in full on the 400k-particle version of the recipe (a
2e5 giant) and on the batched-many box, and on the 4M-particle box by
sampled kernel sums, every group of up to 70,000 members drawn from each
size tier recomputed by the oracle, and batched == plain bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2110_11408_gb300 import cso, synth
from parity_util import assert_matches_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return True


def run(flags, pos, ids, p, giant=None, small=64, huge=None):
    with cso.Context(0, flags=flags) as c:
        if giant:
            cso.cso_set_schedule(c.h, giant, small)
        if huge:
            cso.cso_set_huge_group(c.h, huge)
        return c.find_groups(pos, ids, p)


def test_batched_recipe_at_one_tenth_full_parity(gpu):
    """400k particles, a 2e5 giant: the plain schedule and the batched one
    with clusters above 16,384 and above 2,048 members, and with 16-CTA
    clusters above 16,384, all equal to the oracle."""
    pos, ids, meta = synth.batched(total=400_000, giant=200_000)
    p = cso.cso_params_default(meta["u"])
    a = run(0, pos, ids, p)
    o = assert_matches_oracle(a, pos, ids, meta["u"])
    assert o["stats"]["l0_groups"] > 500
    # clusters above 16,384 and above 2,048 members; then the giant (and
    # every group above 16,384) on 16-CTA clusters
    for giant, huge in ((16384, None), (2048, None), (2048, 16384)):
        b = run(cso.FLAG_BATCHED, pos, ids, p, giant=giant, huge=huge)
        for k in ("sigma", "l0", "l1", "l2"):
            assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a["halos"], b["halos"])


def test_batched_many_full_parity(gpu):
    pos, ids, meta = synth.batched_many()
    p = cso.cso_params_default(meta["u"])
    b = run(cso.FLAG_BATCHED, pos, ids, p, giant=65536, small=64)
    o = assert_matches_oracle(b, pos, ids, meta["u"])
    assert o["stats"]["l0_groups"] > 90_000


def test_batched_config_full_size(gpu):
    """The 4M-particle box in the tuned launch configuration."""
    pos, ids, meta = synth.batched()
    p = cso.cso_params_default(meta["u"])
    po = O.params(meta["u"], np_min_L1=1)
    b = run(cso.FLAG_BATCHED, pos, ids, p, giant=65536)
    a = run(0, pos, ids, p)
    for k in ("sigma", "l0", "l1", "l2"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["halos"], b["halos"])
    rng = np.random.default_rng(5)
    sample = rng.choice(len(pos), 2000, replace=False)
    assert np.array_equal(b["sigma"][sample], O.density_at(pos, po, sample))
    dense = b["l0"] != cso.NO_GROUP
    assert np.all(dense == (b["sigma"] > po.T_L0))
    groups, counts = np.unique(b["l0"][dense], return_counts=True)
    assert counts.max() > 1_500_000
    pick = []
    for lo, hi in ((4096, 70_000), (64, 4096), (1, 64)):
        sel = groups[(counts > lo) & (counts <= hi)]
        pick.append(rng.choice(sel, min(4, sel.size), replace=False))
    members = [np.nonzero(b["l0"] == gid)[0] for gid in np.concatenate(pick)]
    sig_all = O.density_at(pos, po, np.concatenate(members))
    cuts = np.cumsum([0] + [m.size for m in members])
    for k, m in enumerate(members):
        sig = sig_all[cuts[k]:cuts[k + 1]]
        assert np.array_equal(sig, b["sigma"][m])
        l1, l2, halos, _ = O.compaso(pos[m], ids[m], sig, b["l0"][m], po)
        assert np.array_equal(l1, b["l1"][m]) and np.array_equal(l2, b["l2"][m])
