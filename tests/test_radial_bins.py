"""The paper's radial-bin threshold-radius search (Sec. 2.3.4: members binned
outward in steps of sqrt(3)/3 cell sides, a bin skipped while the members
inside it placed at its outer edge still meet the threshold) gives the same
R^2 as the default threshold-count binning, so every output must equal the
oracle's: on the plain schedule, the batched one, with every group above 64
members on clusters, with tiny select tiles, and on the batched recipe with
a 2e5-member group."""
import numpy as np
import pytest

from paper_2110_11408_gb300 import cso, synth
from parity_util import assert_matches_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
R = cso.FLAG_RADIAL_BINS


@pytest.fixture(scope="module")
def tiny():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return synth.tiny()


def run(flags, pos, ids, u, giant=None, small=64):
    with cso.Context(0, flags=flags) as c:
        if giant:
            cso.cso_set_schedule(c.h, giant, small)
        return c.find_groups(pos, ids, cso.cso_params_default(u))


@pytest.mark.parametrize("flags,giant", [(R, None), (R | cso.FLAG_BATCHED, None), (R | cso.FLAG_BATCHED, 64),
                                         (R | cso.FLAG_SELECT_STRESS, None),
                                         (R | cso.FLAG_BATCHED | cso.FLAG_SELECT_STRESS, 64)])
def test_tiny_box(tiny, flags, giant):
    pos, ids, meta = tiny
    assert_matches_oracle(run(flags, pos, ids, meta["u"], giant=giant), pos, ids, meta["u"])


def test_patches_with_select_stress():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for seed in (4, 5):
        pos, ids, meta = synth.patch(extent=18.0, lo=-3.0, seed=seed, nmax=4000)
        g = run(R | cso.FLAG_SELECT_STRESS, pos, ids, meta["u"])
        assert_matches_oracle(g, pos, ids, meta["u"])


def test_batched_recipe_with_a_large_group():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pos, ids, meta = synth.batched(total=400_000, giant=200_000)
    a = run(R | cso.FLAG_BATCHED, pos, ids, meta["u"], giant=16384)
    assert_matches_oracle(a, pos, ids, meta["u"])
    b = run(R, pos, ids, meta["u"])
    for k in ("sigma", "l0", "l1", "l2"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["halos"], b["halos"])
