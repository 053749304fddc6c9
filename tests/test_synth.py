"""The seeded input generators (no GPU): the slab-delivered boxes cover
their box exactly once, in order, reproducibly; the closed-form NFW inverse
agrees with bisection on the mass fraction; the side-1024 slab edges form a
composition of the 512 columns into 256 parts of 1-4."""
import numpy as np

from paper_2110_11408_gb300 import synth

BOX = 1 << 21


def test_slab_box_covers_the_box_once():
    edges = [BOX * k // 8 for k in range(9)]
    b = synth.SlabBox(64, 0.4, 20, 20000, edges, seed=3)
    got = list(b.slabs())
    assert [k for k, _, _ in got] == list(range(8))
    ids = np.concatenate([i for _, _, i in got])
    assert ids.dtype == np.uint64 and ids.size == 64 ** 3
    assert np.array_equal(np.sort(ids), np.arange(64 ** 3, dtype=np.uint64))
    for k, p, _ in got:
        assert p.dtype == np.int32 and (p[:, 0] >= edges[k]).all() and (p[:, 0] < edges[k + 1]).all()
        assert (p >= 0).all() and (p < BOX).all()
    # halo particles take about 60% of the box, as the recipe asks
    assert abs(b.n_halo / b.n - 0.6) < 0.01


def test_slab_box_is_reproducible_in_a_process_pool():
    edges = [0, BOX // 3, BOX // 2, BOX]
    a = list(synth.SlabBox(64, 0.4, 20, 20000, edges, seed=5).slabs())
    b = list(synth.SlabBox(64, 0.4, 20, 20000, edges, seed=5).slabs(workers=3, shuffle_seed=None))
    for (ka, pa, ia), (kb, pb, ib) in zip(a, b):
        assert ka == kb and np.array_equal(pa, pb) and np.array_equal(ia, ib)


def test_closed_form_nfw_inverse_matches_bisection():
    rng = np.random.default_rng(1)
    c = rng.uniform(4.0, 12.0, 20000)
    x_bis = synth.nfw_unit_radii(np.random.default_rng(2), c)
    q = np.random.default_rng(2).random(c.size)
    x_closed = synth.nfw_unit_radii_closed(q, c)
    assert np.abs(x_closed - x_bis).max() < 1e-12
    # enclosed-mass fractions are reproduced
    np.testing.assert_allclose(synth._mu(c * x_closed), q * synth._mu(c), rtol=1e-10, atol=1e-14)


def test_side_1024_edges_are_a_composition():
    e = np.asarray(synth.served1024_edges())
    assert e.size == 257 and e[0] == 0 and e[-1] == BOX
    cols = np.diff(e) // (BOX // 512)
    assert (np.diff(e) % (BOX // 512) == 0).all()
    assert cols.min() >= 1 and cols.max() <= 4 and cols.sum() == 512
