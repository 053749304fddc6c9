"""Pins of the oracle's per-halo summaries and of the L2 level's own
constants (CPU only).

What is checked, and against what:
  * the catalogue row (Sec. 2.2.2 last paragraphs, Table 1): centres of mass
    against exact rational means of hand-built member sets, the L2max choice
    (the first, densest L2 nucleus, not the largest), its member count and
    centre, and the five largest L2 sizes in descending order, on hand-built
    L2 assignments whose answers are written out below;
  * every row of whole pipeline runs against what its own labels define:
    N = #(l1 == id), com = mean member position, n_l2 = number of distinct L2
    labels among the members, l2max = the densest L2 nucleus among them,
    l2max_N and l2max_com from the members labelled with it, top-5 = the five
    largest L2 label counts;
  * L2 uses Delta_L2 and its own stop level: an isolated NFW halo's L2
    radius encloses the particle count the NFW mass profile gives inside
    r_800 (mean enclosed density 800), and lattice top-hats whose central
    kernel density lies between the L1 and L2 stop levels nucleate at L1 but
    not at L2 (Sec. 2.2.2 step 4, App. B.2).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle as O
from paper_2110_11408_gb300 import synth

BOX = 1 << 21
U64 = 32768


def exact_mean(pos, ref):
    """Mean position of `pos` (grid units) as exact rationals, each coordinate
    unwrapped to the periodic image nearest `ref`, then wrapped into the box."""
    d = (pos.astype(np.int64) - np.asarray(ref, np.int64) + BOX // 2) % BOX - BOX // 2
    out = []
    for a in range(3):
        m = Fraction(int(ref[a])) + Fraction(int(d[:, a].sum()), len(pos))
        out.append(float(m % BOX))
    return np.array(out)


# --------------------------------------------------------------------------
# the row on hand-built member sets
# --------------------------------------------------------------------------

def test_com_of_symmetric_lattice_ball_across_the_corner_is_its_centre():
    """A cubic lattice ball about a lattice point next to the box corner (its
    points wrap on all three axes): the centre of mass is the centre exactly,
    whichever member is the nucleus."""
    centre = [1000, BOX - 500, 3]
    pos, ids, _ = synth.lattice_ball(1500, 11, centre)
    assert (pos.max(0) - pos.min(0) > BOX // 2).all()  # wraps on every axis
    n = len(pos)
    members = np.arange(n)
    l0 = np.zeros(n, np.uint64)
    for nuc in (0, n // 3, n - 1):
        row = O.halo_row(pos, ids, l0, U64, nuc, 123456789, members, -np.ones(n), [])
        assert row["N"] == n and row["nucleus_id"] == ids[nuc]
        assert list(row["com"]) == [float(c) for c in centre]
        assert row["n_l2"] == 0 and row["l2max_id"] == O.NONE and row["l2max_N"] == 0
        assert list(row["l2_top5_N"]) == [0] * 5
    assert O.halo_row(pos, ids, l0, U64, 0, 123456789, members, -np.ones(n), [])["R_delta"] == \
        pytest.approx(math.sqrt(123456789) / U64, rel=1e-15)


def test_com_of_asymmetric_set_is_its_exact_mean():
    """A lopsided set of 37 members straddling the corner, the nucleus far
    from the mean: com is the exact mean (a divisor of n - 1, or offsets
    summed from another member without the minimum image, would miss it)."""
    rng = np.random.default_rng(4)
    base = np.array([BOX - 700, 300, BOX - 50])
    off = np.concatenate([rng.integers(-900, 900, (30, 3)), rng.integers(2000, 9000, (7, 3))])
    pos = ((base + off) % BOX).astype(np.int32)
    ids = np.arange(100, 137, dtype=np.uint64)
    n = len(pos)
    l0 = np.full(n, 5, np.uint64)
    want = exact_mean(pos, base)
    for nuc in (0, 33):
        row = O.halo_row(pos, ids, l0, U64, nuc, 10 ** 9, np.arange(n), -np.ones(n), [])
        np.testing.assert_allclose(row["com"], want, rtol=0, atol=1e-7)
        assert row["l0_id"] == 5
    # a mean over n - 1 members would be off by far more than the tolerance
    off_mean = exact_mean(pos[1:], base)
    assert np.abs(off_mean - want).max() > 10


def test_l2max_is_the_first_nucleus_and_top5_the_five_largest():
    """Six L2 haloes accepted in the order 0..5 with sizes 30, 80, 50, 120,
    10, 60 (the first is not the largest, the last not the smallest) and 17
    members in no L2 halo: L2max is nucleus 0 with 30 members, the top five
    sizes are 120, 80, 60, 50, 30, and l2max_com is the mean of nucleus 0's
    own members only."""
    sizes = [30, 80, 50, 120, 10, 60]
    rng = np.random.default_rng(9)
    n = sum(sizes) + 17
    pos = rng.integers(0, 40000, (n, 3)).astype(np.int32)
    pos[:, 0] = (pos[:, 0] - 20000) % BOX  # across the x = 0 face
    ids = rng.permutation(n).astype(np.uint64) + 1000
    slot2 = np.concatenate([np.full(s, q) for q, s in enumerate(sizes)] + [np.full(17, -1)])
    perm = rng.permutation(n)
    slot2 = slot2[perm]
    # each L2 nucleus is one of its own members
    l2nuc = np.array([np.nonzero(slot2 == q)[0][0] for q in range(6)])
    members = np.arange(n)
    l0 = np.zeros(n, np.uint64)
    row = O.halo_row(pos, ids, l0, U64, l2nuc[2], 5 * 10 ** 8, members, slot2, l2nuc)
    assert row["n_l2"] == 6
    assert row["l2max_id"] == ids[l2nuc[0]] and row["l2max_N"] == 30
    assert list(row["l2_top5_N"]) == [120, 80, 60, 50, 30]
    np.testing.assert_allclose(row["l2max_com"], exact_mean(pos[slot2 == 0], pos[l2nuc[0]]), rtol=0, atol=1e-7)
    np.testing.assert_allclose(row["com"], exact_mean(pos, pos[l2nuc[2]]), rtol=0, atol=1e-7)
    # fewer than five L2 haloes: zero-padded
    slot3 = np.where(slot2 >= 3, -1, slot2)
    row3 = O.halo_row(pos, ids, l0, U64, l2nuc[2], 5 * 10 ** 8, members, slot3, l2nuc[:3])
    assert list(row3["l2_top5_N"]) == [80, 50, 30, 0, 0] and row3["n_l2"] == 3


# --------------------------------------------------------------------------
# every catalogue row of whole runs against its own labels
# --------------------------------------------------------------------------

def rows_follow_labels(pos, ids, r):
    sig = r["sigma"]
    for h in r["halos"]:
        m = np.nonzero(r["l1"] == h["nucleus_id"])[0]
        assert h["N"] == m.size
        nuc = np.nonzero(ids == h["nucleus_id"])[0][0]
        np.testing.assert_allclose(h["com"], exact_mean(pos[m], pos[nuc]), rtol=0, atol=1e-6)
        assert h["l0_id"] == r["l0"][nuc]
        lab2 = r["l2"][m]
        labs, counts = np.unique(lab2[lab2 != O.NONE], return_counts=True)
        assert h["n_l2"] == labs.size
        top = sorted(counts.tolist(), reverse=True)[:5]
        assert list(h["l2_top5_N"]) == top + [0] * (5 - len(top))
        if labs.size == 0:
            assert h["l2max_id"] == O.NONE and h["l2max_N"] == 0
            continue
        # L2 nuclei are members labelled with their own id; the densest one
        # (Sigma descending, id ascending) is L2max
        nuc2 = np.nonzero(np.isin(ids, labs))[0]
        best = nuc2[np.lexsort((ids[nuc2], -sig[nuc2]))[0]]
        assert h["l2max_id"] == ids[best]
        mm = m[lab2 == ids[best]]
        assert h["l2max_N"] == mm.size
        np.testing.assert_allclose(h["l2max_com"], exact_mean(pos[mm], pos[best]), rtol=0, atol=1e-6)


@pytest.mark.parametrize("seed", [1, 2])
def test_rows_follow_labels_on_patches(seed):
    pos, ids, _ = synth.patch(extent=16.0, lo=-8.0, seed=seed)
    r = O.find_groups(pos, ids, O.params(U64, np_min_L1=1))
    assert len(r["halos"]) > 10 and (r["halos"]["n_l2"] > 0).any()
    rows_follow_labels(pos, ids, r)


def test_rows_follow_labels_on_the_tiny_box():
    """Box 64 l_mean, 262,144 particles: rows with and without an L2 halo."""
    pos, ids, _ = synth.tiny()
    r = O.find_groups(pos, ids, O.params(U64))
    n2 = r["halos"]["n_l2"]
    assert (n2 == 0).any() and (n2 == 1).any()
    rows_follow_labels(pos, ids, r)


def six_clumps(seed):
    """A uniform ball of radius 1.9 l_mean at 200 times the mean density
    (straddling the x = 0 face) holding six compact clumps of 400, 300, 220,
    160, 170 and 100 particles, one at the centre and five 1 - 1.25 l_mean
    out: one L1 halo with a separate L2 halo per clump."""
    rng = np.random.default_rng(seed)

    def ball(n, r, c):
        return c + synth.isotropic(rng, n) * (rng.random(n) ** (1 / 3) * r * U64)[:, None]

    centre = np.array([BOX - 0.2 * U64, 0.3 * U64, BOX // 2], float)
    parts = [ball(int(round(200 * 4 * math.pi / 3 * 1.9 ** 3)), 1.9, centre)]
    for n, r, dv in ((400, 0.05, [0, 0, 0]), (300, 0.05, [-1.0, 0, 0]), (220, 0.05, [0, 1.0, 0]),
                     (160, 0.04, [0, -1.0, 0]), (170, 0.03, [0, 0, 1.0]), (100, 0.03, [1.25, 0, 0])):
        parts.append(ball(n, r, centre + np.array(dv) * U64))
    pos = np.mod(np.rint(np.concatenate(parts)).astype(np.int64), BOX).astype(np.int32)
    perm = rng.permutation(len(pos))
    return pos[perm], np.arange(len(pos), dtype=np.uint64)[perm]


@pytest.mark.parametrize("seed", [5, 8])
def test_rows_follow_labels_with_several_l2_haloes(seed):
    pos, ids = six_clumps(seed)
    r = O.find_groups(pos, ids, O.params(U64, np_min_L1=1))
    assert r["halos"]["n_l2"].max() >= 6
    rows_follow_labels(pos, ids, r)


def test_rows_follow_labels_on_two_haloes():
    u = U64
    c0 = np.array([BOX - 100] * 3, np.float64)  # the host straddles the corner
    host, hid, hm = synth.nfw_halo(6000, 5.0, u, c0, xmax=1.3, seed=31)
    sat, sid, _ = synth.nfw_halo(700, 9.0, u, c0 + [0.93 * hm["r200"] * u, 0, 0], seed=32, id0=len(host))
    pos, ids = np.concatenate([host, sat]), np.concatenate([hid, sid])
    r = O.find_groups(pos, ids, O.params(u, np_min_L1=1))
    rows_follow_labels(pos, ids, r)


# --------------------------------------------------------------------------
# L2's own constants
# --------------------------------------------------------------------------

def mu(y):
    return math.log1p(y) - y / (1.0 + y)


@pytest.mark.parametrize("seed", [21, 22])
def test_isolated_nfw_l2_radius_is_r800(seed):
    """An isolated NFW halo (c = 6, 20000 particles inside R_200, sampled to
    2 R_200): its L2 halo is the sphere of mean enclosed density 800, so it
    holds N_200 mu(c x_800) / mu(c) particles, x_800 solving
    mu(c x) / mu(c) = 4 x^3 (12,460 here, against ~20,000 for Delta = 200)."""
    c, n200 = 6.0, 20000
    x800 = brentq(lambda x: mu(c * x) / mu(c) - 4.0 * x ** 3, 1e-3, 1.0)
    want = n200 * mu(c * x800) / mu(c)
    pos, ids, _ = synth.nfw_halo(n200, c, U64, [BOX // 2] * 3, xmax=2.0, seed=seed)
    p = O.params(U64, np_min_L1=1)
    sig, _ = O.density(pos, p)
    l1, l2, halos, st = O.compaso(pos, ids, sig, np.zeros(len(pos), np.uint64), p)
    h = halos[np.argmax(halos["N"])]
    assert h["n_l2"] == 1
    # Poisson noise of the count near the crossing is ~1%
    assert h["l2max_N"] == pytest.approx(want, rel=0.04)


def lattice_sigma_max(pos, b2):
    d = pos[:, None, :].astype(np.int64) - pos[None, :, :]
    d = (d + BOX // 2) % BOX - BOX // 2
    d2 = (d * d).sum(-1)
    return int((np.where(d2 < b2, b2 - d2, 0).sum(1) - b2).max())


@pytest.mark.parametrize("a_frac,l1_nucleates,l2_nucleates", [
    (0.16, False, False),  # centre below the L1 stop level (~236 x the mean)
    (0.145, True, False),  # between the L1 and L2 stop levels (~327)
    (0.13, True, True),    # above both (~441)
])
def test_lattice_tophat_stop_levels(a_frac, l1_nucleates, l2_nucleates):
    """Cubic lattice balls (1935 points, spacing a): the kernel density of the
    interior points, computed here by brute force, is placed below, between
    and above the stop levels of L1 (250.84) and L2 (398.18, the SIS rule
    with Delta_L2 = 800).  A level nucleates only above its own level."""
    a = int(a_frac * U64)
    pos, ids, _ = synth.lattice_ball(a, 60, [BOX - 3 * a, 5 * a, BOX // 2])
    p = O.params(U64, np_min_L1=1)
    smax = lattice_sigma_max(pos, p.b2)
    assert (smax > p.T_min_L1) == l1_nucleates
    assert (smax > p.T_min_L2) == l2_nucleates
    r = O.find_groups(pos, ids, p)
    assert (r["stats"]["l1_nuclei"] > 0) == l1_nucleates
    assert (r["stats"]["l2_nuclei"] > 0) == l2_nucleates
    assert ((r["l2"] != O.NONE).any()) == l2_nucleates
