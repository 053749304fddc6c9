"""Pins of the oracle's radial halo statistics (Table 1: r_XX_L2com,
vcirc_max_L2com, rvcirc_max_L2com) against what geometry fixes.

- Cubic lattice balls: shell counts of Z^3 (hand-counted for the first
  shells, enumerated for larger balls) fix every enclosed-fraction radius and
  the circular-velocity peak exactly.
- A singular isothermal sphere, M(<r) = 4 pi A r, encloses the fraction f of
  its particles at r = f R.
- An NFW halo (Sec. 4.2 profile) has the enclosed mass N mu(c x) / mu(c), so
  its half-mass radius solves mu(c x) = mu(c) / 2, and its circular velocity
  peaks at c x = 2.16258 (the root of d/dx [mu(x) / x] = 0).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2110_11408_gb300 import synth

BOX = 1 << 21


def row(nucleus_id, n, centre, n_l2=1, com=None):
    r = np.zeros(1, O.HALO_DTYPE)
    r["nucleus_id"] = nucleus_id
    r["N"] = n
    r["n_l2"] = n_l2
    r["l2max_com"] = np.asarray(centre, np.float64)
    r["com"] = np.asarray(com if com is not None else (5.0, 5.0, 5.0), np.float64)
    return r


def lattice(a, kmax, centre):
    rng = int(math.isqrt(kmax)) + 1
    g = np.arange(-rng, rng + 1)
    i, j, k = np.meshgrid(g, g, g, indexing="ij")
    s = (i * i + j * j + k * k).ravel()
    keep = s <= kmax
    off = np.stack([i.ravel()[keep], j.ravel()[keep], k.ravel()[keep]], axis=1) * a
    pos = (np.asarray(centre, np.int64)[None, :] + off) % BOX
    return pos.astype(np.int32), s[keep]


def test_first_shells_by_hand():
    # shell 0: 1 point, shell 1: 6 points (+-a on one axis), shell 2: 12 points
    a, u = 64, 8192.0
    C = (100, BOX - 30, 7)  # the ball straddles the periodic faces in x and y
    for kmax, n, d_q, vn, vd in [(1, 7, (1, 1, 1, 1), 7, 1), (2, 19, (1, 2, 2, 2), 19, 2)]:
        pos, _ = lattice(a, kmax, C)
        assert len(pos) == n
        r = O.radial(pos, np.full(n, 11, np.uint64), row(11, n, C), u)[0]
        assert tuple(r["centre"]) == C
        assert tuple(r["d_q"]) == tuple(x * a * a for x in d_q)
        assert r["vmax_n"] == vn and r["vmax_d2"] == vd * a * a
        assert r["r_vmax"] == math.sqrt(vd * a * a) / u
        assert r["vmax"] == math.sqrt(vn / (math.sqrt(vd * a * a) / u))


def test_lattice_ball_shell_counts():
    # cumulative shell counts of Z^3 by enumeration fix every statistic
    a, u, kmax = 40, 8192.0, 60
    C = (BOX - 1, 3, BOX // 2)
    pos, s = lattice(a, kmax, C)
    n = len(pos)
    cum = np.cumsum(np.bincount(s, minlength=kmax + 1))
    r = O.radial(pos, np.full(n, 5, np.uint64), row(5, n, C), u)[0]
    for q, f in enumerate(O.RADIAL_PERCENT):
        k = -(-f * n // 100)
        shell = int(np.argmax(cum >= k))
        assert r["d_q"][q] == shell * a * a
    occupied = [t for t in range(1, kmax + 1) if cum[t] > cum[t - 1]]
    best = max(occupied, key=lambda t: (cum[t] ** 2 / t, -t))
    assert r["vmax_n"] == cum[best] and r["vmax_d2"] == best * a * a


def test_centre_choice_rounding_and_members():
    a, u = 64, 8192.0
    C = (5000, 6000, 7000)
    pos1, _ = lattice(a, 5, C)
    pos2, _ = lattice(a, 8, (9000, 9000, 9000))
    pos = np.concatenate([pos2[:20], pos1, pos2[20:]])
    lab = np.concatenate([np.full(20, 2), np.full(len(pos1), 1), np.full(len(pos2) - 20, 2)]).astype(np.uint64)
    perm = np.random.default_rng(3).permutation(len(pos))
    pos, lab = pos[perm], lab[perm]
    rows = np.concatenate([row(1, len(pos1), C), row(2, len(pos2), (9000.0, 9000.0, 9000.0))])
    ref = O.radial(pos, lab, rows, u)
    # without L2 haloes the L1 com is the centre
    rows_l1 = rows.copy()
    rows_l1["n_l2"] = 0
    rows_l1["com"] = rows["l2max_com"]
    rows_l1["l2max_com"] = 0.0
    assert (O.radial(pos, lab, rows_l1, u) == ref).all()
    # the centre is the nearest grid point, wrapped into the box
    rows_r = rows.copy()
    rows_r["l2max_com"][0] = (C[0] + 0.4, C[1] - 0.4, C[2] + 0.49)
    assert (O.radial(pos, lab, rows_r, u) == ref).all()
    rows_r["l2max_com"][0] = (BOX - 0.3, C[1] + 0.6, C[2])
    assert tuple(O.radial(pos, lab, rows_r, u)[0]["centre"]) == (0, C[1] + 1, C[2])
    # each row sees its own members only
    a1 = O.radial(pos1, np.full(len(pos1), 1, np.uint64), rows[:1], u)
    assert (a1 == ref[:1]).all()


def test_sis_quantiles():
    # M(<r) = 4 pi A r: the fraction f of the particles lies inside f R
    u, A, R = 8192, 800.0, 4.0
    centre = (BOX // 3, BOX // 5, BOX - 10)
    pos, ids, meta = synth.sis_ball(A, R, u, centre, seed=9)
    n = meta["n"]
    r = O.radial(pos, np.zeros(n, np.uint64), row(0, n, centre), float(u))[0]
    for q, f in enumerate(O.RADIAL_PERCENT):
        sigma = math.sqrt(f / 100 * (1 - f / 100) / n)
        assert abs(r["r_q"][q] / R - f / 100) < 6 * sigma + 1e-4, (f, r["r_q"][q])


def _mu(y):
    return math.log1p(y) - y / (1.0 + y)


def test_nfw_half_mass_radius_and_vmax():
    u, n200, c = 8192, 200000, 8.0
    centre = (BOX // 2, 17, BOX // 7)
    pos, ids, meta = synth.nfw_halo(n200, c, u, centre, xmax=1.0, seed=21)
    n, r200 = meta["n"], meta["r200"]
    r = O.radial(pos, np.full(n, 3, np.uint64), row(3, n, centre), float(u))[0]
    # half-mass radius: mu(c x) = mu(c) / 2 (bisection on the closed form)
    lo, hi = 0.0, 1.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if _mu(c * mid) < 0.5 * _mu(c) else (lo, mid)
    assert abs(r["r_q"][1] / (lo * r200) - 1) < 0.02
    # V_max^2 = N c mu(x*) / (mu(c) x* R200) at x* = 2.16258 (units G m_p = 1, l_mean)
    xs = 2.16258
    v2 = n * c * _mu(xs) / (_mu(c) * xs * r200)
    assert abs(r["vmax"] / math.sqrt(v2) - 1) < 0.01
    assert abs(r["r_vmax"] / (xs * r200 / c) - 1) < 0.15
    # the enclosed fractions are ordered and inside the truncation radius
    assert np.all(np.diff(r["d_q"]) >= 0) and r["r_q"][3] <= r200 * 1.0001
