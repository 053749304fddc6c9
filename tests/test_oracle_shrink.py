"""Pins of the oracle's shrinking-sphere centre (Sec. 4; Power et al. 2003)
against what geometry fixes.

- A cubic lattice ball about a lattice point is symmetric: the centre of
  mass of every sphere about that point is the point itself, so the centre
  never moves, and the spheres' member counts (lattice points with
  |v|^2 a^2 < R2_i, enumerated) fix the number of steps and where it stops.
- A uniform ball with a dense clump off its centre: the spheres shrink onto
  the clump (the density maximum the method is meant to find).
- An NFW halo started from an off-centre member converges to the profile's
  centre.
- A halo below the stop count keeps its nucleus.
"""
import math

import numpy as np

import oracle as O
from paper_2110_11408_gb300 import synth

BOX = 1 << 21


def row(nucleus_id, n, R2):
    r = np.zeros(1, O.HALO_DTYPE)
    r["nucleus_id"] = nucleus_id
    r["N"] = n
    r["R2"] = R2
    return r


def mi(a):
    return (np.asarray(a, np.int64) + (1 << 20)) % BOX - (1 << 20)


def test_lattice_ball_stays_and_stops_where_counts_say():
    a, kmax = 64, 300
    C = np.array([BOX - 100, 50, BOX // 2], np.int64)
    g = np.arange(-18, 19)
    i, j, k = np.meshgrid(g, g, g, indexing="ij")
    s = (i * i + j * j + k * k).ravel()
    keep = s <= kmax
    off = np.stack([i.ravel()[keep], j.ravel()[keep], k.ravel()[keep]], 1) * a
    pos = ((C[None, :] + off) % BOX).astype(np.int32)
    s = s[keep]
    n = len(pos)
    ids = np.arange(10, 10 + n, dtype=np.uint64)
    nuc = int(ids[np.flatnonzero(s == 0)[0]])
    R2 = (kmax + 1) * a * a
    r = O.shrink_sphere(pos, ids, np.full(n, nuc, np.uint64), row(nuc, n, R2))[0]
    assert tuple(r["centre"]) == tuple(C)
    # expected steps: counts of lattice points strictly inside each sphere
    stop = max(-(-n // 100), O.SHRINK_N_MIN)
    R2i, it = R2, 0
    while True:
        m = int((s * a * a < R2i).sum())
        if m < stop:
            break
        R2i = R2i * 9025 // 10000
        it += 1
    assert (r["iter"], r["n"], r["R2"]) == (it, m, R2i)
    assert it > 10


def test_converges_onto_a_dense_clump():
    rng = np.random.default_rng(4)
    u = 8192
    R = 12.0 * u
    centre = np.array([BOX // 3, BOX // 4, BOX - 5000], np.float64)
    # uniform ball of 40000 particles
    v = rng.normal(size=(40000, 3))
    v *= (R * rng.random(40000) ** (1 / 3) / np.linalg.norm(v, axis=1))[:, None]
    ball = centre + v
    # dense clump: an NFW halo of 8000 particles at 0.5 R from the centre
    clump_c = centre + np.array([0.5 * R, 0.0, 0.0])
    cp, _, _ = synth.nfw_halo(8000, 10.0, u, clump_c, xmax=1.0, seed=5)
    pos = np.concatenate([np.mod(np.rint(ball), BOX).astype(np.int32), cp])
    n = len(pos)
    ids = np.arange(n, dtype=np.uint64)
    r = O.shrink_sphere(pos, ids, np.zeros(n, np.uint64), row(0, n, int((R * 1.01) ** 2)))[0]
    d = np.sqrt((mi(r["centre"] - np.rint(clump_c)) ** 2).sum()) / u
    assert d < 0.1, d  # l_mean units; the clump's R_200 is about 2.1
    assert r["iter"] > 10


def test_nfw_centre_from_an_off_centre_nucleus():
    u, n200, c = 8192, 100000, 8.0
    C = np.array([17, BOX // 2, BOX // 5], np.int64)
    pos, ids, meta = synth.nfw_halo(n200, c, u, C, xmax=1.0, seed=12)
    n = meta["n"]
    r200 = meta["r200"] * u
    d0 = np.sqrt((mi(pos.astype(np.int64) - C) ** 2).sum(1))
    k = int(np.argmin(np.abs(d0 - 0.3 * r200)))  # a member at 0.3 R_200
    nuc = int(ids[k])
    R2 = int((1.3 * r200) ** 2)  # the sphere about the nucleus holds the halo
    r = O.shrink_sphere(pos, ids, np.full(n, nuc, np.uint64), row(nuc, n, R2))[0]
    off = np.sqrt((mi(r["centre"] - C) ** 2).sum()) / r200
    assert off < 0.01, off
    assert r["n"] < max(-(-n // 100), O.SHRINK_N_MIN) and r["iter"] > 20


def test_small_halo_keeps_its_nucleus():
    u = 8192
    pos, ids, meta = synth.nfw_halo(300, 6.0, u, (1000, 2000, 3000), seed=3)
    n = meta["n"]
    nuc = int(ids[7])
    r = O.shrink_sphere(pos, ids, np.full(n, nuc, np.uint64), row(nuc, n, 10 ** 12))[0]
    assert tuple(r["centre"]) == tuple(pos[7]) and r["iter"] == 0 and r["n"] == n
