"""Seeded synthetic particle sets for CompaSO (inputs only).

This module draws positions and ids; it contains none of the group finder's
arithmetic and is the one piece of code shared by the tests, the benchmark and
both sides of every parity check.

Positions live on a periodic grid of 2^21 units per side; a box of ``side``
mean interparticle spacings has u = 2^21 / side grid units per l_mean and
side^3 particles at the mean density.  Haloes are NFW profiles truncated at
R_200 (mean enclosed density 200 times the background), the profile used for
the fits of Sec. 4.2 of the paper (rho ~ 1 / [(r/r_s)(1 + r/r_s)^2]), with
concentrations 4-12 and power-law sizes dN/dN ~ N^-1.9.  Ids are the
generation index; the array order is a seeded shuffle.
"""
import math

import numpy as np

BOX = 1 << 21
FOUR_PI_3 = 4.0 * math.pi / 3.0


def _mu(y):
    return np.log1p(y) - y / (1.0 + y)


def nfw_unit_radii(rng, c, xmax=1.0):
    """Radii r / R_200 in [0, xmax] drawn from NFW profiles of concentration c
    (one draw per entry of c), by bisection on the enclosed-mass fraction."""
    c = np.asarray(c, np.float64)
    q = rng.random(c.size) * _mu(c * xmax)
    lo = np.zeros(c.size)
    hi = np.full(c.size, float(xmax))
    for _ in range(44):
        mid = 0.5 * (lo + hi)
        below = _mu(c * mid) < q
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi)


def isotropic(rng, n):
    z = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def r200(n):
    """R_200 in units of l_mean for a halo of n particles."""
    return (np.asarray(n, np.float64) / (200.0 * FOUR_PI_3)) ** (1.0 / 3.0)


def power_law_sizes(rng, nmin, nmax, slope, count):
    """`count` integer sizes with dN/dN ~ N^slope on [nmin, nmax] (inverse CDF)."""
    a = slope + 1.0
    r = rng.random(count)
    lo, hi = float(nmin) ** a, float(nmax) ** a
    return np.floor((lo + r * (hi - lo)) ** (1.0 / a)).astype(np.int64)


def _halo_points(rng, centres, sizes, conc, u):
    """Particles of NFW haloes: grid-unit float positions (not yet wrapped)."""
    k = np.repeat(np.arange(sizes.size), sizes)
    x = nfw_unit_radii(rng, conc[k])
    rad = x * r200(sizes)[k] * u
    return centres[k] + rad[:, None] * isotropic(rng, k.size)


def _draw_haloes(rng, budget, nmin, nmax, slope, sat_frac, sat_ratio, sat_offset, c_range):
    """Host sizes (and optional satellites) until `budget` particles are used.
    Returns lists (sizes, is_sat, host_index, ratio-offsets)."""
    sizes, conc, parent, offset = [], [], [], []
    used = 0
    done = False
    while not done:
        batch = power_law_sizes(rng, nmin, nmax, slope, 4096)
        cb = rng.uniform(c_range[0], c_range[1], 4096)
        has_sat = rng.random(4096) < sat_frac
        ratio = rng.uniform(sat_ratio[0], sat_ratio[1], 4096)
        off = rng.uniform(sat_offset[0], sat_offset[1], 4096)
        csat = rng.uniform(c_range[0], c_range[1], 4096)
        for t in range(4096):
            n = int(min(batch[t], budget - used))
            if n < nmin:
                done = True  # the remainder goes to the background
                break
            host = len(sizes)
            sizes.append(n); conc.append(cb[t]); parent.append(-1); offset.append(0.0)
            used += n
            if has_sat[t]:
                ns = min(int(round(ratio[t] * n)), budget - used)
                if ns >= nmin:
                    sizes.append(ns); conc.append(csat[t]); parent.append(host); offset.append(off[t])
                    used += ns
    return (np.asarray(sizes, np.int64), np.asarray(conc), np.asarray(parent, np.int64),
            np.asarray(offset))


def nfw_box(side, frac_bg, nmin, nmax, slope=-1.9, sat_frac=0.0, sat_ratio=(0.05, 0.3),
            sat_offset=(0.3, 1.5), c_range=(4.0, 12.0), seed=0, region=None, n_total=None):
    """A periodic box of `side` l_mean: uniform background plus NFW haloes.

    region: optional (lo, extent) in l_mean; the particles then fill only the
    cube [lo, lo + extent)^3 (wrapped), at the mean density, so that small
    cases keep the density contrasts of the full box.
    Returns (pos int32 [n, 3], ids uint64 [n], meta dict)."""
    if BOX % side:
        raise ValueError("side must divide 2^21")
    u = BOX // side
    rng = np.random.default_rng(seed)
    if region is None:
        lo, ext = 0.0, float(side)
    else:
        lo, ext = float(region[0]), float(region[1])
    n = int(n_total) if n_total is not None else int(round(ext ** 3))
    n_bg = int(round(frac_bg * n))
    sizes, conc, parent, offset = _draw_haloes(rng, n - n_bg, nmin, nmax, slope, sat_frac, sat_ratio,
                                               sat_offset, c_range)
    nh = sizes.size
    centres = (lo + rng.random((nh, 3)) * ext) * u
    sat = parent >= 0
    if sat.any():
        dirs = isotropic(rng, int(sat.sum()))
        hp = parent[sat]
        centres[sat] = centres[hp] + (offset[sat] * r200(sizes[hp]) * u)[:, None] * dirs
    pts = _halo_points(rng, centres, sizes, conc, u) if nh else np.zeros((0, 3))
    n_bg = n - int(sizes.sum())
    bg = (lo + rng.random((n_bg, 3)) * ext) * u
    allp = np.concatenate([pts, bg], axis=0)
    pos = np.mod(np.rint(allp).astype(np.int64), BOX).astype(np.int32)
    ids = np.arange(n, dtype=np.uint64)
    perm = rng.permutation(n)
    meta = dict(side=side, u=u, n=n, n_background=n_bg, n_haloes=int(nh), n_satellites=int(sat.sum()),
                halo_particles=int(sizes.sum()), seed=seed)
    return np.ascontiguousarray(pos[perm]), ids[perm], meta


def uniform_box(side, n, seed=0):
    """Poisson (uniform) particles in a box of `side` l_mean."""
    rng = np.random.default_rng(seed)
    pos = rng.integers(0, BOX, size=(n, 3), dtype=np.int64).astype(np.int32)
    return pos, np.arange(n, dtype=np.uint64), dict(side=side, u=BOX // side, n=n, seed=seed)


# Named workloads.  Each is the recipe of one benchmark or test case.
SEED0 = 20211021


def tiny(seed=SEED0):
    """Box 64 l_mean, 64^3 particles: half background, half in NFW haloes of
    20-20000 particles (slope -1.9, c in [4, 12]); haloes are drawn until half
    of the particles are used."""
    return nfw_box(64, 0.5, 20, 20000, seed=seed)


def medium(seed=SEED0 + 1):
    """Box 256 l_mean, 256^3 = 16.8M particles: 40% background, 60% in NFW
    haloes of 20-2e5 particles, 10% of hosts with an NFW satellite of mass
    ratio 0.05-0.3 at 0.3-1.5 R_200."""
    return nfw_box(256, 0.4, 20, 200000, sat_frac=0.1, seed=seed)


def medium_sample(side=128, seed=SEED0 + 11):
    """The medium recipe in a smaller periodic box (same densities and halo
    mixture): a bounded sample of that workload for CPU timing."""
    return nfw_box(side, 0.4, 20, 200000, sat_frac=0.1, seed=seed)


def patch(extent=16.0, lo=-8.0, side=64, frac_bg=0.5, nmin=20, nmax=2000, sat_frac=0.3, seed=1):
    """A small cube of a box at the mean density, straddling the periodic
    corner of the box by default: a few thousand particles for brute-force
    checks."""
    return nfw_box(side, frac_bg, nmin, nmax, sat_frac=sat_frac, seed=seed, region=(lo, extent))


def sis_ball(A, R, u, centre, seed=0):
    """A singular isothermal sphere rho = A / r^2 (l_mean units, unit particle
    mass) truncated at R: M(<r) = 4 pi A r, so r / R is uniform."""
    rng = np.random.default_rng(seed)
    n = int(round(4.0 * math.pi * A * R))
    r = R * rng.random(n) * u
    pts = np.asarray(centre, np.float64)[None, :] + r[:, None] * isotropic(rng, n)
    pos = np.mod(np.rint(pts).astype(np.int64), BOX).astype(np.int32)
    return pos, np.arange(n, dtype=np.uint64), dict(n=n, u=u)


def nfw_halo(n200, c, u, centre, xmax=1.0, seed=0, id0=0):
    """One NFW halo with n200 particles inside R_200, sampled out to xmax R_200."""
    rng = np.random.default_rng(seed)
    n = int(round(n200 * _mu(c * xmax) / _mu(c)))
    x = nfw_unit_radii(rng, np.full(n, float(c)), xmax)
    pts = np.asarray(centre, np.float64)[None, :] + (x * r200(n200) * u)[:, None] * isotropic(rng, n)
    pos = np.mod(np.rint(pts).astype(np.int64), BOX).astype(np.int32)
    return pos, np.arange(id0, id0 + n, dtype=np.uint64), dict(n=n, u=u, r200=float(r200(n200)))


def lattice_ball(a, k_max, centre):
    """Points of a cubic lattice of spacing a (grid units) within squared
    radius k_max a^2 of a lattice point at `centre`."""
    m = int(math.isqrt(k_max))
    r = np.arange(-m, m + 1)
    g = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    g = g[(g * g).sum(1) <= k_max]
    pos = np.mod(np.asarray(centre, np.int64)[None, :] + a * g, BOX).astype(np.int32)
    return pos, np.arange(len(pos), dtype=np.uint64), dict(n=len(pos))
