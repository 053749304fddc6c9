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


# --------------------------------------------------------------------------
# pre-formed groups (the batched workload)
# --------------------------------------------------------------------------

def group_sizes_particle_weighted(rng, nmin, nmax, total, giant=None):
    """Group sizes with equal numbers of particles per logarithmic size
    interval on [nmin, nmax] (dN/dN ~ N^-2), drawn until `total` particles
    are used; `giant` (if given) is the first group.  The last group takes the
    remainder if that is at least nmin (else the remainder is dropped)."""
    sizes = [int(giant)] if giant else []
    used = sum(sizes)
    a, b = 1.0 / nmin, 1.0 / nmax
    while used < total:
        q = rng.random(4096)
        for n in np.floor(1.0 / (a - q * (a - b))).astype(np.int64):
            n = int(min(n, total - used))
            if n < nmin:
                return np.asarray(sizes, np.int64)
            sizes.append(n)
            used += n
            if used >= total:
                break
    return np.asarray(sizes, np.int64)


def _place_spheres(rng, radii, side):
    """Centres (l_mean units) of non-overlapping spheres of the given radii in
    a periodic box, placed largest first by rejection; candidates are checked
    against the spheres registered in the hash cells their bounding box
    covers."""
    order = np.argsort(-radii, kind="stable")
    h = max(2.0 * float(np.median(radii)), 1e-3)
    nh = max(1, int(side // h))
    h = side / nh
    table = {}
    cen = np.zeros((radii.size, 3))

    def cells(c, r):
        lo = np.floor((c - r) / h).astype(np.int64)
        hi = np.floor((c + r) / h).astype(np.int64)
        for x in range(lo[0], hi[0] + 1):
            for y in range(lo[1], hi[1] + 1):
                for z in range(lo[2], hi[2] + 1):
                    yield (x % nh, y % nh, z % nh)

    for i in order:
        r = radii[i]
        for _ in range(10000):
            c = rng.random(3) * side
            near = {j for key in cells(c, r) for j in table.get(key, ())}
            if near:
                js = np.fromiter(near, np.int64)
                d = np.abs(cen[js] - c)
                d = np.minimum(d, side - d)
                if (np.einsum("ij,ij->i", d, d) < (radii[js] + r) ** 2).any():
                    continue
            break
        else:
            raise RuntimeError("cannot place group %d" % i)
        cen[i] = c
        for key in cells(c, r):
            table.setdefault(key, []).append(i)
    return cen


def preformed_groups(side, sizes, max_subs, sub_ratio, c_range=(4.0, 12.0), sub_offset=(0.2, 0.9), margin=0.5,
                     seed=0, min_sub=20):
    """Isolated groups in a periodic box of `side` l_mean (no background).

    Group k has sizes[k] particles: an NFW host truncated at its R_200 and
    0..max_subs NFW subhaloes, each with a mass ratio uniform in sub_ratio
    relative to the host, placed inside the host at sub_offset R_200
    (isotropic), truncated at their own R_200.  Groups sit on non-overlapping
    spheres separated by `margin` l_mean (more than b and l_FoF), so no pair
    of particles of two groups is within reach of the kernel or the linking
    length.  Returns (pos int32 [n, 3], ids uint64 [n], meta)."""
    if BOX % side:
        raise ValueError("side must divide 2^21")
    u = BOX // side
    rng = np.random.default_rng(seed)
    G = sizes.size
    nsub = rng.integers(0, max_subs + 1, G) if max_subs > 0 else np.zeros(G, np.int64)
    comp_n, comp_c, comp_g, comp_off = [], [], [], []
    ext = np.zeros(G)
    for g in range(G):
        ratios = rng.uniform(sub_ratio[0], sub_ratio[1], nsub[g]) if nsub[g] else np.zeros(0)
        host = int(round(sizes[g] / (1.0 + ratios.sum())))
        subs = [int(round(r * host)) for r in ratios]
        subs = [s for s in subs if s >= min_sub]
        host = int(sizes[g] - sum(subs))
        rh = float(r200(host))
        e = rh
        comp_n.append(host); comp_c.append(rng.uniform(*c_range)); comp_g.append(g); comp_off.append(np.zeros(3))
        for s in subs:
            off = rng.uniform(*sub_offset) * rh * isotropic(rng, 1)[0]
            comp_n.append(s); comp_c.append(rng.uniform(*c_range)); comp_g.append(g); comp_off.append(off)
            e = max(e, float(np.linalg.norm(off)) + float(r200(s)))
        ext[g] = e + 0.5 * margin
    centres = _place_spheres(rng, ext, side)
    comp_n = np.asarray(comp_n, np.int64)
    comp_g = np.asarray(comp_g, np.int64)
    cc = (centres[comp_g] + np.asarray(comp_off)) * u
    pts = _halo_points(rng, cc, comp_n, np.asarray(comp_c), u)
    n = int(comp_n.sum())
    pos = np.mod(np.rint(pts).astype(np.int64), BOX).astype(np.int32)
    ids = np.arange(n, dtype=np.uint64)
    perm = rng.permutation(n)
    meta = dict(side=side, u=u, n=n, groups=int(G), components=int(comp_n.size), largest=int(sizes.max()),
                seed=seed)
    return np.ascontiguousarray(pos[perm]), ids[perm], meta


def batched(seed=SEED0 + 3, total=4_000_000, giant=2_000_000):
    """About 4M particles as pre-formed groups of uneven size in a box of side
    256 l_mean: sizes with equal particles per logarithmic interval on
    [35, 2e6] and one forced group of 2e6, each group an NFW host plus 0-5
    NFW subhaloes of mass ratio 0.01-0.3."""
    rng = np.random.default_rng(seed)
    sizes = group_sizes_particle_weighted(rng, 35, 2_000_000, total, giant=giant)
    return preformed_groups(256, sizes, 5, (0.01, 0.3), seed=seed + 1)


def batched_many(seed=SEED0 + 4, groups=100_000):
    """100,000 small pre-formed groups (single NFW haloes of 35-45 particles,
    about 4M particles) in a box of side 256 l_mean."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(35, 46, groups)
    return preformed_groups(256, sizes, 0, (0.0, 0.0), seed=seed + 1)


# --------------------------------------------------------------------------
# boxes delivered as x-slabs (the served workloads)
# --------------------------------------------------------------------------

def nfw_unit_radii_closed(q, c):
    """Radii r / R_200 of NFW profiles of concentration c at enclosed-mass
    fractions q * mu(c), by the closed-form inverse of mu(y) = ln(1 + y) -
    y / (1 + y): with t = 1 / (1 + y), t - ln t = 1 + m, so
    t = -W0(-exp(-1 - m)) (principal branch of Lambert's W)."""
    from scipy.special import lambertw
    c = np.asarray(c, np.float64)
    m = np.asarray(q, np.float64) * _mu(c)
    t = -lambertw(-np.exp(-1.0 - m), 0).real
    return (1.0 / t - 1.0) / c


class SlabBox:
    """A periodic box of `side` l_mean of the NFW-halo recipe (uniform
    background plus NFW haloes with optional satellites, as nfw_box), cut
    into x-slabs at the grid coordinates `edges` (0 = edges[0] < ... <
    edges[-1] = 2^21) and generated slab by slab with bounded memory.

    The halo catalogue (sizes, concentrations, centres) is drawn first.  The
    haloes whose centre lies in slab j form chunk j; a chunk's particles are
    drawn from a generator seeded by (seed, j), so any chunk can be made in any
    order (or in another process) and gives the same particles, which are
    routed to the slabs they fall in.  Background particles of slab k come
    from a generator seeded by (seed, k).  Ids: halo particles are numbered
    chunk by chunk, then the background slab by slab.  NFW radii use the
    closed-form inverse of the mass fraction."""

    def __init__(self, side, frac_bg, nmin, nmax, edges, slope=-1.9, sat_frac=0.1, sat_ratio=(0.05, 0.3),
                 sat_offset=(0.3, 1.5), c_range=(4.0, 12.0), seed=0):
        if BOX % side:
            raise ValueError("side must divide 2^21")
        self.side, self.u, self.seed = side, BOX // side, seed
        self.edges = np.asarray(edges, np.int64)
        assert self.edges[0] == 0 and self.edges[-1] == BOX and np.all(np.diff(self.edges) > 0)
        self.nslab = self.edges.size - 1
        n = side ** 3
        self.n = n
        rng = np.random.default_rng(seed)
        sizes, conc, parent, offset = _draw_haloes(rng, n - int(round(frac_bg * n)), nmin, nmax, slope, sat_frac,
                                                   sat_ratio, sat_offset, c_range)
        nh = sizes.size
        centres = rng.random((nh, 3)) * side
        sat = parent >= 0
        if sat.any():
            dirs = isotropic(rng, int(sat.sum()))
            hp = parent[sat]
            centres[sat] = centres[hp] + (offset[sat] * r200(sizes[hp]))[:, None] * dirs
        centres = np.mod(centres, side)
        self.sizes, self.conc, self.centres = sizes, conc, centres * self.u  # centres in grid units
        self.n_halo = int(sizes.sum())
        self.n_bg = n - self.n_halo
        # chunks: haloes by the slab holding their centre
        cx = self.centres[:, 0]
        self.chunk_of = np.clip(np.searchsorted(self.edges, cx, side="right") - 1, 0, self.nslab - 1)
        order = np.argsort(self.chunk_of, kind="stable")
        self.halo_order = order
        self.chunk_start = np.searchsorted(self.chunk_of[order], np.arange(self.nslab + 1))
        pc = np.zeros(self.nslab + 1, np.int64)
        np.add.at(pc, self.chunk_of + 1, sizes)
        self.chunk_id0 = np.cumsum(pc)  # first id of each chunk
        # the slabs a chunk can reach (haloes extend at most R_200 from their centre)
        ext = r200(sizes) * self.u
        self.chunk_reach = []
        for j in range(self.nslab):
            hs = order[self.chunk_start[j]:self.chunk_start[j + 1]]
            if hs.size == 0:
                self.chunk_reach.append(())
                continue
            lo = float((cx[hs] - ext[hs]).min()) - 2.0
            hi = float((cx[hs] + ext[hs]).max()) + 2.0
            self.chunk_reach.append(tuple(sorted(self._slabs_in(lo, hi))))
        self.needs = [[] for _ in range(self.nslab)]
        for j, ks in enumerate(self.chunk_reach):
            for k in ks:
                self.needs[k].append(j)
        width = np.diff(self.edges).astype(np.float64)
        bg = np.floor(self.n_bg * width / BOX).astype(np.int64)
        bg[-1] += self.n_bg - int(bg.sum())
        self.bg_count = bg
        self.bg_id0 = self.n_halo + np.concatenate([[0], np.cumsum(bg)])

    def _slabs_in(self, lo, hi):
        """Slabs meeting the x interval [lo, hi) (grid units, may wrap)."""
        out = set()
        for a, b in ((lo, hi), (lo + BOX, hi + BOX), (lo - BOX, hi - BOX)):
            a, b = max(a, 0.0), min(b, float(BOX))
            if a >= b:
                continue
            k0 = int(np.searchsorted(self.edges, a, side="right") - 1)
            k1 = int(np.searchsorted(self.edges, b, side="left"))
            out.update(range(max(k0, 0), min(k1, self.nslab)))
        return out

    def chunk(self, j):
        """Particles of the haloes of chunk j: {slab: (pos int32 [m, 3], ids uint64 [m])}."""
        hs = self.halo_order[self.chunk_start[j]:self.chunk_start[j + 1]]
        if hs.size == 0:
            return {}
        rng = np.random.default_rng([self.seed, 1, j])
        sizes = self.sizes[hs]
        k = np.repeat(np.arange(hs.size), sizes)
        x = nfw_unit_radii_closed(rng.random(k.size), self.conc[hs][k])
        rad = x * r200(sizes)[k] * self.u
        pts = self.centres[hs][k] + rad[:, None] * isotropic(rng, k.size)
        pos = np.mod(np.rint(pts).astype(np.int64), BOX).astype(np.int32)
        ids = np.uint64(self.chunk_id0[j]) + np.arange(k.size, dtype=np.uint64)
        dest = np.searchsorted(self.edges, pos[:, 0], side="right") - 1
        out = {}
        for s in np.unique(dest):
            m = dest == s
            out[int(s)] = (pos[m], ids[m])
        return out

    def background(self, k):
        rng = np.random.default_rng([self.seed, 2, k])
        m = int(self.bg_count[k])
        x = rng.integers(self.edges[k], self.edges[k + 1], m)
        yz = rng.integers(0, BOX, (m, 2))
        pos = np.column_stack([x, yz]).astype(np.int32)
        return pos, np.uint64(self.bg_id0[k]) + np.arange(m, dtype=np.uint64)

    def slabs(self, workers=1, shuffle_seed=None):
        """Yield (k, pos, ids) for k = 0 .. nslab - 1, in order.  workers > 1
        draws chunks in a pool of spawned processes, a few slabs ahead."""
        pending = {}  # slab -> list of (pos, ids)
        done = set()
        pool = None
        futs = {}
        if workers > 1:
            import concurrent.futures as cf
            import multiprocessing as mp
            pool = cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))

        def submit(j):
            if j in done or j in futs:
                return
            futs[j] = pool.submit(_slab_box_chunk, self, j) if pool else None

        try:
            for k in range(self.nslab):
                if pool:
                    for kk in range(k, min(k + 2 * workers, self.nslab)):
                        for j in self.needs[kk]:
                            submit(j)
                for j in self.needs[k]:
                    if j in done:
                        continue
                    parts = futs.pop(j).result() if (pool and j in futs) else self.chunk(j)
                    futs.pop(j, None)
                    done.add(j)
                    for s, v in parts.items():
                        pending.setdefault(s, []).append(v)
                bp, bi = self.background(k)
                got = pending.pop(k, [])
                pos = np.concatenate([bp] + [p for p, _ in got])
                ids = np.concatenate([bi] + [i for _, i in got])
                if shuffle_seed is not None:
                    perm = np.random.default_rng([shuffle_seed, k]).permutation(len(pos))
                    pos, ids = pos[perm], ids[perm]
                yield k, np.ascontiguousarray(pos), ids
        finally:
            if pool:
                pool.shutdown(wait=True, cancel_futures=True)


def _slab_box_chunk(box, j):
    return box.chunk(j)


def served512(seed=SEED0 + 5):
    """Box 512 l_mean, 512^3 = 134M particles: 40% background, 60% in NFW
    haloes of 20-2e6 particles (slope -1.9), 10% with satellites, delivered
    as 64 x-slabs of 8 l_mean (~2.1M particles each)."""
    edges = [BOX * k // 64 for k in range(65)]
    return SlabBox(512, 0.4, 20, 2_000_000, edges, seed=seed)


def served1024_edges(seed=SEED0 + 6):
    """x-slab edges of the side-1024 stream: the 512 columns of 2 l_mean are
    cut into 256 slabs of 1-4 columns by a seeded composition."""
    rng = np.random.default_rng(seed)
    parts = np.full(256, 2, np.int64)  # 512 columns; seeded moves of one column keep the sum and the range
    src = rng.integers(0, 256, 8192)
    dst = rng.integers(0, 256, 8192)
    for i, j in zip(src, dst):
        if i != j and parts[i] > 1 and parts[j] < 4:
            parts[i] -= 1
            parts[j] += 1
    cols = np.concatenate([[0], np.cumsum(parts)])
    return [int(c) * (BOX // 512) for c in cols]


def served1024(seed=SEED0 + 7):
    """Box 1024 l_mean, 1024^3 = 1.07e9 particles (12.9 GB of positions): the
    same mixture with haloes up to 1e7 particles, delivered as 256 x-slabs of
    1-4 columns of 2 l_mean."""
    return SlabBox(1024, 0.4, 20, 10_000_000, served1024_edges(), seed=seed)
