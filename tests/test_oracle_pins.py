"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these compares the oracle with itself: each checks it against a
closed form printed in the paper (App. B.2), a textbook or library routine
(exact rational arithmetic, scipy connected components, numerical
quadrature, lattice shell counts), a geometric statement of the competitive
rule (Sec. 2.2.2 step 3, Eq. 3), or brute force on tiny inputs.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate, special
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import oracle as O
from paper_2110_11408_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
BOX = 1 << 21
U64 = 32768  # grid units per l_mean in a box of 64 l_mean


def mi(a):
    a = np.asarray(a, np.int64)
    return (a + (1 << 20)) % BOX - (1 << 20)


def brute_d2(pos):
    p = pos.astype(np.int64)
    d = np.zeros((len(p), len(p)), np.int64)
    for a in range(3):
        x = mi(p[:, None, a] - p[None, :, a])
        d += x * x
    return d


# --------------------------------------------------------------------------
# derived thresholds (Sec. 2.2.1, Sec. 2.2.2 step 4, App. B.2)
# --------------------------------------------------------------------------

def test_sis_central_density_matches_quadrature():
    """Step 4's stop level is the kernel density at the centre of an SIS of 35
    particles inside the radius enclosing Delta times the mean; check the
    closed form 5A/b^2 against direct quadrature of the kernel-weighted SIS
    normalised by the kernel volume (2/5)(4pi/3) b^3 (App. B.2)."""
    L = O.lib()
    for delta in (200.0, 800.0, 258.2):
        b = 0.4
        R = (35.0 / (delta * 4.0 * math.pi / 3.0)) ** (1.0 / 3.0)
        A = 35.0 / (4.0 * math.pi * R)  # M(<R) = 4 pi A R = 35
        num, _ = integrate.quad(lambda r: (1 - r * r / (b * b)) * A / (r * r) * 4 * math.pi * r * r, 0, b)
        den = 0.4 * 4.0 * math.pi / 3.0 * b ** 3
        got = L.orc_sis_central_density(35.0, delta, b)
        assert got == pytest.approx(num / den, rel=1e-9)
    assert L.orc_sis_central_density(35.0, 200.0, 0.4) == pytest.approx(250.84, abs=0.01)


def test_sis_r200m_worked_example():
    """App. B.2: an SIS with N_200m = 40 has R_200m ~ 0.36 l_mean."""
    g = GOLD["sis_r200m_for_n40"]
    assert (g["n"] / (200 * 4 * math.pi / 3)) ** (1 / 3) == pytest.approx(g["value"], abs=0.005)


def test_derived_integers():
    p = O.params(U64)
    assert p.b2 == round((0.4 * U64) ** 2)
    assert p.lfof2 == (U64 // 4) ** 2
    # dense <=> Delta > 60 with Delta = Sigma / (b2 (2/5)(4pi/3) (b/l)^3)
    nbar_unit = 0.4 * 4 * math.pi / 3 * (math.sqrt(p.b2) / U64) ** 3
    assert p.T_L0 == math.floor(60 * nbar_unit * p.b2) or abs(p.T_L0 - 60 * nbar_unit * p.b2) < 2
    assert p.T_min_L1 > p.T_L0 and p.T_min_L2 > p.T_min_L1


# --------------------------------------------------------------------------
# density (Sec. 2.2.1, Eq. 1; App. B.2)
# --------------------------------------------------------------------------

def test_density_brute_force_patch_across_periodic_corner():
    pos, ids, _ = synth.patch(extent=12.0, lo=-6.0, seed=3)
    p = O.params(U64)
    d = brute_d2(pos)
    np.fill_diagonal(d, np.iinfo(np.int64).max)
    expect = np.where(d < p.b2, p.b2 - d, 0).sum(1)
    got, pairs = O.density(pos, p)
    assert np.array_equal(got, expect)
    assert pairs == int((d < p.b2).sum())
    got_b, _ = O.density(pos, p, brute=True)
    assert np.array_equal(got_b, expect)


def test_density_include_self_adds_exactly_b2():
    pos, ids, _ = synth.patch(extent=8.0, lo=20.0, seed=4)
    p0 = O.params(U64)
    p1 = O.params(U64, include_self=1)
    s0, _ = O.density(pos, p0)
    s1, _ = O.density(pos, p1)
    assert np.array_equal(s1 - s0, np.full(len(pos), p0.b2))


@pytest.mark.parametrize("delta,golden", [(1.0, None), (60.0, "uniform_count_at_delta60")])
def test_density_uniform_field_mean_and_variance(delta, golden):
    """App. B.2: in a uniform field of density Delta the kernel count has mean
    N = (2/5)(4pi/3) b^3 Delta and variance (4/7) N."""
    side = 64
    u = BOX // side
    if delta == 1.0:
        pos, _, _ = synth.uniform_box(side, 262144, seed=7)
    else:
        # density 60 inside a cube of 10 l_mean, measured away from its faces
        rng = np.random.default_rng(8)
        n = int(60 * 10 ** 3)
        pos = (rng.random((n, 3)) * 10 * u).astype(np.int32) + 4 * u
    p = O.params(u)
    sig, _ = O.density(pos, p)
    W = sig / p.b2
    if delta == 60.0:
        x = pos.astype(np.int64) - 4 * u
        inner = np.all((x > u) & (x < 9 * u), axis=1)
        W = W[inner]
    b = math.sqrt(p.b2) / u
    nbar = 0.4 * 4 * math.pi / 3 * b ** 3 * delta
    assert W.mean() == pytest.approx(nbar, rel=0.02)
    assert W.var() / nbar == pytest.approx(GOLD["uniform_var_over_mean"]["value"], rel=0.05)
    if golden:
        assert nbar == pytest.approx(GOLD[golden]["value"], abs=0.05)


def sis_ratio_closed_form(x):
    """App. B.2: smoothed SIS over true SIS density at r = x b."""
    if x > 1:
        return special.hyp2f1(1, 0.5, 3.5, 1 / x ** 2)
    return 5 * x ** 2 * special.hyp2f1(1, -1.5, 1.5, x ** 2)


def test_sis_closed_form_matches_printed_numbers():
    assert sis_ratio_closed_form(1.0 - 1e-12) == pytest.approx(GOLD["sis_ratio_at_b"]["value"], abs=0.01)
    xs = np.linspace(0.3, 3, 2701)
    r = np.array([sis_ratio_closed_form(x) for x in xs])
    assert r.max() == pytest.approx(GOLD["sis_ratio_peak"]["value"], abs=0.02)
    assert xs[r.argmax()] == pytest.approx(GOLD["sis_ratio_peak"]["r_over_b"], abs=0.05)
    cross = xs[np.argmax(r > 1)]
    assert cross == pytest.approx(GOLD["sis_ratio_unity_crossing"]["r_over_b"], abs=0.015)


def test_density_of_sis_follows_smoothed_profile():
    """Kernel densities of particles in a dense SIS follow App. B.2's
    convolution of the SIS with W: ratio 1.25 at b, ~1.45 near 0.8 b."""
    u = U64
    A = 655.0
    R = 1.6
    c = np.array([BOX // 2] * 3, np.float64)
    pos, ids, meta = synth.sis_ball(A, R, u, c, seed=11)
    p = O.params(u)
    sig, _ = O.density(pos, p)
    b = math.sqrt(p.b2) / u
    nb = 0.4 * 4 * math.pi / 3 * b ** 3
    r = np.sqrt(((pos - c) ** 2).sum(1)) / u
    for x in (0.5, 0.8, 1.0, 1.5, 2.0):
        sel = np.abs(r / b - x) < 0.04
        ratio = (sig[sel] / p.b2 / nb) / (A / r[sel] ** 2)
        assert ratio.mean() == pytest.approx(sis_ratio_closed_form(x), rel=0.03), x


# --------------------------------------------------------------------------
# L0: modified FoF (Sec. 2.2.1)
# --------------------------------------------------------------------------

def test_fof_matches_connected_components():
    pos, ids, _ = synth.patch(extent=14.0, lo=-7.0, seed=5, frac_bg=0.3)
    p = O.params(U64)
    sig, _ = O.density(pos, p)
    l0, links = O.fof(pos, ids, sig, p)
    dense = sig > p.T_L0
    d = brute_d2(pos)
    adj = (d < p.lfof2) & dense[:, None] & dense[None, :]
    np.fill_diagonal(adj, False)
    assert links == int(adj.sum())
    ii, jj = np.nonzero(adj)
    g = coo_matrix((np.ones(ii.size), (ii, jj)), shape=(len(pos), len(pos)))
    ncomp, comp = connected_components(g, directed=False)
    expect = np.full(len(pos), O.NONE, np.uint64)
    for cidx in np.unique(comp[dense]):
        m = dense & (comp == cidx)
        expect[m] = ids[m].min()
    assert np.array_equal(l0, expect)
    l0b, _ = O.fof(pos, ids, sig, p, brute=True)
    assert np.array_equal(l0b, expect)


def test_fof_all_dense_is_plain_fof():
    """With the density cut at zero every particle is dense: plain FoF."""
    pos, ids, _ = synth.patch(extent=10.0, lo=3.0, seed=6)
    p = O.params(U64, delta_L0=-1.0)
    sig, _ = O.density(pos, p)
    l0, _ = O.fof(pos, ids, sig, p)
    d = brute_d2(pos)
    adj = d < p.lfof2
    np.fill_diagonal(adj, False)
    _, comp = connected_components(coo_matrix(adj), directed=False)
    for cidx in np.unique(comp):
        m = comp == cidx
        assert np.all(l0[m] == ids[m].min())


# --------------------------------------------------------------------------
# threshold radius search (Sec. 2.2.2 step 1, Sec. 2.3.3)
# --------------------------------------------------------------------------

def test_exact_predicate_against_rationals():
    rng = np.random.default_rng(1)
    p = O.params(U64)
    for K in (p.K_L1, p.K_L2, 3.0, 1e-3):
        Kf = Fraction(K)
        for _ in range(300):
            n = int(rng.integers(0, 1 << 24))
            # put d^3 near the boundary n^2 u^6 / K
            d0 = (n * n * U64 ** 6 / K) ** (1 / 3) if n else 0.0
            d = max(0, int(d0) + int(rng.integers(-2, 3)))
            want = n * n * U64 ** 6 < Kf * d ** 3
            assert O.pred(n, d, K, U64) == want, (n, d, K)


# lattice shell multiplicities r_3(k): number of integer vectors with |v|^2 = k
def r3(kmax):
    m = int(math.isqrt(kmax))
    r = np.arange(-m, m + 1)
    g = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    return np.bincount((g * g).sum(1), minlength=kmax + 1)[: kmax + 1]


def test_r3_is_textbook_sequence():
    # number of representations of k as a sum of three squares (k = 0..10)
    assert list(r3(10)) == [1, 6, 12, 8, 6, 24, 24, 0, 12, 30, 24]


@pytest.mark.parametrize("a_frac", [0.05, 0.08, 0.12, 0.3])
def test_r_search_on_cubic_lattice(a_frac):
    """Nucleus at a lattice point: the enclosed count just inside k a^2 is the
    sum of r_3(j) for j < k, so R^2 is the first occupied shell k a^2 with
    (sum_{j<k} r_3(j))^2 u^6 < K (k a^2)^3."""
    u = U64
    a = int(a_frac * u)
    kmax = 60
    pos, ids, _ = synth.lattice_ball(a, kmax, [BOX // 2] * 3)
    p = O.params(u)
    d = ((pos.astype(np.int64) - BOX // 2) ** 2).sum(1)
    got = O.r_search(d, p.K_L1, u)
    counts = r3(kmax)
    K = Fraction(p.K_L1)
    enclosed = 0
    want = None
    for k in range(kmax + 1):
        if counts[k] and k > 0 and enclosed ** 2 * u ** 6 < K * (k * a * a) ** 3:
            want = k * a * a
            break
        enclosed += int(counts[k])
    if want is None:  # exhaustion: smallest D beyond the last shell with N^2 u^6 < K D^3
        N = int(counts.sum())
        want = int((Fraction(N * N * u ** 6) / K) ** Fraction(1, 3)) - 2
        while not (N * N * u ** 6 < K * want ** 3 and want > int(d.max())):
            want += 1
    assert got == want


def test_r_search_exhaustion_closed_form():
    """A top-hat denser than Delta everywhere: R^3 = N / (Delta 4pi/3) beyond
    its edge (enclosed count fixed at N)."""
    u = U64
    pos, _, _ = synth.lattice_ball(int(0.05 * u), 30, [0, 0, 0])
    p = O.params(u)
    d = (mi(pos.astype(np.int64)) ** 2).sum(1)
    N = len(pos)
    got = O.r_search(d, p.K_L1, u)
    r_closed = (N / (200 * 4 * math.pi / 3)) ** (1 / 3) * u
    assert got > d.max()
    assert math.sqrt(got) == pytest.approx(r_closed, abs=1.0)


def test_isolated_nfw_recovers_r200():
    """An isolated NFW halo (c = 6, 20000 particles inside R_200, sampled to
    2 R_200) in one L0 group: R_L1 at Delta = 200 is R_200 up to Poisson noise."""
    u = U64
    c = [BOX // 2] * 3
    pos, ids, meta = synth.nfw_halo(20000, 6.0, u, c, xmax=2.0, seed=21)
    p = O.params(u, np_min_L1=1)
    sig, _ = O.density(pos, p)
    l0 = np.zeros(len(pos), np.uint64)
    l1, l2, halos, st = O.compaso(pos, ids, sig, l0, p)
    h = halos[np.argmax(halos["N"])]
    assert math.sqrt(h["R2"]) / u == pytest.approx(meta["r200"], rel=0.02)


# --------------------------------------------------------------------------
# competitive assignment, eligibility, nesting (Sec. 2.2.2 steps 1-3, Eq. 3)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def two_haloes():
    u = U64
    c0 = np.array([BOX // 2] * 3, np.float64)
    host, hid, hm = synth.nfw_halo(6000, 5.0, u, c0, xmax=1.3, seed=31)
    off = np.array([0.93 * hm["r200"] * u, 0.0, 0.0])
    sat, sid, sm = synth.nfw_halo(700, 9.0, u, c0 + off, xmax=1.0, seed=32, id0=len(host))
    pos = np.concatenate([host, sat])
    ids = np.concatenate([hid, sid])
    p = O.params(u, np_min_L1=1)
    r = O.find_groups(pos, ids, p)
    return pos, ids, p, r


def test_two_haloes_deblend_by_apollonius_rule(two_haloes):
    """For two nuclei A (first) and B (later) of one group, a particle inside
    both spheres and no other belongs to B iff R_B^2 d_A >= c R_A^2 d_B."""
    pos, ids, p, r = two_haloes
    H = r["halos"]
    order = np.argsort(-H["N"])
    A, B = H[order[0]], H[order[1]]
    assert A["l0_id"] == B["l0_id"]
    P = pos.astype(np.int64)
    pa = P[ids == A["nucleus_id"]][0]
    pb = P[ids == B["nucleus_id"]][0]
    others = [P[ids == h["nucleus_id"]][0] for h in H if h["nucleus_id"] not in (A["nucleus_id"], B["nucleus_id"])]
    oR2 = [int(h["R2"]) for h in H if h["nucleus_id"] not in (A["nucleus_id"], B["nucleus_id"])]
    dA = (mi(P - pa) ** 2).sum(1)
    dB = (mi(P - pb) ** 2).sum(1)
    RA, RB = int(A["R2"]), int(B["R2"])
    checked = 0
    for i in range(len(P)):
        if not (dA[i] < RA and dB[i] < RB) or r["l0"][i] != A["l0_id"]:
            continue
        if any(int((mi(P[i] - q) ** 2).sum()) < R2 for q, R2 in zip(others, oR2)):
            continue
        in_b = RB * int(dA[i]) * p.roche_den >= p.roche_num * RA * int(dB[i])
        assert r["l1"][i] == (B["nucleus_id"] if in_b else A["nucleus_id"]), i
        checked += 1
    assert checked > 50


def test_nuclei_respect_eligibility_and_nesting(two_haloes):
    pos, ids, p, r = two_haloes
    check_invariants(pos, ids, p, r)


def check_invariants(pos, ids, p, r):
    l0, l1, l2, sig = r["l0"], r["l1"], r["l2"], r["sigma"]
    NONE = O.NONE
    idx = {int(i): k for k, i in enumerate(ids)}
    assert np.all(l0[l1 != NONE] != NONE)  # L1 inside L0
    assert np.all(l1[l2 != NONE] != NONE)  # L2 inside L1
    for h in np.unique(l1[l1 != NONE]):
        m = l1 == h
        assert len(np.unique(l0[m])) == 1
        assert l1[idx[int(h)]] == h  # a nucleus is never stolen
    for h in np.unique(l2[l2 != NONE]):
        m = l2 == h
        assert len(np.unique(l1[m])) == 1
        assert l2[idx[int(h)]] == h
    H = r["halos"]
    P = pos.astype(np.int64)
    d_all = brute_d2(pos) if len(pos) <= 12000 else None
    key = lambda i: (-int(sig[i]), int(ids[i]))
    for h in H:
        k = idx[int(h["nucleus_id"])]
        # step 4: every nucleus is above the stop level
        assert sig[k] > p.T_min_L1
        if d_all is not None:
            # step 2: a nucleus is denser than every other member of its group within b
            near = np.nonzero((d_all[k] < p.b2) & (l0 == l0[k]))[0]
            assert all(key(q) > key(k) for q in near if q != k)
            # step 1: members lie inside R; group particles inside R belong to some halo
            m = l1 == h["nucleus_id"]
            assert np.all(d_all[k][m] < h["R2"])
            inside = (d_all[k] < h["R2"]) & (l0 == l0[k])
            assert np.all(l1[inside] != NONE)
    # step 1: the densest particle of every group above the stop level is a nucleus
    for g in np.unique(l0[l0 != NONE]):
        m = np.nonzero(l0 == g)[0]
        top = min(m, key=key)
        if sig[top] > p.T_min_L1:
            assert l1[top] == ids[top]
    # eligibility: a later nucleus never lies inside alpha R of an earlier one of its group
    for g in np.unique(H["l0_id"]):
        hs = H[H["l0_id"] == g]
        keys = sorted(hs, key=lambda h: (-sig[idx[int(h["nucleus_id"])]], int(h["nucleus_id"])))
        for a in range(len(keys)):
            for b in range(a + 1, len(keys)):
                pa = P[idx[int(keys[a]["nucleus_id"])]]
                pb = P[idx[int(keys[b]["nucleus_id"])]]
                d = int((mi(pb - pa) ** 2).sum())
                assert p.alpha_den ** 2 * d >= p.alpha_num ** 2 * int(keys[a]["R2"])


def test_pipeline_invariants_and_order_independence():
    pos, ids, _ = synth.patch(extent=16.0, lo=-8.0, seed=41)
    p = O.params(U64, np_min_L1=1)
    r = O.find_groups(pos, ids, p)
    check_invariants(pos, ids, p, r)
    perm = np.random.default_rng(2).permutation(len(pos))
    r2 = O.find_groups(pos[perm], ids[perm], p)
    for k in ("sigma", "l0", "l1", "l2"):
        assert np.array_equal(r[k][perm], r2[k]), k
    assert np.array_equal(r["halos"], r2["halos"])


@pytest.mark.parametrize("kw", [dict(alpha=(7, 10)), dict(alpha=(9, 10)), dict(l_fof=0.30),
                                dict(delta_L0=40.0)])
def test_parameter_variants_run_and_nest(kw):
    """App. B.1 variants: alpha = 0.7 / 0.9, l_FoF = 0.30, Delta_L0 = 40."""
    pos, ids, _ = synth.patch(extent=14.0, lo=5.0, seed=43)
    p = O.params(U64, np_min_L1=1, **kw)
    r = O.find_groups(pos, ids, p)
    check_invariants(pos, ids, p, r)


def test_eligibility_radius_controls_satellite_nucleus(two_haloes):
    """Step 1: the satellite sits at 0.93 R_200 of the host, outside 0.8 R_L1
    but inside 0.95 R_L1, so it is a nucleus at alpha = 0.8 and not at 0.95."""
    pos, ids, p, r = two_haloes
    assert len(r["halos"]) >= 2
    p95 = O.params(p.u, np_min_L1=1, alpha=(19, 20))
    r95 = O.find_groups(pos, ids, p95)
    assert len(r95["halos"]) < len(r["halos"])


# --------------------------------------------------------------------------
# redshift scaling of the thresholds (Sec. 2.3.1, Eq. 2)
# --------------------------------------------------------------------------

def test_cosmology_scaling_reproduces_table1():
    g = GOLD["table1_thresholds_z05"]
    d0, d1, d2, lf = O.cosmology(g["omega_m0"], g["z"])
    assert d1 == pytest.approx(g["delta_L1"], rel=1e-3)
    assert d2 == pytest.approx(g["delta_L2"], rel=1e-3)
    assert d0 == pytest.approx(g["delta_L0"], rel=1e-3)
    assert lf == pytest.approx(0.25 * (d1 / 200) ** (-1 / 3), rel=1e-12)


def test_cosmology_scaling_einstein_de_sitter_limit():
    """Omega_m = 1 at all times: x = 0, Delta_base = 18 pi^2, so the
    Einstein-de Sitter values 60 / 200 / 800 and l_FoF = 0.25 come back."""
    for z in (0.0, 0.5, 3.0):
        d0, d1, d2, lf = O.cosmology(1.0, z)
        assert (d0, d1, d2, lf) == pytest.approx((60.0, 200.0, 800.0, 0.25), rel=1e-12)
