"""GPU path vs the CPU oracle, through the C ABI.

Integer outputs (kernel sums, L0/L1/L2 labels, nucleus ids, N, R^2) must be
bit-identical; FP64 halo statistics (centres of mass, R_Delta) within 1e-9
relative (the path accumulates them exactly in integers, so they agree far
below the 1e-6 bar).
"""
import numpy as np
import pytest

import oracle as O
from paper_2110_11408_gb300 import cso, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
BOX = 1 << 21
U64 = 32768


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cso.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_stress():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cso.Context(0, flags=cso.FLAG_SELECT_STRESS)
    yield c
    c.close()


def both_params(u, **kw):
    return cso.cso_params_default(u, **kw), O.params(u, **kw)


def assert_same(g, o, n_sample_fp=None):
    for k in ("sigma", "l0", "l1", "l2"):
        a, b = g[k], o[k]
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError("%s differs at %d of %d entries, first %s: gpu %s oracle %s"
                                 % (k, bad.size, a.size, bad[:5], a[bad[:5]], b[bad[:5]]))
    H, Ho = g["halos"], o["halos"]
    assert len(H) == len(Ho), (len(H), len(Ho))
    for f in ("nucleus_id", "N", "R2", "l2max_id", "l2max_N", "l2_top5_N", "n_l2", "l0_id"):
        assert np.array_equal(H[f], Ho[f]), f
    for f in ("com", "l2max_com", "R_delta"):
        np.testing.assert_allclose(H[f], Ho[f], rtol=1e-9, atol=1e-9 * BOX)


_MEDIUM = {}


def medium_box():
    """The benchmark box (side 256, 16.8M particles), drawn once per session."""
    if "box" not in _MEDIUM:
        _MEDIUM["box"] = synth.medium()
    return _MEDIUM["box"]


def check_groups_against_oracle(g, pos, ids, po, pick, u, radial=True):
    """L1/L2 labels and catalogue rows of the L0 groups `pick` of a GPU run
    `g`, each recomputed by the oracle on exactly its own members, with
    their kernel sums from the oracle on the full box."""
    members = [np.nonzero(g["l0"] == gid)[0] for gid in pick]
    # one oracle density pass over all members of all picked groups
    sig_all = O.density_at(pos, po, np.concatenate(members))
    cuts = np.cumsum([0] + [m.size for m in members])
    for k, gid in enumerate(pick):
        m = members[k]
        sig = sig_all[cuts[k]:cuts[k + 1]]
        assert np.array_equal(sig, g["sigma"][m])
        l1, l2, halos, _ = O.compaso(pos[m], ids[m], sig, g["l0"][m], po)
        assert np.array_equal(l1, g["l1"][m]), "L1 of group %d (%d members)" % (gid, m.size)
        assert np.array_equal(l2, g["l2"][m]), "L2 of group %d (%d members)" % (gid, m.size)
        sel = np.isin(g["halos"]["nucleus_id"], halos["nucleus_id"])
        mine = g["halos"][sel]
        assert len(mine) == len(halos)
        for f in ("nucleus_id", "N", "R2", "l2max_id", "l2max_N", "l2_top5_N", "n_l2", "l0_id"):
            assert np.array_equal(mine[f], halos[f]), f
        for f in ("com", "l2max_com", "R_delta"):
            np.testing.assert_allclose(mine[f], halos[f], rtol=1e-9, atol=1e-9 * BOX)
        if radial:
            # radial statistics of the same rows, from the oracle's own labels
            assert_same_radial(g["radial"][sel], O.radial(pos[m], l1, halos, u),
                               O.shrink_sphere(pos[m], ids[m], l1, halos))


def run_both(ctx, pos, ids, u=U64, on_device=True, **kw):
    pg, po = both_params(u, **kw)
    g = ctx.find_groups(pos, ids, pg, on_device=on_device)
    o = O.find_groups(pos, ids, po)
    return g, o


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_patch_across_periodic_corner(ctx, seed):
    pos, ids, _ = synth.patch(extent=16.0, lo=-8.0, seed=seed)
    g, o = run_both(ctx, pos, ids)
    assert_same(g, o)
    assert o["stats"]["l1_nuclei"] > 5


def test_patch_select_stress(ctx_stress):
    """Tiny select tiles force every branch of the radius search (window
    narrowing, single-value bins, bins without the answer, exhaustion)."""
    for seed in (4, 5):
        pos, ids, _ = synth.patch(extent=18.0, lo=-3.0, seed=seed, nmax=4000)
        g, o = run_both(ctx_stress, pos, ids)
        assert_same(g, o)


def test_tiny_box_full_parity(ctx):
    """Box 64 l_mean, 262,144 particles, ~850 NFW haloes: every output."""
    pos, ids, meta = synth.tiny()
    g, o = run_both(ctx, pos, ids)
    assert_same(g, o)
    st = ctx.stats()
    assert st["dense"] == o["stats"]["dense"]
    assert st["l0_groups"] == o["stats"]["l0_groups"]
    assert st["l1_nuclei"] == o["stats"]["l1_nuclei"]
    assert st["l2_nuclei"] == o["stats"]["l2_nuclei"]
    assert st["l1_work"] == o["stats"]["l1_work"]


def test_tiny_box_select_stress(ctx_stress):
    pos, ids, meta = synth.tiny()
    g, o = run_both(ctx_stress, pos, ids)
    assert_same(g, o)


def test_host_buffers_match_device_buffers(ctx):
    pos, ids, _ = synth.patch(extent=20.0, lo=30.0, seed=7)
    p, _ = both_params(U64)
    a = ctx.find_groups(pos, ids, p, on_device=True)
    b = ctx.find_groups(pos, ids, p, on_device=False)
    for k in ("sigma", "l0", "l1", "l2"):
        assert np.array_equal(a[k], b[k])
    assert np.array_equal(a["halos"], b["halos"])


def test_input_order_does_not_matter(ctx):
    pos, ids, _ = synth.patch(extent=16.0, lo=10.0, seed=8)
    p, _ = both_params(U64)
    a = ctx.find_groups(pos, ids, p)
    perm = np.random.default_rng(0).permutation(len(pos))
    b = ctx.find_groups(pos[perm], ids[perm], p)
    for k in ("sigma", "l0", "l1", "l2"):
        assert np.array_equal(a[k][perm], b[k])
    assert np.array_equal(a["halos"], b["halos"])


@pytest.mark.parametrize("kw", [dict(alpha=(7, 10)), dict(alpha=(9, 10)), dict(l_fof=0.30),
                                dict(delta_L0=40.0), dict(roche=(1, 1)), dict(include_self=1),
                                dict(np_min_L1=1)])
def test_parameter_variants(ctx, kw):
    pos, ids, _ = synth.patch(extent=16.0, lo=-8.0, seed=9)
    g, o = run_both(ctx, pos, ids, **kw)
    assert_same(g, o)


def test_box_sizes(ctx):
    """Other grids: box 128 (u = 16384) and box 256 (u = 8192) patches."""
    for side in (128, 256):
        pos, ids, _ = synth.patch(extent=14.0, lo=-5.0, side=side, seed=10)
        g, o = run_both(ctx, pos, ids, u=BOX // side)
        assert_same(g, o)


def test_edge_cases(ctx):
    p, po = both_params(U64)
    # empty input
    e = ctx.find_groups(np.zeros((0, 3), np.int32), np.zeros(0, np.uint64), p)
    assert e["n_halos"] == 0 and all(e[k].size == 0 for k in ("l0", "l1", "l2", "sigma"))
    # one particle
    one = ctx.find_groups(np.array([[5, 6, 7]], np.int32), np.array([42], np.uint64), p)
    assert one["sigma"][0] == 0 and one["l0"][0] == cso.NO_GROUP
    # many particles on one spot: equal Sigma everywhere, ties broken by id
    pos = np.full((300, 3), 1000, np.int32)
    ids = np.random.default_rng(1).permutation(300).astype(np.uint64) + 7
    g, o = run_both(ctx, pos, ids, np_min_L1=1)
    assert_same(g, o)
    # a cubic lattice (many equal distances), straddling the box corner
    lat, lid, _ = synth.lattice_ball(int(0.06 * U64), 150, [0, 0, 0])
    g, o = run_both(ctx, lat, lid, np_min_L1=1)
    assert_same(g, o)


@pytest.mark.parametrize("bad", [[BOX, 0, 0], [0, BOX, 0], [0, 0, BOX], [5, -1, 7], [5, 7, -(1 << 30)],
                                 [-(1 << 31), 1 << 30, 3]])
def test_rejects_positions_outside_grid(ctx, bad):
    """Any coordinate outside [0, 2^21) fails the request with CSO_ERR_ARG;
    the rejected particle is binned and stored at cell 0, so every kernel of
    the failed request still indexes inside its tables (patch particles
    around it exercise density and FoF on the same run)."""
    p, _ = both_params(U64)
    pos, ids, _ = synth.patch(extent=6.0, lo=-3.0, seed=2)
    pos = np.concatenate([pos, np.array([bad], np.int32)])
    ids = np.arange(len(pos), dtype=np.uint64)
    with pytest.raises(cso.CsoError) as e:
        ctx.find_groups(pos, ids, p)
    assert e.value.rc == cso.CSO_ERR_ARG
    # the context stays usable
    g, o = run_both(ctx, pos[:-1], ids[:-1])
    assert_same(g, o)


def test_rejects_requests_of_2_31_particles(ctx):
    """n >= 2^31 - 1 is refused before anything is read."""
    p, _ = both_params(U64)
    b = cso.Buffers(np.zeros((1, 3), np.int32), np.zeros(1, np.uint64), False)
    b.cin.n = (1 << 31) - 1
    assert cso.lib().cso_find_groups(ctx.h, b.cin, p, b.cout) == cso.CSO_ERR_ARG
    assert "too large" in cso.cso_last_error()


def test_capacity_error_reports_needed_rows(ctx):
    pos, ids, _ = synth.patch(extent=16.0, lo=-8.0, seed=1)
    p, _ = both_params(U64, np_min_L1=1)
    b = cso.Buffers(pos, ids, on_device=False, halo_cap=1)
    rc = cso.lib().cso_find_groups(ctx.h, b.cin, p, b.cout)
    assert rc == cso.CSO_ERR_CAPACITY and b.cout.n_halos > 1


def test_medium_box_sampled_parity(ctx):
    """Box 256 l_mean, 16.8M particles (the benchmark workload), in the
    benchmark's launch configuration: kernel sums of 3000 sampled particles,
    L0 consistency of sampled dense particles, and L1/L2 labels and catalogue
    rows of 40 sampled L0 groups, each recomputed by the oracle on exactly
    its own members (their kernel sums from the oracle on the full box)."""
    from scipy.spatial import cKDTree
    pos, ids, meta = medium_box()
    p, po = both_params(meta["u"], np_min_L1=1)
    g = ctx.find_groups(pos, ids, p, radial=True)
    rng = np.random.default_rng(3)
    n = len(pos)
    sample = rng.choice(n, 3000, replace=False)
    assert np.array_equal(g["sigma"][sample], O.density_at(pos, po, sample))
    dense = g["sigma"] > po.T_L0
    assert np.all((g["l0"] != cso.NO_GROUP) == dense)
    tree = cKDTree(pos.astype(np.float64), boxsize=float(BOX))
    ds = sample[dense[sample]]
    for i, nb in zip(ds, tree.query_ball_point(pos[ds].astype(np.float64), np.sqrt(po.lfof2) - 1e-6)):
        nb = np.asarray(nb)
        nb = nb[dense[nb]]
        d2 = (((pos[nb].astype(np.int64) - pos[i] + BOX // 2) % BOX - BOX // 2) ** 2).sum(1)
        assert np.all(g["l0"][nb[d2 < po.lfof2]] == g["l0"][i])
    groups, counts = np.unique(g["l0"][dense], return_counts=True)
    big = groups[counts >= 200]
    pick = np.concatenate([rng.choice(big, 20, replace=False), rng.choice(groups, 20, replace=False)])
    check_groups_against_oracle(g, pos, ids, po, pick, meta["u"])


def assert_same_radial(a, b, ss):
    assert len(a) == len(b) == len(ss)
    for f, fo in (("ss_centre", "centre"), ("ss_n", "n"), ("ss_R2", "R2"), ("ss_iter", "iter")):
        if not np.array_equal(a[f], ss[fo]):
            bad = np.nonzero(np.any((a[f] != ss[fo]).reshape(len(a), -1), axis=1))[0]
            raise AssertionError("shrinking sphere %s differs in %d of %d rows, first %s: gpu %s oracle %s"
                                 % (f, bad.size, len(a), bad[:3], a[f][bad[:3]], ss[fo][bad[:3]]))
    for f in O.RADIAL_DTYPE.names:
        if not np.array_equal(a[f], b[f]):
            bad = np.nonzero(np.any((a[f] != b[f]).reshape(len(a), -1), axis=1))[0]
            raise AssertionError("radial %s differs in %d of %d rows, first %s: gpu %s oracle %s"
                                 % (f, bad.size, len(a), bad[:3], a[f][bad[:3]], b[f][bad[:3]]))


def test_radial_statistics_tiny_box(ctx):
    """r_25/50/75/98 and V_max of every catalogue row, bit-identical; rows
    with and without L2 haloes (the two centre choices) both occur."""
    pos, ids, meta = synth.tiny()
    pg, po = both_params(U64)
    g = ctx.find_groups(pos, ids, pg, on_device=True, radial=True)
    o = O.find_groups(pos, ids, po)
    assert_same(g, o)
    assert_same_radial(g["radial"], O.radial(pos, o["l1"], o["halos"], U64),
                       O.shrink_sphere(pos, ids, o["l1"], o["halos"]))
    assert (o["halos"]["n_l2"] == 0).any() and (o["halos"]["n_l2"] > 0).any()
    assert (g["radial"]["ss_iter"] > 0).any()
    h = ctx.find_groups(pos, ids, pg, on_device=False, radial=True)
    assert np.array_equal(h["radial"], g["radial"])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_radial_statistics_across_periodic_corner(ctx, seed):
    pos, ids, _ = synth.patch(extent=16.0, lo=-8.0, seed=seed)
    pg, po = both_params(U64, np_min_L1=1)
    g = ctx.find_groups(pos, ids, pg, radial=True)
    o = O.find_groups(pos, ids, po)
    assert_same(g, o)
    assert_same_radial(g["radial"], O.radial(pos, o["l1"], o["halos"], U64),
                       O.shrink_sphere(pos, ids, o["l1"], o["halos"], n_min=cso.SHRINK_N_MIN))


def test_radial_rejected_for_slab_requests(ctx):
    pos, ids, _ = synth.patch(extent=8.0, lo=0.0, seed=1)
    p = cso.cso_params_default(U64)
    b = cso.Buffers(pos, ids, False, want=("l0", "radial"), x_lo=0, x_hi=1 << 16, request_id=77)
    with pytest.raises(cso.CsoError) as e:
        cso.cso_submit(ctx.h, b, p)
    assert e.value.rc == cso.CSO_ERR_ARG


# --------------------------------------------------------------------------
# batched schedule: warp per small group, block per medium, 1024-thread
# block per giant, largest first, giants on a second stream
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def ctx_batched():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = cso.Context(0, flags=cso.FLAG_BATCHED)
    yield c
    c.close()


def test_batched_tiny_full_parity(ctx_batched):
    pos, ids, meta = synth.tiny()
    g, o = run_both(ctx_batched, pos, ids)
    assert_same(g, o)


@pytest.mark.parametrize("seed", [1, 2])
def test_batched_patch_parity(ctx_batched, seed):
    pos, ids, _ = synth.patch(extent=16.0, lo=-8.0, seed=seed)
    g, o = run_both(ctx_batched, pos, ids, np_min_L1=1)
    assert_same(g, o)


def test_batched_select_stress():
    c = cso.Context(0, flags=cso.FLAG_BATCHED | cso.FLAG_SELECT_STRESS)
    try:
        pos, ids, _ = synth.patch(extent=18.0, lo=-3.0, seed=4, nmax=4000)
        g, o = run_both(c, pos, ids)
        assert_same(g, o)
    finally:
        c.close()


def test_batched_medium_box_giant_groups_parity():
    """The batched schedule in the benchmark's tuned configuration (groups
    above 65,536 members on 8-CTA clusters, above 4,096 on 1024-thread
    blocks, up to 64 on warps) on the 16.8M-particle box, against the oracle:
    the five largest L0 groups (cluster tier), four of the 1024-thread tier,
    four of the 256-thread tier and four warp groups, each recomputed on its
    own members."""
    pos, ids, meta = medium_box()
    p, po = both_params(meta["u"], np_min_L1=1)
    c = cso.Context(0, flags=cso.FLAG_BATCHED)
    try:
        cso.cso_set_schedule(c.h, 65536, 64)
        g = c.find_groups(pos, ids, p, radial=True)
    finally:
        c.close()
    dense = g["l0"] != cso.NO_GROUP
    groups, counts = np.unique(g["l0"][dense], return_counts=True)
    order = np.argsort(-counts)
    rng = np.random.default_rng(11)
    giants = groups[order[:5]]
    assert counts[order[0]] > 65536
    tiers = [giants]
    for lo, hi in ((4096, 65536), (64, 4096), (1, 64)):
        sel = groups[(counts > lo) & (counts <= hi)]
        tiers.append(rng.choice(sel, min(4, sel.size), replace=False))
    check_groups_against_oracle(g, pos, ids, po, np.concatenate(tiers), meta["u"])


def test_batched_equals_plain_on_medium_box(ctx, ctx_batched):
    """Same labels and catalogue, bit for bit, from both schedules on the
    16.8M-particle benchmark box."""
    pos, ids, meta = medium_box()
    p = cso.cso_params_default(meta["u"])
    dpos = torch.from_numpy(pos).cuda()
    dids = torch.from_numpy(ids.view(np.int64)).cuda()
    a = ctx.find_groups(dpos, dids, p)
    b = ctx_batched.find_groups(dpos, dids, p)
    for k in ("sigma", "l0", "l1", "l2"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["halos"], b["halos"])


def test_redshift_scaled_thresholds(ctx):
    """Parity with the thresholds of Table 1's box (z = 0.5, Omega_m = 0.315)."""
    pos, ids, _ = synth.patch(extent=16.0, lo=-8.0, seed=12)
    p = cso.cso_params_cosmology(cso.cso_params_default(U64), 0.315, 0.5)
    po = O.params(U64, delta_L0=p.delta_L0, delta_L1=p.delta_L1, delta_L2=p.delta_L2, l_fof=p.l_fof)
    g = ctx.find_groups(pos, ids, p)
    o = O.find_groups(pos, ids, po)
    assert_same(g, o)


def test_autotuned_schedule_keeps_results(ctx_batched):
    pos, ids, meta = synth.tiny(seed=5)
    p, po = both_params(U64)
    b = cso.Buffers(pos, ids, False)
    giant, small = cso.cso_autotune(ctx_batched.h, b, p)
    assert giant in (4096, 8192, 16384, 65536, 262144) and small in (32, 64)
    g = ctx_batched.find_groups(pos, ids, p)
    o = O.find_groups(pos, ids, po)
    assert_same(g, o)
    assert_same(b.result(), o)


def test_cluster_path_for_every_group_above_64():
    """Giant threshold 64: every group above 64 members runs on an 8-CTA
    thread-block cluster (DSMEM histogram merge, leader-driven select)."""
    c = cso.Context(0, flags=cso.FLAG_BATCHED)
    try:
        cso.cso_set_schedule(c.h, 64, 64)
        pos, ids, meta = synth.tiny()
        g, o = run_both(c, pos, ids)
        assert_same(g, o)
    finally:
        c.close()


def test_huge_cluster_path_for_every_group_above_64():
    """Giant and huge thresholds 64: every group above 64 members runs on a
    16-CTA thread-block cluster (a non-portable size; 8-CTA clusters where
    the device cannot hold one), plain and under select stress."""
    for flags in (cso.FLAG_BATCHED, cso.FLAG_BATCHED | cso.FLAG_SELECT_STRESS):
        c = cso.Context(0, flags=flags)
        try:
            cso.cso_set_schedule(c.h, 64, 64)
            cso.cso_set_huge_group(c.h, 64)
            pos, ids, meta = synth.tiny()
            g, o = run_both(c, pos, ids)
            assert_same(g, o)
        finally:
            c.close()


def test_cluster_path_select_stress():
    c = cso.Context(0, flags=cso.FLAG_BATCHED | cso.FLAG_SELECT_STRESS)
    try:
        cso.cso_set_schedule(c.h, 64, 8)
        for seed in (4, 6):
            pos, ids, _ = synth.patch(extent=18.0, lo=-3.0, seed=seed, nmax=4000)
            g, o = run_both(c, pos, ids)
            assert_same(g, o)
    finally:
        c.close()


def test_batched_level_stages_as_cuda_graphs():
    """CSO_FLAG_GRAPH: the level stages captured once and replayed give the
    oracle's results on every call (a capture, then replays of it)."""
    pos, ids, meta = synth.tiny()
    p, po = both_params(U64)
    o = O.find_groups(pos, ids, po)
    c = cso.Context(0, flags=cso.FLAG_BATCHED | cso.FLAG_GRAPH)
    try:
        dpos = torch.from_numpy(pos).cuda()
        dids = torch.from_numpy(ids.view(np.int64)).cuda()
        for _ in range(3):
            g = c.find_groups(dpos, dids, p)
            assert_same(g, o)
        # another box in the same context: a new capture, same parity
        pos2, ids2, _ = synth.patch(extent=16.0, lo=-8.0, seed=2)
        g2, o2 = run_both(c, pos2, ids2)
        assert_same(g2, o2)
    finally:
        c.close()
