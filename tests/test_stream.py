"""Slab stream: a box delivered as x-slabs, with ghost columns and open L0
groups kept on the device between slabs, gives exactly the labels and
catalogue of the whole box processed at once."""
import numpy as np
import pytest

from paper_2110_11408_gb300 import cso, synth
from parity_util import assert_matches_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BOX = 1 << 21


@pytest.fixture(scope="module")
def box():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pos, ids, meta = synth.tiny(seed=77)
    p = cso.cso_params_default(meta["u"])
    with cso.Context(0) as ctx:
        whole = ctx.find_groups(pos, ids, p, halo_cap=len(pos) // 10)
    # the whole-box result every slab stream is compared with is the oracle's
    assert_matches_oracle(whole, pos, ids, meta["u"])
    return pos, ids, p, whole


def run_stream(ctx, pos, ids, p, edges, stream_id, on_device=True):
    bufs, tickets = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (pos[:, 0] >= lo) & (pos[:, 0] < hi)
        sp, si = pos[m], ids[m]
        if on_device:
            sp = torch.from_numpy(np.ascontiguousarray(sp)).cuda()
            si = torch.from_numpy(np.ascontiguousarray(si).view(np.int64)).cuda()
        b = cso.Buffers(sp, si, on_device, halo_cap=len(pos) // 20 + 16, x_lo=lo, x_hi=hi, request_id=stream_id,
                        out_device=True)
        b.mask = m
        bufs.append(b)
        tickets.append(ctx.submit(b, p))
    return bufs, tickets


def check_stream(ctx, bufs, tickets, pos, whole):
    halos = []
    for b, t in zip(bufs, tickets):
        done, rc = ctx.wait(t)
        assert done and rc == cso.CSO_OK, cso.cso_last_error()
        r = b.result()
        for k in ("sigma", "l0", "l1", "l2"):
            a = r[k]
            ref = whole[k][b.mask]
            if not np.array_equal(a, ref):
                bad = np.nonzero(a != ref)[0]
                raise AssertionError("%s differs at %d of %d slab particles" % (k, bad.size, a.size))
        halos.append(r["halos"])
    h = np.concatenate(halos)
    h = h[np.argsort(h["nucleus_id"])]
    assert np.array_equal(h, whole["halos"])


@pytest.mark.parametrize("nslab", [1, 4, 16])
def test_equal_slabs(box, nslab):
    pos, ids, p, whole = box
    edges = [BOX * k // nslab for k in range(nslab + 1)]
    with cso.Context(0, flags=cso.FLAG_SLOTS(2)) as ctx:
        bufs, tickets = run_stream(ctx, pos, ids, p, edges, stream_id=nslab)
        check_stream(ctx, bufs, tickets, pos, whole)


def test_uneven_slabs_off_the_cell_grid_with_host_inputs(box):
    pos, ids, p, whole = box
    rng = np.random.default_rng(5)
    cuts = np.sort(rng.choice(np.arange(1, BOX), 22, replace=False))
    edges = [0] + [int(c) for c in cuts] + [BOX]
    with cso.Context(0, flags=cso.FLAG_SLOTS(3) | cso.FLAG_BATCHED) as ctx:
        bufs, tickets = run_stream(ctx, pos, ids, p, edges, stream_id=9, on_device=False)
        check_stream(ctx, bufs, tickets, pos, whole)


def test_two_streams_and_whole_boxes_in_the_mix(box):
    pos, ids, p, whole = box
    pos2, ids2, meta2 = synth.tiny(seed=78)
    with cso.Context(0) as ctx:
        whole2 = ctx.find_groups(pos2, ids2, p, halo_cap=len(pos2) // 10)
    assert_matches_oracle(whole2, pos2, ids2, meta2["u"])
    with cso.Context(0, flags=cso.FLAG_SLOTS(4)) as ctx:
        e1 = [BOX * k // 8 for k in range(9)]
        e2 = [BOX * k // 5 for k in range(6)]
        b1, t1 = run_stream(ctx, pos, ids, p, e1, stream_id=101)
        wb = cso.Buffers(pos2, ids2, False, halo_cap=len(pos2) // 10)
        tw = ctx.submit(wb, p)
        b2, t2 = run_stream(ctx, pos2, ids2, p, e2, stream_id=102)
        check_stream(ctx, b1, t1, pos, whole)
        check_stream(ctx, b2, t2, pos2, whole2)
        done, rc = ctx.wait(tw)
        assert done and rc == cso.CSO_OK
        r = wb.result()
        for k in ("sigma", "l0", "l1", "l2"):
            assert np.array_equal(r[k], whole2[k])


def test_out_of_order_slab_is_refused(box):
    pos, ids, p, whole = box
    with cso.Context(0, flags=cso.FLAG_SLOTS(1)) as ctx:
        m = pos[:, 0] < BOX // 4
        b0 = cso.Buffers(pos[m], ids[m], False, x_lo=0, x_hi=BOX // 4, request_id=5, out_device=True)
        t0 = ctx.submit(b0, p)
        m2 = (pos[:, 0] >= BOX // 2) & (pos[:, 0] < 3 * BOX // 4)
        b2 = cso.Buffers(pos[m2], ids[m2], False, x_lo=BOX // 2, x_hi=3 * BOX // 4, request_id=5, out_device=True)
        t2 = ctx.submit(b2, p)
        done, rc = ctx.wait(t2)
        assert done and rc == cso.CSO_ERR_STATE
