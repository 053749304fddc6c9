"""Served path: continuous batching of requests on one GPU.

Requests submitted together are admitted onto worker slots while memory
allows and run concurrently; each must give exactly what it gives alone.
"""
import numpy as np
import pytest

from paper_2110_11408_gb300 import cso, synth
from parity_util import assert_matches_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def boxes():
    out = [synth.tiny()]
    for seed, ext, side in [(11, 16.0, 64), (12, 20.0, 64), (13, 14.0, 128), (14, 18.0, 64), (15, 12.0, 256)]:
        out.append(synth.patch(extent=ext, lo=-4.0, side=side, seed=seed))
    return out


@pytest.fixture(scope="module")
def alone():
    """Each box computed alone, and checked against the oracle, so that
    "the same in the mix as alone" also means "the same as the oracle"."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    res = []
    with cso.Context(0) as ctx:
        for pos, ids, meta in boxes():
            p = cso.cso_params_default(meta["u"])
            r = ctx.find_groups(pos, ids, p)
            assert_matches_oracle(r, pos, ids, meta["u"])
            res.append(r)
    return res


def same(a, b):
    for k in ("sigma", "l0", "l1", "l2"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["halos"], b["halos"])


@pytest.mark.parametrize("flags", [cso.FLAG_SLOTS(4), cso.FLAG_SLOTS(3) | cso.FLAG_BATCHED])
def test_requests_in_the_mix_equal_alone(alone, flags):
    with cso.Context(0, flags=flags) as ctx:
        bufs, tickets = [], []
        for pos, ids, meta in boxes():
            p = cso.cso_params_default(meta["u"])
            b = cso.Buffers(torch.from_numpy(pos).cuda(), torch.from_numpy(ids.view(np.int64)).cuda(), True)
            bufs.append(b)
            tickets.append(ctx.submit(b, p))
        for t in tickets:
            done, rc = ctx.wait(t)
            assert done and rc == cso.CSO_OK, cso.cso_last_error()
        for b, ref in zip(bufs, alone):
            same(b.result(), ref)
        times = [cso.cso_ticket_times(ctx.h, t) for t in tickets]
        assert all(s <= a <= d for s, a, d in times)


def test_budget_admits_one_request_at_a_time():
    """Three 262k-particle boxes (about 230 MB of workspace each) under a
    400 MB budget: never two at once, and each result as computed alone."""
    data = [synth.tiny(seed=s) for s in (101, 102, 103)]
    with cso.Context(0) as ctx:
        ref = [ctx.find_groups(pos, ids, cso.cso_params_default(meta["u"])) for pos, ids, meta in data]
    for r, (pos, ids, meta) in zip(ref, data):
        assert_matches_oracle(r, pos, ids, meta["u"])
    with cso.Context(0, budget_bytes=(400 << 20), flags=cso.FLAG_SLOTS(3)) as ctx:
        bufs, tickets = [], []
        for pos, ids, meta in data:
            b = cso.Buffers(pos, ids, False)
            bufs.append(b)
            tickets.append(ctx.submit(b, cso.cso_params_default(meta["u"])))
        for t in tickets:
            done, rc = ctx.wait(t)
            assert done and rc == cso.CSO_OK
        for b, r in zip(bufs, ref):
            same(b.result(), r)
        iv = sorted(cso.cso_ticket_times(ctx.h, t)[1:] for t in tickets)
        for (s0, d0), (s1, d1) in zip(iv, iv[1:]):
            assert s1 >= d0  # admitted only after the previous one finished


def test_request_over_budget_is_refused():
    pos, ids, meta = synth.tiny()
    with cso.Context(0, budget_bytes=(32 << 20)) as ctx:
        b = cso.Buffers(pos, ids, False)
        with pytest.raises(cso.CsoError) as e:
            ctx.submit(b, cso.cso_params_default(meta["u"]))
        assert e.value.rc == cso.CSO_ERR_BUDGET


def test_bad_request_fails_alone(alone):
    good = boxes()[1]
    bad_pos = good[0].copy()
    bad_pos[5, 0] = 1 << 21  # off the grid
    with cso.Context(0, flags=cso.FLAG_SLOTS(2)) as ctx:
        p = cso.cso_params_default(good[2]["u"])
        b_bad = cso.Buffers(bad_pos, good[1], False)
        b_good = cso.Buffers(good[0], good[1], False)
        t_bad = ctx.submit(b_bad, p)
        t_good = ctx.submit(b_good, p)
        done, rc = ctx.wait(t_bad)
        assert done and rc == cso.CSO_ERR_ARG
        done, rc = ctx.wait(t_good)
        assert done and rc == cso.CSO_OK
        same(b_good.result(), alone[1])
        done, rc = ctx.wait(987654)
        assert rc == cso.CSO_ERR_STATE and not done


def test_bounded_poll_times_out_then_completes():
    """A positive timeout that passes before the request is done returns
    CSO_ERR_TIMEOUT with done = 0; the ticket stays valid and completes."""
    pos, ids, meta = synth.tiny(seed=104)
    with cso.Context(0, flags=cso.FLAG_SLOTS(1)) as ctx:
        b = cso.Buffers(pos, ids, False)
        t = ctx.submit(b, cso.cso_params_default(meta["u"]))
        done, rc = ctx.wait(t, timeout_us=1)
        # a 262k-particle request takes milliseconds; 1 us cannot cover it
        assert (not done and rc == cso.CSO_ERR_TIMEOUT) or (done and rc == cso.CSO_OK)
        assert ctx.wait(t, timeout_us=0)[1] == cso.CSO_OK  # a plain test never times out
        done, rc = ctx.wait(t)
        assert done and rc == cso.CSO_OK
