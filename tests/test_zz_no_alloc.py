"""cso_density_static: kernel densities for callers that cannot allocate
device memory (their memory belongs to their own pool, or an allocation
would synchronise the device in the middle of a time step).

The entry point keeps its scratch in a fixed array in device memory; its
densities must equal those of the allocating path (cso_find_groups) bit for
bit, call after call, since the array keeps each call's leftovers.  This file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2110_11408_gb300 import cso, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def static_density(pos_dev, params, stream=None):
    L = cso.lib()
    L.cso_density_static.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(cso.CsoParams),
                                     ctypes.c_void_p, ctypes.c_void_p]
    n = int(pos_dev.shape[0])
    out = torch.full((n,), -1, dtype=torch.int64, device=pos_dev.device)
    rc = L.cso_density_static(pos_dev.data_ptr() if n else None, n, ctypes.byref(params),
                              out.data_ptr() if n else None, stream)
    return rc, out


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def test_static_density_matches_allocating_path(dev):
    cases = [synth.tiny(), synth.patch(extent=16.0, lo=-8.0, seed=3)]
    with cso.Context(0) as ctx:
        for pos, ids, meta in cases:
            p = cso.cso_params_default(meta["u"])
            ref = ctx.find_groups(pos, ids, p)["sigma"]
            dpos = torch.from_numpy(pos).to(dev)
            for _ in range(2):  # two calls in a row share the scratch array
                rc, out = static_density(dpos, p)
                assert rc == cso.CSO_OK, cso.cso_last_error()
                torch.cuda.synchronize()
                assert np.array_equal(out.cpu().numpy(), ref)


def test_static_density_on_a_caller_stream(dev):
    pos, ids, meta = synth.patch(extent=12.0, lo=20.0, seed=5)
    p = cso.cso_params_default(meta["u"])
    with cso.Context(0) as ctx:
        ref = ctx.find_groups(pos, ids, p)["sigma"]
    s = torch.cuda.Stream()
    rc, out = static_density(torch.from_numpy(pos).to(dev), p, ctypes.c_void_p(s.cuda_stream))
    assert rc == cso.CSO_OK
    assert np.array_equal(out.cpu().numpy(), ref)


def test_static_density_rejects_oversized_requests(dev):
    p = cso.cso_params_default(32768)
    L = cso.lib()
    L.cso_density_static.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(cso.CsoParams),
                                     ctypes.c_void_p, ctypes.c_void_p]
    dummy = torch.zeros((1, 3), dtype=torch.int32, device=dev)
    out = torch.zeros(1, dtype=torch.int64, device=dev)
    rc = L.cso_density_static(dummy.data_ptr(), (1 << 20) + 1, ctypes.byref(p), out.data_ptr(), None)
    assert rc == cso.CSO_ERR_ARG and "static limit" in cso.cso_last_error()
    fine = cso.cso_params_default(16384)  # box 128: 320^3 cells, beyond the table limit
    rc = L.cso_density_static(dummy.data_ptr(), 1, ctypes.byref(fine), out.data_ptr(), None)
    assert rc == cso.CSO_ERR_ARG and "cells exceed" in cso.cso_last_error()


def test_static_density_at_its_documented_limits(dev):
    """2^20 particles (the particle limit) in a box of 64 l_mean per side (the
    largest cell table the limit admits at the default b): the scratch array
    holds the cell table, the sorted copy and the binning scratch of the
    largest request, and the sums equal the allocating path's."""
    pos, ids, meta = synth.nfw_box(64, 0.5, 20, 20000, seed=41, n_total=1 << 20)
    assert len(pos) == cso.CSO_STATIC_MAX_N
    p = cso.cso_params_default(meta["u"])
    with cso.Context(0) as ctx:
        ref = ctx.find_groups(pos, ids, p)["sigma"]
    dpos = torch.from_numpy(pos).to(dev)
    for _ in range(2):
        rc, out = static_density(dpos, p)
        assert rc == cso.CSO_OK, cso.cso_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
