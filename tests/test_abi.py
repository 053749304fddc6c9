"""The C-ABI library loads, exports every entry point its header declares,
and its host-side parameter derivation agrees bit for bit with the oracle's
independent derivation (no GPU needed)."""
import ctypes
import os
import re

import pytest

import oracle as O
from paper_2110_11408_gb300 import cso

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(cso_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    L = cso.lib()
    names = declared_functions()
    assert {"cso_init", "cso_params_derive", "cso_find_groups", "cso_submit", "cso_poll", "cso_free"} <= names
    for nm in names:
        assert hasattr(L, nm), nm


@pytest.mark.parametrize("u", [32768, 16384, 8192, 4096, 2048])
@pytest.mark.parametrize("kw", [{}, dict(alpha=(7, 10)), dict(l_fof=0.30), dict(delta_L0=40.0),
                                dict(delta_L1=258.2, delta_L2=1033.0, delta_L0=77.5)])
def test_derived_parameters_match_oracle(u, kw):
    p = cso.cso_params_default(u, **kw)
    q = O.params(u, **kw)
    for f in ("b2", "lfof2", "T_L0", "T_min_L1", "T_min_L2"):
        assert getattr(p, f) == getattr(q, f), f
    assert p.K_L1 == q.K_L1 and p.K_L2 == q.K_L2


def test_invalid_parameters_rejected():
    p = cso.cso_params_default(32768)
    p.l_mean_grid = 32768.5
    with pytest.raises(cso.CsoError):
        cso.cso_params_derive(p)
    p = cso.cso_params_default(32768)
    p.grid_bits = 20
    with pytest.raises(cso.CsoError):
        cso.cso_params_derive(p)


def test_struct_layout_matches_header():
    # offsets of the ctypes mirror follow the C declaration order with natural alignment
    assert ctypes.sizeof(cso.CsoParams) == 4 + 4 + 8 * 6 + 4 * 6 + 8 * 5 + 8 * 2
    assert ctypes.sizeof(cso.CsoHalo) == 8 * 19
    assert ctypes.sizeof(cso.CsoInput) == 8 + 8 + 8 + 4 + 4 + 4 + 4 + 8
    assert ctypes.sizeof(cso.CsoOutput) == 8 * 5 + 8 + 8 + 4 + 4 + 8
    assert cso.RADIAL_DTYPE.itemsize == 8 * 21
    # the compiled library agrees on every layout
    sizes = (ctypes.c_int64 * 5)()
    assert cso.lib().cso_struct_sizes(sizes, 5) == 5
    assert list(sizes) == [ctypes.sizeof(cso.CsoParams), ctypes.sizeof(cso.CsoHalo), ctypes.sizeof(cso.CsoInput),
                           ctypes.sizeof(cso.CsoOutput), cso.RADIAL_DTYPE.itemsize]


def test_cosmology_scaling_matches_oracle():
    for om, z in ((0.315, 0.5), (0.3, 0.0), (0.25, 2.0), (1.0, 1.0)):
        p = cso.cso_params_cosmology(cso.cso_params_default(8192), om, z)
        ref = O.cosmology(om, z)
        assert (p.delta_L0, p.delta_L1, p.delta_L2, p.l_fof) == pytest.approx(ref, rel=1e-12)


def test_probe_rejects_a_short_result_buffer():
    # argument checks come before any device call, so this runs without a GPU
    out = (ctypes.c_double * 2)()
    assert cso.lib().cso_probe_peaks(0, out, 2) == cso.CSO_ERR_ARG
    assert b"3 results" in cso.lib().cso_last_error()


def test_schedule_setters_check_their_arguments():
    # argument checks come before any context use, so these run without a GPU
    L = cso.lib()
    assert L.cso_set_schedule(None, 32, 64) == cso.CSO_ERR_ARG
    assert L.cso_set_schedule(None, 16384, 0) == cso.CSO_ERR_ARG
    assert L.cso_set_huge_group(None, 1 << 19) == cso.CSO_ERR_ARG
    assert L.cso_set_huge_group(None, 63) == cso.CSO_ERR_ARG
