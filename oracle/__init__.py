"""CompaSO oracle loader — TEST INFRASTRUCTURE ONLY.

Loads ``libcso_oracle.so`` (plain C, built from ``cso_oracle.c`` beside this
file) through ctypes.  The oracle is a slow, single-threaded CPU statement of
the CompaSO algorithm of Hadzhiyska et al. 2021 (Sec. 2.2), used only by the
test suite, the smoke check and the benchmark's CPU-baseline leg.  The product
library never imports, links or runs anything here, and nothing here imports
the product package.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cso_oracle.c")
_LIB = os.path.join(_HERE, "libcso_oracle.so")

NONE = np.uint64(0xFFFFFFFFFFFFFFFF)

ST_NAMES = ["pairs_b", "pairs_fof", "dense", "l0_groups", "l1_nuclei", "l1_work",
            "l2_nuclei", "l2_work", "l1_halos_cat"]


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("u", ctypes.c_int64),
        ("b_kernel", ctypes.c_double), ("l_fof", ctypes.c_double),
        ("delta_L0", ctypes.c_double), ("delta_L1", ctypes.c_double), ("delta_L2", ctypes.c_double),
        ("alpha_num", ctypes.c_int32), ("alpha_den", ctypes.c_int32),
        ("roche_num", ctypes.c_int32), ("roche_den", ctypes.c_int32),
        ("np_min_density", ctypes.c_int32), ("np_min_L1", ctypes.c_int32),
        ("include_self", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("b2", ctypes.c_int64), ("lfof2", ctypes.c_int64), ("T_L0", ctypes.c_int64),
        ("T_min_L1", ctypes.c_int64), ("T_min_L2", ctypes.c_int64),
        ("K_L1", ctypes.c_double), ("K_L2", ctypes.c_double),
    ]


class OrcHalo(ctypes.Structure):
    _fields_ = [
        ("nucleus_id", ctypes.c_uint64), ("N", ctypes.c_int64), ("R2", ctypes.c_int64),
        ("R_delta", ctypes.c_double), ("com", ctypes.c_double * 3),
        ("l2max_id", ctypes.c_uint64), ("l2max_N", ctypes.c_int64), ("l2max_com", ctypes.c_double * 3),
        ("l2_top5_N", ctypes.c_int64 * 5), ("n_l2", ctypes.c_int64), ("l0_id", ctypes.c_uint64),
    ]


HALO_DTYPE = np.dtype([
    ("nucleus_id", np.uint64), ("N", np.int64), ("R2", np.int64), ("R_delta", np.float64),
    ("com", np.float64, 3), ("l2max_id", np.uint64), ("l2max_N", np.int64),
    ("l2max_com", np.float64, 3), ("l2_top5_N", np.int64, 5), ("n_l2", np.int64),
    ("l0_id", np.uint64),
])


RADIAL_DTYPE = np.dtype([
    ("centre", np.int64, 3), ("d_q", np.int64, 4), ("r_q", np.float64, 4), ("vmax_n", np.int64),
    ("vmax_d2", np.int64), ("vmax", np.float64), ("r_vmax", np.float64),
])

# fractions of the members enclosed by r_q (Table 1, r_XX_L2com)
RADIAL_PERCENT = (25, 50, 75, 98)

SHRINK_DTYPE = np.dtype([("centre", np.int64, 3), ("n", np.int64), ("R2", np.int64), ("iter", np.int64)])

# the shrinking sphere stops below max(ceil(N / 100), SHRINK_N_MIN) members (Sec. 4)
SHRINK_N_MIN = 700


def build(force=False):
    """Compile the oracle with gcc (plain -O2, no tuning)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        L.orc_derive.argtypes = [P(OrcParams)]
        L.orc_sis_central_density.argtypes = [ctypes.c_double] * 3
        L.orc_sis_central_density.restype = ctypes.c_double
        L.orc_cosmology.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        L.orc_pred.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_int64]
        L.orc_pred.restype = ctypes.c_int
        L.orc_r_search.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int64]
        L.orc_r_search.restype = ctypes.c_int64
        L.orc_density.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(OrcParams), ctypes.c_int, ctypes.c_void_p]
        L.orc_density.restype = ctypes.c_int64
        L.orc_density_at.argtypes = [ctypes.c_void_p, ctypes.c_int64, P(OrcParams), ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_void_p]
        L.orc_density_at.restype = ctypes.c_int64
        L.orc_fof.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                              P(OrcParams), ctypes.c_int, ctypes.c_void_p]
        L.orc_fof.restype = ctypes.c_int64
        L.orc_compaso.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_int64, P(OrcParams), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_int64), ctypes.c_void_p]
        L.orc_find_groups.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, P(OrcParams),
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_int64), ctypes.c_void_p]
        L.orc_halo_row.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                   ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.c_void_p, ctypes.c_void_p]
        L.orc_halo_row.restype = None
        L.orc_radial.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                 ctypes.c_int64, ctypes.c_double, ctypes.c_void_p]
        assert L.orc_sizeof_halo() == ctypes.sizeof(OrcHalo) == HALO_DTYPE.itemsize
        assert L.orc_sizeof_radial() == RADIAL_DTYPE.itemsize
        L.orc_shrink_sphere.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
        assert L.orc_sizeof_shrink() == SHRINK_DTYPE.itemsize
        assert L.orc_sizeof_params() == ctypes.sizeof(OrcParams)
        assert L.orc_stats_count() == len(ST_NAMES)
        _lib = L
    return _lib


def params(u, b_kernel=0.4, l_fof=0.25, delta_L0=60.0, delta_L1=200.0, delta_L2=800.0,
           alpha=(4, 5), roche=(2, 1), np_min_density=35, np_min_L1=35, include_self=0):
    """Paper defaults (Table 1, Einstein-de Sitter thresholds of Sec. 2.3.1);
    returns the parameter block with its derived integer thresholds."""
    p = OrcParams(u=int(u), b_kernel=b_kernel, l_fof=l_fof, delta_L0=delta_L0,
                  delta_L1=delta_L1, delta_L2=delta_L2, alpha_num=alpha[0], alpha_den=alpha[1],
                  roche_num=roche[0], roche_den=roche[1], np_min_density=np_min_density,
                  np_min_L1=np_min_L1, include_self=include_self)
    if lib().orc_derive(ctypes.byref(p)) != 0:
        raise ValueError("bad oracle parameters")
    return p


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pos(pos):
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    assert pos.ndim == 2 and pos.shape[1] == 3
    return pos


def cosmology(omega_m0, z):
    """(Delta_L0, Delta_L1, Delta_L2, l_FoF) at redshift z."""
    out = np.zeros(4)
    lib().orc_cosmology(float(omega_m0), float(z), _ptr(out))
    return tuple(out.tolist())


def pred(n, d, K, u):
    return bool(lib().orc_pred(int(n), int(d), float(K), int(u)))


def r_search(d, K, u):
    d = np.ascontiguousarray(d, dtype=np.int64)
    return int(lib().orc_r_search(_ptr(d), d.size, float(K), int(u)))


def density(pos, p, brute=False):
    pos = _pos(pos)
    sigma = np.empty(pos.shape[0], np.int64)
    pairs = lib().orc_density(_ptr(pos), pos.shape[0], ctypes.byref(p), int(brute), _ptr(sigma))
    return sigma, int(pairs)


def density_at(pos, p, which):
    pos = _pos(pos)
    which = np.ascontiguousarray(which, dtype=np.int64)
    sigma = np.empty(which.size, np.int64)
    lib().orc_density_at(_ptr(pos), pos.shape[0], ctypes.byref(p), _ptr(which), which.size, _ptr(sigma))
    return sigma


def fof(pos, ids, sigma, p, brute=False):
    pos = _pos(pos)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    sigma = np.ascontiguousarray(sigma, dtype=np.int64)
    l0 = np.empty(pos.shape[0], np.uint64)
    links = lib().orc_fof(_ptr(pos), _ptr(ids), _ptr(sigma), pos.shape[0], ctypes.byref(p), int(brute), _ptr(l0))
    return l0, int(links)


def _halos(n_cap):
    return np.zeros(max(int(n_cap), 1), HALO_DTYPE)


def compaso(pos, ids, sigma, l0, p):
    pos = _pos(pos)
    n = pos.shape[0]
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    sigma = np.ascontiguousarray(sigma, dtype=np.int64)
    l0 = np.ascontiguousarray(l0, dtype=np.uint64)
    l1 = np.empty(n, np.uint64)
    l2 = np.empty(n, np.uint64)
    st = np.zeros(len(ST_NAMES), np.int64)
    cap = max(16, n // 35 + 1)
    halos = _halos(cap)
    nh = ctypes.c_int64(0)
    rc = lib().orc_compaso(_ptr(pos), _ptr(ids), _ptr(sigma), _ptr(l0), n, ctypes.byref(p), _ptr(l1),
                           _ptr(l2), _ptr(halos), cap, ctypes.byref(nh), _ptr(st))
    assert rc == 0, rc
    return l1, l2, halos[:nh.value].copy(), dict(zip(ST_NAMES, st.tolist()))


def find_groups(pos, ids, p):
    """Whole path: Sigma, L0, L1, L2 labels (input order) and the L1 catalogue."""
    pos = _pos(pos)
    n = pos.shape[0]
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    sigma = np.empty(n, np.int64)
    l0 = np.empty(n, np.uint64)
    l1 = np.empty(n, np.uint64)
    l2 = np.empty(n, np.uint64)
    st = np.zeros(len(ST_NAMES), np.int64)
    cap = max(16, n // 35 + 1)
    halos = _halos(cap)
    nh = ctypes.c_int64(0)
    rc = lib().orc_find_groups(_ptr(pos), _ptr(ids), n, ctypes.byref(p), _ptr(sigma), _ptr(l0), _ptr(l1),
                               _ptr(l2), _ptr(halos), cap, ctypes.byref(nh), _ptr(st))
    if rc != 0:
        raise RuntimeError("oracle failed: %d" % rc)
    return dict(sigma=sigma, l0=l0, l1=l1, l2=l2, halos=halos[:nh.value].copy(),
                stats=dict(zip(ST_NAMES, st.tolist())))


def halo_row(pos, ids, l0, u, nucleus, R2, members, slot2, l2_nuclei):
    """One catalogue row of an L1 halo from its members (particle indices,
    the nucleus among them), the L1 nucleus and squared radius, and the L2
    assignment inside it: slot2[m] = ordinal of the L2 nucleus of member m
    (-1: none), l2_nuclei = particle indices of the L2 nuclei in acceptance
    order (densest first)."""
    pos = _pos(pos)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    l0 = np.ascontiguousarray(l0, dtype=np.uint64)
    members = np.ascontiguousarray(members, dtype=np.int64)
    slot2 = np.ascontiguousarray(slot2, dtype=np.int64)
    l2_nuclei = np.ascontiguousarray(l2_nuclei, dtype=np.int64)
    assert members.size == slot2.size and members.size > 0
    assert slot2.max() < l2_nuclei.size
    out = np.zeros(1, HALO_DTYPE)
    lib().orc_halo_row(_ptr(pos), _ptr(ids), _ptr(l0), int(u), int(nucleus), int(R2), _ptr(members), members.size,
                       _ptr(slot2), l2_nuclei.size, _ptr(l2_nuclei), _ptr(out))
    return out[0]


def radial(pos, l1, halos, u):
    """Radial statistics of catalogue rows (r_25/50/75/98 and V_max about the
    L2max centre of mass), members taken from the L1 labels."""
    pos = _pos(pos)
    l1 = np.ascontiguousarray(l1, dtype=np.uint64)
    halos = np.ascontiguousarray(halos, dtype=HALO_DTYPE)
    out = np.zeros(max(halos.size, 1), RADIAL_DTYPE)
    rc = lib().orc_radial(_ptr(pos), _ptr(l1), pos.shape[0], _ptr(halos), halos.size, float(u), _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle radial: a row has no members")
    return out[:halos.size].copy()


def shrink_sphere(pos, ids, l1, halos, n_min=SHRINK_N_MIN):
    """Shrinking-sphere centre of every catalogue row (Sec. 4): from the L1
    nucleus and radius, 5% smaller spheres about the rounded centre of mass
    until fewer than max(ceil(N / 100), n_min) members remain."""
    pos = _pos(pos)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    l1 = np.ascontiguousarray(l1, dtype=np.uint64)
    halos = np.ascontiguousarray(halos, dtype=HALO_DTYPE)
    out = np.zeros(max(halos.size, 1), SHRINK_DTYPE)
    rc = lib().orc_shrink_sphere(_ptr(pos), _ptr(ids), _ptr(l1), pos.shape[0], _ptr(halos), halos.size,
                                 int(n_min), _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle shrink_sphere: a row's nucleus is not among its members")
    return out[:halos.size].copy()
