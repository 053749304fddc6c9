"""Thin ctypes binding of the CompaSO C ABI (``include/cso.h``).

Argument marshalling only: every step of the group finder runs in the CUDA
kernels of ``libcso.so``.  Entry points keep the C names (cso_init,
cso_params_default, cso_params_derive, cso_find_groups, cso_submit, cso_poll,
cso_free).  Device buffers are torch CUDA tensors (torch provides device
memory and streams only); host buffers are numpy arrays.

If the library is missing, importing this module raises: there is no CPU
fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcso.so")

CSO_OK = 0
CSO_ERR_ARG = -1
CSO_ERR_BUDGET = -2
CSO_ERR_CAPACITY = -3
CSO_ERR_TIMEOUT = -4
CSO_ERR_CUDA = -5
CSO_EAGAIN = -6
CSO_ERR_STATE = -7
NO_GROUP = np.uint64(0xFFFFFFFFFFFFFFFF)
# limits of cso_density_static (include/cso.h)
CSO_STATIC_MAX_N = 1 << 20
CSO_STATIC_MAX_CELLS = 1 << 22

FLAG_BATCHED = 1
FLAG_GRAPH = 4
FLAG_RADIAL_BINS = 32
FLAG_TIMING = 2
FLAG_COUNT_PAIRS = 8
FLAG_SELECT_STRESS = 16


def FLAG_SLOTS(k):
    """served path: number of concurrent worker slots (1..15)"""
    return (int(k) & 0xF) << 8

STAT_NAMES = ["n", "dense", "l0_groups", "l1_nuclei", "l2_nuclei", "catalogue_rows", "pairs_b", "l1_work",
              "l2_work", "workspace_bytes", "launches"]


class CsoParams(ctypes.Structure):
    _fields_ = [
        ("grid_bits", ctypes.c_int32), ("include_self", ctypes.c_int32),
        ("l_mean_grid", ctypes.c_double), ("b_kernel", ctypes.c_double), ("l_fof", ctypes.c_double),
        ("delta_L0", ctypes.c_double), ("delta_L1", ctypes.c_double), ("delta_L2", ctypes.c_double),
        ("alpha_num", ctypes.c_int32), ("alpha_den", ctypes.c_int32),
        ("roche_num", ctypes.c_int32), ("roche_den", ctypes.c_int32),
        ("np_min_density", ctypes.c_int32), ("np_min_L1", ctypes.c_int32),
        ("b2", ctypes.c_int64), ("lfof2", ctypes.c_int64), ("T_L0", ctypes.c_int64),
        ("T_min_L1", ctypes.c_int64), ("T_min_L2", ctypes.c_int64),
        ("K_L1", ctypes.c_double), ("K_L2", ctypes.c_double),
    ]


class CsoHalo(ctypes.Structure):
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
assert HALO_DTYPE.itemsize == ctypes.sizeof(CsoHalo)


# one row of radial statistics (cso_radial): exact squared radii about the
# grid point nearest the L2max com and the circular-velocity peak
RADIAL_DTYPE = np.dtype([
    ("centre", np.int64, 3), ("d_q", np.int64, 4), ("r_q", np.float64, 4), ("vmax_n", np.int64),
    ("vmax_d2", np.int64), ("vmax", np.float64), ("r_vmax", np.float64),
    ("ss_centre", np.int64, 3), ("ss_n", np.int64), ("ss_R2", np.int64), ("ss_iter", np.int64),
])

# the shrinking sphere stops below max(ceil(N / 100), SHRINK_N_MIN) members
SHRINK_N_MIN = 700


class CsoInput(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_void_p), ("ids", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("on_device", ctypes.c_int32), ("x_lo", ctypes.c_int32), ("x_hi", ctypes.c_int32),
                ("request_id", ctypes.c_uint64)]


class CsoOutput(ctypes.Structure):
    _fields_ = [("l0", ctypes.c_void_p), ("l1", ctypes.c_void_p), ("l2", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("halos", ctypes.c_void_p), ("halo_cap", ctypes.c_int64),
                ("n_halos", ctypes.c_int64), ("on_device", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("radial", ctypes.c_void_p)]


class CsoError(RuntimeError):
    def __init__(self, rc, where):
        super().__init__("%s failed (%d): %s" % (where, rc, cso_last_error()))
        self.rc = rc


_lib = None


def lib(build_if_missing=True):
    """The loaded libcso.so (built in-tree on first use if absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise ImportError("libcso.so is not built (run __graft_entry__.build())")
            _build.build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.cso_init.argtypes = [P(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t, ctypes.c_uint32]
        L.cso_params_default.argtypes = [P(CsoParams), ctypes.c_double]
        L.cso_params_derive.argtypes = [P(CsoParams)]
        L.cso_autotune.argtypes = [ctypes.c_void_p, P(CsoInput), P(CsoParams), P(CsoOutput), P(ctypes.c_int32),
                                   P(ctypes.c_int32)]
        L.cso_params_cosmology.argtypes = [P(CsoParams), ctypes.c_double, ctypes.c_double]
        L.cso_find_groups.argtypes = [ctypes.c_void_p, P(CsoInput), P(CsoParams), P(CsoOutput)]
        L.cso_submit.argtypes = [ctypes.c_void_p, P(CsoInput), P(CsoParams), P(CsoOutput), P(ctypes.c_uint64)]
        L.cso_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_int32), ctypes.c_int32]
        L.cso_free.argtypes = [ctypes.c_void_p]
        L.cso_free.restype = None
        L.cso_stream.argtypes = [ctypes.c_void_p]
        L.cso_stream.restype = ctypes.c_void_p
        L.cso_stage_times.argtypes = [ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_char_p), ctypes.c_int]
        L.cso_last_stats.argtypes = [ctypes.c_void_p, P(ctypes.c_int64), ctypes.c_int]
        L.cso_last_error.restype = ctypes.c_char_p
        L.cso_ticket_times.argtypes = [ctypes.c_void_p, ctypes.c_uint64, P(ctypes.c_double), P(ctypes.c_double),
                                       P(ctypes.c_double)]
        L.cso_clock.restype = ctypes.c_double
        L.cso_struct_sizes.argtypes = [P(ctypes.c_int64), ctypes.c_int]
        L.cso_probe_peaks.argtypes = [ctypes.c_int, P(ctypes.c_double), ctypes.c_int]
        L.cso_density.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, P(CsoParams),
                                  ctypes.c_void_p, ctypes.c_int32]
        L.cso_fof.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                              P(CsoParams), ctypes.c_void_p, ctypes.c_int32]
        L.cso_levels.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_int64, P(CsoParams), P(CsoOutput)]
        _lib = L
    return _lib


def cso_last_error():
    return lib().cso_last_error().decode()


def _check(rc, where, ok=(CSO_OK,)):
    if rc not in ok:
        raise CsoError(rc, where)
    return rc


# --------------------------------------------------------------------------
# entry points (same names as the C ABI)
# --------------------------------------------------------------------------

def cso_init(device=0, budget_bytes=0, flags=0):
    h = ctypes.c_void_p()
    _check(lib().cso_init(ctypes.byref(h), int(device), int(budget_bytes), int(flags)), "cso_init")
    return h


def cso_free(ctx):
    if ctx:
        lib().cso_free(ctx)


def cso_params_default(l_mean_grid, **kw):
    """Paper defaults for u = l_mean_grid; keyword overrides of primary fields
    (alpha=(num, den) and roche=(num, den) accepted), then re-derived."""
    p = CsoParams()
    _check(lib().cso_params_default(ctypes.byref(p), float(l_mean_grid)), "cso_params_default")
    if "alpha" in kw:
        p.alpha_num, p.alpha_den = kw.pop("alpha")
    if "roche" in kw:
        p.roche_num, p.roche_den = kw.pop("roche")
    for k, v in kw.items():
        setattr(p, k, v)
    return cso_params_derive(p)


def cso_params_cosmology(p, omega_m0, z):
    """Thresholds and linking length at redshift z (flat LambdaCDM)."""
    _check(lib().cso_params_cosmology(ctypes.byref(p), float(omega_m0), float(z)), "cso_params_cosmology")
    return p


def cso_params_derive(p):
    _check(lib().cso_params_derive(ctypes.byref(p)), "cso_params_derive")
    return p


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()  # torch tensor


class Buffers:
    """Inputs/outputs of one request: torch CUDA tensors or numpy arrays."""

    def __init__(self, pos, ids, on_device, halo_cap=None, want=("l0", "l1", "l2", "sigma"), x_lo=0, x_hi=0,
                 request_id=0, out_device=None):
        n = int(pos.shape[0])
        self.n = n
        self.on_device = on_device
        self.out_device = on_device if out_device is None else bool(out_device)
        self.halo_cap = int(halo_cap if halo_cap is not None else max(16, n // 35 + 1))
        self.pos, self.ids = pos, ids
        if self.out_device:
            import torch
            dev = pos.device if on_device else torch.device("cuda", torch.cuda.current_device())
            mk = lambda: torch.empty(n, dtype=torch.int64, device=dev)
            self.halos = torch.empty(self.halo_cap * HALO_DTYPE.itemsize, dtype=torch.uint8, device=dev)
            self.radial = (torch.empty(self.halo_cap * RADIAL_DTYPE.itemsize, dtype=torch.uint8, device=dev)
                           if "radial" in want else None)
        else:
            mk = lambda: np.empty(n, np.uint64)
            self.halos = np.empty(self.halo_cap, HALO_DTYPE)
            self.radial = np.empty(self.halo_cap, RADIAL_DTYPE) if "radial" in want else None
        self.out = {k: mk() for k in want if k != "radial"}
        # x_hi > 0: the x-slab [x_lo, x_hi) of a box streamed under `request_id`
        self.cin = CsoInput(pos=_ptr(pos), ids=_ptr(ids), n=n, on_device=int(on_device), x_lo=int(x_lo),
                            x_hi=int(x_hi), request_id=int(request_id))
        self.cout = CsoOutput(l0=_ptr(self.out.get("l0")), l1=_ptr(self.out.get("l1")),
                              l2=_ptr(self.out.get("l2")), sigma=_ptr(self.out.get("sigma")),
                              halos=_ptr(self.halos), halo_cap=self.halo_cap, n_halos=0,
                              on_device=int(self.out_device), radial=_ptr(self.radial))

    def result(self):
        """Outputs as numpy (copies device tensors to the host)."""
        r = {}
        for k, v in self.out.items():
            a = v.cpu().numpy() if self.out_device else v
            r[k] = a.view(np.int64) if k == "sigma" else a.view(np.uint64)
        nh = int(self.cout.n_halos)
        if self.out_device:
            raw = self.halos[: min(nh, self.halo_cap) * HALO_DTYPE.itemsize].cpu().numpy()
            r["halos"] = raw.view(HALO_DTYPE).copy()
        else:
            r["halos"] = self.halos[: min(nh, self.halo_cap)].copy()
        if self.radial is not None:
            m = min(nh, self.halo_cap)
            if self.out_device:
                r["radial"] = self.radial[: m * RADIAL_DTYPE.itemsize].cpu().numpy().view(RADIAL_DTYPE).copy()
            else:
                r["radial"] = self.radial[:m].copy()
        r["n_halos"] = nh
        return r


def cso_find_groups(ctx, buffers, params):
    rc = lib().cso_find_groups(ctx, ctypes.byref(buffers.cin), ctypes.byref(params), ctypes.byref(buffers.cout))
    _check(rc, "cso_find_groups")
    return rc


def cso_density(ctx, pos, n_query, params):
    """Kernel sums of the first n_query particles of pos (numpy int32 [n, 3]),
    every particle a neighbour; numpy int64 [n_query]."""
    pos = np.ascontiguousarray(pos, np.int32)
    out = np.empty(int(n_query), np.int64)
    _check(lib().cso_density(ctx, _ptr(pos), pos.shape[0], int(n_query), ctypes.byref(params), _ptr(out), 0),
           "cso_density")
    return out


def cso_fof(ctx, pos, ids, sigma, params):
    """L0 labels (smallest id of the group, NO_GROUP if not dense) of the given
    particles with the given kernel sums; numpy uint64 [n]."""
    pos = np.ascontiguousarray(pos, np.int32)
    ids = np.ascontiguousarray(ids).view(np.uint64)
    sigma = np.ascontiguousarray(sigma, np.int64)
    out = np.empty(pos.shape[0], np.uint64)
    _check(lib().cso_fof(ctx, _ptr(pos), _ptr(ids), _ptr(sigma), pos.shape[0], ctypes.byref(params), _ptr(out), 0),
           "cso_fof")
    return out


def cso_levels(ctx, pos, ids, sigma, l0, params, halo_cap=None):
    """L1 and L2 labels and the catalogue inside the groups that the labels
    l0 define; returns (l1, l2, halos) as numpy arrays."""
    pos = np.ascontiguousarray(pos, np.int32)
    ids = np.ascontiguousarray(ids).view(np.uint64)
    sigma = np.ascontiguousarray(sigma, np.int64)
    l0 = np.ascontiguousarray(l0).view(np.uint64)
    n = pos.shape[0]
    cap = int(halo_cap if halo_cap is not None else max(16, n // 35 + 1))
    l1 = np.empty(n, np.uint64)
    l2 = np.empty(n, np.uint64)
    halos = np.empty(cap, HALO_DTYPE)
    out = CsoOutput(l0=None, l1=_ptr(l1), l2=_ptr(l2), sigma=None, halos=_ptr(halos), halo_cap=cap, n_halos=0,
                    on_device=0, radial=None)
    _check(lib().cso_levels(ctx, _ptr(pos), _ptr(ids), _ptr(sigma), _ptr(l0), n, ctypes.byref(params),
                            ctypes.byref(out)), "cso_levels")
    return l1, l2, halos[:out.n_halos].copy()


def cso_autotune(ctx, buffers, params):
    """Pick the batched schedule's size bins by timing this request; returns
    (giant, small)."""
    g, s = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().cso_autotune(ctx, ctypes.byref(buffers.cin), ctypes.byref(params), ctypes.byref(buffers.cout),
                              ctypes.byref(g), ctypes.byref(s)), "cso_autotune")
    return g.value, s.value


def cso_set_schedule(ctx, giant, small):
    _check(lib().cso_set_schedule(ctx, int(giant), int(small)), "cso_set_schedule")


def cso_set_huge_group(ctx, huge):
    _check(lib().cso_set_huge_group(ctx, int(huge)), "cso_set_huge_group")


def cso_submit(ctx, buffers, params):
    t = ctypes.c_uint64()
    rc = lib().cso_submit(ctx, ctypes.byref(buffers.cin), ctypes.byref(params), ctypes.byref(buffers.cout),
                          ctypes.byref(t))
    _check(rc, "cso_submit", ok=(CSO_OK, CSO_EAGAIN))
    return t.value


def cso_poll(ctx, ticket, timeout_us=-1):
    done = ctypes.c_int32()
    rc = lib().cso_poll(ctx, ctypes.c_uint64(ticket), ctypes.byref(done), int(timeout_us))
    return bool(done.value), rc


def cso_ticket_times(ctx, ticket):
    """(t_submit, t_start, t_done) of a finished ticket, host steady clock (s)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().cso_ticket_times(ctx, ctypes.c_uint64(ticket), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "cso_ticket_times")
    return a.value, b.value, c.value


def cso_clock():
    return lib().cso_clock()


def cso_stream(ctx):
    return lib().cso_stream(ctx)


def cso_stage_times(ctx):
    ms = (ctypes.c_double * 16)()
    names = (ctypes.c_char_p * 16)()
    k = lib().cso_stage_times(ctx, ms, names, 16)
    return {names[i].decode(): ms[i] for i in range(k)}


def cso_last_stats(ctx):
    a = (ctypes.c_int64 * len(STAT_NAMES))()
    k = lib().cso_last_stats(ctx, a, len(STAT_NAMES))
    return {STAT_NAMES[i]: int(a[i]) for i in range(k)}


# --------------------------------------------------------------------------
# convenience
# --------------------------------------------------------------------------

class Context:
    """Owns a cso_ctx; find_groups() runs one box through the C ABI."""

    def __init__(self, device=0, budget_bytes=0, flags=0):
        self.h = cso_init(device, budget_bytes, flags)

    def close(self):
        if self.h:
            cso_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def find_groups(self, pos, ids, params, on_device=None, halo_cap=None, radial=False):
        """pos int32 [n, 3], ids uint64/int64 [n] (numpy -> host path, torch
        CUDA -> device path).  Returns numpy outputs; radial=True adds the
        radial statistics of every catalogue row."""
        if on_device is None:
            on_device = not isinstance(pos, np.ndarray)
        if on_device and isinstance(pos, np.ndarray):
            import torch
            pos = torch.from_numpy(np.ascontiguousarray(pos, np.int32)).cuda()
            ids = torch.from_numpy(np.ascontiguousarray(ids).view(np.int64)).cuda()
        if not on_device:
            pos = np.ascontiguousarray(pos, np.int32)
            ids = np.ascontiguousarray(ids).view(np.uint64)
        want = ("l0", "l1", "l2", "sigma") + (("radial",) if radial else ())
        b = Buffers(pos, ids, on_device, halo_cap=halo_cap, want=want)
        cso_find_groups(self.h, b, params)
        return b.result()

    def submit(self, buffers, params):
        """Served path: queue one request; keep `buffers` alive until done."""
        return cso_submit(self.h, buffers, params)

    def wait(self, ticket, timeout_us=-1):
        done, rc = cso_poll(self.h, ticket, timeout_us)
        return done, rc

    def stage_times(self):
        return cso_stage_times(self.h)

    def stats(self):
        return cso_last_stats(self.h)


def cso_probe_peaks(device=0):
    """Measured pipe rates: integer add/xor and multiply-add (Tops/s), and
    broadcast 128-bit shared-memory loads (TB/s delivered to lanes)."""
    a = (ctypes.c_double * 3)()
    _check(lib().cso_probe_peaks(int(device), a, 3), "cso_probe_peaks")
    return {"alu_tops": a[0], "imad_tops": a[1], "lds_broadcast_tbs": a[2]}
