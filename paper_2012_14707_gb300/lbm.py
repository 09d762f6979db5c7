"""ctypes binding of liblbm.so (include/lbm.h), argument marshalling only.

The module-level functions carry the C names (`lbm_create`, `lbm_step`,
`lbm_fields`, `lbm_residual`, ...) and take numpy arrays or raw device
pointers; every step of the computation runs in the CUDA library.  There is
no fallback: if liblbm.so is missing or fails to load, the first call raises.
`Solver` is a small convenience wrapper around one handle.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ENOMEM, LBM_EIO = range(7)
LBM_FP64, LBM_FP32, LBM_BF16, LBM_FP16 = 0, 1, 2, 3
L_MODES = {"paper": 0, "zero": 1, "gamma": 2, "2gamma": 3, "gamma2": 4, "gamma2+gamma": 5,
           "fixed": 6}
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "bf16": LBM_BF16, "fp16": LBM_FP16}

# Every entry point include/lbm.h declares.
EXPORTS = ("lbm_params_default", "lbm_create", "lbm_step", "lbm_fields", "lbm_residual",
           "lbm_set_fields",
           "lbm_run_to", "lbm_get_f", "lbm_set_f", "lbm_link_params", "lbm_get_info",
           "lbm_precompute", "lbm_residual_noalloc", "lbm_save", "lbm_load", "lbm_destroy",
           "lbm_last_error",
           "lbm_batch_create", "lbm_batch_reset", "lbm_batch_run_to", "lbm_batch_fields",
           "lbm_batch_set_fields",
           "lbm_batch_info", "lbm_batch_set_launch", "lbm_batch_destroy", "lbm_batch_last_error",
           "lbm_net_create", "lbm_net_num_params", "lbm_net_set_params", "lbm_net_get_params",
           "lbm_net_forward", "lbm_net_gradients", "lbm_net_train_step", "lbm_net_destroy",
           "lbm_net_last_error")


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


class Domain(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("H", ctypes.c_double), ("ax", ctypes.c_double), ("ay", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("L1", ctypes.c_double), ("L2", ctypes.c_double),
                ("E", ctypes.c_double), ("l_clamp", ctypes.c_double),
                ("tau_rho", ctypes.c_double), ("tau_j", ctypes.c_double),
                ("tau_e", ctypes.c_double), ("tau_eps", ctypes.c_double),
                ("tau_s", ctypes.c_double), ("tau_q", ctypes.c_double),
                ("r_value", ctypes.c_double), ("l_value", ctypes.c_double),
                ("l_mode", ctypes.c_int32), ("diffuse_mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("residual_every", ctypes.c_int32),
                ("storage_scale", ctypes.c_double), ("collision", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("mass_mode", ctypes.c_int32),
                ("residual_mode", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_fluid", ctypes.c_int64),
                ("n_links", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("tau_s", ctypes.c_double), ("tau_q", ctypes.c_double), ("E", ctypes.c_double),
                ("E_max", ctypes.c_double), ("L1", ctypes.c_double), ("L2", ctypes.c_double),
                ("n_clamped", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("precision", ctypes.c_int32), ("pitch", ctypes.c_int32),
                ("exact_mass", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Domain3D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("periodic_z", ctypes.c_int32), ("H", ctypes.c_double), ("ax", ctypes.c_double),
                ("ay", ctypes.c_double), ("az", ctypes.c_double)]


class CaseDesc(ctypes.Structure):
    _fields_ = [("dom", Domain), ("solid", ctypes.c_void_p), ("n_links", ctypes.c_size_t),
                ("link_x", ctypes.c_void_p), ("link_y", ctypes.c_void_p),
                ("link_dir", ctypes.c_void_p), ("link_q", ctypes.c_void_p),
                ("link_ubx", ctypes.c_void_p), ("link_uby", ctypes.c_void_p),
                ("Kn", ctypes.c_double), ("params", Params)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblbm.so once and declare every signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2012_14707_gb300.build.build()")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.lbm_params_default.argtypes = [ctypes.POINTER(Params)]
    lib.lbm_params_default.restype = None
    lib.lbm_create.argtypes = [ctypes.POINTER(Domain), ctypes.POINTER(ctypes.c_uint8), ctypes.c_size_t,
                               ip, ip, ip, dp, dp, dp, ctypes.c_double, ctypes.POINTER(Params),
                               ctypes.POINTER(H)]
    lib.lbm_step.argtypes = [H, ctypes.c_int64]
    lib.lbm_fields.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.lbm_residual.argtypes = [H, dp, dp]
    lib.lbm_run_to.argtypes = [H, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), dp]
    lib.lbm_get_f.argtypes = [H, dp]
    lib.lbm_set_f.argtypes = [H, dp]
    lib.lbm_link_params.argtypes = [H, dp, dp]
    lib.lbm_set_fields.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    lib.lbm_set_fields.restype = ctypes.c_int
    lib.lbm_get_info.argtypes = [H, ctypes.POINTER(Info)]
    lib.lbm_precompute.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(Params),
                                   ctypes.c_size_t, ip, dp, dp, dp, dp, dp, ctypes.POINTER(Info)]
    lib.lbm_residual_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_void_p, dp, dp]
    lib.lbm3d_create.argtypes = [ctypes.POINTER(Domain3D), ctypes.POINTER(ctypes.c_uint8),
                                 ctypes.c_size_t, ip, ip, ip, ip, dp, dp, ctypes.c_double,
                                 ctypes.POINTER(Params), ctypes.POINTER(H)]
    lib.lbm3d_step.argtypes = [H, ctypes.c_int64]
    lib.lbm3d_residual.argtypes = [H, dp, dp]
    lib.lbm3d_get_f.argtypes = [H, dp]
    lib.lbm3d_set_f.argtypes = [H, dp]
    lib.lbm3d_link_params.argtypes = [H, dp, dp]
    lib.lbm3d_get_info.argtypes = [H, ctypes.POINTER(Info)]
    lib.lbm3d_fields.argtypes = [H, dp, dp, dp, dp]
    lib.lbm3d_destroy.argtypes = [H]
    lib.lbm3d_destroy.restype = None
    lib.lbm3d_last_error.argtypes = [H]
    lib.lbm3d_last_error.restype = ctypes.c_char_p
    lib.lbm_save.argtypes = [H, ctypes.c_char_p]
    lib.lbm_load.argtypes = [H, ctypes.c_char_p]
    lib.lbm_destroy.argtypes = [H]
    lib.lbm_destroy.restype = None
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.lbm_batch_create.argtypes = [ctypes.POINTER(CaseDesc), ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.POINTER(H)]
    lib.lbm_batch_reset.argtypes = [H]
    lib.lbm_batch_run_to.argtypes = [H, ctypes.c_double, ctypes.c_int64, ctypes.c_int32, i64p, dp,
                                     i64p]
    lib.lbm_batch_fields.argtypes = [H, ctypes.c_int32, dp, dp, dp]
    lib.lbm_batch_set_fields.argtypes = [H, ctypes.c_int32, dp, dp, dp]
    lib.lbm_batch_set_fields.restype = ctypes.c_int
    lib.lbm_batch_info.argtypes = [H, i64p, i64p, ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int32)]
    lib.lbm_batch_set_launch.argtypes = [H, ctypes.c_int32, ctypes.c_int32]
    lib.lbm_batch_set_launch.restype = ctypes.c_int
    lib.lbm_batch_destroy.argtypes = [H]
    lib.lbm_batch_destroy.restype = None
    lib.lbm_batch_last_error.argtypes = [H]
    lib.lbm_batch_last_error.restype = ctypes.c_char_p
    for name in ("lbm_batch_create", "lbm_batch_reset", "lbm_batch_run_to", "lbm_batch_fields",
                 "lbm_batch_info"):
        getattr(lib, name).restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    lib.lbm_net_create.argtypes = [ctypes.c_int32] * 8 + [ctypes.c_uint64, ctypes.c_void_p,
                                                          ctypes.POINTER(H)]
    lib.lbm_net_num_params.argtypes = [H]
    lib.lbm_net_num_params.restype = ctypes.c_int64
    lib.lbm_net_set_params.argtypes = [H, fp, ctypes.c_int64]
    lib.lbm_net_get_params.argtypes = [H, fp, ctypes.c_int64]
    lib.lbm_net_forward.argtypes = [H, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    lib.lbm_net_gradients.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, fp, dp]
    lib.lbm_net_train_step.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_float, dp]
    lib.lbm_net_destroy.argtypes = [H]
    lib.lbm_net_destroy.restype = None
    lib.lbm_net_last_error.argtypes = [H]
    lib.lbm_net_last_error.restype = ctypes.c_char_p
    for name in ("lbm_net_create", "lbm_net_set_params", "lbm_net_get_params", "lbm_net_forward",
                 "lbm_net_gradients", "lbm_net_train_step"):
        getattr(lib, name).restype = ctypes.c_int
    lib.lbm_last_error.argtypes = [H]
    lib.lbm_last_error.restype = ctypes.c_char_p
    for name in ("lbm_create", "lbm_step", "lbm_fields", "lbm_residual", "lbm_run_to",
                 "lbm_get_f", "lbm_set_f", "lbm_link_params", "lbm_get_info", "lbm_precompute",
                 "lbm_residual_noalloc"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, h=None):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_last_error(h).decode())
    return rc


# --------------------------------------------------------------------------
# the C entry points under their own names
# --------------------------------------------------------------------------

def lbm_params_default() -> Params:
    p = Params()
    load().lbm_params_default(ctypes.byref(p))
    return p


def lbm_create(nx, ny, periodic_x, periodic_y, H, ax, ay, solid, link_x, link_y, link_dir,
               link_q, link_ubx, link_uby, Kn, params: Params):
    """Returns an opaque handle (int); raises LbmError on failure."""
    lib = load()
    dom = Domain(int(nx), int(ny), int(bool(periodic_x)), int(bool(periodic_y)), float(H),
                 float(ax), float(ay))
    solid = np.ascontiguousarray(solid, np.uint8).reshape(-1)
    if solid.size != int(nx) * int(ny):
        raise ValueError("solid mask must hold nx*ny entries")
    arrs = [np.ascontiguousarray(a, t) for a, t in
            ((link_x, np.int32), (link_y, np.int32), (link_dir, np.int32),
             (link_q, np.float64), (link_ubx, np.float64), (link_uby, np.float64))]
    n = arrs[0].size
    if any(a.size != n for a in arrs):
        raise ValueError("link arrays differ in length")
    ip = ctypes.POINTER(ctypes.c_int32)
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(dom), solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n,
                        arrs[0].ctypes.data_as(ip), arrs[1].ctypes.data_as(ip),
                        arrs[2].ctypes.data_as(ip), _dp(arrs[3]), _dp(arrs[4]), _dp(arrs[5]),
                        float(Kn), ctypes.byref(params), ctypes.byref(h))
    _check(rc, None)
    return h.value


def lbm_step(h, n: int):
    _check(load().lbm_step(h, int(n)), h)


def lbm_fields(h, rho, ux, uy, on_device: bool = False):
    """Host numpy arrays (float64, nx*ny) or device pointers (int) when
    on_device; None skips a field."""
    lib = load()
    if on_device:
        _check(lib.lbm_fields(h, rho, ux, uy, 1), h)
        return
    ptr = [None if a is None else a.ctypes.data for a in (rho, ux, uy)]
    for a in (rho, ux, uy):
        if a is not None and (a.dtype != np.float64 or not a.flags.c_contiguous):
            raise ValueError("field arrays must be C-contiguous float64")
    _check(lib.lbm_fields(h, ptr[0], ptr[1], ptr[2], 0), h)


def lbm_residual(h):
    """Returns (residual, mass); raises LbmError(LBM_EUNSTABLE) on non-finite state."""
    r, m = ctypes.c_double(), ctypes.c_double()
    _check(load().lbm_residual(h, ctypes.byref(r), ctypes.byref(m)), h)
    return r.value, m.value


def lbm_run_to(h, tol: float, max_steps: int):
    done, res = ctypes.c_int64(), ctypes.c_double()
    _check(load().lbm_run_to(h, float(tol), int(max_steps), ctypes.byref(done), ctypes.byref(res)), h)
    return done.value, res.value


def lbm_get_f(h, out: np.ndarray):
    _check(load().lbm_get_f(h, _dp(out)), h)


def lbm_set_f(h, f: np.ndarray):
    f = np.ascontiguousarray(f, np.float64)
    _check(load().lbm_set_f(h, _dp(f)), h)


def lbm_save(h, path: str):
    """Checkpoint the solver state to `path` (see include/lbm.h)."""
    _check(load().lbm_save(h, os.fsencode(path)), h)


def lbm_load(h, path: str):
    """Resume from a checkpoint of the same case."""
    _check(load().lbm_load(h, os.fsencode(path)), h)


def lbm_set_fields(h, rho, ux, uy, on_device: bool = False):
    """Warm start from density / velocity fields (host float64 arrays of
    nx*ny, or device pointers when on_device)."""
    lib = load()
    if on_device:
        _check(lib.lbm_set_fields(h, rho, ux, uy, 1), h)
        return
    arrs = [np.ascontiguousarray(a, np.float64).reshape(-1) for a in (rho, ux, uy)]
    _check(lib.lbm_set_fields(h, arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data, 0), h)


def lbm_link_params(h, n_links: int):
    r, l = np.empty(n_links), np.empty(n_links)
    _check(load().lbm_link_params(h, _dp(r), _dp(l)), h)
    return r, l


def lbm_get_info(h) -> Info:
    info = Info()
    _check(load().lbm_get_info(h, ctypes.byref(info)), h)
    return info


def lbm_precompute(Kn, H, params: Params, link_dir, link_q, link_ubx=None, link_uby=None):
    """Host-only FP64 precompute: returns (r, l, info)."""
    d = np.ascontiguousarray(link_dir, np.int32)
    q = np.ascontiguousarray(link_q, np.float64)
    ubx = np.zeros_like(q) if link_ubx is None else np.ascontiguousarray(link_ubx, np.float64)
    uby = np.zeros_like(q) if link_uby is None else np.ascontiguousarray(link_uby, np.float64)
    r, l = np.empty(q.size), np.empty(q.size)
    info = Info()
    _check(load().lbm_precompute(float(Kn), float(H), ctypes.byref(params), q.size,
                                 d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(q), _dp(ubx),
                                 _dp(uby), _dp(r), _dp(l), ctypes.byref(info)), None)
    return r, l, info


def lbm_residual_noalloc(f_cur_ptr: int, f_prev_ptr: int, solid_ptr: int, nx: int, ny: int,
                         ax: float, ay: float, stream: int | None = None):
    """Residual and mass of caller-held device state without any device
    allocation (see include/lbm.h).  Pointers are device addresses: f_cur and
    f_prev 9*nx*ny float64 populations in the lbm_get_f layout, solid nx*ny
    uint8.  Returns (residual, mass)."""
    r, m = ctypes.c_double(), ctypes.c_double()
    _check(load().lbm_residual_noalloc(f_cur_ptr, f_prev_ptr, solid_ptr, int(nx), int(ny),
                                       float(ax), float(ay), stream, ctypes.byref(r),
                                       ctypes.byref(m)), None)
    return r.value, m.value


def lbm_destroy(h):
    if h:
        load().lbm_destroy(h)


def lbm_last_error(h=None) -> str:
    return load().lbm_last_error(h).decode()


# --------------------------------------------------------------------------
# convenience wrapper
# --------------------------------------------------------------------------

class Solver:
    """One case on the GPU.

    `case` is a `cases.Case`.  Keyword arguments override the parameter
    defaults of include/lbm.h: precision ("fp32" | "fp64" | "bf16" | "fp16"), l_mode (a name of
    L_MODES or a float for a fixed l), r (fixed r), tau_q, tau_s, E, L1, L2,
    sigma, diffuse_mode, residual_every, stream (a cudaStream_t as int),
    mass_mode (FP32: 0 auto, 1 always, -1 never the exact-mass step),
    residual_mode (0 one-step, 1 interval residual).
    """

    def __init__(self, case, precision="fp32", l_mode="paper", r=None, tau_q=None, tau_s=None,
                 E=None, L1=None, L2=None, sigma=1.0, diffuse_mode=0, residual_every=100,
                 stream=None, tau_e=1.1, tau_eps=1.2, l_clamp=-0.4, storage_scale=0.0,
                 bgk=False, mass_mode=0, residual_mode=0):
        p = lbm_params_default()
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if isinstance(l_mode, str):
            p.l_mode = L_MODES[l_mode]
        else:
            p.l_mode = L_MODES["fixed"]
            p.l_value = float(l_mode)
        nan = math.nan
        p.r_value = nan if r is None else float(r)
        p.tau_q = nan if tau_q is None else float(tau_q)
        p.tau_s = nan if tau_s is None else float(tau_s)
        p.E = nan if E is None else float(E)
        p.L1 = nan if L1 is None else float(L1)
        p.L2 = nan if L2 is None else float(L2)
        p.sigma = float(sigma)
        p.tau_e, p.tau_eps, p.l_clamp = float(tau_e), float(tau_eps), float(l_clamp)
        p.diffuse_mode = int(diffuse_mode)
        p.residual_every = int(residual_every)
        p.storage_scale = float(storage_scale)
        p.collision = 1 if bgk else 0
        p.stream = stream
        p.mass_mode = int(mass_mode)
        p.residual_mode = int(residual_mode)
        self.case = case
        self.params = p
        self.h = None
        self.h = lbm_create(case.nx, case.ny, case.periodic_x, case.periodic_y, case.H, case.ax,
                            case.ay, case.solid, case.link_x, case.link_y, case.link_dir,
                            case.link_q, case.link_ubx, case.link_uby, case.Kn, p)

    def close(self):
        if self.h:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lbm_step(self.h, n)

    def residual(self):
        return lbm_residual(self.h)

    def run_to(self, tol, max_steps):
        return lbm_run_to(self.h, tol, max_steps)

    def fields(self):
        n = self.case.nx * self.case.ny
        rho, ux, uy = np.empty(n), np.empty(n), np.empty(n)
        lbm_fields(self.h, rho, ux, uy)
        s = (self.case.ny, self.case.nx)
        return rho.reshape(s), ux.reshape(s), uy.reshape(s)

    def get_f(self):
        f = np.empty((9, self.case.ny, self.case.nx))
        lbm_get_f(self.h, f)
        return f

    def set_f(self, f):
        lbm_set_f(self.h, f)

    def save(self, path: str):
        lbm_save(self.h, path)

    def load(self, path: str):
        lbm_load(self.h, path)

    def link_params(self):
        return lbm_link_params(self.h, self.case.n_links)

    def set_fields(self, rho, ux, uy):
        lbm_set_fields(self.h, rho, ux, uy)

    def info(self) -> Info:
        return lbm_get_info(self.h)


# --------------------------------------------------------------------------
# batched solver
# --------------------------------------------------------------------------

def _bcheck(rc, b=None):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_batch_last_error(b).decode())


def make_params(**kw) -> Params:
    """lbm_params_t with the keyword overrides of `Solver`."""
    p = lbm_params_default()
    l_mode = kw.pop("l_mode", "paper")
    if isinstance(l_mode, str):
        p.l_mode = L_MODES[l_mode]
    else:
        p.l_mode = L_MODES["fixed"]
        p.l_value = float(l_mode)
    for key, field in (("r", "r_value"), ("tau_q", "tau_q"), ("tau_s", "tau_s"), ("E", "E"),
                       ("L1", "L1"), ("L2", "L2")):
        v = kw.pop(key, None)
        setattr(p, field, math.nan if v is None else float(v))
    if kw.pop("bgk", False):
        p.collision = 1
    for key in ("sigma", "diffuse_mode", "tau_e", "tau_eps", "l_clamp", "storage_scale",
                "mass_mode", "residual_mode"):
        if key in kw:
            setattr(p, key, kw.pop(key))
    if kw:
        raise TypeError(f"unknown parameters {sorted(kw)}")
    return p


class Batch:
    """Many cases advanced together (lbm_batch_*).  `cases` is a list of
    `cases.Case`; `params` an optional list of keyword dicts (see
    `Solver`) per case."""

    def __init__(self, case_list, precision="fp32", params=None, stream=None):
        lib = load()
        self.cases = list(case_list)
        n = len(self.cases)
        descs = (CaseDesc * n)()
        self._keep = []
        for k, c in enumerate(self.cases):
            arrs = [np.ascontiguousarray(c.solid, np.uint8).reshape(-1),
                    np.ascontiguousarray(c.link_x, np.int32), np.ascontiguousarray(c.link_y, np.int32),
                    np.ascontiguousarray(c.link_dir, np.int32),
                    np.ascontiguousarray(c.link_q, np.float64),
                    np.ascontiguousarray(c.link_ubx, np.float64),
                    np.ascontiguousarray(c.link_uby, np.float64)]
            self._keep.append(arrs)
            d = descs[k]
            d.dom = Domain(c.nx, c.ny, int(c.periodic_x), int(c.periodic_y), c.H, c.ax, c.ay)
            d.solid = arrs[0].ctypes.data
            d.n_links = c.n_links
            d.link_x, d.link_y, d.link_dir = (arrs[1].ctypes.data, arrs[2].ctypes.data,
                                              arrs[3].ctypes.data)
            d.link_q, d.link_ubx, d.link_uby = (arrs[4].ctypes.data, arrs[5].ctypes.data,
                                                arrs[6].ctypes.data)
            d.Kn = c.Kn
            d.params = make_params(**(params[k] if params else {}))
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        _bcheck(lib.lbm_batch_create(descs, n, prec, stream, ctypes.byref(h)))
        self.h = h.value
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            load().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _bcheck(load().lbm_batch_reset(self.h), self.h)

    def run_to(self, tol: float, max_steps: int, check_every: int = 100):
        """Returns (steps per case, residual per case, total steps)."""
        n = len(self.cases)
        steps = np.zeros(n, np.int64)
        res = np.zeros(n)
        tot = ctypes.c_int64()
        _bcheck(load().lbm_batch_run_to(self.h, float(tol), int(max_steps), int(check_every),
                                        steps.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        _dp(res), ctypes.byref(tot)), self.h)
        return steps, res, tot.value

    def fields(self, k: int):
        c = self.cases[k]
        n = c.nx * c.ny
        rho, ux, uy = np.empty(n), np.empty(n), np.empty(n)
        _bcheck(load().lbm_batch_fields(self.h, int(k), _dp(rho), _dp(ux), _dp(uy)), self.h)
        s = (c.ny, c.nx)
        return rho.reshape(s), ux.reshape(s), uy.reshape(s)

    def set_fields(self, k: int, rho, ux, uy):
        arrs = [np.ascontiguousarray(a, np.float64).reshape(-1) for a in (rho, ux, uy)]
        _bcheck(load().lbm_batch_set_fields(self.h, int(k), _dp(arrs[0]), _dp(arrs[1]),
                                            _dp(arrs[2])), self.h)

    def info(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        t, nt = ctypes.c_int32(), ctypes.c_int32()
        _bcheck(load().lbm_batch_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t),
                                      ctypes.byref(nt)), self.h)
        return dict(total_nodes=a.value, total_fluid=b.value, cta_threads=t.value, n_ctas=nt.value)

    def set_launch(self, cta_threads: int, l2_prefetch: bool):
        """Override the autotuned launch shape (lbm_batch_set_launch)."""
        _bcheck(load().lbm_batch_set_launch(self.h, int(cta_threads), int(bool(l2_prefetch))),
                self.h)


# --------------------------------------------------------------------------
# warm-start network
# --------------------------------------------------------------------------

def _ncheck(rc, n=None):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_net_last_error(n).decode())


class Net:
    """The warm-start encoder-decoder (lbm_net_*).  Inputs and outputs are
    device pointers (int) to NHWC FP32 arrays, e.g. torch tensors'
    data_ptr()."""

    def __init__(self, H, W, base=32, levels=4, c_in=3, c_out=3, precision="bf16", max_batch=8,
                 seed=0, stream=None):
        lib = load()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        _ncheck(lib.lbm_net_create(base, levels, c_in, c_out, prec, max_batch, H, W, seed, stream,
                                   ctypes.byref(h)))
        self.h = h.value
        self.H, self.W, self.c_in, self.c_out, self.max_batch = H, W, c_in, c_out, max_batch

    def _call(self, rc):
        """Status check of a network call.  LBM_ETIMEOUT leaves the network
        unspecified (a tensor-core kernel gave up on a bounded wait): it is
        destroyed, and later calls fail."""
        if rc == LBM_ETIMEOUT:
            msg = load().lbm_net_last_error(self.h).decode()
            self.close()
            raise LbmError(rc, msg + " (network destroyed)")
        _ncheck(rc, self.h)

    def _live(self):
        if not getattr(self, "h", None):
            raise LbmError(LBM_EINVAL, "network was destroyed")
        return self.h

    @property
    def n_params(self) -> int:
        return int(load().lbm_net_num_params(self._live()))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, np.float32)
        self._call(load().lbm_net_get_params(self._live(),
                                             p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        self._call(load().lbm_net_set_params(self._live(),
                                             p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size))

    def forward(self, x_ptr: int, n: int, y_ptr: int):
        self._call(load().lbm_net_forward(self._live(), x_ptr, int(n), y_ptr))

    def gradients(self, x_ptr: int, t_ptr: int, n: int):
        g = np.empty(self.n_params, np.float32)
        loss = ctypes.c_double()
        self._call(load().lbm_net_gradients(self._live(), x_ptr, t_ptr, int(n),
                                            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                            ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, x_ptr: int, t_ptr: int, n: int, lr: float) -> float:
        loss = ctypes.c_double()
        self._call(load().lbm_net_train_step(self._live(), x_ptr, t_ptr, int(n), float(lr),
                                             ctypes.byref(loss)))
        return loss.value

    def close(self):
        if getattr(self, "h", None):
            load().lbm_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# three dimensions (lbm3d_*)
# --------------------------------------------------------------------------

def _check3(rc, h=None):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm3d_last_error(h).decode())


class Solver3D:
    """One D3Q19 case (`cases.Case3D`) on the GPU.  Keyword arguments as for
    `Solver` (precision "fp64" or "fp32")."""

    def __init__(self, case, precision="fp32", stream=None, **kw):
        lib = load()
        p = make_params(**kw)
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.stream = stream
        self.case = case
        px, py, pz = (int(bool(v)) for v in case.periodic)
        dom = Domain3D(case.nx, case.ny, case.nz, px, py, pz, float(case.H), *(float(v) for v in case.a))
        solid = np.ascontiguousarray(case.solid, np.uint8).reshape(-1)
        arrs = [np.ascontiguousarray(a, t) for a, t in
                ((case.link_x, np.int32), (case.link_y, np.int32), (case.link_z, np.int32),
                 (case.link_dir, np.int32), (case.link_q, np.float64))]
        ub = np.ascontiguousarray(case.link_ub, np.float64).reshape(-1)
        self._keep = (solid, arrs, ub)
        ip = ctypes.POINTER(ctypes.c_int32)
        h = ctypes.c_void_p()
        rc = lib.lbm3d_create(ctypes.byref(dom), solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                              arrs[0].size, *(a.ctypes.data_as(ip) for a in arrs[:4]),
                              _dp(arrs[4]), _dp(ub), float(case.Kn), ctypes.byref(p), ctypes.byref(h))
        _check3(rc, None)
        self.h = h.value

    def step(self, n=1):
        _check3(load().lbm3d_step(self.h, int(n)), self.h)

    def residual(self):
        r, m = ctypes.c_double(), ctypes.c_double()
        _check3(load().lbm3d_residual(self.h, ctypes.byref(r), ctypes.byref(m)), self.h)
        return r.value, m.value

    def get_f(self):
        c = self.case
        f = np.empty((19, c.nz, c.ny, c.nx))
        _check3(load().lbm3d_get_f(self.h, _dp(f)), self.h)
        return f

    def set_f(self, f):
        f = np.ascontiguousarray(f, np.float64)
        _check3(load().lbm3d_set_f(self.h, _dp(f)), self.h)

    def fields(self):
        """(rho, ux, uy, uz) [nz, ny, nx] (lbm3d_fields); solid nodes 0."""
        c = self.case
        out = [np.empty((c.nz, c.ny, c.nx)) for _ in range(4)]
        _check3(load().lbm3d_fields(self.h, *(_dp(a) for a in out)), self.h)
        return tuple(out)

    def run_to(self, tol, max_steps, every=100):
        done, res = 0, math.inf
        while done < max_steps:
            self.step(every)
            done += every
            res = self.residual()[0]
            if res < tol:
                break
        return done, res

    def link_params(self):
        n = self.case.n_links
        r, l = np.empty(n), np.empty(n)
        _check3(load().lbm3d_link_params(self.h, _dp(r), _dp(l)), self.h)
        return r, l

    def info(self) -> Info:
        """lbm3d_get_info: sizes, parameters, device bytes, exact_mass."""
        info = Info()
        _check3(load().lbm3d_get_info(self.h, ctypes.byref(info)), self.h)
        return info

    def close(self):
        if getattr(self, "h", None):
            load().lbm3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
