"""FP64 CPU oracle of the slip-wall D2Q9 MRT lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY: the tests, `__graft_entry__.smoke()` and the CPU
baseline leg of `bench.py` use it; the product path never does.  It shares
no code with the CUDA library (`paper_2012_14707_gb300`): the parameter
formulas are in `oracle.params`, the time stepping in `lbm_oracle.c`.

Parity status per function (what pins it is in tests/test_oracle_*.py):
  * parameter formulas -- pinned (cross-identities between independently
    printed equations, the slip law of Eq. PhyscPoiSlip).
  * collision + forcing -- pinned (moment identities, conservation, rest
    state, momentum gain per step).
  * boundary scheme -- pinned (halfway bounce-back no-slip parabola at the
    magic parameter, Zhao no-slip parabola, slip Poiseuille closed forms for
    tuned and untuned parameters).
  * boundary scheme with the Maxwell part at the printed wall velocity
    (diffuse_mode 1) -- pinned per node by the wall relation of the Sec. 3.B
    channel analysis carried out for that reading
    (params.wall_recursion_coefficients_printed): plane Couette, untuned
    Poiseuille, and force plus moving wall with unequal walls.
  * curved walls (Couette) -- pinned only to within discretisation error
    (error against Eq. EqAnaMicro falls under refinement).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import params  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_LIB_OMP = os.path.join(_HERE, "liblbm_oracle_omp.so")
_SRC3 = os.path.join(_HERE, "lbm3d_oracle.c")
_LIB3 = os.path.join(_HERE, "liblbm3d_oracle.so")
_libs = {}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no target-specific flags,
    no contraction into FMAs), twice from the same source: single-threaded,
    and with OpenMP over the row loops of a step (bitwise the same results).
    Returns the single-threaded library's path."""
    for lib, src, extra in ((_LIB, _SRC, []), (_LIB_OMP, _SRC, ["-fopenmp"]), (_LIB3, _SRC3, [])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", *extra, "-shared",
                                   "-fPIC", "-o", tmp, src, "-lm"])
            os.replace(tmp, lib)
    return _LIB


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _load(threaded: bool = False):
    if threaded not in _libs:
        build()
        lib = ctypes.CDLL(_LIB_OMP if threaded else _LIB)
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        up = ctypes.POINTER(ctypes.c_uint8)
        lib.olbm_create.restype = P
        lib.olbm_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, up,
                                    ctypes.c_double, ctypes.c_double, dp, ctypes.c_int, ip, ip, ip,
                                    dp, dp, dp, dp, dp, ctypes.c_int]
        lib.olbm_step.argtypes = [P, ctypes.c_long]
        lib.olbm_fields.argtypes = [P, dp, dp, dp]
        lib.olbm_residual.argtypes = [P, dp, dp]
        lib.olbm_residual_interval.argtypes = [P, dp]
        lib.olbm_get_f.argtypes = [P, dp]
        lib.olbm_set_f.argtypes = [P, dp]
        lib.olbm_get_fpost.argtypes = [P, dp]
        lib.olbm_get_minv.argtypes = [P, dp]
        lib.olbm_steps.restype = ctypes.c_long
        lib.olbm_steps.argtypes = [P]
        lib.olbm_destroy.argtypes = [P]
        lib.olbm_set_threads.argtypes = [ctypes.c_int]
        lib.olbm_threads.restype = ctypes.c_int
        _libs[threaded] = lib
    return _libs[threaded]


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleLBM:
    """One case on the CPU in FP64.

    `par` is an `oracle.params.Parameters`; per-link r and l come from it
    unless `link_r` / `link_l` are given.  `diffuse_mode` 0 evaluates the
    Maxwell part of Eq. EqNewBDSC at the fluid velocity of x_f (the reading
    under which the analysis of Sec. 3.B holds), 1 at the wall velocity u_b
    (the equation as printed).  `threads` > 1 runs the OpenMP build of the
    same source on that many threads (bitwise the same states).
    """

    def __init__(self, case, par, link_r=None, link_l=None, diffuse_mode=0, threads=1):
        self._lib = lib = _load(threads > 1)
        if threads > 1:
            lib.olbm_set_threads(int(threads))
        self.threads = int(lib.olbm_threads())
        self.case = case
        self.par = par
        g = np.ascontiguousarray(case.link_q, np.float64)
        r, l = par.per_link(g)
        if link_l is not None:
            l = np.asarray(link_l, np.float64) * np.ones_like(g)
        if link_r is not None:
            r = np.asarray(link_r, np.float64) * np.ones_like(g)
        self.link_r = np.ascontiguousarray(r, np.float64)
        self.link_l = np.ascontiguousarray(l, np.float64)
        self._keep = [np.ascontiguousarray(case.solid, np.uint8), par.relaxation_times(),
                      np.ascontiguousarray(case.link_x, np.int32),
                      np.ascontiguousarray(case.link_y, np.int32),
                      np.ascontiguousarray(case.link_dir, np.int32), self.link_r, self.link_l, g,
                      np.ascontiguousarray(case.link_ubx, np.float64),
                      np.ascontiguousarray(case.link_uby, np.float64)]
        k = self._keep
        ip = ctypes.POINTER(ctypes.c_int32)
        self._h = lib.olbm_create(
            case.nx, case.ny, int(case.periodic_x), int(case.periodic_y),
            k[0].ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), case.ax, case.ay, _dp(k[1]),
            case.n_links, k[2].ctypes.data_as(ip), k[3].ctypes.data_as(ip),
            k[4].ctypes.data_as(ip), _dp(k[5]), _dp(k[6]), _dp(k[7]), _dp(k[8]), _dp(k[9]),
            int(diffuse_mode))
        if not self._h:
            raise ValueError("oracle rejected the case (bad link set or parameters)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.olbm_destroy(h)
            self._h = None

    def step(self, n: int = 1):
        self._lib.olbm_step(self._h, int(n))

    @property
    def steps(self) -> int:
        return int(self._lib.olbm_steps(self._h))

    def fields(self):
        n = self.case.nx * self.case.ny
        rho, ux, uy = np.empty(n), np.empty(n), np.empty(n)
        self._lib.olbm_fields(self._h, _dp(rho), _dp(ux), _dp(uy))
        s = (self.case.ny, self.case.nx)
        return rho.reshape(s), ux.reshape(s), uy.reshape(s)

    def residual(self):
        res = ctypes.c_double()
        mass = ctypes.c_double()
        self._lib.olbm_residual(self._h, ctypes.byref(res), ctypes.byref(mass))
        return res.value, mass.value

    def residual_interval(self) -> float:
        """||u^n - u^m|| / ((n - m) ||u^n||): the mean change per step since
        the previous call (since the initial state for the first)."""
        res = ctypes.c_double()
        self._lib.olbm_residual_interval(self._h, ctypes.byref(res))
        return res.value

    def get_f(self) -> np.ndarray:
        f = np.empty((9, self.case.ny, self.case.nx))
        self._lib.olbm_get_f(self._h, _dp(f))
        return f

    def get_fpost(self) -> np.ndarray:
        f = np.empty((9, self.case.ny, self.case.nx))
        self._lib.olbm_get_fpost(self._h, _dp(f))
        return f

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, np.float64).reshape(9, self.case.ny, self.case.nx)
        self._lib.olbm_set_f(self._h, _dp(f))

    def minv(self) -> np.ndarray:
        m = np.empty((9, 9))
        self._lib.olbm_get_minv(self._h, _dp(m))
        return m

    def run_to(self, tol: float, max_steps: int, every: int = 100, interval: bool = False):
        """Step in chunks of `every` until the residual (one-step, or the
        interval residual over each chunk) is below tol; returns steps done."""
        done = 0
        while done < max_steps:
            self.step(every)
            done += every
            res = self.residual_interval() if interval else self.residual()[0]
            if res < tol:
                break
        return done


def _load3d():
    if "3d" not in _libs:
        build()
        lib = ctypes.CDLL(_LIB3)
        P = ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        up = ctypes.POINTER(ctypes.c_uint8)
        c_int, c_d = ctypes.c_int, ctypes.c_double
        lib.o3d_create.restype = P
        lib.o3d_create.argtypes = [c_int, c_int, c_int, c_int, c_int, c_int, up, c_d, c_d, c_d, dp,
                                   c_int, ip, ip, ip, ip, dp, dp, dp, dp, c_int]
        lib.o3d_step.argtypes = [P, ctypes.c_long]
        lib.o3d_fields.argtypes = [P, dp, dp, dp, dp]
        lib.o3d_residual.argtypes = [P, dp, dp]
        lib.o3d_get_f.argtypes = [P, dp]
        lib.o3d_set_f.argtypes = [P, dp]
        lib.o3d_get_m.argtypes = [P, dp]
        lib.o3d_lattice.argtypes = [ip, dp]
        lib.o3d_steps.restype = ctypes.c_long
        lib.o3d_steps.argtypes = [P]
        lib.o3d_destroy.argtypes = [P]
        _libs["3d"] = lib
    return _libs["3d"]


def d3q19_lattice():
    """(c [19, 3] int, w [19]) as the 3-D oracle uses them."""
    c = np.empty((19, 3), np.int32)
    w = np.empty(19)
    _load3d().o3d_lattice(c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(w))
    return c, w


class OracleLBM3D:
    """One D3Q19 case (`cases.Case3D`) on the CPU in FP64, with the per-link
    r and l of `par` (an `oracle.params.Parameters`, the formulas of Sec. 3.B
    applied unchanged in three dimensions) and the D3Q19 relaxation times of
    `par.relaxation_times_d3q19()`."""

    def __init__(self, case, par, diffuse_mode=0, link_r=None, link_l=None):
        lib = self._lib = _load3d()
        self.case = case
        g = np.ascontiguousarray(case.link_q, np.float64)
        r, l = par.per_link(g)
        if link_l is not None:
            l = np.asarray(link_l, np.float64) * np.ones_like(g)
        if link_r is not None:
            r = np.asarray(link_r, np.float64) * np.ones_like(g)
        ip = ctypes.POINTER(ctypes.c_int32)
        k = self._keep = [np.ascontiguousarray(case.solid, np.uint8), par.relaxation_times_d3q19(),
                          np.ascontiguousarray(case.link_x, np.int32),
                          np.ascontiguousarray(case.link_y, np.int32),
                          np.ascontiguousarray(case.link_z, np.int32),
                          np.ascontiguousarray(case.link_dir, np.int32),
                          np.ascontiguousarray(r, np.float64), np.ascontiguousarray(l, np.float64), g,
                          np.ascontiguousarray(case.link_ub, np.float64)]
        self.link_r, self.link_l = k[6], k[7]
        px, py, pz = (int(v) for v in case.periodic)
        ax, ay, az = case.a
        self._h = lib.o3d_create(case.nx, case.ny, case.nz, px, py, pz,
                                 k[0].ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ax, ay, az,
                                 _dp(k[1]), case.n_links, k[2].ctypes.data_as(ip),
                                 k[3].ctypes.data_as(ip), k[4].ctypes.data_as(ip),
                                 k[5].ctypes.data_as(ip), _dp(k[6]), _dp(k[7]), _dp(k[8]), _dp(k[9]),
                                 int(diffuse_mode))
        if not self._h:
            raise ValueError("oracle rejected the 3-D case (bad link set or parameters)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.o3d_destroy(h)
            self._h = None

    def step(self, n: int = 1):
        self._lib.o3d_step(self._h, int(n))

    @property
    def steps(self) -> int:
        return int(self._lib.o3d_steps(self._h))

    def fields(self):
        c = self.case
        n = c.nx * c.ny * c.nz
        out = [np.empty(n) for _ in range(4)]
        self._lib.o3d_fields(self._h, *(_dp(a) for a in out))
        return tuple(a.reshape(c.nz, c.ny, c.nx) for a in out)

    def residual(self):
        res, mass = ctypes.c_double(), ctypes.c_double()
        self._lib.o3d_residual(self._h, ctypes.byref(res), ctypes.byref(mass))
        return res.value, mass.value

    def get_f(self) -> np.ndarray:
        c = self.case
        f = np.empty((19, c.nz, c.ny, c.nx))
        self._lib.o3d_get_f(self._h, _dp(f))
        return f

    def set_f(self, f: np.ndarray):
        c = self.case
        f = np.ascontiguousarray(f, np.float64).reshape(19, c.nz, c.ny, c.nx)
        self._lib.o3d_set_f(self._h, _dp(f))

    def moment_matrix(self) -> np.ndarray:
        m = np.empty((19, 19))
        self._lib.o3d_get_m(self._h, _dp(m))
        return m

    def run_to(self, tol: float, max_steps: int, every: int = 100):
        done = 0
        while done < max_steps:
            self.step(every)
            done += every
            if self.residual()[0] < tol:
                break
        return done
