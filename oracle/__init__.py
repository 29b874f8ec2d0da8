"""CPU oracle for the CSWENO-limited RKDG method -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It wraps ``oracle.c`` (plain FP64 C, single-threaded,
compiled with ``-ffp-contract=off`` so that no fused multiply-add changes its rounding)
through ctypes and shares nothing with the CUDA library.

Modal arrays use the library's public layout ``[cell][var][mode]`` with
``cell = iy * nx + ix``; 2D modes are ordered by total degree, then by the y-degree.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against
the paper's printed constants (Sec. 3, P2 tables and smoothness indicators), closed
forms, invariants or brute force.  The P3 limiter constants have no printed values;
they are pinned by an independent derivation and by polynomial reproduction only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PDE_BURGERS, PDE_EULER = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_DMR = 0, 1, 2
IC_SINE, IC_RIEMANN1D, IC_QUADRANT, IC_DENSITY_WAVE = 0, 1, 2, 3
IC_DMR = 6


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` beside it (plain gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", _LIB_PATH + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("pde", ctypes.c_int), ("N", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("bc", ctypes.c_int),
                ("xL", ctypes.c_double), ("xR", ctypes.c_double),
                ("yL", ctypes.c_double), ("yR", ctypes.c_double), ("gamma", ctypes.c_double),
                ("t", ctypes.c_double), ("bcp", ctypes.c_double * 11)]


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.POINTER(ctypes.c_long)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            M = ctypes.POINTER(_Mesh)
            l.or_rhs.argtypes = [M, _D, _D]
            l.or_rk_stage.argtypes = [M, ctypes.c_int, ctypes.c_double, _D, _D, _D]
            l.or_flag_tvb.argtypes = [M, _D, ctypes.c_double, _U8, _L]
            l.or_flag_tvb.restype = ctypes.c_long
            l.or_flag_tvb_cells.argtypes = [M, _D, ctypes.c_double, _U8, _U8, _L]
            l.or_flag_tvb_cells.restype = ctypes.c_long
            l.or_flag_kxrcf_cells.argtypes = [M, _D, _U8, _U8, _L, _D]
            l.or_flag_kxrcf_cells.restype = ctypes.c_long
            l.or_weno_points.argtypes = [ctypes.c_int, ctypes.c_int, _D, ctypes.c_double, _D]
            l.or_csweno_limit.argtypes = [M, _D, _U8, _D, ctypes.c_double]
            l.or_step.argtypes = [M, ctypes.c_double, _D, ctypes.c_double, ctypes.c_int, ctypes.c_double, _L]
            l.or_step.restype = ctypes.c_long
            l.or_step_pp.argtypes = [M, ctypes.c_double, _D, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_double, _L, _L, _L]
            l.or_step_pp.restype = ctypes.c_long
            l.or_positivity_limit.argtypes = [M, _D, ctypes.c_double, _L]
            l.or_flag_kxrcf.argtypes = [M, _D, _U8, _L, _D]
            l.or_flag_kxrcf.restype = ctypes.c_long
            l.or_step_ind.argtypes = [M, ctypes.c_double, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_double, _L, _L, _L]
            l.or_step_ind.restype = ctypes.c_long
            l.or_positivity_limit.restype = ctypes.c_long
            l.or_max_wavespeed.argtypes = [M, _D, _D]
            l.or_project_ic.argtypes = [M, ctypes.c_int, _D, _D]
            l.or_euler_eigen.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, _D, _D, _D]
            l.or_weno_export.argtypes = [ctypes.c_int, _D, _D, _D, _D, _D, _D, _D, _I, _D]
            l.or_weno_export_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, _D, _D,
                                           _D, _I, _D]
            l.or_parent_weno_limit.argtypes = [M, _D, _U8, _D, ctypes.c_double]
            l.or_step_gen.argtypes = [M, ctypes.c_double, _D, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_double, _L, _L, _L]
            l.or_step_gen.restype = ctypes.c_long
            l.or_max_wavespeed_points.argtypes = [M, _D, _D]
            l.or_max_wavespeed_points.restype = ctypes.c_int
            l.or_dg_export.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D]
            _lib = l
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def nmodes(dim: int, N: int) -> int:
    return N + 1 if dim == 1 else (N + 1) * (N + 2) // 2


def nvars(dim: int, pde: int) -> int:
    return 1 if pde == PDE_BURGERS else (3 if dim == 1 else 4)


def mode_ab(dim: int, N: int):
    """(a, b) degrees of every mode in storage order."""
    if dim == 1:
        return [(n, 0) for n in range(N + 1)]
    out = []
    for d in range(N + 1):
        for b in range(d + 1):
            out.append((d - b, b))
    return out


class Mesh:
    """One mesh instance: dim 1 or 2, pde, degree N, nx x ny cells on the box, bc."""

    def __init__(self, dim, pde, N, nx, ny=1, box=(0.0, 1.0, 0.0, 1.0), bc=BC_PERIODIC, gamma=1.4, bcp=None):
        """bc = BC_DMR (2D Euler): bcp holds the double Mach reflection data -- post-shock
        (rho, u, v, p), pre-shock (rho, u, v, p), and a, b, c of the shock line
        x_s(y, t) = a + b y + c t; the attribute t is the time of the states passed."""
        if dim == 1:
            ny = 1
        self.dim, self.pde, self.N, self.nx, self.ny, self.bc = dim, pde, N, nx, ny, bc
        self.box = tuple(float(b) for b in box)
        assert len(self.box) == 4
        self.gamma = float(gamma)
        self.bcp = [0.0] * 11 if bcp is None else [float(x) for x in bcp]
        assert len(self.bcp) == 11
        self.t = 0.0
        self._m = _Mesh(dim, pde, N, nx, ny, bc, *self.box, self.gamma, 0.0, (ctypes.c_double * 11)(*self.bcp))
        self.nv = nvars(dim, pde)
        self.np = nmodes(dim, N)
        self.shape = (nx * ny, self.nv, self.np)

    @property
    def h(self):
        xL, xR, yL, yR = self.box
        return ((xR - xL) / self.nx, (yR - yL) / self.ny if self.dim == 2 else None)

    def _ref(self):
        self._m.t = float(self.t)
        return ctypes.byref(self._m)

    def zeros(self):
        return np.zeros(self.shape, dtype=np.float64)

    def _chk(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.size == self.nx * self.ny * self.nv * self.np
        return u.reshape(self.shape)

    def rhs(self, u):
        u = self._chk(u)
        L = self.zeros()
        lib().or_rhs(self._ref(), _dp(u), _dp(L))
        return L

    def rk_stage(self, stage, dt, un, us):
        un, us = self._chk(un), self._chk(us)
        out = self.zeros()
        lib().or_rk_stage(self._ref(), stage, dt, _dp(un), _dp(us), _dp(out))
        return out

    def flag_tvb(self, u, M=0.01, near_cells=False):
        """TVB flags: (flags, n_flagged, n_near), plus the per-cell near-threshold bytes
        when near_cells is set."""
        u = self._chk(u)
        fl = np.zeros(self.nx * self.ny, dtype=np.uint8)
        nc = np.zeros(self.nx * self.ny, dtype=np.uint8)
        near = ctypes.c_long(0)
        n = lib().or_flag_tvb_cells(self._ref(), _dp(u), M, fl.ctypes.data_as(_U8), nc.ctypes.data_as(_U8),
                                    ctypes.byref(near))
        if near_cells:
            return fl, int(n), int(near.value), nc
        return fl, int(n), int(near.value)

    def limit(self, u, flags, eps=1e-6):
        u = self._chk(u)
        fl = np.ascontiguousarray(flags, dtype=np.uint8)
        out = self.zeros()
        lib().or_csweno_limit(self._ref(), _dp(u), fl.ctypes.data_as(_U8), _dp(out), eps)
        return out

    def step(self, u, dt, M=0.01, limit=True, eps=1e-6):
        """One SSP-RK3 step, limiter after each stage. Returns (u_new, n_flagged, n_near)."""
        u = self._chk(u).copy()
        near = ctypes.c_long(0)
        nf = lib().or_step(self._ref(), dt, _dp(u), M, int(limit), eps, ctypes.byref(near))
        return u, int(nf), int(near.value)

    def flag_kxrcf(self, u, near_cells=False):
        """KXRCF troubled-cell flags. Returns (flags, n_flagged, n_near, ratio), ratio the
        largest indicator value over the indicator variables of each cell, plus the per-cell
        near-threshold bytes when near_cells is set."""
        u = self._chk(u)
        flags = np.zeros(self.nx * self.ny, dtype=np.uint8)
        nc = np.zeros(self.nx * self.ny, dtype=np.uint8)
        ratio = np.zeros(self.nx * self.ny)
        near = ctypes.c_long(0)
        nf = lib().or_flag_kxrcf_cells(self._ref(), _dp(u), flags.ctypes.data_as(_U8), nc.ctypes.data_as(_U8),
                                       ctypes.byref(near), _dp(ratio))
        if near_cells:
            return flags, int(nf), int(near.value), ratio, nc
        return flags, int(nf), int(near.value), ratio

    def parent_limit(self, u, flags, eps=1e-6):
        """Parent WENO limiter (whole cells j-N..j+N) on the flagged cells (Jacobi)."""
        u = self._chk(u)
        out = np.empty_like(u)
        fl = np.ascontiguousarray(flags, dtype=np.uint8)
        lib().or_parent_weno_limit(self._ref(), _dp(u), fl.ctypes.data_as(_U8), _dp(out), eps)
        return out

    def step_gen(self, u, dt, indicator="tvb", limiter="csweno", M=0.01, eps=1e-6, pp=False, pp_eps=1e-13):
        """SSP-RK3 step with indicator "tvb"/"kxrcf" and limiter "csweno"/"parent"/"none".
        Returns (u_new, n_flagged, n_near, n_changed, n_bad)."""
        ind = {"tvb": 0, "kxrcf": 2}[indicator]
        lim = {"none": 0, "csweno": 1, "parent": 2}[limiter]
        u = self._chk(u).copy()
        near, npp, bad = ctypes.c_long(0), ctypes.c_long(0), ctypes.c_long(0)
        nf = lib().or_step_gen(self._ref(), dt, _dp(u), ind, M, lim, eps, int(pp), pp_eps, ctypes.byref(near),
                               ctypes.byref(npp), ctypes.byref(bad))
        return u, int(nf), int(near.value), int(npp.value), int(bad.value)

    def step_ind(self, u, dt, indicator="tvb", M=0.01, limit=True, eps=1e-6, pp=False, pp_eps=1e-13):
        """SSP-RK3 step with indicator "tvb" or "kxrcf" (and the optional positivity scaling).
        Returns (u_new, n_flagged, n_near, n_changed, n_bad)."""
        ind = {"tvb": 0, "kxrcf": 2}[indicator]
        u = self._chk(u).copy()
        near, npp, bad = ctypes.c_long(0), ctypes.c_long(0), ctypes.c_long(0)
        nf = lib().or_step_ind(self._ref(), dt, _dp(u), ind, M, int(limit), eps, int(pp), pp_eps,
                               ctypes.byref(near), ctypes.byref(npp), ctypes.byref(bad))
        return u, int(nf), int(near.value), int(npp.value), int(bad.value)

    def positivity_limit(self, u, eps0=1e-13):
        """Zhang-Shu positivity-preserving scaling (Euler). Returns (u_new, cells changed,
        cells with an inadmissible mean)."""
        u = self._chk(u).copy()
        bad = ctypes.c_long(0)
        n = lib().or_positivity_limit(self._ref(), _dp(u), eps0, ctypes.byref(bad))
        if n < 0:
            raise ValueError("the positivity-preserving scaling is defined for the Euler equations")
        return u, int(n), int(bad.value)

    def step_pp(self, u, dt, M=0.01, limit=True, eps=1e-6, pp=True, pp_eps=1e-13):
        """SSP-RK3 step with the positivity-preserving scaling after each stage's limiter.
        Returns (u_new, n_flagged, n_near, n_changed, n_bad)."""
        u = self._chk(u).copy()
        near, npp, bad = ctypes.c_long(0), ctypes.c_long(0), ctypes.c_long(0)
        nf = lib().or_step_pp(self._ref(), dt, _dp(u), M, int(limit), eps, int(pp), pp_eps, ctypes.byref(near),
                              ctypes.byref(npp), ctypes.byref(bad))
        return u, int(nf), int(near.value), int(npp.value), int(bad.value)

    def max_wavespeed(self, u):
        u = self._chk(u)
        out = np.zeros(2)
        lib().or_max_wavespeed(self._ref(), _dp(u), _dp(out))
        return out

    def max_wavespeed_points(self, u):
        """Largest |v_d| + c over the positivity check points (Euler), per direction."""
        u = self._chk(u)
        out = np.zeros(2)
        if lib().or_max_wavespeed_points(self._ref(), _dp(u), _dp(out)) != 0:
            raise ValueError("defined for the Euler equations")
        return out

    def project_ic(self, kind, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        out = self.zeros()
        lib().or_project_ic(self._ref(), kind, _dp(p), _dp(out))
        return out


def euler_eigen(dim, gamma, direction, u):
    nv = 3 if dim == 1 else 4
    u = np.ascontiguousarray(u, dtype=np.float64)
    R = np.zeros((nv, nv))
    L = np.zeros((nv, nv))
    lib().or_euler_eigen(dim, gamma, direction, _dp(u), _dp(R), _dp(L))
    return R, L


def weno_points(N: int, avg, eps: float = 1e-6, parent: bool = False):
    """Point values at the Step 1 points from 2N+1 stencil averages (Steps 2-5)."""
    a = np.ascontiguousarray(avg, dtype=np.float64)
    assert a.shape == (2 * N + 1,)
    out = np.zeros(2 if N == 1 else 4)
    lib().or_weno_points(N, int(parent), _dp(a), eps, _dp(out))
    return out


def weno_tables(N: int, parent: bool = False, points=None):
    """The CSWENO tables the oracle derived for degree N (Sec. 3, Steps 1-4); parent: the
    full-width stencil of the parent WENO limiter; points: reconstruction points r in
    [-1, 1] instead of the Step 1 points."""
    ns = 2 * N + 1
    ng = (2 if N == 1 else 4) if points is None else len(points)
    pt, wt = np.zeros(ng), np.zeros(ng)
    C = np.zeros((N + 1, ng, ns))
    D = np.zeros((ng, ns))
    gam = np.zeros((ng, N + 1))
    B = np.zeros((N + 1, ns, ns))
    SA = np.zeros((ns, N + 1))
    OFF = np.zeros(ns, dtype=np.int32)
    resid = ctypes.c_double(0)
    rin = np.ascontiguousarray(points if points is not None else [0.0], dtype=np.float64)
    lib().or_weno_export_g(N, int(parent), 0 if points is None else ng, _dp(rin), _dp(pt), _dp(wt), _dp(C), _dp(D),
                           _dp(gam), _dp(B), _dp(SA), OFF.ctypes.data_as(_I), ctypes.byref(resid))
    return dict(pt=pt, wt=wt, C=C, D=D, gam=gam, B=B, SA=SA, OFF=OFF, resid=resid.value)


def dg_tables(N: int, nq: int):
    x, w = np.zeros(nq), np.zeros(nq)
    P, dP = np.zeros((nq, N + 1)), np.zeros((nq, N + 1))
    lib().or_dg_export(N, nq, _dp(x), _dp(w), _dp(P), _dp(dP))
    return x, w, P, dP
