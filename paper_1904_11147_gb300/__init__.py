"""GB300-native RKDG + compact subcell WENO (CSWENO) limiter.

Python binding of the C ABI in ``include/dg.h`` (ctypes; argument marshalling only --
every step of the method runs in the CUDA kernels of ``libcswenodg.so``).  There is no
CPU fallback: if the library cannot be loaded, importing ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcswenodg.so")

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_EPOSITIVITY, DG_ETIMEOUT, DG_ESTATE = range(7)
BURGERS, EULER = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_DMR = 0, 1, 2
IND_TVB, IND_MLP, IND_KXRCF = 0, 1, 2
LIM_CSWENO, LIM_PARENT = 0, 1
IC_SINE, IC_RIEMANN1D, IC_QUADRANT, IC_DENSITY_WAVE = 0, 1, 2, 3
IC_DMR = 6
STATUS_NAMES = {0: "DG_OK", 1: "DG_EINVAL", 2: "DG_ENOMEM", 3: "DG_ECUDA", 4: "DG_EPOSITIVITY",
                5: "DG_ETIMEOUT", 6: "DG_ESTATE"}

_lock = threading.Lock()
_lib = None


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def lib():
    """Load (building first if needed) the CUDA library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                from . import build as _b
                _b.build()
            l = ctypes.CDLL(LIB_PATH)
            D, I, P = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_void_p
            l.dg_mesh_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, I, I, D,
                                         ctypes.c_int, ctypes.c_double, P, ctypes.POINTER(P)]
            l.dg_mesh_destroy.argtypes = [P]
            l.dg_mesh_size.argtypes = [P]
            l.dg_mesh_size.restype = ctypes.c_size_t
            l.dg_set_modes.argtypes = [P, P, ctypes.c_size_t, ctypes.c_int]
            l.dg_get_modes.argtypes = [P, P, ctypes.c_size_t, ctypes.c_int]
            l.dg_project_ic.argtypes = [P, ctypes.c_int, D, ctypes.c_int]
            l.dg_set_dt.argtypes = [P, D]
            l.dg_rk_stage.argtypes = [P, ctypes.c_int, ctypes.c_double]
            l.dg_flag_cells.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_uint8)]
            l.dg_cswenolimit.argtypes = [P]
            l.dg_step.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_double]
            l.dg_max_wavespeed.argtypes = [P, D]
            l.dg_kernel_launches.argtypes = [P]
            l.dg_kernel_launches.restype = ctypes.c_int64
            l.dg_last_error.restype = ctypes.c_char_p
            l.dg_limiter_tables.argtypes = [ctypes.c_int, D, D, D, D, D, D]
            F = ctypes.POINTER(ctypes.c_float)
            l.dg_mlp_features.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
            l.dg_mlp_create.argtypes = [ctypes.c_int, ctypes.c_uint64, P, ctypes.POINTER(P)]
            l.dg_mlp_destroy.argtypes = [P]
            l.dg_mlp_param_count.argtypes = [P]
            l.dg_mlp_param_count.restype = ctypes.c_size_t
            l.dg_mlp_get_params.argtypes = [P, F, ctypes.c_size_t]
            l.dg_mlp_set_params.argtypes = [P, F, ctypes.c_size_t]
            l.dg_mlp_grad.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_float, F, F]
            l.dg_mlp_train_step.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_float, ctypes.c_float, F]
            l.dg_set_indicator_mlp.argtypes = [P, P, ctypes.c_float]
            l.dg_mlp_predict.argtypes = [P, P, ctypes.c_int64, P]
            l.dg_positivity_report.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
            l.dg_positivity_report.restype = ctypes.c_int
            l.dg_flag_statistics.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
            l.dg_flag_statistics.restype = ctypes.c_int
            l.dg_autotune.argtypes = [P, ctypes.c_double, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]
            l.dg_autotune.restype = ctypes.c_int
            l.dg_indicator_logits.argtypes = [P, P]
            l.dg_refined_arith.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, P]
            l.dg_set_boundary_data.argtypes = [P, D, ctypes.c_int]
            l.dg_set_boundary_data.restype = ctypes.c_int
            l.dg_set_time.argtypes = [P, D]
            l.dg_set_time.restype = ctypes.c_int
            l.dg_get_time.argtypes = [P, D]
            l.dg_get_time.restype = ctypes.c_int
            l.dg_refined_arith.restype = ctypes.c_int
            l.dg_harvest.argtypes = [P, ctypes.c_double, P, P, P]
            l.dg_positivity_limit.argtypes = [P, ctypes.c_double]
            l.dg_parent_wenolimit.argtypes = [P]
            l.dg_max_wavespeed_points.argtypes = [P, D]
            l.dg_set_limiter.argtypes = [P, ctypes.c_int]
            l.dg_set_positivity.argtypes = [P, ctypes.c_int, ctypes.c_double]
            l.dg_positivity_counts.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                               ctypes.c_int]
            for name in ("dg_mesh_create", "dg_mesh_destroy", "dg_set_modes", "dg_get_modes", "dg_project_ic",
                         "dg_set_dt", "dg_rk_stage", "dg_flag_cells", "dg_cswenolimit", "dg_step",
                         "dg_max_wavespeed", "dg_limiter_tables", "dg_mlp_create", "dg_mlp_destroy",
                         "dg_mlp_get_params", "dg_mlp_set_params", "dg_mlp_grad", "dg_mlp_train_step",
                         "dg_set_indicator_mlp", "dg_indicator_logits", "dg_harvest", "dg_mlp_predict",
                         "dg_positivity_limit", "dg_set_positivity", "dg_positivity_counts",
                         "dg_parent_wenolimit", "dg_set_limiter", "dg_max_wavespeed_points"):
                getattr(l, name).restype = ctypes.c_int
            _lib = l
    return _lib


def _check(status):
    if status != DG_OK:
        raise DGError(status, lib().dg_last_error().decode(errors="replace"))


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def limiter_tables(N: int):
    """The CSWENO tables the library derived for degree N (host-only call)."""
    ng = 2 if N == 1 else 4
    n1 = N + 1
    rp, rw = np.zeros(ng), np.zeros(ng)
    C = np.zeros((n1, ng, n1))
    gam = np.zeros((ng, n1))
    B = np.zeros((n1, n1, n1))
    SA = np.zeros((2 * N + 1, n1))
    _check(lib().dg_limiter_tables(N, _dp(rp), _dp(rw), _dp(C), _dp(gam), _dp(B), _dp(SA)))
    return dict(pt=rp, wt=rw, C=C, gam=gam, B=B, SA=SA)


class Mesh:
    """A batch of meshes on the current CUDA device (see ``dg_mesh_create``).

    ``stream`` is a raw ``cudaStream_t`` value (e.g. ``torch.cuda.current_stream().cuda_stream``)
    or 0 for the legacy default stream.
    """

    def __init__(self, dim, pde, N, nx, ny=None, box=None, bc=BC_PERIODIC, gamma=1.4, stream=0):
        nx = [int(v) for v in np.atleast_1d(nx)]
        n_inst = len(nx)
        ny = [1] * n_inst if (ny is None or dim == 1) else [int(v) for v in np.atleast_1d(ny)]
        if box is None:
            box = [(0.0, 1.0, 0.0, 1.0)] * n_inst
        box = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(n_inst, 4))
        self.dim, self.pde, self.N, self.n_inst, self.bc = dim, pde, N, n_inst, bc
        self.nx, self.ny, self.box = nx, ny, box
        self.nv = 1 if pde == BURGERS else (3 if dim == 1 else 4)
        self.np = N + 1 if dim == 1 else (N + 1) * (N + 2) // 2
        self.cells = sum(a * b for a, b in zip(nx, ny))
        self._h = ctypes.c_void_p()
        nxa = (ctypes.c_int * n_inst)(*nx)
        nya = (ctypes.c_int * n_inst)(*ny)
        _check(lib().dg_mesh_create(dim, pde, N, n_inst, nxa, nya, _dp(box), bc, gamma,
                                    ctypes.c_void_p(int(stream)), ctypes.byref(self._h)))
        self.size = int(lib().dg_mesh_size(self._h))

    def close(self):
        if self._h:
            lib().dg_mesh_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- data movement --------------------------------------------------------------------
    def set_modes(self, modes):
        """modes: numpy array (host) or a CUDA tensor (device), layout [cell][var][mode]."""
        if hasattr(modes, "is_cuda") and modes.is_cuda:
            assert modes.is_contiguous() and modes.numel() == self.size and str(modes.dtype) == "torch.float64"
            _check(lib().dg_set_modes(self._h, ctypes.c_void_p(modes.data_ptr()), self.size, 1))
            return
        if hasattr(modes, "numpy"):
            assert str(modes.dtype) == "torch.float64" and modes.is_contiguous() and modes.numel() == self.size
            _check(lib().dg_set_modes(self._h, ctypes.c_void_p(modes.data_ptr()), self.size, 0))
            return
        a = np.ascontiguousarray(modes, dtype=np.float64)
        assert a.size == self.size
        _check(lib().dg_set_modes(self._h, a.ctypes.data_as(ctypes.c_void_p), self.size, 0))

    def get_modes(self, out=None):
        """Returns a numpy array [cell][var][mode], or fills ``out`` (numpy or CUDA tensor)."""
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            _check(lib().dg_get_modes(self._h, ctypes.c_void_p(out.data_ptr()), self.size, 1))
            return out
        if out is not None and hasattr(out, "numpy"):
            _check(lib().dg_get_modes(self._h, ctypes.c_void_p(out.data_ptr()), self.size, 0))
            return out
        a = np.empty((self.cells, self.nv, self.np)) if out is None else out
        _check(lib().dg_get_modes(self._h, a.ctypes.data_as(ctypes.c_void_p), self.size, 0))
        return a

    def project_ic(self, ic, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(self.n_inst, -1))
        _check(lib().dg_project_ic(self._h, ic, _dp(p), p.shape[1]))

    def set_dt(self, dt):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (self.n_inst,)))
        _check(lib().dg_set_dt(self._h, _dp(d)))

    def set_boundary_data(self, p):
        """dg_set_boundary_data (BC_DMR meshes): post-shock and pre-shock (rho, u, v, p), then
        a, b, c of the shock line x_s(y, t) = a + b y + c t."""
        a = np.ascontiguousarray(p, dtype=np.float64)
        _check(lib().dg_set_boundary_data(self._h, _dp(a), a.size))

    def set_time(self, t):
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(t, dtype=np.float64), (self.n_inst,)))
        _check(lib().dg_set_time(self._h, _dp(d)))

    def get_time(self):
        d = np.zeros(self.n_inst)
        _check(lib().dg_get_time(self._h, _dp(d)))
        return d

    # -- the method ----------------------------------------------------------------------
    def rk_stage(self, stage, dt):
        _check(lib().dg_rk_stage(self._h, stage, dt))

    def flag_cells(self, indicator=IND_TVB, M=0.01, want=False, near_cells=False):
        """dg_flag_cells.  want: return (troubled bytes, n_flagged, n_near); near_cells: also
        the per-cell near-threshold bytes (bit 1 of the library's flag bytes)."""
        if not (want or near_cells):
            _check(lib().dg_flag_cells(self._h, indicator, M, None, None, None))
            return None
        nf, nn = ctypes.c_int64(0), ctypes.c_int64(0)
        fl = np.zeros(self.cells, dtype=np.uint8)
        _check(lib().dg_flag_cells(self._h, indicator, M, ctypes.byref(nf), ctypes.byref(nn),
                                   fl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))
        if near_cells:
            return fl & 1, int(nf.value), int(nn.value), (fl >> 1) & 1
        return fl & 1, int(nf.value), int(nn.value)

    def cswenolimit(self):
        _check(lib().dg_cswenolimit(self._h))

    def step(self, dt, indicator=IND_TVB, M=0.01):
        _check(lib().dg_step(self._h, dt, indicator, M))

    def parent_wenolimit(self):
        """Parent WENO limiter on the flagged cells (see dg_parent_wenolimit)."""
        _check(lib().dg_parent_wenolimit(self._h))

    def set_limiter(self, limiter):
        """Limiter of step() with the TVB / KXRCF indicators: LIM_CSWENO or LIM_PARENT."""
        _check(lib().dg_set_limiter(self._h, int(limiter)))

    def positivity_limit(self, eps0=1e-13):
        """Positivity-preserving scaling of the current state (see dg_positivity_limit)."""
        _check(lib().dg_positivity_limit(self._h, eps0))

    def set_positivity(self, enable=True, eps0=1e-13):
        """Apply the positivity-preserving scaling after every stage's limiter in step()."""
        _check(lib().dg_set_positivity(self._h, int(enable), eps0))

    def positivity_counts(self, reset=False):
        """(cells changed, cells with an inadmissible mean) by the scaling so far."""
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        lib().dg_positivity_counts(self._h, ctypes.byref(a), ctypes.byref(b), int(reset))
        return int(a.value), int(b.value)

    def max_wavespeed(self, points=False):
        """[n_inst][2] largest wave speeds per direction, over the cell means or (points,
        Euler) over the positivity check points."""
        out = np.zeros(2 * self.n_inst)
        fn = lib().dg_max_wavespeed_points if points else lib().dg_max_wavespeed
        _check(fn(self._h, _dp(out)))
        return out.reshape(self.n_inst, 2)

    @property
    def launches(self):
        return int(lib().dg_kernel_launches(self._h))

    # -- learned indicator -------------------------------------------------------------
    def harvest(self, X, flags, change, M=0.01):
        """Features, TVB flags and the limiter's relative change of the current state into
        CUDA tensors (float32, uint8, float32), then limits the state with the TVB indicator."""
        _check(lib().dg_harvest(self._h, M, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(flags.data_ptr()),
                                ctypes.c_void_p(change.data_ptr())))

    def set_indicator(self, net, tau=0.0):
        _check(lib().dg_set_indicator_mlp(self._h, net._h, tau))

    def autotune(self, dt):
        """Chooses the stage form (split, or fused with its tile height and launch form) and
        the limiter grid on this mesh (see dg_autotune); returns (tile rows, 0 for the split
        stage; limiter blocks per SM; persistent)."""
        a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().dg_autotune(self._h, dt, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return int(a.value), int(b.value), int(c.value)

    def flag_statistics(self, reset=False):
        """(TVB-flagged, limited, passes) totals over the dg_step limiter passes."""
        a, b, c = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().dg_flag_statistics(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), int(reset)))
        return int(a.value), int(b.value), int(c.value)

    def positivity_report(self):
        """(fallbacks, failures) of the learned indicator's positivity screen."""
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        lib().dg_positivity_report(self._h, ctypes.byref(a), ctypes.byref(b))
        return int(a.value), int(b.value)

    def logits(self, out):
        _check(lib().dg_indicator_logits(self._h, ctypes.c_void_p(out.data_ptr())))
        return out


def refined_arith(op, x, out, stream=0):
    """dg_refined_arith on CUDA float64 tensors: op 0 reciprocal, 1 square root."""
    _check(lib().dg_refined_arith(int(op), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  x.numel(), ctypes.c_void_p(int(stream))))
    return out


def n_features(dim, pde, N):
    return int(lib().dg_mlp_features(dim, pde, N))


class MLP:
    """The learned indicator's network (see dg_mlp_create); inputs are CUDA tensors."""

    def __init__(self, n_features, seed=0, stream=0):
        self._h = ctypes.c_void_p()
        _check(lib().dg_mlp_create(int(n_features), int(seed), ctypes.c_void_p(int(stream)), ctypes.byref(self._h)))
        self.F = int(n_features)
        self.P = int(lib().dg_mlp_param_count(self._h))

    def close(self):
        if self._h:
            lib().dg_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros(self.P, dtype=np.float32)
        _check(lib().dg_mlp_get_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.P))
        return out

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        assert a.size == self.P
        _check(lib().dg_mlp_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), self.P))

    def grad(self, X, y, pos_weight=1.0):
        g = np.zeros(self.P, dtype=np.float32)
        loss = ctypes.c_float(0)
        _check(lib().dg_mlp_grad(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()), X.shape[0],
                                 pos_weight, g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)))
        return g, float(loss.value)

    def predict(self, X, out):
        _check(lib().dg_mlp_predict(self._h, ctypes.c_void_p(X.data_ptr()), X.shape[0], ctypes.c_void_p(out.data_ptr())))
        return out

    def train_step(self, X, y, pos_weight=1.0, lr=1e-3, want_loss=False):
        loss = ctypes.c_float(0)
        _check(lib().dg_mlp_train_step(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       X.shape[0], pos_weight, lr, ctypes.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None
