"""The entry point that allocates no device memory (dg_cswenolimit_noalloc).

It exists for callers that must not allocate once they run (an application whose memory
manager already holds the GPU memory, a loop where cudaMalloc/cudaFree could block or
synchronise, a plugin host that forbids allocation after start-up).  It runs the TVB
indicator and the CSWENO limiter with all scratch in a fixed device array inside the
library; its results must equal, bit for bit, those of the mesh-based calls
(dg_flag_cells + dg_cswenolimit), on calls in a row (the array keeps the previous call's
contents), up to the largest mesh it accepts.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import paper_1904_11147_gb300 as dgl
from paper_1904_11147_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _entry():
    l = dgl.lib()
    f = l.dg_cswenolimit_noalloc
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    return l, f


def _mesh_based(dim, pde, N, nx, ny, box, bc, u):
    g = dgl.Mesh(dim, pde, N, [nx], [ny], [box], bc=bc)
    g.set_modes(u)
    fl, nf, nn = g.flag_cells(dgl.IND_TVB, 0.01, want=True)
    g.cswenolimit()
    out = g.get_modes()
    g.close()
    return out, nf, nn


def _untroubled(dim, pde, N, nx, ny):
    """Random cell means with higher modes far below M h^2: every face deviation stays inside
    the TVB bound, so no cell is troubled."""
    rng = np.random.default_rng(77)
    u = W.random_modes(dim, pde, N, nx * ny, rng, smooth=0.02)
    h = min(1.0 / nx, 1.0 / ny) if dim == 2 else 1.0 / nx
    u[:, :, 1:] = 1e-3 * 0.01 * h * h * rng.uniform(-1.0, 1.0, u[:, :, 1:].shape)
    return u


# the last case is the largest mesh the entry point accepts (128 x 128 = DG_NOALLOC_MAX_CELLS)
# with the largest per-cell state (2D Euler P3), so every scratch region is used to its end
@pytest.mark.parametrize("dim,pde,N,nx,ny,bc", [(2, 1, 2, 96, 80, 1), (2, 0, 3, 70, 45, 0), (1, 1, 3, 613, 1, 1),
                                                (2, 1, 3, 128, 128, 1)])
def test_noalloc_matches_mesh_entry_points_twice(dim, pde, N, nx, ny, bc):
    """Two calls in a row on different data: the same kernels as dg_flag_cells +
    dg_cswenolimit on the same input, so the limited state is bitwise equal and so are the
    troubled and near-threshold counts; in place gives the same.  A third call on smooth
    data without a troubled cell returns its input unchanged."""
    import torch
    l, f = _entry()
    box = np.array([0.0, 1.0, 0.0, 1.0])
    bp = box.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    V = 1 if pde == 0 else (3 if dim == 1 else 4)
    NP = N + 1 if dim == 1 else (N + 1) * (N + 2) // 2
    assert nx * ny <= 16384
    for call in range(3):
        if call < 2:
            rng = np.random.default_rng(4000 + call + 10 * N)
            u = W.random_modes(dim, pde, N, nx * ny, rng, smooth=0.15 if pde == 0 else 0.02)
        else:
            u = _untroubled(dim, pde, N, nx, ny)
        ref, nf_ref, nn_ref = _mesh_based(dim, pde, N, nx, ny, box, bc, u)
        # planes [var*NP + mode][cell] on the device
        planes = torch.from_numpy(np.ascontiguousarray(u.reshape(nx * ny, V * NP).T)).cuda()
        out = torch.empty_like(planes)
        nf, nn = ctypes.c_int64(-1), ctypes.c_int64(-1)
        s = f(dim, pde, N, nx, ny, bp, bc, 1.4, 0.01, planes.data_ptr(), out.data_ptr(), ctypes.byref(nf),
              ctypes.byref(nn), None)
        assert s == dgl.DG_OK, l.dg_last_error()
        torch.cuda.synchronize()
        got = out.cpu().numpy().T.reshape(nx * ny, V, NP)
        assert nf.value == nf_ref and nn.value == nn_ref
        assert (nf_ref > 0) if call < 2 else (nf_ref == 0)
        assert np.array_equal(got, ref), (call, float(np.abs(got - ref).max()))
        if call == 2:
            assert np.array_equal(got, u)
        # in place gives the same
        s = f(dim, pde, N, nx, ny, bp, bc, 1.4, 0.01, planes.data_ptr(), planes.data_ptr(), None, None, None)
        assert s == dgl.DG_OK
        torch.cuda.synchronize()
        got2 = planes.cpu().numpy().T.reshape(nx * ny, V, NP)
        assert np.array_equal(got2, ref)


def test_noalloc_rejects_large_meshes_and_allocates_nothing():
    import torch
    l, f = _entry()
    box = np.array([0.0, 1.0, 0.0, 1.0])
    bp = box.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    n = 129  # 129 x 129 > 16384 cells
    x = torch.zeros(24 * n * n, dtype=torch.float64, device="cuda")
    s = f(2, 1, 2, n, n, bp, 1, 1.4, 0.01, x.data_ptr(), x.data_ptr(), None, None, None)
    assert s == dgl.DG_EINVAL
    assert b"exceeds" in l.dg_last_error()
    # after the first call on the device, further calls leave the free device memory alone
    m = 64
    rng = np.random.default_rng(9)
    u = W.random_modes(2, 1, 2, m * m, rng, smooth=0.02)
    planes = torch.from_numpy(np.ascontiguousarray(u.reshape(m * m, 24).T)).cuda()
    out = torch.empty_like(planes)
    assert f(2, 1, 2, m, m, bp, 1, 1.4, 0.01, planes.data_ptr(), out.data_ptr(), None, None, None) == dgl.DG_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert f(2, 1, 2, m, m, bp, 1, 1.4, 0.01, planes.data_ptr(), out.data_ptr(), None, None, None) == dgl.DG_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
