"""The parent WENO limiter (dg_parent_wenolimit, DG_LIM_PARENT) against the oracle: one call
on random states of every kind, and stage-by-stage runs with it."""
import numpy as np
import pytest

import oracle
import paper_1904_11147_gb300 as dgl
from paper_1904_11147_gb300 import workloads as W
from shadow_util import shadow_stages

pytestmark = pytest.mark.gpu

CASES = [(d, p, n) for d in (1, 2) for p in (0, 1) for n in (1, 2, 3)]


@pytest.mark.parametrize("dim,pde,N", CASES)
@pytest.mark.parametrize("bc", [0, 1])
def test_parent_limiter_parity(dim, pde, N, bc):
    nx, ny = (613, 1) if dim == 1 else (70, 45)
    o = oracle.Mesh(dim, pde, N, nx, ny, box=(0.0, 1.3, 0.0, 0.9), bc=bc)
    g = dgl.Mesh(dim, pde, N, [nx], [ny], [(0.0, 1.3, 0.0, 0.9)], bc=bc)
    rng = np.random.default_rng(700 + 10 * dim + 3 * pde + N)
    u = W.random_modes(dim, pde, N, nx * ny, rng, smooth=0.15 if pde == 0 else 0.02)
    g.set_modes(u)
    fl, nf, _ = g.flag_cells(dgl.IND_TVB, 0.01, want=True)
    assert nf > 0  # the Euler cases flag every cell, boundary cells included (reflected ghosts)
    g.parent_wenolimit()
    ref = o.parent_limit(u, fl)
    got = g.get_modes()
    assert np.array_equal(got[:, :, 0], u[:, :, 0])
    scale = np.maximum(np.abs(ref).max(axis=(0, 2)), 1e-300)
    d = float((np.abs(got - ref).max(axis=(0, 2)) / scale).max())
    assert d <= 1e-11, d


def test_parent_argument_errors():
    g = dgl.Mesh(2, 0, 3, [3], [10], [(0.0, 1.0, 0.0, 1.0)])
    with pytest.raises(dgl.DGError):
        g.set_limiter(dgl.LIM_PARENT)  # 3 cells < N + 1 = 4
    g.set_modes(np.zeros((30, 1, 10)))
    g.flag_cells(dgl.IND_TVB, 0.01)
    with pytest.raises(dgl.DGError):
        g.parent_wenolimit()
    with pytest.raises(dgl.DGError):
        g.set_limiter(7)


@pytest.mark.parametrize("name", ["sod_p2_k200", "sod_p3_k200", "quadrant_p2_40", "quadrant_p3_24"])
def test_parent_shadow(name):
    import torch
    st = torch.cuda.Stream()
    if name.startswith("sod"):
        N = int(name[5])
        w = W.shock_tube("sod", 200, N)
        o = oracle.Mesh(1, 1, N, 200, box=w.box[0], bc=w.bc)
        g = dgl.Mesh(1, 1, N, [200], None, w.box, bc=w.bc, stream=st.cuda_stream)
        u0 = o.project_ic(w.ic, w.params[0])
        dt = 0.1 * (1 / 200) / o.max_wavespeed(u0)[0]
        steps = 100
    else:
        N = 2 if "p2" in name else 3
        n = 40 if N == 2 else 24
        w = W.euler_2d_quadrant(n, N, seed=1907 if N == 3 else 1904)
        o = oracle.Mesh(2, 1, N, n, n, box=w.box[0], bc=w.bc)
        g = dgl.Mesh(2, 1, N, [n], [n], w.box, bc=w.bc, stream=st.cuda_stream)
        u0 = o.project_ic(w.ic, w.params[0])
        ws = o.max_wavespeed(u0)
        dt = 0.1 / (ws[0] * n + ws[1] * n)
        steps = 30
    with torch.cuda.stream(st):
        ws_, wl, nf, done, _ = shadow_stages(o, g, u0, dt, steps, limiter="parent")
    print(name, "parent WENO: worst stage %.2e, worst limited %.2e, flagged %d" % (ws_, wl, nf))
    assert done == steps and nf > 0
