"""The positivity-preserving scaling (dg_positivity_limit, dg_set_positivity) against the
oracle: one call on states with many inadmissible check points, and SSP-RK3 runs with the
scaling after every stage's limiter on problems that lose positivity without it."""
import numpy as np
import pytest

import oracle
import paper_1904_11147_gb300 as dgl
from paper_1904_11147_gb300 import workloads as W
from shadow_util import shadow_stages

pytestmark = pytest.mark.gpu


def _rel(a, b):
    scale = np.maximum(np.abs(b).max(axis=(0, 2)), 1e-300)
    return float((np.abs(np.asarray(a).reshape(b.shape) - b).max(axis=(0, 2)) / scale).max())


def _hostile(dim, N, ncell, rng):
    """Admissible means with large random higher modes."""
    u = W.random_modes(dim, 1, N, ncell, rng, smooth=0.0)
    for k in range(1, u.shape[2]):
        u[:, :, k] = rng.uniform(-0.6, 0.6, u[:, :, 0].shape) * np.abs(u[:, :, 0]) / k
    return u


@pytest.mark.parametrize("dim,N", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
@pytest.mark.parametrize("eps0", [1e-13, 1e-6])
def test_positivity_limit_parity(dim, N, eps0):
    nx, ny = (1000, 1) if dim == 1 else (61, 37)  # ragged against the 128-thread blocks
    o = oracle.Mesh(dim, 1, N, nx, ny, box=(0, 1, 0, 1), bc=1)
    g = dgl.Mesh(dim, 1, N, [nx], [ny], [(0.0, 1.0, 0.0, 1.0)], bc=1)
    rng = np.random.default_rng(100 + 10 * dim + N)
    u = _hostile(dim, N, nx * ny, rng)
    u[5, 0, 0] = -u[5, 0, 0]  # one inadmissible mean
    g.set_modes(u)
    g.positivity_limit(eps0)
    got = g.get_modes()
    ref, n, bad = o.positivity_limit(u, eps0)
    assert bad == 1 and n > nx * ny // 10
    assert g.positivity_counts() == (n, bad)
    assert np.array_equal(got[:, :, 0], u[:, :, 0])
    unchanged = np.all(ref == u, axis=(1, 2))
    assert np.array_equal(got[unchanged], u[unchanged])  # untouched cells bitwise
    assert _rel(got, ref) <= 1e-12, _rel(got, ref)


@pytest.mark.parametrize("dim,N", [(1, 2), (2, 2), (2, 3)])
def test_fp32_screen_at_the_threshold(dim, N):
    """Cells at rest whose smallest check-point density or pressure lies just below or just
    above eps (relative offsets down to 1e-7, far inside the FP32 screen's margin yet
    resolved by FP64) beside cells the screen clears: the screen may send a cell to the
    FP64 pass but must never skip one that needs scaling, so the changed cells and the
    scaled state equal the oracle's (unchanged cells bitwise)."""
    eps0, gam = 1e-6, 1.4
    offs = [-1e-3, -1e-5, -1e-7, 1e-7, 1e-5, 1e-3, 1.0, 1e3, 1e5]
    ab = oracle.mode_ab(dim, N) if dim == 2 else [(k, 0) for k in range(N + 1)]
    lin = ab.index((1, 0))  # linear in x: extreme at the check points x = -1, 1
    psi0, psi1 = 1 / np.sqrt(2), np.sqrt(1.5)
    c0 = psi0 * psi0 if dim == 2 else psi0  # cell mean = U_0 c0
    k1 = psi1 * psi0 if dim == 2 else psi1  # |phi_lin| at x = -1, 1
    E = dim + 1
    cells = []
    for var in (0, E):  # density, then energy (pressure (gamma - 1) E at rest)
        for off in offs:
            for mean in (1.0, 0.5):
                u = np.zeros((dim + 2, len(ab)))
                u[0, 0] = mean / c0
                u[E, 0] = mean / (gam - 1) / c0
                drop = mean - eps0 * (1 + off)  # the mean minus the smallest point value
                u[var, lin] = drop / k1 if var == 0 else drop / ((gam - 1) * k1)
                cells.append(u)
    u = np.array(cells)
    n = len(cells)
    o = oracle.Mesh(dim, 1, N, n, 1, box=(0, 1, 0, 1), bc=1)
    g = dgl.Mesh(dim, 1, N, [n], [1], [(0.0, 1.0, 0.0, 1.0)], bc=1)
    g.set_modes(u)
    g.positivity_limit(eps0)
    got = g.get_modes()
    ref, changed, bad = o.positivity_limit(u, eps0)
    assert bad == 0 and g.positivity_counts() == (changed, 0)
    assert changed == 2 * 2 * sum(1 for off in offs if off < 0), changed
    unchanged = np.all(ref == u, axis=(1, 2))
    assert np.array_equal(got[unchanged], u[unchanged])
    assert _rel(got, ref) <= 1e-12


def test_positivity_argument_errors():
    g = dgl.Mesh(1, 0, 2, [16], None, [(0.0, 1.0, 0.0, 1.0)])
    with pytest.raises(dgl.DGError):
        g.positivity_limit()
    with pytest.raises(dgl.DGError):
        g.set_positivity(True)
    e = dgl.Mesh(1, 1, 2, [16], None, [(0.0, 1.0, 0.0, 1.0)])
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(dgl.DGError):
            e.positivity_limit(bad)


def test_step_with_scaling_tube_p3_k800():
    """Seeded random tube 10 (density ratio near 10), P3, K = 800: without the scaling both
    sides reach a negative density in the second step; with it, 100 steps stay admissible
    and match the oracle step by step."""
    w = W.shock_tube("random", 800, 3, index=10)
    o = oracle.Mesh(1, 1, 3, 800, box=w.box[0], bc=w.bc)
    import torch
    st = torch.cuda.Stream()
    g = dgl.Mesh(1, 1, 3, [800], None, w.box, bc=w.bc, stream=st.cuda_stream)
    u0 = o.project_ic(w.ic, w.params[0])
    dt = 0.1 * (1 / 800) / o.max_wavespeed(u0)[0]
    with torch.cuda.stream(st):
        ws, wl, nf, done, _ = shadow_stages(o, g, u0, dt, 100, pp_eps=1e-13)
    gc, gbad = g.positivity_counts()
    print("tube 10 with scaling: worst stage %.2e, worst limited/scaled %.2e, cells scaled %d" % (ws, wl, gc))
    assert done == 100 and gc > 0 and gbad == 0


def test_step_with_scaling_quadrant_p3():
    """2D Euler P3 four-quadrant problem (seed 31) on 38 x 38: the plain method reaches a
    negative pressure within 5 steps; with the scaling 30 steps stay admissible and match
    the oracle step by step (CUDA graph path, six extra launches per step: the FP32 screen
    and the FP64 scaling after each stage)."""
    n = 38
    w = W.euler_2d_quadrant(n, 3, seed=31)
    o = oracle.Mesh(2, 1, 3, n, n, box=w.box[0], bc=w.bc)
    import torch
    st = torch.cuda.Stream()
    g = dgl.Mesh(2, 1, 3, [n], [n], w.box, bc=w.bc, stream=st.cuda_stream)
    u0 = o.project_ic(w.ic, w.params[0])
    ws = o.max_wavespeed(u0)
    dt = 0.1 / (ws[0] * n + ws[1] * n)
    with torch.cuda.stream(st):
        ws, wl, nf, done, _ = shadow_stages(o, g, u0, dt, 30, pp_eps=1e-13)
    gc, gbad = g.positivity_counts()
    print("quadrant seed 31 with scaling: worst stage %.2e, worst limited/scaled %.2e, cells scaled %d"
          % (ws, wl, gc))
    assert done == 30 and gc > 0 and gbad == 0
    before = g.launches
    g.step(dt)
    g.set_positivity(False)
    g.step(dt)
    assert g.launches - before == 2 * 18 + 6


def _points(dim, N):
    gl = np.array([-1.0, 1.0]) if N == 1 else np.array([-1.0, 0.0, 1.0])
    if dim == 1:
        return [(x, None) for x in gl]
    g, _ = np.polynomial.legendre.leggauss(N + 1)
    return [(r, s) for r in g for s in gl] + [(r, s) for r in gl for s in g]


def _cell_bound(dim, N, u, gam=1.4):
    """max over cells of (max |v_d| + max c) over each cell's check points (numpy)."""
    ab = oracle.mode_ab(dim, N) if dim == 2 else [(k, 0) for k in range(N + 1)]

    def psi(n, x):
        c = np.zeros(n + 1)
        c[n] = 1.0
        return np.sqrt((2 * n + 1) / 2) * np.polynomial.legendre.legval(x, c)

    pts = _points(dim, N)
    Phi = np.array([[psi(a, r) * (psi(b, s) if dim == 2 else 1.0) for a, b in ab] for r, s in pts])
    q = np.einsum("cvk,pk->cpv", u, Phi)
    rho = q[..., 0]
    kin = q[..., 1] ** 2 + (q[..., 2] ** 2 if dim == 2 else 0.0)
    c2 = gam * (gam - 1) * (q[..., -1] - 0.5 * kin / rho) / rho
    ok = c2 >= 0
    cs = np.sqrt(np.where(ok, c2, 0.0).max(axis=1))
    return [np.max(np.where(ok, np.abs(q[..., 1 + d] / rho), 0.0).max(axis=1) + cs) for d in range(dim)]


@pytest.mark.parametrize("dim,N", [(1, 2), (1, 3), (2, 2), (2, 3)])
def test_max_wavespeed_points_parity(dim, N):
    """dg_max_wavespeed_points per instance, on three instances whose cells share warps (two
    with large higher modes and non-admissible points, one nearly uniform).  The
    kernel takes, per cell, max |v_d| + max c over the check points (one square root per
    cell): an upper bound of the oracle's pointwise maximum of |v_d| + c, which any
    admissible time step may use, and at most twice it (max|v| + max c <= 2 max(|v| + c)).
    Checked: oracle <= GPU <= 2 oracle (up to rounding), and GPU = the numpy evaluation of
    the cell bound."""
    sizes = [(331, 1), (250, 1), (97, 1)] if dim == 1 else [(33, 17), (20, 40), (16, 9)]
    g = dgl.Mesh(dim, 1, N, [s[0] for s in sizes], [s[1] for s in sizes], [(0.0, 1.0, 0.0, 1.0)] * 3, bc=1)
    rng = np.random.default_rng(60 + 10 * dim + N)
    us = [_hostile(dim, N, nx * ny, rng) for nx, ny in sizes[:2]]
    # a uniform flow with 1e-9 perturbations: every cell's FP32 bounds overlap the maximum
    # (the FP32 screen keeps them all for the FP64 pass)
    flat = np.zeros_like(_hostile(dim, N, sizes[2][0] * sizes[2][1], rng))
    flat[:, :, 0] = us[0][0, :, 0]
    flat *= 1 + 1e-9 * rng.standard_normal(flat.shape)
    us.append(flat)
    g.set_modes(np.concatenate(us))
    got = g.max_wavespeed(points=True)
    for i, ((nx, ny), u) in enumerate(zip(sizes, us)):
        o = oracle.Mesh(dim, 1, N, nx, ny, box=(0, 1, 0, 1), bc=1)
        ref = o.max_wavespeed_points(u)[:dim]
        # (1e-13: the kernel's refined reciprocal and square root differ from IEEE by an ulp or two)
        assert np.all(got[i, :dim] >= ref * (1 - 1e-13)), (got[i, :dim], ref)
        assert np.all(got[i, :dim] <= 2 * ref * (1 + 1e-13)), (got[i, :dim], ref)
        np.testing.assert_allclose(got[i, :dim], _cell_bound(dim, N, u), rtol=1e-13)


def test_batched_p3_quadrants_stay_admissible():
    """The batched 2D Euler P3 workload scaled down 8x (256 instances of 16^2..128^2): with
    the positivity-preserving scaling and each step's time step from the check-point wave
    speeds (CFL 0.1), every instance stays admissible for 30 steps (without them 73 of the
    256 instances of the 4x-scaled workload fail within 23 steps)."""
    import torch
    w = W.euler_2d_batched()
    nx = [max(8, 2 * (s // 16)) for s in w.nx]
    st = torch.cuda.Stream()
    m = dgl.Mesh(2, 1, 3, nx, nx, w.box, bc=w.bc, stream=st.cuda_stream)
    m.project_ic(w.ic, w.params)
    m.set_positivity(True)
    h = np.array([1.0 / a for a in nx])
    with torch.cuda.stream(st):
        for _ in range(30):
            sp = m.max_wavespeed(points=True)
            m.set_dt(0.1 / (sp[:, 0] / h + sp[:, 1] / h))
            m.step(0.0)
    u = m.get_modes()
    assert np.isfinite(u).all()
    changed, bad = m.positivity_counts()
    assert bad == 0 and changed > 0
