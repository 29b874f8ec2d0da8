"""Host checks of the error margins behind the two FP32 screens of the positivity code
(`csrc/dg_positivity.cu`), on the CPU: an FP32 emulation (numpy float32, the modes
truncated to FP32 as the kernels truncate them, the point values summed in another order
than the kernels sum them) of

- the scaling's screen: every cell it clears must be one that the oracle's Zhang-Shu
  scaling leaves unchanged;
- the wave-speed bounds: lo <= the FP64 cell value max |v_d| + max c <= hi, for every cell
  and direction (hi may be infinite);

on random states with large higher modes, near-vacuum and non-admissible points and cells
built to sit at the screens' margins, P1-P3 in 1D and 2D.  A margin taken too small (a
plausible mistake in the bounds) makes one of these fail."""
import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle
from paper_1904_11147_gb300 import workloads as W

GAM = 1.4
DELTA = np.float32(1.0 / 65536.0)


def _psi(n, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return np.sqrt((2 * n + 1) / 2) * Lg.legval(x, c)


def _modes(dim, N):
    return oracle.mode_ab(dim, N) if dim == 2 else [(k, 0) for k in range(N + 1)]


def _points(dim, N):
    """The check points: Gauss-Lobatto in 1D; (Gauss x Gauss-Lobatto) u (Gauss-Lobatto x
    Gauss) in 2D."""
    gl = np.array([-1.0, 1.0]) if N == 1 else np.array([-1.0, 0.0, 1.0])
    if dim == 1:
        return [(x, 0.0) for x in gl]
    g, _ = Lg.leggauss(N + 1)
    return [(r, s) for r in g for s in gl] + [(r, s) for r in gl for s in g]


def _phi(dim, N):
    ab = _modes(dim, N)
    return np.array([[_psi(a, r) * (_psi(b, s) if dim == 2 else 1.0) for a, b in ab] for r, s in _points(dim, N)])


def d2f_trunc(x):
    """double -> float by truncation of the significand, as the kernels convert."""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    sign = ((b >> np.uint64(32)) & np.uint64(0x80000000)).astype(np.uint32)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023 + 127
    man = ((b >> np.uint64(29)) & np.uint64(0x7FFFFF)).astype(np.uint32)
    out = sign | (np.clip(e, 0, 255).astype(np.uint32) << np.uint32(23)) | man
    out = np.where(e <= 0, sign, out)
    out = np.where(e >= 255, sign | np.uint32(0x7F800000), out)
    return out.astype(np.uint32).view(np.float32)


def _fp32_points(dim, N, u):
    """Point values [cell, point, var] in FP32 and the bounds S_v = delta sum_k |U_vk| psi_a(1) psi_b(1)."""
    ab = _modes(dim, N)
    u32 = d2f_trunc(u.reshape(-1)).reshape(u.shape)
    phi32 = _phi(dim, N).astype(np.float32)
    w = np.einsum("cvk,pk->cpv", u32, phi32).astype(np.float32)
    p1 = np.array([np.nextafter(np.float32(abs(_psi(n, 1.0))), np.float32(np.inf)) for n in range(N + 1)],
                  dtype=np.float32)
    pk = np.array([p1[a] * (p1[b] if dim == 2 else np.float32(1)) for a, b in ab], dtype=np.float32)
    S = (np.abs(u32) * pk[None, None, :]).sum(axis=2, dtype=np.float32)
    return w, S


def screen_clears(dim, N, u, eps0):
    """The scaling's FP32 screen per cell (the caller's guards included)."""
    V = dim + 2
    c0 = 0.5 if dim == 2 else 1 / np.sqrt(2)
    ub = u[:, :, 0] * c0
    pb = (GAM - 1) * (ub[:, -1] - 0.5 * (ub[:, 1:V - 1] ** 2).sum(axis=1) / ub[:, 0])
    eps = np.minimum(np.minimum(eps0, ub[:, 0]), pb)
    w, S = _fp32_points(dim, N, u)
    gm1 = np.float32(GAM - 1)
    e32 = eps.astype(np.float32)
    sm2 = (S[:, 1:V - 1] ** 2).sum(axis=1, dtype=np.float32)
    B = gm1 * (S[:, -1] * S[:, 0] + sm2) + e32 * S[:, 0]
    rho_min = e32 + DELTA * S[:, 0]
    q_min = np.float32(4) * DELTA * B
    k2 = (w[:, :, 1:V - 1] ** 2).sum(axis=2, dtype=np.float32)
    q = gm1 * (w[:, :, -1] * w[:, :, 0] - np.float32(0.5) * k2) - e32[:, None] * w[:, :, 0]
    with np.errstate(all="ignore"):
        ok = (w[:, :, 0] > rho_min[:, None]).all(axis=1) & (q > q_min[:, None]).all(axis=1)
        ok &= (B < np.float32(1e30)) & (S[:, 0] < np.float32(1e15))
    return ok & (ub[:, 0] >= 1e-10) & (pb >= 1e-10)


def speed_bounds(dim, N, u):
    """lo, hi [cell, dim] of max |v_d| + max c over the check points, as the kernel forms them."""
    V = dim + 2
    w, S0 = _fp32_points(dim, N, u)
    S = DELTA * S0
    gm1, gam = np.float32(GAM - 1), np.float32(GAM)
    with np.errstate(all="ignore"):
        rl = w[:, :, 0] - S[:, None, 0]
        ru = w[:, :, 0] + S[:, None, 0]
        unb = ~(rl > 0).all(axis=1) | ~(S0 < np.float32(1e15)).all(axis=1)
        mu = np.abs(w[:, :, 1:V - 1]) + S[:, None, 1:V - 1]
        ml = np.maximum(np.abs(w[:, :, 1:V - 1]) - S[:, None, 1:V - 1], np.float32(0))
        m2l = (ml ** 2).sum(axis=2, dtype=np.float32)
        m2u = (mu ** 2).sum(axis=2, dtype=np.float32)
        pu = gm1 * ((w[:, :, -1] + S[:, None, -1]) - np.float32(0.5) * m2l / ru)
        pl = gm1 * ((w[:, :, -1] - S[:, None, -1]) - np.float32(0.5) * m2u / rl)
        good = rl > 0
        inc_hi = good & (pu >= 0)
        inc_lo = good & (pl > 0)
        c2hi = np.where(inc_hi, gam * pu / rl, np.float32(0)).max(axis=1)
        c2lo = np.where(inc_lo, gam * pl / ru, np.float32(0)).max(axis=1)
        vhi = np.where(inc_hi[:, :, None], mu / rl[:, :, None], np.float32(0)).max(axis=1)
        vlo = np.where(inc_lo[:, :, None], ml / ru[:, :, None], np.float32(0)).max(axis=1)
    lo = (vlo + np.sqrt(c2lo)[:, None]) * np.float32(1 - 1 / 4096)
    hi = (vhi + np.sqrt(c2hi)[:, None]) * np.float32(1 + 1 / 4096)
    hi = np.where(unb[:, None], np.float32(np.inf), hi)
    return lo, hi


def cell_speed(dim, N, u):
    """The FP64 cell value: max |v_d| + max c over the check points with c^2 >= 0."""
    V = dim + 2
    q = np.einsum("cvk,pk->cpv", u, _phi(dim, N))
    with np.errstate(all="ignore"):
        rho = q[..., 0]
        kin = (q[..., 1:V - 1] ** 2).sum(axis=2)
        c2 = GAM * (GAM - 1) * (q[..., -1] - 0.5 * kin / rho) / rho
        ok = c2 >= 0
        cs = np.sqrt(np.where(ok, c2, 0.0).max(axis=1))
        v = np.where(ok[:, :, None], np.abs(q[..., 1:V - 1] / rho[:, :, None]), 0.0).max(axis=1)
    return v + cs[:, None]


def _states(dim, N, rng):
    """Random cells with large higher modes (many need scaling, some have non-admissible
    points), near-vacuum cells, and cells at rest whose smallest check-point density or
    pressure sits within a few screen margins of eps."""
    n = 600
    u = W.random_modes(dim, 1, N, n, rng, smooth=0.0)
    for k in range(1, u.shape[2]):
        u[:, :, k] = rng.uniform(-0.6, 0.6, u[:, :, 0].shape) * np.abs(u[:, :, 0]) / k
    u[: n // 6] *= 10.0 ** rng.uniform(-9, -3, (n // 6, 1, 1))  # near vacuum, same shape
    ab = _modes(dim, N)
    lin = ab.index((1, 0))
    c0 = 0.5 if dim == 2 else 1 / np.sqrt(2)
    k1 = abs(_psi(1, 1.0)) * (abs(_psi(0, 0.0)) if dim == 2 else 1.0)
    E = dim + 1
    extra = []
    for var in (0, E):
        for kappa in np.linspace(-3.0, 3.0, 61):
            v = np.zeros((dim + 2, len(ab)))
            v[0, 0] = 1.0 / c0
            v[E, 0] = 1.0 / (GAM - 1) / c0
            S = DELTA * (1.0 + 1.0 / (GAM - 1))  # the order of the density / energy bounds
            drop = 1.0 - (1e-13 + kappa * float(S) * (1.0 + rng.uniform(0, 1)))
            v[var, lin] = drop / k1 if var == 0 else drop / ((GAM - 1) * k1)
            extra.append(v)
    return np.concatenate([u, np.array(extra)])


@pytest.mark.parametrize("dim,N", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_scaling_screen_clears_only_unchanged_cells(dim, N):
    rng = np.random.default_rng(1000 + 10 * dim + N)
    u = _states(dim, N, rng)
    o = oracle.Mesh(dim, 1, N, len(u), 1, box=(0, 1, 0, 1), bc=1)
    eps0 = 1e-13
    ref, changed, _ = o.positivity_limit(u, eps0)
    unchanged = np.all(ref == u, axis=(1, 2))
    clear = screen_clears(dim, N, u, eps0)
    assert not (clear & ~unchanged).any(), np.nonzero(clear & ~unchanged)[0][:10]
    # the screen is not vacuous: it clears most admissible cells and the scaling changes some
    assert clear.sum() > 0.3 * unchanged.sum() and changed > 20


@pytest.mark.parametrize("dim,N", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_wave_speed_bounds_enclose_the_fp64_value(dim, N):
    rng = np.random.default_rng(2000 + 10 * dim + N)
    u = _states(dim, N, rng)
    lo, hi = speed_bounds(dim, N, u)
    ex = cell_speed(dim, N, u)
    assert np.all(lo[:, :dim] <= ex), np.nonzero(~(lo[:, :dim] <= ex))[0][:10]
    assert np.all(ex <= hi[:, :dim]), np.nonzero(~(ex <= hi[:, :dim]))[0][:10]
    # useful away from vacuum: on the random cells of ordinary density (not the first
    # sixth, scaled towards vacuum) most upper bounds are finite and within 1 % of the value
    sel = np.arange(len(u)) >= 100
    sel[600:] = False
    fin = sel & np.isfinite(hi[:, 0])
    assert fin.sum() > 0.5 * sel.sum()
    assert np.mean(hi[fin, 0] <= ex[fin, 0] * 1.01) > 0.9
