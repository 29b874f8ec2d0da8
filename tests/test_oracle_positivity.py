"""Pins of the oracle's positivity-preserving scaling (Zhang and Shu, ref. [zs3] of the
paper, added to the limiter in Example 11): closed forms for one-variable cases, exact
preservation of the means, admissibility and minimality at the check points evaluated
here with numpy's Legendre module (independent of the oracle's basis code)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle
from paper_1904_11147_gb300 import workloads as W

G = 1.4


def _psi(n, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt((2 * n + 1) / 2) * Lg.legval(np.asarray(x, dtype=float), c)


def _points(dim, N):
    """The published check set: Gauss-Lobatto (L points, 2L-3 >= N) in 1D; in 2D the
    union of Gauss x Gauss-Lobatto and Gauss-Lobatto x Gauss with N+1 Gauss points."""
    gl = np.array([-1.0, 1.0]) if N == 1 else np.array([-1.0, 0.0, 1.0])
    if dim == 1:
        return [(x, None) for x in gl]
    g, _ = Lg.leggauss(N + 1)
    return [(r, s) for r in g for s in gl] + [(r, s) for r in gl for s in g]


def _basis(dim, N, pts):
    if dim == 1:
        return np.array([[_psi(k, r) for k in range(N + 1)] for r, _ in pts])
    ab = oracle.mode_ab(2, N)
    return np.array([[_psi(a, r) * _psi(b, s) for a, b in ab] for r, s in pts])


def _pressure(q):
    k = q[..., 1] ** 2 + (q[..., 2] ** 2 if q.shape[-1] == 4 else 0.0)
    return (G - 1) * (q[..., -1] - 0.5 * k / q[..., 0])


def _values(u, Phi):
    return np.einsum("cvk,pk->cpv", u, Phi)


def _mesh(dim, N, n=6):
    return oracle.Mesh(dim, 1, N, n, n if dim == 2 else 1, box=(0, 1, 0, 1), bc=1)


def test_density_closed_form_1d():
    """P1, rho = 1 + s x with rho(-1) = -1/2, u = 0, p = 1: theta1 = (1 - eps)/(1 + 1/2)
    and the pressure needs no scaling."""
    m = _mesh(1, 1, 1)
    eps = 1e-13
    c0 = _psi(0, 0.0)
    u = np.zeros((1, 3, 2))
    u[0, 0, 0] = 1.0 / c0
    u[0, 0, 1] = 1.5 / _psi(1, 1.0)  # rho(+-1) = 1 +- 1.5
    u[0, 2, 0] = 2.5 / c0  # E = p/(g-1)
    out, n, bad = m.positivity_limit(u, eps)
    assert (n, bad) == (1, 0)
    th1 = (1.0 - eps) / (1.0 + 0.5)
    assert out[0, 0, 1] == pytest.approx(th1 * u[0, 0, 1], rel=1e-15)
    assert out[0, 0, 0] == u[0, 0, 0] and out[0, 2, 0] == u[0, 2, 0] and out[0, 2, 1] == 0.0


def test_pressure_closed_form_1d():
    """Constant rho = 1, m = 0 and a linear E with p(-1) = -0.2: p is linear in t along the
    segment, so theta2 = (pbar - eps) / (pbar - p_q), shifted by the 1e-12 margin."""
    m = _mesh(1, 2, 1)
    eps = 1e-13
    c0 = _psi(0, 0.0)
    u = np.zeros((1, 3, 3))
    u[0, 0, 0] = 1.0 / c0
    Ebar, pq = 2.5, -0.2
    u[0, 2, 0] = Ebar / c0
    u[0, 2, 1] = (Ebar - pq / (G - 1)) / _psi(1, 1.0)  # E(-1) = pq/(g-1)
    out, n, bad = m.positivity_limit(u, eps)
    assert (n, bad) == (1, 0)
    pbar = (G - 1) * Ebar
    th2 = (pbar - eps) / (pbar - pq) * (1 - 1e-12)
    assert out[0, 2, 1] == pytest.approx(th2 * u[0, 2, 1], rel=1e-13)
    assert out[0, 0, 1] == 0.0 and out[0, 2, 0] == u[0, 2, 0]


@pytest.mark.parametrize("dim,N", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
def test_admissible_states_unchanged(dim, N):
    m = _mesh(dim, N)
    w = W.euler_2d_quadrant(6, N) if dim == 2 else W.shock_tube("sod", 6, N)
    u = m.project_ic(w.ic, w.params[0])
    out, n, bad = m.positivity_limit(u)
    assert (n, bad) == (0, 0) and np.array_equal(out, u)


def _hostile(dim, N, ncell, rng):
    """Admissible means with large random higher modes (many points inadmissible)."""
    u = W.random_modes(dim, 1, N, ncell, rng, smooth=0.0)
    NP = u.shape[2]
    for k in range(1, NP):
        u[:, :, k] = rng.uniform(-0.6, 0.6, u[:, :, 0].shape) * np.abs(u[:, :, 0]) / k
    return u


@pytest.mark.parametrize("dim,N", [(1, 1), (1, 2), (1, 3), (2, 1), (2, 2), (2, 3)])
@pytest.mark.parametrize("eps0", [1e-13, 1e-6])
def test_scaling_admissible_minimal_mean_preserving(dim, N, eps0):
    m = _mesh(dim, N, 7)
    rng = np.random.default_rng(40 + 10 * dim + N)
    u = _hostile(dim, N, m.nx * m.ny, rng)
    Phi = _basis(dim, N, _points(dim, N))
    q0 = _values(u, Phi)
    assert ((q0[..., 0] < 0) | (_pressure(q0) < 0)).any()
    out, n, bad = m.positivity_limit(u, eps0)
    assert bad == 0 and n > 0
    assert np.array_equal(out[:, :, 0], u[:, :, 0])  # means untouched, bitwise
    c0 = _psi(0, 0.0) ** dim
    q = _values(out, Phi)
    nchanged = 0
    for c in range(u.shape[0]):
        ub = u[c, :, 0] * c0
        eps = min(eps0, ub[0], _pressure(ub))
        assert q[c, :, 0].min() >= eps * (1 - 1e-9)
        assert _pressure(q[c]).min() >= eps - 1e-14 * abs(ub[-1])
        # one factor per variable on the modes n >= 1: theta1 theta2 for rho, theta2 else
        ratios = []
        for v in range(u.shape[1]):
            nz = np.abs(u[c, v, 1:]) > 1e-300
            r = out[c, v, 1:][nz] / u[c, v, 1:][nz]
            assert np.allclose(r, r[0], rtol=1e-13, atol=0)
            ratios.append(r[0])
        th2 = ratios[1]
        assert np.allclose(ratios[1:], th2, rtol=1e-13, atol=0)
        # theta1 from its closed form with the minimum density found here
        rmin = q0[c, :, 0].min()
        th1 = 1.0 if rmin >= eps else (ub[0] - eps) / (ub[0] - rmin)
        assert ratios[0] == pytest.approx(th1 * th2, rel=1e-12, abs=1e-15)
        # theta2 is the largest admissible factor: bisection on the density-scaled state
        u1 = u[c].copy()
        u1[0, 1:] *= th1
        def ok(t):
            ut = u1.copy()
            ut[:, 1:] *= t
            qt = _values(ut[None], Phi)[0]
            return _pressure(qt).min() >= eps
        if ok(1.0):
            assert th2 == 1.0
        else:
            lo, hi = 0.0, 1.0
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                lo, hi = (mid, hi) if ok(mid) else (lo, mid)
            assert th2 <= hi and th2 == pytest.approx(lo, rel=1e-9, abs=1e-12)
            nchanged += 1
        nchanged += th1 < 1.0 and th2 == 1.0
    assert nchanged == n


def test_inadmissible_mean_is_left_alone_and_counted():
    m = _mesh(2, 2, 3)
    w = W.euler_2d_quadrant(3, 2)
    u = m.project_ic(w.ic, w.params[0])
    u[4, 3, 0] = -abs(u[4, 3, 0])  # negative energy mean: no admissible state
    u[4, 0, 1] = 0.3
    out, n, bad = m.positivity_limit(u)
    assert bad == 1 and np.array_equal(out[4], u[4])


def test_burgers_is_rejected():
    m = oracle.Mesh(1, 0, 2, 4)
    with pytest.raises(ValueError):
        m.positivity_limit(m.zeros())


def test_step_with_scaling_keeps_check_points_admissible():
    """A strong P3 shock tube (seeded tube 10, density ratio near 10) loses positivity in its
    second step without the scaling; with it the state stays admissible at every check
    point over 30 steps."""
    w = W.shock_tube("random", 200, 3, index=10)
    m = oracle.Mesh(1, 1, 3, 200, box=w.box[0], bc=w.bc)
    u0 = m.project_ic(w.ic, w.params[0])
    dt = 0.1 * (1 / 200) / m.max_wavespeed(u0)[0]
    u, *_ = m.step_pp(u0, dt, pp=False)
    assert not np.isfinite(m.step(u, dt)[0]).all() or not np.isfinite(u).all()
    Phi = _basis(1, 3, _points(1, 3))
    u = u0
    for _ in range(30):
        u, nf, near, npp, bad = m.step_pp(u, dt)
        assert bad == 0
        q = _values(u, Phi)
        assert q[..., 0].min() > 0 and _pressure(q).min() > 0


@pytest.mark.parametrize("dim,N", [(1, 1), (1, 3), (2, 2), (2, 3)])
def test_max_wavespeed_points(dim, N):
    """The largest |v_d| + c over the check points (Zhang and Shu's time-step condition
    uses the wave speeds of these point values): equal to the mean-based speed for
    piecewise-constant data, and to an independent numpy evaluation of the pointwise
    maximum (points without a real sound speed, gamma p / rho < 0, skipped) on states with
    many non-admissible points."""
    m = _mesh(dim, N, 7)
    rng = np.random.default_rng(90 + 10 * dim + N)
    u = W.random_modes(dim, 1, N, m.nx * m.ny, rng, smooth=0.0)
    np.testing.assert_array_equal(m.max_wavespeed_points(u), m.max_wavespeed(u))
    u = _hostile(dim, N, m.nx * m.ny, rng)
    q = _values(u, _basis(dim, N, _points(dim, N)))
    rho, p = q[..., 0], _pressure(q)
    c2 = G * p / rho
    ok = c2 >= 0
    want = [np.max(np.where(ok, np.abs(q[..., 1 + d] / rho) + np.sqrt(np.where(ok, c2, 0.0)), 0.0))
            for d in range(dim)]
    got = m.max_wavespeed_points(u)[:dim]
    np.testing.assert_allclose(got, want, rtol=1e-12)
