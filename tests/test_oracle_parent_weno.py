"""Pins of the oracle's parent WENO limiter (Qiu and Shu, ref. [qs1]; the paper's main
comparison in Sec. 4): on the uniform full-width stencil the derived tables are the
textbook WENO3/5/7 ones (Jiang-Shu reconstruction rows, linear weights and smoothness
indicators), the limiter coincides with CSWENO for P1 (the paper notes the two are the
same there), reproduces polynomials, keeps the means, and reaches N cells out."""
import math

import numpy as np
import pytest

import oracle
from paper_1904_11147_gb300 import workloads as W


def test_weno5_rows_weights_and_smoothness_indicators():
    t = oracle.weno_tables(2, parent=True, points=[-1.0, 1.0])
    # reconstruction at x_{j+1/2} (r = +1) from the averages f_{j-2} .. f_{j+2}
    C = t["C"][:, 1, :] * 6.0
    np.testing.assert_allclose(C[0], [2, -7, 11, 0, 0], atol=1e-13)
    np.testing.assert_allclose(C[1], [0, -1, 5, 2, 0], atol=1e-13)
    np.testing.assert_allclose(C[2], [0, 0, 2, 5, -1], atol=1e-13)
    np.testing.assert_allclose(t["gam"][1], [0.1, 0.6, 0.3], atol=1e-14)
    np.testing.assert_allclose(t["gam"][0], [0.3, 0.6, 0.1], atol=1e-14)
    # Jiang-Shu: beta_0 = 13/12 (f0 - 2 f1 + f2)^2 + 1/4 (f0 - 4 f1 + 3 f2)^2, etc.
    rng = np.random.default_rng(0)
    for _ in range(5):
        f = rng.normal(size=5)
        js = [13 / 12 * (f[0] - 2 * f[1] + f[2]) ** 2 + 0.25 * (f[0] - 4 * f[1] + 3 * f[2]) ** 2,
              13 / 12 * (f[1] - 2 * f[2] + f[3]) ** 2 + 0.25 * (f[1] - f[3]) ** 2,
              13 / 12 * (f[2] - 2 * f[3] + f[4]) ** 2 + 0.25 * (3 * f[2] - 4 * f[3] + f[4]) ** 2]
        for i in range(3):
            assert f @ t["B"][i] @ f == pytest.approx(js[i], rel=1e-12)


def test_weno3_and_weno7_boundary_weights():
    t1 = oracle.weno_tables(1, parent=True, points=[1.0])
    np.testing.assert_allclose(t1["gam"][0], [1 / 3, 2 / 3], atol=1e-15)
    np.testing.assert_allclose(t1["C"][:, 0, :] * 2, [[-1, 3, 0], [0, 1, 1]], atol=1e-14)
    t3 = oracle.weno_tables(3, parent=True, points=[1.0])
    np.testing.assert_allclose(t3["gam"][0] * 35, [1, 12, 18, 4], atol=1e-12)
    assert t3["resid"] < 1e-14


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("pde", [0, 1])
def test_p1_parent_equals_csweno(dim, pde):
    """For P1 the subcells of CSWENO are the whole neighbours: both limiters agree."""
    nx, ny = (40, 1) if dim == 1 else (9, 7)
    m = oracle.Mesh(dim, pde, 1, nx, ny, bc=1)
    rng = np.random.default_rng(7 + dim + pde)
    u = W.random_modes(dim, pde, 1, nx * ny, rng, smooth=0.3 if pde == 0 else 0.02)
    fl = np.ones(nx * ny, dtype=np.uint8)
    a = m.limit(u, fl)
    b = m.parent_limit(u, fl)
    np.testing.assert_allclose(b, a, rtol=0, atol=1e-14 * np.abs(a).max())


def _poly_modes(dim, N, nx, ny, coef):
    """Exact modes (Eq. (2) by a Gauss rule exact for the degree) of the polynomial
    sum_ab coef[a, b] x^a y^b on the unit box."""
    from numpy.polynomial import legendre as Lg
    xq, wq = Lg.leggauss(N + 3)
    psi = lambda n, r: math.sqrt((2 * n + 1) / 2) * Lg.legval(r, np.eye(n + 1)[n])
    ab = [(k, 0) for k in range(N + 1)] if dim == 1 else oracle.mode_ab(2, N)
    hx, hy = 1.0 / nx, 1.0 / ny
    u = np.zeros((nx * ny, 1, len(ab)))
    for iy in range(ny):
        for ix in range(nx):
            X = (ix + 0.5 + 0.5 * xq) * hx
            if dim == 1:
                P = sum(coef[a, 0] * X ** a for a in range(N + 1))
                for k in range(N + 1):
                    u[ix, 0, k] = np.sum(wq * P * psi(k, xq))
            else:
                Y = (iy + 0.5 + 0.5 * xq) * hy
                P = sum(coef[a, b] * np.outer(Y ** b, X ** a) for a in range(N + 1) for b in range(N + 1 - a))
                for k, (a, b) in enumerate(ab):
                    u[iy * nx + ix, 0, k] = np.einsum("y,x,yx,y,x->", wq, wq, P, psi(b, xq), psi(a, xq))
    return u


@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("dim", [1, 2])
def test_parent_reproduces_polynomials_and_keeps_means(N, dim):
    """A global polynomial of degree N is a fixed point of the limiter (every stencil
    reproduces it) on cells whose stencil stays inside the mesh; means are kept bitwise."""
    nx, ny = (16, 1) if dim == 1 else (11, 10)
    m = oracle.Mesh(dim, 0, N, nx, ny, box=(0.0, 1.0, 0.0, 1.0), bc=1)
    rng = np.random.default_rng(N + 10 * dim)
    u = _poly_modes(dim, N, nx, ny, rng.normal(size=(N + 1, N + 1)))
    fl = np.zeros(nx * ny, dtype=np.uint8)
    inner = [iy * nx + ix for iy in range(ny) for ix in range(nx)
             if N <= ix < nx - N and (dim == 1 or N <= iy < ny - N)]
    fl[inner] = 1
    out = m.parent_limit(u, fl)
    assert np.array_equal(out[:, :, 0], u[:, :, 0])
    np.testing.assert_allclose(out[inner], u[inner], rtol=0, atol=1e-10 * np.abs(u).max())


def test_parent_reach():
    """P2: the limited modes of cell j depend on the mean of cell j+2 but not on its
    higher modes, and CSWENO ignores cell j+2 altogether."""
    K, j = 20, 9
    m = oracle.Mesh(1, 0, 2, K, bc=0)
    rng = np.random.default_rng(3)
    u = W.random_modes(1, 0, 2, K, rng, smooth=0.3)
    fl = np.zeros(K, dtype=np.uint8)
    fl[j] = 1
    base_p, base_c = m.parent_limit(u, fl), m.limit(u, fl)
    v = u.copy()
    v[j + 2, 0, 1:] += 0.3
    assert np.array_equal(m.parent_limit(v, fl)[j], base_p[j])
    v = u.copy()
    v[j + 2, 0, 0] += 0.3
    assert not np.array_equal(m.parent_limit(v, fl)[j], base_p[j])
    assert np.array_equal(m.limit(v, fl)[j], base_c[j])
