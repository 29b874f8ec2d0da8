"""Pins for the oracle's CSWENO limiter (Sec. 3, Steps 1-6, characteristic fields, 2D)."""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npl

import oracle
from paper_1904_11147_gb300 import workloads as W


def _psi(n, r):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt((2 * n + 1) / 2.0) * npl.legval(r, c)


def _project_poly_1d(coeffs_per_var, N, K, box):
    """Modes of global polynomials (numpy quadrature, exact for these degrees)."""
    xL, xR = box
    h = (xR - xL) / K
    xs, ws = npl.leggauss(N + 3)
    u = np.zeros((K, len(coeffs_per_var), N + 1))
    for c in range(K):
        x = xL + h * (c + 0.5 * (1 + xs))
        for v, cf in enumerate(coeffs_per_var):
            val = np.polynomial.Polynomial(cf)(x)
            for n in range(N + 1):
                u[c, v, n] = np.sum(ws * val * _psi(n, xs))
    return u


def _project_poly_2d(funcs, N, nx, ny, box):
    xL, xR, yL, yR = box
    hx, hy = (xR - xL) / nx, (yR - yL) / ny
    xs, ws = npl.leggauss(N + 3)
    ab = oracle.mode_ab(2, N)
    u = np.zeros((nx * ny, len(funcs), len(ab)))
    for iy in range(ny):
        for ix in range(nx):
            X = xL + hx * (ix + 0.5 * (1 + xs))[None, :]
            Y = yL + hy * (iy + 0.5 * (1 + xs))[:, None]
            for v, f in enumerate(funcs):
                val = f(X, Y)
                for k, (a, b) in enumerate(ab):
                    Wk = ws[None, :] * ws[:, None] * _psi(a, xs)[None, :] * _psi(b, xs)[:, None]
                    u[iy * nx + ix, v, k] = np.sum(Wk * val)
    return u


@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("pde", [0, 1])
def test_limiter_reproduces_global_polynomials_1d(N, pde):
    """Each p_i reproduces polynomials of degree <= N and the nonlinear weights sum to one,
    so a troubled cell inside one global polynomial of degree <= N gets its own modes back
    (Steps 2-6); the characteristic transform is linear and changes nothing."""
    K = 9
    rng = np.random.default_rng(N)
    if pde == 0:
        polys = [rng.normal(size=N + 1)]
    else:
        rho = np.concatenate([[1.0], 0.1 * rng.normal(size=N)])
        mom = np.concatenate([[0.3], 0.1 * rng.normal(size=N)])
        E = np.concatenate([[3.0], 0.1 * rng.normal(size=N)])
        polys = [rho, mom, E]
    m = oracle.Mesh(1, pde, N, K, box=(-1, 1, 0, 1))
    u = _project_poly_1d(polys, N, K, (-1, 1))
    flags = np.zeros(K, np.uint8)
    flags[1:-1] = 1  # the periodic wrap breaks the polynomial at the two end cells
    out = m.limit(u, flags)
    np.testing.assert_allclose(out[1:-1], u[1:-1], rtol=0, atol=1e-12)
    assert np.array_equal(out[:, :, 0], u[:, :, 0])


@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("pde", [0, 1])
def test_limiter_reproduces_global_polynomials_2d(N, pde):
    """2D, dimension by dimension on the (2N+1)^2 subcell grid (x sweep then y sweep, then
    the tensor projection): polynomials of total degree <= N are reproduced."""
    nx, ny = 6, 5
    rng = np.random.default_rng(20 + N)
    terms = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]

    def rand_poly(c0, scale):
        cf = {t: (c0 if t == (0, 0) else scale * rng.normal()) for t in terms}
        return lambda X, Y: sum(v * X ** a * Y ** b for (a, b), v in cf.items())
    if pde == 0:
        funcs = [rand_poly(0.3, 1.0)]
    else:
        funcs = [rand_poly(1.0, 0.1), rand_poly(0.2, 0.1), rand_poly(-0.3, 0.1), rand_poly(3.0, 0.1)]
    box = (-1, 1, -1, 1)
    m = oracle.Mesh(2, pde, N, nx, ny, box=box)
    u = _project_poly_2d(funcs, N, nx, ny, box)
    fl = np.zeros((ny, nx), np.uint8)
    fl[1:-1, 1:-1] = 1
    out = m.limit(u, fl.reshape(-1))
    inner = fl.reshape(-1) == 1
    np.testing.assert_allclose(out[inner], u[inner], rtol=0, atol=1e-11)
    assert np.array_equal(out[:, :, 0], u[:, :, 0])
    assert np.array_equal(out[~inner], u[~inner])


@pytest.mark.parametrize("dim,pde,N", [(1, 0, 2), (1, 1, 3), (2, 0, 2), (2, 1, 2), (2, 1, 3)])
def test_limiter_jacobi_and_mean(dim, pde, N):
    """The cell average is kept bitwise (Sec. 3: "we retain the cell average"), unflagged
    cells are untouched, and the update is Jacobi: limiting a cell never changes what
    another flagged cell sees (flagging cells one at a time gives the same result)."""
    rng = np.random.default_rng(100 + N)
    nx, ny = (30, 1) if dim == 1 else (7, 6)
    m = oracle.Mesh(dim, pde, N, nx, ny, bc=oracle.BC_OUTFLOW)
    u = W.random_modes(dim, pde, N, nx * ny, rng, smooth=0.2)
    fl = (rng.uniform(size=nx * ny) < 0.4).astype(np.uint8)
    out = m.limit(u, fl)
    assert np.array_equal(out[:, :, 0], u[:, :, 0])
    assert np.array_equal(out[fl == 0], u[fl == 0])
    assert not np.allclose(out[fl == 1], u[fl == 1])
    single = u.copy()
    for c in np.nonzero(fl)[0]:
        f1 = np.zeros_like(fl)
        f1[c] = 1
        single[c] = m.limit(u, f1)[c]
    assert np.array_equal(single, out)


def test_limiter_removes_oscillation_at_a_jump():
    """A P2 step with an overshooting slope: after limiting, the reconstructed point values
    of the troubled cell stay within the range of the neighbouring means (essentially
    non-oscillatory), while the mean is kept."""
    K = 10
    m = oracle.Mesh(1, 0, 2, K, box=(0, 1, 0, 1), bc=oracle.BC_OUTFLOW)
    u = np.zeros((K, 1, 3))
    u[:5, 0, 0] = math.sqrt(2) * 1.0
    u[5:, 0, 0] = 0.0
    u[4, 0, 1] = -0.4  # large slope in the cell before the jump
    u[4, 0, 2] = 0.2
    fl, n, _ = m.flag_tvb(u)
    assert fl[4] == 1
    out = m.limit(u, fl)
    r = np.linspace(-1, 1, 21)
    vals = sum(out[4, 0, k] * _psi(k, r) for k in range(3))
    assert vals.max() < 1.0 + 0.05 and vals.min() > -0.05


def test_p3_negative_weight_split_matches_linear_reconstruction():
    """Where the P3 linear weights are negative the split of Shi, Hu and Shu is used; with
    equal smoothness indicators (a global polynomial of degree 6 cannot be represented,
    but a huge epsilon makes the weights linear) the result must equal Q at the points,
    i.e. the sigma+/sigma- recombination reproduces gamma exactly."""
    t = oracle.weno_tables(3)
    K = 5
    m = oracle.Mesh(1, 0, 3, K, box=(0, 1, 0, 1))
    rng = np.random.default_rng(9)
    u = rng.normal(size=(K, 1, 4))
    fl = np.zeros(K, np.uint8)
    fl[2] = 1
    out = m.limit(u, fl, eps=1e15)
    # stencil averages
    avg = np.zeros(7)
    for k in range(7):
        src = u[2 + t["OFF"][k], 0]
        avg[k] = src @ t["SA"][k]
    q = t["D"] @ avg
    ref = np.array([np.sum(t["wt"] * q * np.array([_psi(n, r) for r in t["pt"]])) for n in range(4)])
    np.testing.assert_allclose(out[2, 0, 1:], ref[1:], rtol=0, atol=1e-12)
