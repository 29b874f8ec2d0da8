"""Pins for the oracle's DG operator, time stepping, indicator and exact solutions
(Sec. 2, Eqs. (2)-(7); Sec. 3 last paragraph; Sec. 4.1 Examples 1-3; Examples 7-8)."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npl
from scipy import integrate

import oracle
from oracle.exact import burgers_exact, l1_linf_1d, l1_linf_2d, riemann_exact
from paper_1904_11147_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _psi(n, r):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt((2 * n + 1) / 2.0) * npl.legval(r, c)


def _dpsi(n, r):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt((2 * n + 1) / 2.0) * npl.legval(r, npl.legder(c))


# ------------------------------------------------------------------ brute force, 1D Burgers
@pytest.mark.parametrize("N", [1, 2])
def test_rhs_1d_burgers_brute_force(N):
    """Eq. (5) written out with exact (adaptive) integrals on a 5-cell mesh; for N <= 2 the
    oracle's (N+1)-point rule is exact for f(u_h) psi', so the two agree to rounding."""
    K, h = 5, 0.4
    m = oracle.Mesh(1, 0, N, K, box=(0.0, K * h, 0, 1))
    rng = np.random.default_rng(3)
    u = rng.normal(size=(K, 1, N + 1))
    L = m.rhs(u)

    def uh(c, r):
        return sum(u[c % K, 0, n] * _psi(n, r) for n in range(N + 1))

    def fstar(a, b):  # LLF
        al = max(abs(a), abs(b))
        return 0.5 * (0.5 * a * a + 0.5 * b * b) - 0.5 * al * (b - a)

    for c in range(K):
        fr = fstar(uh(c, 1.0), uh(c + 1, -1.0))
        fl = fstar(uh(c - 1, 1.0), uh(c, -1.0))
        for i in range(N + 1):
            vol, _ = integrate.quad(lambda r: 0.5 * uh(c, r) ** 2 * _dpsi(i, r), -1, 1, epsabs=1e-14)
            ref = (2 / h) * (vol - (fr * _psi(i, 1.0) - fl * _psi(i, -1.0)))
            assert abs(L[c, 0, i] - ref) <= 1e-12 * max(1, abs(ref))


# ------------------------------------------------------------------ 2D reduces to 1D
@pytest.mark.parametrize("pde", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("direction", [0, 1])
def test_rhs_2d_reduces_to_1d(pde, N, direction):
    """Data constant in one direction: the 2D operator must act like the 1D one on the
    modes (a,0) (or (0,b)), which carry a factor sqrt(2) = 2 psi_0 from the constant
    direction; all other modes of L vanish.  For Euler the 1D system is embedded with a
    zero transverse momentum."""
    K = 6
    rng = np.random.default_rng(11 + N)
    u1 = W.random_modes(1, pde, N, K, rng, blocks=2)
    m1 = oracle.Mesh(1, pde, N, K, box=(0, 1.2, 0, 1))
    L1 = m1.rhs(u1)
    nx, ny = (K, 3) if direction == 0 else (3, K)
    m2 = oracle.Mesh(2, pde, N, nx, ny, box=(0, 1.2 if direction == 0 else 0.6, 0, 0.6 if direction == 0 else 1.2))
    ab = oracle.mode_ab(2, N)
    nv2 = m2.nv
    u2 = m2.zeros().reshape(ny, nx, nv2, m2.np)
    var_map = [0] if pde == 0 else ([0, 1, 3] if direction == 0 else [0, 2, 3])
    for k, (a, b) in enumerate(ab):
        n = a if direction == 0 else b
        other = b if direction == 0 else a
        if other != 0:
            continue
        for j in range(3):
            for c in range(K):
                for v1, v2 in enumerate(var_map):
                    if direction == 0:
                        u2[j, c, v2, k] = math.sqrt(2) * u1[c, v1, n]
                    else:
                        u2[c, j, v2, k] = math.sqrt(2) * u1[c, v1, n]
    L2 = m2.rhs(u2.reshape(-1, nv2, m2.np)).reshape(ny, nx, nv2, m2.np)
    for k, (a, b) in enumerate(ab):
        n = a if direction == 0 else b
        other = b if direction == 0 else a
        for j in range(3):
            for c in range(K):
                got = L2[j, c] if direction == 0 else L2[c, j]
                for v1, v2 in enumerate(var_map):
                    ref = math.sqrt(2) * L1[c, v1, n] if other == 0 else 0.0
                    assert abs(got[v2, k] - ref) <= 1e-11 * max(1, np.abs(L1).max())
                if pde == 1:
                    t = 2 if direction == 0 else 1
                    assert abs(got[t, k]) <= 1e-11 * max(1, np.abs(L1).max())


def test_free_stream_and_conservation():
    """A constant state is steady (L = 0 to rounding), and the limited SSP-RK3 step
    conserves the cell averages on a periodic mesh (sum of U_0 unchanged)."""
    m = oracle.Mesh(2, 1, 2, 7, 5, box=(0, 1, 0, 1))
    u = m.zeros()
    u[:, :, 0] = 2 * np.array([1.2, 0.3, -0.4, 3.0])
    assert np.abs(m.rhs(u)).max() < 1e-12
    rng = np.random.default_rng(5)
    for dim, pde, N in [(1, 0, 2), (1, 1, 3), (2, 0, 2), (2, 1, 2), (2, 1, 3)]:
        nx, ny = (40, 1) if dim == 1 else (10, 8)  # the quadrant lines fall on faces
        m = oracle.Mesh(dim, pde, N, nx, ny)
        if pde == 0 or dim == 1:
            u = W.random_modes(dim, pde, N, nx * ny, rng)
        else:
            # a four-quadrant Riemann problem: random piecewise-constant 2D Euler data can
            # make the limited P3 polynomials lose positivity at a quadrature point (the
            # method has no positivity-preserving step), and the flux then has no real
            # sound speed
            w = W.euler_2d_quadrant(nx, N)
            u = m.project_ic(w.ic, w.params[0])
        un, nf, _ = m.step(u, 1e-3)
        assert np.isfinite(un).all()
        assert nf > 0
        np.testing.assert_allclose(un[:, :, 0].sum(axis=0), u[:, :, 0].sum(axis=0), rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------------ initial projection
@pytest.mark.parametrize("dim", [1, 2])
def test_project_ic_is_l2_projection(dim):
    """Eq. (2) for the initial data: mode n is int u0 psi_n over the reference cell.
    Checked against numpy quadrature of high order."""
    N = 3
    m = oracle.Mesh(dim, 1, N, 5, 4 if dim == 2 else 1, box=(0, 2, 0, 1.5))
    p = [1.0, 0.2, 1.3, 0.7, 0.7, 0.3, 1.0]
    u = m.project_ic(W.IC_DENSITY_WAVE, p)
    xs, ws = npl.leggauss(N + 4)
    hx = 2 / 5
    if dim == 1:
        for c in range(5):
            x = hx * (c + 0.5 * (1 + xs))
            rho = 1.0 + 0.2 * np.sin(1.3 * x)
            for n in range(N + 1):
                assert abs(u[c, 0, n] - np.sum(ws * rho * _psi(n, xs))) < 1e-14
                assert abs(u[c, 1, n] - 0.7 * np.sum(ws * rho * _psi(n, xs))) < 1e-14
        return
    hy = 1.5 / 4
    ab = oracle.mode_ab(2, N)
    for iy in range(4):
        for ix in range(5):
            X = hx * (ix + 0.5 * (1 + xs))[None, :]
            Y = hy * (iy + 0.5 * (1 + xs))[:, None]
            rho = 1.0 + 0.2 * np.sin(1.3 * X + 0.7 * Y)
            E = 1.0 / 0.4 + 0.5 * rho * (0.49 + 0.09)
            for k, (a, b) in enumerate(ab):
                Wk = ws[None, :] * ws[:, None] * _psi(a, xs)[None, :] * _psi(b, xs)[:, None]
                assert abs(u[iy * 5 + ix, 0, k] - np.sum(Wk * rho)) < 1e-14
                assert abs(u[iy * 5 + ix, 3, k] - np.sum(Wk * E)) < 1e-13


# ------------------------------------------------------------------ TVB indicator
def _cells_from_means_and_slopes(means, slopes):
    """1D P1 modes for cells with the given means and face-to-face differences."""
    u = np.zeros((len(means), 1, 2))
    u[:, 0, 0] = np.asarray(means) * math.sqrt(2)
    # u(+1) - u(-1) = 2 U_1 psi_1(1) = 2 U_1 sqrt(3/2)
    u[:, 0, 1] = np.asarray(slopes) / (2 * math.sqrt(1.5))
    return u


def test_tvb_minmod_cases():
    """Cockburn-Shu modified minmod: flag when mt(a1, a2, a3) != a1, mt = a1 if
    |a1| <= M h^2 else minmod.  Hand-made cases on a periodic 1D P1 mesh."""
    K, h = 8, 1.0 / 8
    m = oracle.Mesh(1, 0, 1, K, box=(0, 1, 0, 1))
    # a global line with slope 1: face deviation h/2 < mean differences h -> no flags
    means = h * np.arange(K) + 0.0
    u = _cells_from_means_and_slopes(means, [h] * K)
    fl, n, _ = m.flag_tvb(u, M=0.0)
    # periodic wrap makes cells 0 and K-1 see a jump, interior cells are clean
    assert list(fl[1:-1]) == [0] * (K - 2)
    # a local extremum with a slope: signs of the mean differences disagree -> flag
    means = np.zeros(K)
    means[3] = 1.0
    u = _cells_from_means_and_slopes(means, [0, 0, 0, 0.5, 0, 0, 0, 0])
    fl, n, _ = m.flag_tvb(u, M=0.0)
    assert fl[3] == 1 and n >= 1
    # the same extremum with |a1| below M h^2 is left alone
    fl2, _, _ = m.flag_tvb(u, M=0.25 / (h * h) * 1.01)
    assert fl2[3] == 0
    # slope larger than the mean differences (same signs): minmod picks the smaller -> flag
    means = h * np.arange(K) * 1.0
    slopes = [h] * K
    slopes[4] = 3 * h
    u = _cells_from_means_and_slopes(means, slopes)
    fl, _, _ = m.flag_tvb(u, M=0.0)
    assert fl[4] == 1 and fl[2] == 0
    # constant data: nothing flagged, and no near-threshold comparisons
    u = _cells_from_means_and_slopes(np.ones(K), np.zeros(K))
    fl, n, near = m.flag_tvb(u, M=0.01)
    assert n == 0


def test_tvb_2d_uses_both_directions():
    """A jump in y only must flag cells along it through the y test."""
    n = 8
    m = oracle.Mesh(2, 0, 1, n, n, box=(0, 1, 0, 1), bc=1)
    u = m.zeros().reshape(n, n, 1, 3)
    u[: n // 2, :, 0, 0] = 2 * 1.0
    u[n // 2:, :, 0, 0] = 2 * 0.0
    u[n // 2, :, 0, 2] = 0.3  # a y-slope in the row above the jump
    fl, cnt, _ = m.flag_tvb(u.reshape(-1, 1, 3), M=0.0)
    fl = fl.reshape(n, n)
    assert fl[n // 2].all() and cnt == n


# ------------------------------------------------------------------ Euler eigenvectors
@pytest.mark.parametrize("dim,direction", [(1, 0), (2, 0), (2, 1)])
def test_euler_eigenvectors(dim, direction):
    """L R = I and R diag(lambda) L = the flux Jacobian (finite differences of the flux
    written here from Eqs. (21)/(23))."""
    g = 1.4
    if dim == 1:
        rho, vx, p = 0.8, 0.3, 1.1
        u = np.array([rho, rho * vx, p / (g - 1) + 0.5 * rho * vx ** 2])

        def flux(U):
            r, mm, E = U
            pr = (g - 1) * (E - 0.5 * mm * mm / r)
            return np.array([mm, mm * mm / r + pr, (E + pr) * mm / r])
        vn = vx
    else:
        rho, vx, vy, p = 0.8, 0.3, -0.6, 1.1
        u = np.array([rho, rho * vx, rho * vy, p / (g - 1) + 0.5 * rho * (vx ** 2 + vy ** 2)])

        def flux(U):
            r, mx, my, E = U
            pr = (g - 1) * (E - 0.5 * (mx * mx + my * my) / r)
            vel = (mx if direction == 0 else my) / r
            f = vel * U + np.array([0, pr if direction == 0 else 0, pr if direction == 1 else 0, pr * vel])
            return f
        vn = vx if direction == 0 else vy
    R, L = oracle.euler_eigen(dim, g, direction, u)
    np.testing.assert_allclose(L @ R, np.eye(len(u)), atol=1e-13)
    c = math.sqrt(g * p / rho)
    lam = [vn - c] + [vn] * (len(u) - 2) + [vn + c]
    J = np.zeros((len(u), len(u)))
    for j in range(len(u)):
        e = np.zeros(len(u))
        e[j] = 1e-6
        J[:, j] = (flux(u + e) - flux(u - e)) / 2e-6
    np.testing.assert_allclose(R @ np.diag(lam) @ L, J, atol=1e-7)


# ------------------------------------------------------------------ exact solutions
def test_burgers_exact_solution():
    """The characteristic solution satisfies u = u0(x - u t) and the PDE (finite differences)."""
    x = np.linspace(-1, 1, 41)
    t = 0.3 / math.pi
    u = burgers_exact(x, t, 0.5, 1.0, math.pi)
    np.testing.assert_allclose(u, 0.5 + np.sin(math.pi * (x - u * t)), atol=1e-14)
    e = 1e-6
    ut = (burgers_exact(x, t + e, 0.5, 1.0, math.pi) - burgers_exact(x, t - e, 0.5, 1.0, math.pi)) / (2 * e)
    ux = (burgers_exact(x + e, t, 0.5, 1.0, math.pi) - burgers_exact(x - e, t, 0.5, 1.0, math.pi)) / (2 * e)
    assert np.abs(ut + u * ux).max() < 1e-6


@pytest.mark.parametrize("WL,WR", [((1, 0, 1), (0.125, 0, 0.1)), ((0.445, 0.698, 3.528), (0.5, 0, 0.571))])
def test_riemann_exact_jump_conditions(WL, WR):
    """Sod and Lax: across the right shock the Rankine-Hugoniot conditions hold; across the
    contact pressure and velocity are continuous; left of the contact the left rarefaction
    is isentropic (p / rho^gamma constant)."""
    g = 1.4
    xi = np.linspace(-2.5, 2.5, 20001)
    rho, u, p, (ps, us) = riemann_exact(WL, WR, g, xi)
    E = p / (g - 1) + 0.5 * rho * u * u
    # right shock: locate the jump to the right state
    i = np.max(np.nonzero(np.abs(rho - WR[0]) > 1e-9)[0])
    S = 0.5 * (xi[i] + xi[i + 1])
    a = np.array([rho[i], rho[i] * u[i], E[i]])
    b = np.array([rho[i + 1], rho[i + 1] * u[i + 1], E[i + 1]])

    def fl(U, pr):
        return np.array([U[1], U[1] ** 2 / U[0] + pr, (U[2] + pr) * U[1] / U[0]])
    np.testing.assert_allclose(fl(a, p[i]) - fl(b, p[i + 1]), S * (a - b), atol=2e-3)
    assert abs(p[i] - ps) < 1e-12 and abs(u[i] - us) < 1e-12
    left = xi < us - 1e-3
    s = p[left] / rho[left] ** g
    np.testing.assert_allclose(s, s[0], rtol=1e-10)


# ------------------------------------------------------------------ accuracy / convergence
def _table1():
    rows = {}
    for line in open(os.path.join(GOLD, "table1_burgers1d.txt")):
        line = line.split("#")[0].strip()
        if line:
            N, K, a, b = line.split()
            rows[(int(N), int(K))] = (float(a), float(b))
    return rows


@pytest.mark.parametrize("N", [1, 2, 3])
def test_burgers_1d_design_order_and_table1(N):
    """Example 1 (rescaled to [-1,1]: x' = x/pi, t' = t/pi leaves the errors unchanged):
    errors at t = 0.5 converge at about N+1 with the limiter, and stay within a factor 4 of
    Table 1 (whose mesh is perturbed and whose indicator is KXRCF)."""
    tab = _table1()
    errs = []
    Ks = (20, 40, 80)
    for K in Ks:
        m = oracle.Mesh(1, 0, N, K, box=(-1, 1, 0, 1))
        u = m.project_ic(W.IC_SINE, [0.5, 1.0, math.pi, 0.0])
        T = 0.5 / math.pi
        n = int(math.ceil(T / (0.1 * (2 / K) / 1.5)))
        for _ in range(n):
            u, _, _ = m.step(u, T / n)
        l1, _ = l1_linf_1d(m, u, lambda x: burgers_exact(x, T, 0.5, 1.0, math.pi))
        errs.append(l1)
        assert tab[(N, K)][1] / 4 < l1 < tab[(N, K)][1] * 4
    order = math.log2(errs[-2] / errs[-1])
    assert N + 0.6 < order < N + 1.8


def test_euler_2d_density_wave_order():
    """Example 3 (smooth 2D Euler, periodic, exact rho = 1 + 0.2 sin(x+y-t)): the P1 and P2
    limited schemes converge at about N+1 (short final time to keep the test cheap)."""
    for N in (1, 2):
        errs = []
        for K in (8, 16):
            m = oracle.Mesh(2, 1, N, K, K, box=(0, 2 * math.pi, 0, 2 * math.pi))
            u = m.project_ic(W.IC_DENSITY_WAVE, [1.0, 0.2, 1.0, 1.0, 0.7, 0.3, 1.0])
            T = 0.3
            h = 2 * math.pi / K
            ws = m.max_wavespeed(u)
            n = int(math.ceil(T / (0.1 / (ws[0] / h + ws[1] / h))))
            for _ in range(n):
                u, _, _ = m.step(u, T / n)
            l1, _ = l1_linf_2d(m, u, lambda X, Y: 1 + 0.2 * np.sin(X + Y - T))
            errs.append(l1)
        order = math.log2(errs[0] / errs[1])
        assert order > N + 0.5, (N, errs)


def test_sod_converges_to_exact_riemann_solution():
    """Example 7 (Sod): the P2 density L1 error against the exact solution falls with K."""
    errs = []
    for K in (50, 100):
        m = oracle.Mesh(1, 1, 2, K, box=(0, 1, 0, 1), bc=oracle.BC_OUTFLOW)
        u = m.project_ic(W.IC_RIEMANN1D, [1, 0, 1, 0.125, 0, 0.1, 0.5])
        t, T, h = 0.0, 0.2, 1.0 / K
        while t < T - 1e-14:
            dt = min(0.1 * h / m.max_wavespeed(u)[0], T - t)
            u, _, _ = m.step(u, dt)
            t += dt
        l1, _ = l1_linf_1d(m, u, lambda x: riemann_exact((1, 0, 1), (0.125, 0, 0.1), 1.4, (x - 0.5) / T)[0])
        errs.append(l1)
    assert errs[1] < 0.7 * errs[0] and errs[1] < 6e-3


def _table4():
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "table4_vortex.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                N, K, a, b = line.split()
                rows[(int(N), int(K))] = (float(a), float(b))
    return rows


@pytest.mark.parametrize("N", [1, 2])
def test_isentropic_vortex_against_table4(N):
    """Example 4 (domain [0,10] x [-5,5], our reading): the unlimited scheme's density L1
    errors at t = 2 on 20^2 and 40^2 meshes are within 2.5x of Table 4 (whose mesh is
    non-uniform) and converge at about N+1; the projected initial state matches the
    printed exact solution."""
    from oracle.exact import l1_linf_2d, vortex_exact
    tab = _table4()
    errs = []
    for n in (20, 40):
        w = W.isentropic_vortex(n, N)
        m = oracle.Mesh(2, 1, N, n, n, box=w.box[0], bc=w.bc)
        u = m.project_ic(w.ic, w.params[0])
        l10, _ = l1_linf_2d(m, u, lambda X, Y: vortex_exact(X, Y, 0.0)[0])
        assert l10 < tab[(N, n)][0]
        ws = m.max_wavespeed(u)
        ns = int(math.ceil(2.0 / (0.1 / (ws[0] * n / 10 + ws[1] * n / 10))))
        for _ in range(ns):
            u, _, _ = m.step(u, 2.0 / ns, limit=False)
        l1, _ = l1_linf_2d(m, u, lambda X, Y: vortex_exact(X, Y, 2.0)[0])
        assert tab[(N, n)][0] / 2.5 < l1 < tab[(N, n)][0] * 2.5, (N, n, l1)
        errs.append(l1)
    assert N + 0.6 < math.log2(errs[0] / errs[1]) < N + 1.8


# ------------------------------------------------------------------ sensitivity to rounding
@pytest.mark.parametrize("name,p3", [("sod_p2_k200", False), ("sod_p3_k200", True),
                                     ("euler2d_quadrant_p2_40", False), ("euler2d_quadrant_p3_24", True)])
def test_oracle_sensitivity_to_one_ulp(name, p3):
    """The oracle against itself, 100 steps, from inputs that differ by one unit in the last
    place in the mean of one troubled cell.  With P2 the two runs stay within 1e-13 of each
    other; with P3 the difference grows by orders of magnitude (the split of negative linear
    weights and smoothness forms with large entries amplify it, and once a TVB decision
    flips the runs limit different cells): past 1e-9 on the Sod tube and past 1e-4 on the
    quadrant problem.  So no second FP64 implementation that rounds differently can keep a
    fixed 1e-11 bar over 100 P3 steps; the GPU parity tests hold it to this envelope."""
    from parity_cases import oracle_case, perturbed_mean, reference_run, rel
    o, u0, dt = oracle_case(name)
    ref = reference_run(o, u0, dt, 100)
    u = perturbed_mean(o, u0, dt)
    track = []
    for k in range(100):
        u, _, _ = o.step(u, dt)
        track.append(rel(u, ref[k]))
    print(name, "1-ulp growth:", ["%.1e" % x for x in track[::10]], "%.1e" % track[-1])
    assert track[0] <= 1e-14
    if p3:
        assert max(track) >= (1e-4 if "quadrant" in name else 1e-9), track[::10]
    else:
        assert max(track) <= 1e-13, track[::10]
