"""Pins of the oracle's KXRCF troubled-cell indicator (the paper's own choice, Sec. 3 step 1,
after Krivodonova et al.): closed forms on piecewise-constant data, the published
convergence rates of the indicator (it decays on smooth data and grows like
h^-(N+1)/2 at a discontinuity), exact invariances, and the effect on Example 1."""
import math

import numpy as np
import pytest

import oracle
from oracle.exact import burgers_exact, l1_linf_1d
from paper_1904_11147_gb300 import workloads as W


def _const_modes(means, dim, N, nv):
    """Modes of piecewise-constant data with the given cell means [cells, nv]."""
    c0 = (1 / math.sqrt(2)) ** dim
    np_ = N + 1 if dim == 1 else (N + 1) * (N + 2) // 2
    u = np.zeros((means.shape[0], nv, np_))
    u[:, :, 0] = means / c0
    return u


@pytest.mark.parametrize("N", [1, 2, 3])
def test_piecewise_constant_closed_form_1d(N):
    """Burgers, means only: the inflow face is the left one where ubar > 0, the right one
    where ubar < 0, none where ubar = 0; I = |ubar_j - ubar_nb| / ((h/2)^((N+1)/2) |ubar_j|)."""
    K = 12
    rng = np.random.default_rng(N)
    ub = rng.uniform(-1, 1, K)
    ub[3] = 0.0
    m = oracle.Mesh(1, 0, N, K, box=(0.0, 3.0, 0, 1), bc=0)
    fl, nf, _, ratio = m.flag_kxrcf(_const_modes(ub[:, None], 1, N, 1))
    h = 3.0 / K
    for j in range(K):
        if ub[j] > 0:
            want = abs(ub[j] - ub[j - 1]) / ((h / 2) ** ((N + 1) / 2) * abs(ub[j]))
        elif ub[j] < 0:
            want = abs(ub[j] - ub[(j + 1) % K]) / ((h / 2) ** ((N + 1) / 2) * abs(ub[j]))
        else:
            want = 0.0
        assert ratio[j] == pytest.approx(want, rel=1e-13)
        assert fl[j] == (want > 1)
    assert nf == int((ratio > 1).sum())


@pytest.mark.parametrize("N", [1, 3])
def test_piecewise_constant_closed_form_2d(N):
    """Burgers in 2D (f' = g' = u): with ubar > 0 the inflow faces are W and S, with
    ubar < 0 E and N; I = |hy (u_j - u_x') + hx (u_j - u_y')| / (r^((N+1)/2) (hx + hy) |u_j|)
    with r = sqrt(hx^2 + hy^2) / 2."""
    nx, ny = 7, 5
    rng = np.random.default_rng(10 + N)
    ub = rng.uniform(-1, 1, (ny, nx))
    m = oracle.Mesh(2, 0, N, nx, ny, box=(0.0, 1.4, 0.0, 2.0), bc=0)
    fl, nf, _, ratio = m.flag_kxrcf(_const_modes(ub.reshape(-1, 1), 2, N, 1))
    hx, hy = 1.4 / nx, 2.0 / ny
    r = 0.5 * math.sqrt(hx * hx + hy * hy)
    for iy in range(ny):
        for ix in range(nx):
            u = ub[iy, ix]
            if u > 0:
                num = hy * (u - ub[iy, ix - 1]) + hx * (u - ub[iy - 1, ix])
            else:
                num = hy * (u - ub[iy, (ix + 1) % nx]) + hx * (u - ub[(iy + 1) % ny, ix])
            want = abs(num) / (r ** ((N + 1) / 2) * (hx + hy) * abs(u))
            assert ratio[iy * nx + ix] == pytest.approx(want, rel=1e-12)


def test_euler_uses_density_and_energy_and_momentum_sign():
    """1D Euler, means only: the mean momentum's sign picks the inflow face and the larger
    of the density and energy indicators decides."""
    K, N = 10, 2
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.5, 2.0, K)
    vel = rng.uniform(-1, 1, K)
    E = rng.uniform(1.0, 3.0, K)
    means = np.stack([rho, rho * vel, E], axis=1)
    m = oracle.Mesh(1, 1, N, K, box=(0.0, 1.0, 0, 1), bc=0)
    _, _, _, ratio = m.flag_kxrcf(_const_modes(means, 1, N, 3))
    hp = (0.5 / K) ** ((N + 1) / 2)
    for j in range(K):
        nb = j - 1 if vel[j] > 0 else (j + 1) % K
        want = max(abs(rho[j] - rho[nb]) / (hp * rho[j]), abs(E[j] - E[nb]) / (hp * E[j]))
        assert ratio[j] == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("N,factor", [(1, 4.0), (2, 2 ** 1.5), (3, 8.0)])
def test_smooth_data_rates(N, factor):
    """On a smooth projection (|u| bounded away from 0) the face jumps of the L2 projection
    are O(h^(N+1)) for even N and O(h^(N+2)) for odd N (the leading error modes of the two
    neighbours cancel), so max I falls by 2^((N+1)/2), resp. 2^((N+3)/2), per halving of h."""
    r = []
    for K in (40, 80, 160):
        m = oracle.Mesh(1, 0, N, K, box=(-1, 1, 0, 1))
        u = m.project_ic(W.IC_SINE, [2.0, 1.0, math.pi, 0.0])
        fl, nf, _, ratio = m.flag_kxrcf(u)
        assert nf == 0
        r.append(ratio.max())
    for a, b in zip(r, r[1:]):
        assert a / b == pytest.approx(factor, rel=0.03)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_discontinuity_rate(N):
    """A jump inside a cell keeps an O(1) face jump: max I grows by 2^((N+1)/2) per halving
    of h, and the cells at the jump are flagged."""
    r = []
    for K in (20, 40, 80):
        m = oracle.Mesh(1, 1, N, K, box=(0, 1, 0, 1), bc=1)
        u = m.project_ic(W.IC_RIEMANN1D, [1.0, 0.5, 1.0, 0.125, 0.5, 0.1, 0.5 + 0.3 / K])
        fl, nf, _, ratio = m.flag_kxrcf(u)
        assert fl[K // 2] == 1
        r.append(ratio.max())
    for a, b in zip(r, r[1:]):
        assert b / a == pytest.approx(2 ** ((N + 1) / 2), rel=1e-3)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_mirror_and_scale_invariance(N):
    """Burgers is invariant under u(x) -> -u(-x): the indicator of the mirrored data is the
    mirrored indicator, bitwise.  Euler data scaled by 2 (density, momentum, energy) keeps
    the velocity and every ratio, bitwise."""
    K = 30
    rng = np.random.default_rng(20 + N)
    m = oracle.Mesh(1, 0, N, K, box=(-1, 1, 0, 1), bc=0)
    u = W.random_modes(1, 0, N, K, rng, smooth=0.3)
    _, _, _, r1 = m.flag_kxrcf(u)
    sign = np.array([(-1.0) ** (k + 1) for k in range(N + 1)])
    _, _, _, r2 = m.flag_kxrcf(u[::-1] * sign)
    assert np.array_equal(r1, r2[::-1])
    e = oracle.Mesh(1, 1, N, K, box=(0, 1, 0, 1), bc=1)
    ue = W.random_modes(1, 1, N, K, rng, smooth=0.05)
    _, _, _, r3 = e.flag_kxrcf(ue)
    _, _, _, r4 = e.flag_kxrcf(2.0 * ue)
    assert np.array_equal(r3, r4)


def test_example1_errors_against_table1():
    """Example 1 with the KXRCF indicator: the smooth solution is hardly ever flagged, so
    the limited errors stay near the unlimited ones, as in Table 1 (whose mesh is randomly
    perturbed by 10 %: the values agree within a factor 2.5)."""
    rows = {}
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "table1_burgers1d.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                N, K, a, b = line.split()
                rows[(int(N), int(K))] = float(b)
    T = 0.5 / math.pi
    for N in (2, 3):
        for K in (20, 40, 80):
            m = oracle.Mesh(1, 0, N, K, box=(-1, 1, 0, 1))
            u = m.project_ic(W.IC_SINE, [0.5, 1.0, math.pi, 0.0])
            n = int(math.ceil(T / (0.1 * (2 / K) / 1.5)))
            for _ in range(n):
                u, _, _, _, _ = m.step_ind(u, T / n, "kxrcf")
            l1, _ = l1_linf_1d(m, u, lambda x: burgers_exact(x, T, 0.5, 1.0, math.pi))
            assert rows[(N, K)] / 2.5 < l1 < rows[(N, K)] * 2.5, (N, K, l1, rows[(N, K)])
