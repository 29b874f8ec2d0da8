"""Pins for the nonlinear part of the oracle's CSWENO limiter and for its indicator window.

- Eqs. (14)-(15) (Sec. 3, Steps 4-5): on step data whose jump lies inside one stencil
  only, two smoothness indicators vanish and the reconstruction has a closed form in the
  third weight; the expected values come from the printed P2 tables and smoothness
  indicators (tests/golden), not from the oracle's own tables.  A worked P2 case at
  r = -1/sqrt(5) is evaluated in 50-digit decimal arithmetic from the same printed values.
- The 2D limiter (the dimension-by-dimension reading of the 2D paragraph of Sec. 3): on
  data constant in x it must equal the 1D limiter applied in y, and vice versa, which
  fixes that the y sweep uses the y-Jacobian eigenvectors and the x sweep the x ones.
- The near-threshold window of the TVB indicator: 1e-12 relative.
"""
import math
import os
import re
from decimal import Decimal, getcontext

import numpy as np
import pytest
from numpy.polynomial import legendre as npl

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS = 1e-6


# ----------------------------------------------------------------------------- printed P2 data
def _dec(expr, s5):
    """Evaluates one printed entry (integers, s5, + - * / and parentheses) in Decimal."""
    py = re.sub(r"(?<![\w*])(\d+)", r'D("\1")', expr)
    return eval(py, {"D": Decimal, "s5": s5})


def _printed_tables(exact=False):
    """{point r: (rows p0 p1 p2 over the five averages, gamma)} from the printed tables."""
    getcontext().prec = 50
    s5 = Decimal(5).sqrt() if exact else math.sqrt(5.0)
    out, cur = {}, None
    for line in open(os.path.join(GOLD, "p2_cswenotables.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("point"):
            key = line.split("=")[1].strip()
            cur = out.setdefault(key, {"rows": [], "gamma": None})
        elif line.startswith("row") and not line.startswith("row Q"):
            vals = line.split(":")[1].split(",")
            cur["rows"].append([_dec(v.strip(), s5) if exact else eval(v, {"s5": s5}) for v in vals])
        elif line.startswith("gamma"):
            vals = line.split(":")[1].split(",")
            cur["gamma"] = [_dec(v.strip(), s5) if exact else eval(v, {"s5": s5}) for v in vals]
    return out


def _printed_betas(avg, exact=False):
    env = dict(zip("abcde", avg))
    out = []
    for line in open(os.path.join(GOLD, "p2_smoothness.txt")):
        line = line.split("#")[0].strip()
        if line.startswith("beta"):
            expr = line.split(":")[1]
            if exact:
                expr = re.sub(r"(?<![\w*])(\d+)", r'D("\1")', expr)
                out.append(eval(expr, {"D": Decimal, **env}))
            else:
                out.append(eval(expr, env))
    return out


_POINT_VALUE = {"-1": -1.0, "-1/sqrt(5)": -1 / math.sqrt(5.0), "1/sqrt(5)": 1 / math.sqrt(5.0), "1": 1.0}


def _step_points():
    """The oracle's Step 1 points for P2, in its output order."""
    return np.asarray(oracle.weno_tables(2)["pt"])


# ----------------------------------------------------------------------------- ENO closed form
@pytest.mark.parametrize("side", ["right", "left"])
@pytest.mark.parametrize("c0,J,rtol", [(0.0, 2.0 ** -10, 1e-12), (0.0, -(2.0 ** -7), 1e-12),
                                       (0.25, 2.0 ** -10, 1e-8)])
def test_p2_eno_weights_closed_form(side, c0, J, rtol):
    """Averages (c0, c0, c0, c0, c0 + J): only stencil S_2 = (I_j, I_j3, I_j4) sees the jump,
    so beta_0 = beta_1 = 0, p_0 = p_1 = c0 and Eq. (15) gives
        u_G - c0 = omega_2 (p_2(x_G) - c0),
        omega_2 = [g2/(eps+b2)^2] / [(g0+g1)/eps^2 + g2/(eps+b2)^2]
    at every Step 1 point, with eps = 1e-6 and the exponent 2 of Eq. (14).  The mirror case
    (jump between I_j1 and I_j2) leaves only S_0 with a non-zero indicator."""
    tabs = _printed_tables()
    avg = [c0, c0, c0, c0, c0 + J] if side == "right" else [c0 + J, c0, c0, c0, c0]
    b = _printed_betas(avg)
    k = 2 if side == "right" else 0
    others = [i for i in range(3) if i != k]
    assert b[others[0]] == 0.0 and b[others[1]] == 0.0
    got = oracle.weno_points(2, np.array(avg), EPS)
    pts = _step_points()
    assert len(pts) == 4
    for key, tab in tabs.items():
        g = int(np.argmin(np.abs(pts - _POINT_VALUE[key])))
        assert abs(pts[g] - _POINT_VALUE[key]) < 1e-15
        gam = tab["gamma"]
        pk = sum(r * a for r, a in zip(tab["rows"][k], avg))
        wk = gam[k] / (EPS + b[k]) ** 2
        omega = wk / ((gam[others[0]] + gam[others[1]]) / EPS ** 2 + wk)
        want = omega * (pk - c0)
        assert abs((got[g] - c0) - want) <= rtol * abs(want), (key, got[g] - c0, want)


def test_p2_eno_weights_through_the_limiter():
    """The same step reached through or_csweno_limit on modes (1D Burgers P2): cells j-1 and
    j constant c0, cell j+1 linear with half-averages c0 and c0 + J, so the subcell averages
    of Fig. 1 are (c0, c0, c0, c0, c0 + J); the troubled cell's modes 1..2 are the Step 6
    projection U_n = sum_G w_G u_G psi_n(r_G) (4-point Gauss-Lobatto weights 1/6, 5/6,
    5/6, 1/6) of the closed-form point values."""
    c0, J = 0.0, 2.0 ** -10
    m = oracle.Mesh(1, 0, 2, 3, box=(0.0, 3.0, 0.0, 1.0))
    u = m.zeros()
    u[0, 0, 0] = u[1, 0, 0] = c0 * math.sqrt(2.0)
    a, bb = c0 + 0.5 * J, J  # u = a + bb r on cell j+1: half-averages a -+ bb/2
    u[2, 0, 0] = a * math.sqrt(2.0)
    u[2, 0, 1] = bb * math.sqrt(2.0 / 3.0)
    out = m.limit(u, np.array([0, 1, 0], dtype=np.uint8))
    tabs = _printed_tables()
    avg = [c0, c0, c0, c0, c0 + J]
    b = _printed_betas(avg)
    r = {"-1": -1.0, "-1/sqrt(5)": -1 / math.sqrt(5), "1/sqrt(5)": 1 / math.sqrt(5), "1": 1.0}
    w = {"-1": 1 / 6, "-1/sqrt(5)": 5 / 6, "1/sqrt(5)": 5 / 6, "1": 1 / 6}
    want = np.zeros(3)
    for key, tab in tabs.items():
        gam = tab["gamma"]
        p2 = sum(x * y for x, y in zip(tab["rows"][2], avg))
        w2 = gam[2] / (EPS + b[2]) ** 2
        uG = c0 + w2 / ((gam[0] + gam[1]) / EPS ** 2 + w2) * (p2 - c0)
        for n in (1, 2):
            c = np.zeros(n + 1)
            c[n] = 1.0
            want[n] += w[key] * uG * math.sqrt((2 * n + 1) / 2) * npl.legval(r[key], c)
    np.testing.assert_allclose(out[1, 0, 1:], want[1:], rtol=1e-9, atol=0)
    assert out[1, 0, 0] == u[1, 0, 0]


def test_p2_worked_case_at_inner_point():
    """A worked P2 case at r = -1/sqrt(5) (Sec. 3, Step 5) with all three weights active:
    averages (1, 1.5, 1.25, 0.75, 1) (x1e-3 around 2), evaluated from the printed T^4 rows,
    gamma = ((235-33 sqrt5)/950, 48/95, (235+33 sqrt5)/950) and beta_0..beta_2 in 50-digit
    decimal arithmetic, eps = 1e-6."""
    getcontext().prec = 50
    tabs = _printed_tables(exact=True)
    tab = tabs["-1/sqrt(5)"]
    base = Decimal(2)
    scale = Decimal("0.001")
    avg_d = [base + scale * Decimal(x) for x in ("1", "1.5", "1.25", "0.75", "1")]
    avg_d = [a - avg_d[2] for a in avg_d]  # centred at the troubled cell (exact)
    centre = base + scale * Decimal("1.25")
    b = _printed_betas(avg_d, exact=True)
    eps = Decimal("0.000001")
    p = [sum(r * a for r, a in zip(row, avg_d)) for row in tab["rows"]]
    wb = [g / (eps + bi) ** 2 for g, bi in zip(tab["gamma"], b)]
    want = centre + sum(w * pi for w, pi in zip(wb, p)) / sum(wb)
    avg = np.array([float(base + scale * Decimal(x)) for x in ("1", "1.5", "1.25", "0.75", "1")])
    got = oracle.weno_points(2, avg, 1e-6)
    pts = _step_points()
    g = int(np.argmin(np.abs(pts + 1 / math.sqrt(5))))
    # all three nonlinear weights are far from 0 and 1 here
    om = [float(w / sum(wb)) for w in wb]
    assert min(om) > 1e-3, om
    assert abs(got[g] - float(want)) <= 4e-16 * float(abs(want)), (got[g], float(want))


# ----------------------------------------------------------------------------- 2D -> 1D
def _profile_1d(rng, K, N, nv):
    """Piecewise-constant states with jumps plus small higher modes (1D modes per cell)."""
    u = np.zeros((K, nv, N + 1))
    rho = np.where(np.arange(K) < K // 2, 1.0, 0.3) * rng.uniform(0.8, 1.2, K)
    vel = np.where(np.arange(K) < K // 3, 0.4, -0.2) + 0.05 * rng.standard_normal(K)
    p = np.where(np.arange(K) < 2 * K // 3, 1.0, 0.15) * rng.uniform(0.9, 1.1, K)
    if nv == 1:
        prim = [rho]
    else:
        prim = [rho, rho * vel, p / 0.4 + 0.5 * rho * vel ** 2]
    for v in range(nv):
        u[:, v, 0] = prim[v] * math.sqrt(2.0)
        for n in range(1, N + 1):
            u[:, v, n] = 0.02 * rng.standard_normal(K) * abs(prim[v]).mean() / n
    return u


@pytest.mark.parametrize("pde", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("direction", ["y", "x"])
def test_2d_limiter_reduces_to_1d(pde, N, direction):
    """Data constant in x (resp. y): the 2D limiter equals the 1D limiter along y (resp.
    x).  With zero transverse velocity the 2D characteristic fields along the sweep
    direction are the 1D Euler fields of (rho, rho v_n, E) plus a passive shear field equal
    to the transverse momentum, here zero; the other sweep sees constant rows and returns
    them.  A 2D limiter that used the x eigenvectors in the y sweep (or the reverse) fails."""
    K, nt = 11, 4
    rng = np.random.default_rng(7 + 10 * N + pde + (100 if direction == "x" else 0))
    nv1 = 1 if pde == 0 else 3
    u1 = _profile_1d(rng, K, N, nv1)
    m1 = oracle.Mesh(1, pde, N, K, box=(0.0, 1.1, 0.0, 1.0), bc=1)
    flags1 = np.ones(K, dtype=np.uint8)
    lim1 = m1.limit(u1, flags1)
    nx, ny = (nt, K) if direction == "y" else (K, nt)
    m2 = oracle.Mesh(2, pde, N, nx, ny, box=(0.0, 0.4 if direction == "y" else 1.1, 0.0,
                                                1.1 if direction == "y" else 0.4), bc=1)
    ab = oracle.mode_ab(2, N)
    nv2 = 1 if pde == 0 else 4
    # variable map 1D -> 2D: rho, normal momentum, E; the transverse momentum is zero
    vmap = [0] if pde == 0 else ([0, 2, 3] if direction == "y" else [0, 1, 3])
    u2 = np.zeros((nx * ny, nv2, len(ab)))
    for iy in range(ny):
        for ix in range(nx):
            c1 = iy if direction == "y" else ix
            for k, (a, b) in enumerate(ab):
                n1, t = (b, a) if direction == "y" else (a, b)
                if t != 0:
                    continue
                for v1, v2 in enumerate(vmap):
                    u2[iy * nx + ix, v2, k] = u1[c1, v1, n1] * math.sqrt(2.0)
    lim2 = m2.limit(u2, np.ones(nx * ny, dtype=np.uint8))
    scale = np.abs(lim1).max()
    for iy in range(ny):
        for ix in range(nx):
            c1 = iy if direction == "y" else ix
            for k, (a, b) in enumerate(ab):
                n1, t = (b, a) if direction == "y" else (a, b)
                for v2 in range(nv2):
                    got = lim2[iy * nx + ix, v2, k]
                    if t == 0 and v2 in vmap:
                        want = lim1[c1, vmap.index(v2), n1] * math.sqrt(2.0)
                    else:
                        want = 0.0
                    assert abs(got - want) <= 1e-12 * scale, (ix, iy, v2, (a, b), got, want)
    # the limiter changed the data, so the comparison is not trivially the identity
    assert np.abs(lim1 - u1).max() > 1e-3 * scale


# ----------------------------------------------------------------------------- near window
def _near_case(rel, binade_top):
    """1D Burgers P2, outflow, three cells: cell 1 has u+~ = u-~ = a1 = M h^2 (1 + rel),
    neighbour mean differences 10 a1 (no other comparison is near)."""
    m = oracle.Mesh(1, 0, 2, 3, box=(0.0, 3.0, 0.0, 1.0), bc=1)
    Mh2 = (2.0 - 2.0 ** -40) if binade_top else (1.0 + 2.0 ** -40)  # just below / above 2 and 1
    Mh2 *= 2.0 ** -20
    a1 = Mh2 * (1.0 + rel)
    u = m.zeros()
    D = 10.0 * a1
    for c in range(3):
        u[c, 0, 0] = (c - 1) * D * math.sqrt(2.0)
    u[1, 0, 1] = a1 / math.sqrt(1.5)
    fl, nf, nn, nc = m.flag_tvb(u, M=Mh2, near_cells=True)  # h = 1
    return fl, nn, nc


@pytest.mark.parametrize("binade_top", [False, True])
def test_tvb_near_window_is_1e12_relative(binade_top):
    """|a1| vs M h^2 within 1e-12 relative is near; 1.5e-12 is not, wherever in its binade
    the threshold lies (a window of 8192 units in the last place would call 1.5e-12 near
    just above a power of two and miss 0.95e-12 just below one)."""
    for rel, near in [(0.5e-12, 1), (0.95e-12, 1), (-0.95e-12, 1), (1.5e-12, 0), (-1.5e-12, 0), (1e-9, 0)]:
        fl, nn, nc = _near_case(rel, binade_top)
        assert nn == near and nc[1] == near and nc[0] == 0 and nc[2] == 0, (rel, nn, nc)
        assert fl[1] == 0  # minmod(a1, 10 a1, 10 a1) = a1 above the threshold; below it a1 is kept


def test_tvb_near_window_sign_test():
    """A neighbour mean difference within 1e-12 of the largest magnitude in the comparison
    makes the minmod sign decision near; 2e-12 does not."""
    m = oracle.Mesh(1, 0, 2, 3, box=(0.0, 3.0, 0.0, 1.0), bc=1)
    a1 = 1.0
    for rel, near in [(0.5e-12, 1), (2e-12, 0)]:
        u = m.zeros()
        means = [0.0, 10.0 * rel, 10.0 * rel + 10.0]  # a3 = mean1 - mean0 = 10 rel; a2 = 10
        for c in range(3):
            u[c, 0, 0] = means[c] * math.sqrt(2.0)
        u[1, 0, 1] = a1 / math.sqrt(1.5)
        fl, nf, nn, nc = m.flag_tvb(u, M=1e-6, near_cells=True)
        assert nc[1] == near, (rel, nc)
