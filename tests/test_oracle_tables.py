"""Pins for the oracle's basis, quadrature and CSWENO tables (Sec. 2 and Sec. 3, Steps 1-4).

Each check compares what the oracle derived with something fixed independently of it:
the paper's printed P2 constants, closed forms, numpy's own Gauss/Legendre routines, or
an independent derivation (primitive-function interpolation) written here.
"""
import math
import os
import re

import numpy as np
import pytest
from numpy.polynomial import legendre as npl

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _psi_np(n, r):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt((2 * n + 1) / 2.0) * npl.legval(r, c)


# ----------------------------------------------------------------------------- basis
@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("nq", [2, 3, 4, 5, 6, 7])
def test_gauss_rule_and_basis_against_numpy(N, nq):
    x, w, P, dP = oracle.dg_tables(N, nq)
    xr, wr = npl.leggauss(nq)
    np.testing.assert_allclose(x, xr, rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, wr, rtol=0, atol=1e-15)
    for n in range(N + 1):
        np.testing.assert_allclose(P[:, n], _psi_np(n, xr), rtol=0, atol=1e-14)
        c = np.zeros(n + 1)
        c[n] = 1.0
        np.testing.assert_allclose(dP[:, n], math.sqrt((2 * n + 1) / 2) * npl.legval(xr, npl.legder(c)),
                                   rtol=0, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_basis_orthonormal_mass_matrix(N):
    """Sec. 2, Eq. (6): with the orthonormalised basis, M = (h/2) I, i.e. the reference
    mass matrix is the identity.  The oracle's N+1 point rule integrates degree 2N exactly."""
    x, w, P, dP = oracle.dg_tables(N, N + 1)
    M = (P * w[:, None]).T @ P
    np.testing.assert_allclose(M, np.eye(N + 1), atol=1e-14)
    # stiffness S_ij = int psi_i psi_j' (Eq. (7)): closed form via numpy's own series
    S = (P * w[:, None]).T @ dP
    for i in range(N + 1):
        for j in range(N + 1):
            ci = np.zeros(i + 1); ci[i] = math.sqrt((2 * i + 1) / 2)
            cj = np.zeros(j + 1); cj[j] = math.sqrt((2 * j + 1) / 2)
            prod = npl.legmul(ci, npl.legder(cj)) if j > 0 else np.zeros(1)
            integ = npl.legint(prod)
            exact = npl.legval(1.0, integ) - npl.legval(-1.0, integ)
            assert abs(S[i, j] - exact) < 1e-13


# ----------------------------------------------------------------------------- P2 printed
def _parse_tables(path):
    pts, cur = [], None
    env = {"s5": math.sqrt(5.0), "sqrt": math.sqrt}
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("point"):
            cur = {"rows": [], "gamma": None, "r": eval(line.split("=")[1], env)}
            pts.append(cur)
        elif line.startswith("row"):
            cur["rows"].append([eval(v, env) for v in line.split(":")[1].split(",")])
        elif line.startswith("gamma"):
            cur["gamma"] = [eval(v, env) for v in line.split(":")[1].split(",")]
    return pts


def test_p2_tables_match_printed_values():
    """Sec. 3, Step 3: T^3..T^6 and the linear weights for P2 at the four Gauss-Lobatto
    points, as printed (with the two sign corrections recorded in the fixture)."""
    t = oracle.weno_tables(2)
    printed = _parse_tables(os.path.join(GOLD, "p2_cswenotables.txt"))
    np.testing.assert_allclose(t["pt"], [p["r"] for p in printed], atol=1e-15)
    np.testing.assert_allclose(t["wt"], [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    for g, p in enumerate(printed):
        rows = np.array(p["rows"])
        for i in range(3):
            np.testing.assert_allclose(t["C"][i, g], rows[i], atol=2e-15)
        np.testing.assert_allclose(t["D"][g], rows[3], atol=2e-15)
        np.testing.assert_allclose(t["gam"][g], p["gamma"], atol=2e-15)


def test_p2_printed_typos_break_constant_reproduction():
    """The two printed entries that the fixture corrects do break the row-sum identity,
    which is why they are read as sign slips."""
    printed = _parse_tables(os.path.join(GOLD, "p2_cswenotables.txt"))
    as_printed_row3 = np.array(printed[0]["rows"][2]); as_printed_row3[4] = -0.75
    as_printed_row1 = np.array(printed[3]["rows"][0]); as_printed_row1[0] = -0.75
    assert abs(as_printed_row3.sum() - 1) > 1
    assert abs(as_printed_row1.sum() - 1) > 1
    for p in printed:
        for row in p["rows"]:
            assert abs(sum(row) - 1) < 1e-14


def test_p2_smoothness_indicators_match_printed():
    """Sec. 3, Step 4: the printed closed forms of beta_0, beta_1, beta_2 for P2."""
    t = oracle.weno_tables(2)
    forms = {}
    for line in open(os.path.join(GOLD, "p2_smoothness.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split(":", 1)
            forms[k.strip()] = v.strip()
    rng = np.random.default_rng(7)
    for _ in range(50):
        avg = rng.normal(size=5)
        env = dict(zip("abcde", avg))
        for i in range(3):
            ref = eval(forms["beta%d" % i], {}, env)
            got = avg @ t["B"][i] @ avg
            assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


# ----------------------------------------------------------------------------- P1 closed form
def test_p1_is_plain_weno3():
    """Sec. 3: for P1 the stencil is three whole cells (standard WENO3 at the two Gauss
    points).  Closed forms: gamma = (1/2, 1/2); beta_0 = (u_j - u_{j-1})^2,
    beta_1 = (u_{j+1} - u_j)^2; p_0 = u_j + (u_j - u_{j-1}) xi, p_1 = u_j + (u_{j+1} - u_j) xi."""
    t = oracle.weno_tables(1)
    np.testing.assert_allclose(t["pt"], [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-16)
    np.testing.assert_allclose(t["wt"], [1, 1], atol=1e-15)
    np.testing.assert_allclose(t["gam"], [[0.5, 0.5], [0.5, 0.5]], atol=1e-15)
    np.testing.assert_allclose(t["B"][0], [[1, -1, 0], [-1, 1, 0], [0, 0, 0]], atol=1e-15)
    np.testing.assert_allclose(t["B"][1], [[0, 0, 0], [0, 1, -1], [0, -1, 1]], atol=1e-15)
    for g, r in enumerate(t["pt"]):
        xi = r / 2
        np.testing.assert_allclose(t["C"][0, g], [-xi, 1 + xi, 0], atol=1e-15)
        np.testing.assert_allclose(t["C"][1, g], [0, 1 - xi, xi], atol=1e-15)
    np.testing.assert_allclose(t["SA"][:, 0], [1 / math.sqrt(2)] * 3, atol=1e-16)
    np.testing.assert_allclose(t["SA"][:, 1], [0, 0, 0], atol=1e-16)


# ----------------------------------------------------------------------------- invariants
def _independent_rows(edges, x):
    """Weights w_k with p(x) = sum_k w_k avg_k for the polynomial of degree n-1 whose cell
    averages match, by differentiating the Lagrange interpolant of the primitive
    function through the n+1 cell edges (not the oracle's moment-matrix solve)."""
    e = np.asarray(edges, dtype=float)
    n = len(e) - 1
    w = np.zeros(n)
    for m in range(1, n + 1):
        # derivative of the Lagrange basis polynomial l_m at x
        others = [e[j] for j in range(n + 1) if j != m]
        denom = np.prod([e[m] - o for o in others])
        dl = 0.0
        for skip in range(len(others)):
            dl += np.prod([x - o for j, o in enumerate(others) if j != skip])
        dl /= denom
        for k in range(m):
            w[k] += (e[k + 1] - e[k]) * dl
    return w


def _edges(N):
    return [-1.5 + k / N for k in range(N + 1)] + [0.5] + [0.5 + k / N for k in range(1, N + 1)]


@pytest.mark.parametrize("N", [1, 2, 3])
def test_tables_against_independent_derivation(N):
    """Steps 2-3 for every order, including the P3 thirds (no printed values exist for P3,
    so this is the pin): rows from primitive-function interpolation, weights by least
    squares over all 2N+1 columns of Eq. (8)."""
    t = oracle.weno_tables(N)
    e = _edges(N)
    for g, r in enumerate(t["pt"]):
        xi = r / 2
        for i in range(N + 1):
            w = _independent_rows(e[i:i + N + 2], xi)
            ref = np.zeros(2 * N + 1)
            ref[i:i + N + 1] = w
            np.testing.assert_allclose(t["C"][i, g], ref, atol=5e-14)
        np.testing.assert_allclose(t["D"][g], _independent_rows(e, xi), atol=5e-13)
        A = np.stack([t["C"][i, g] for i in range(N + 1)], axis=1)
        gam, *_ = np.linalg.lstsq(A, t["D"][g], rcond=None)
        np.testing.assert_allclose(t["gam"][g], gam, atol=5e-13)
        assert abs(t["gam"][g].sum() - 1) < 1e-14
    assert t["resid"] < 1e-14


def test_p3_negative_weights_at_inner_points():
    """With thirds, P3 has a negative linear weight at the two inner Gauss points; the
    oracle handles them with the split of Shi, Hu and Shu (checked in the limiter tests)."""
    t = oracle.weno_tables(3)
    assert (t["gam"][[0, 3]] > 0).all()
    assert t["gam"][1, 3] < 0 and t["gam"][2, 0] < 0
    np.testing.assert_allclose(t["gam"][1], [0.0505247, 0.2707219, 1.3735460, -0.6947926], atol=1e-6)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_tables_reproduce_polynomials(N):
    """p_i reproduces every polynomial of degree <= N and Q every one of degree <= 2N
    (Step 2): exact cell averages in, exact point values out."""
    t = oracle.weno_tables(N)
    e = np.array(_edges(N))
    rng = np.random.default_rng(N)
    for deg in range(2 * N + 1):
        c = rng.normal(size=deg + 1)
        P = np.polynomial.Polynomial(c)
        I = P.integ()
        avg = (I(e[1:]) - I(e[:-1])) / (e[1:] - e[:-1])
        for g, r in enumerate(t["pt"]):
            assert abs(t["D"][g] @ avg - P(r / 2)) < 1e-12
            if deg <= N:
                for i in range(N + 1):
                    assert abs(t["C"][i, g] @ avg - P(r / 2)) < 1e-12


@pytest.mark.parametrize("N", [1, 2, 3])
def test_smoothness_indicator_definition(N):
    """Eq. (13) evaluated by numpy on the fitted polynomial (independent of the B matrices)."""
    t = oracle.weno_tables(N)
    e = np.array(_edges(N))
    rng = np.random.default_rng(10 + N)
    for _ in range(5):
        avg = rng.normal(size=2 * N + 1)
        for i in range(N + 1):
            cells = slice(i, i + N + 1)
            ee = e[i:i + N + 2]
            # solve for monomial coefficients in xi by exact averages
            A = np.array([[(ee[k + 1] ** (j + 1) - ee[k] ** (j + 1)) / ((j + 1) * (ee[k + 1] - ee[k]))
                           for j in range(N + 1)] for k in range(N + 1)])
            P = np.polynomial.Polynomial(np.linalg.solve(A, avg[cells]))
            beta = 0.0
            for l in range(1, N + 1):
                d = P.deriv(l)
                sq = (d * d).integ()
                beta += sq(0.5) - sq(-0.5)
            got = avg @ t["B"][i] @ avg
            assert abs(got - beta) <= 1e-10 * max(1, abs(beta))


@pytest.mark.parametrize("N", [1, 2, 3])
def test_subcell_averages(N):
    """Fig. 1: the subcell averages are averages of the neighbour's DG polynomial over
    its N equal parts (halves for P2); the troubled cell stays whole."""
    t = oracle.weno_tables(N)
    for k in range(2 * N + 1):
        if k == N:
            a, b = -1.0, 1.0
        else:
            q = k if k < N else k - N - 1
            a, b = -1 + 2 * q / N, -1 + 2 * (q + 1) / N
        xs, ws = npl.leggauss(8)
        xm = 0.5 * (a + b) + 0.5 * (b - a) * xs
        for n in range(N + 1):
            ref = 0.5 * np.sum(ws * _psi_np(n, xm))
            assert abs(t["SA"][k, n] - ref) < 1e-14
    assert list(t["OFF"]) == [-1] * N + [0] + [1] * N
