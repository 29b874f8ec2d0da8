"""Exact solutions used to pin the oracle -- TEST INFRASTRUCTURE ONLY.

* Burgers (Examples 1, 2 and 5): u(x, t) = u0(x - u t) solved by Newton-Raphson on the
  characteristics, as the paper prescribes for its accuracy tables (Sec. 4.1); valid
  before the shock forms.
* Euler Riemann problem (Examples 7, 8): the exact solution of the ideal-gas Riemann
  problem, written from the Rankine-Hugoniot and isentropic relations (a Newton
  iteration on the star pressure, then sampling of the self-similar fan).
* Error norms (Sec. 4.1 does not define them; our reading): the domain-averaged L1
  error and the L-infinity error at N+3 Gauss points per direction per cell.
"""
from __future__ import annotations

import numpy as np


def burgers_exact(x, t, a=0.5, A=1.0, k=1.0, tol=1e-15):
    """u(x,t) for u_t + (u^2/2)_x = 0, u0 = a + A sin(k x), before shock formation."""
    x = np.asarray(x, dtype=np.float64)
    u = a + A * np.sin(k * x)
    for _ in range(100):
        s = k * (x - u * t)
        F = u - a - A * np.sin(s)
        dF = 1.0 + A * k * t * np.cos(s)
        du = F / dF
        u = u - du
        if np.max(np.abs(du)) < tol:
            break
    return u


def riemann_exact(WL, WR, gamma, xi):
    """Exact solution of the 1D Euler Riemann problem at similarity coordinates xi = x/t.

    WL, WR: (rho, u, p).  Returns (rho, u, p) arrays.  Assumes no vacuum generation.
    """
    rL, uL, pL = WL
    rR, uR, pR = WR
    g = gamma
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)

    def f(p, r, pk, ck):
        if p > pk:  # shock
            Ak, Bk = 2.0 / ((g + 1) * r), (g - 1) / (g + 1) * pk
            q = np.sqrt(Ak / (p + Bk))
            return (p - pk) * q, q * (1 - 0.5 * (p - pk) / (p + Bk))
        # rarefaction
        e = (g - 1) / (2 * g)
        val = 2 * ck / (g - 1) * ((p / pk) ** e - 1)
        der = 1.0 / (r * ck) * (p / pk) ** (-(g + 1) / (2 * g))
        return val, der

    p = max(1e-8, 0.5 * (pL + pR))
    for _ in range(200):
        fL, dL = f(p, rL, pL, cL)
        fR, dR = f(p, rR, pR, cR)
        F = fL + fR + (uR - uL)
        dp = F / (dL + dR)
        pn = max(p - dp, 1e-12)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = f(p, rL, pL, cL)
    fR, _ = f(p, rR, pR, cR)
    us = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    ps = p
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    pr = np.empty_like(xi)
    gm = (g - 1) / (g + 1)
    for i, s in np.ndenumerate(xi):
        if s <= us:  # left of contact
            if ps > pL:  # left shock
                rs = rL * (ps / pL + gm) / (gm * ps / pL + 1)
                S = uL - cL * np.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                val = (rL, uL, pL) if s < S else (rs, us, ps)
            else:  # left rarefaction
                rs = rL * (ps / pL) ** (1 / g)
                cs = cL * (ps / pL) ** ((g - 1) / (2 * g))
                if s < uL - cL:
                    val = (rL, uL, pL)
                elif s > us - cs:
                    val = (rs, us, ps)
                else:
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    uu = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    rr = rL * (c / cL) ** (2 / (g - 1))
                    val = (rr, uu, pL * (c / cL) ** (2 * g / (g - 1)))
        else:
            if ps > pR:  # right shock
                rs = rR * (ps / pR + gm) / (gm * ps / pR + 1)
                S = uR + cR * np.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                val = (rR, uR, pR) if s > S else (rs, us, ps)
            else:
                rs = rR * (ps / pR) ** (1 / g)
                cs = cR * (ps / pR) ** ((g - 1) / (2 * g))
                if s > uR + cR:
                    val = (rR, uR, pR)
                elif s < us + cs:
                    val = (rs, us, ps)
                else:
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    uu = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    rr = rR * (c / cR) ** (2 / (g - 1))
                    val = (rr, uu, pR * (c / cR) ** (2 * g / (g - 1)))
        rho[i], u[i], pr[i] = val
    return rho, u, pr, (ps, us)


def vortex_exact(x, y, t, x0=5.0, y0=0.0, beta=5.0, gamma=1.4):
    """Example 4's printed exact solution: the isentropic vortex advected with speed 1 in
    x; returns (rho, u, v, p) at the points (x, y) and time t."""
    dx, dy = x - x0 - t, y - y0
    e = np.exp(1.0 - (dx * dx + dy * dy))
    rho = (1.0 - (gamma - 1.0) * beta ** 2 * e * e / (16.0 * gamma * np.pi ** 2)) ** (1.0 / (gamma - 1.0))
    u = 1.0 - beta * e * dy / (2.0 * np.pi)
    v = beta * e * dx / (2.0 * np.pi)
    return rho, u, v, rho ** gamma


def eval_points(mesh, u, nq):
    """Values of the modal solution at nq Gauss points per direction per cell.

    Uses numpy's Gauss-Legendre rule and Legendre series (independent of the oracle's
    own tables).  Returns (x, [y,] values[cell, var, q...], weights).
    """
    from numpy.polynomial import legendre as npl

    xq, wq = npl.leggauss(nq)
    N = mesh.N

    def psi(n, r):
        c = np.zeros(n + 1)
        c[n] = 1.0
        return np.sqrt((2 * n + 1) / 2.0) * npl.legval(r, c)

    u = np.asarray(u).reshape(mesh.shape)
    xL, xR, yL, yR = mesh.box
    hx = (xR - xL) / mesh.nx
    if mesh.dim == 1:
        V = np.stack([psi(n, xq) for n in range(N + 1)], axis=1)  # q x n
        vals = np.einsum("cvn,qn->cvq", u, V)
        xc = xL + hx * (np.arange(mesh.nx)[:, None] + 0.5 * (1 + xq[None, :]))
        return xc, vals, wq
    hy = (yR - yL) / mesh.ny
    ab = [(d - b, b) for d in range(N + 1) for b in range(d + 1)]
    Px = np.stack([psi(n, xq) for n in range(N + 1)], axis=1)
    V = np.stack([np.einsum("i,j->ij", Px[:, a], Px[:, b]) for a, b in ab], axis=-1)  # qy? -> (qx,qy,k)
    vals = np.einsum("cvk,xyk->cvyx", u, V)
    ix = np.arange(mesh.nx)
    iy = np.arange(mesh.ny)
    X = xL + hx * (ix[:, None] + 0.5 * (1 + xq[None, :]))  # nx x q
    Y = yL + hy * (iy[:, None] + 0.5 * (1 + xq[None, :]))
    return (X, Y), vals, wq


def l1_linf_1d(mesh, u, exact_fn, var=0, nq=None):
    """Domain-averaged L1 and max-norm errors of variable var against exact_fn(x)."""
    nq = nq or mesh.N + 3
    xc, vals, wq = eval_points(mesh, u, nq)
    err = np.abs(vals[:, var, :] - exact_fn(xc))
    l1 = np.sum(err * wq[None, :]) / (2.0 * mesh.nx)
    return l1, err.max()


def l1_linf_2d(mesh, u, exact_fn, var=0, nq=None):
    nq = nq or mesh.N + 3
    (X, Y), vals, wq = eval_points(mesh, u, nq)
    nx, ny = mesh.nx, mesh.ny
    v = vals[:, var].reshape(ny, nx, nq, nq)  # iy, ix, qy, qx
    Xg = X[None, :, None, :]
    Yg = Y[:, None, :, None]
    err = np.abs(v - exact_fn(Xg, Yg))
    W = wq[:, None] * wq[None, :]
    l1 = np.sum(err * W[None, None]) / (4.0 * nx * ny)
    return l1, err.max()
