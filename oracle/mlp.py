"""Learned troubled-cell indicator, FP64 reference -- TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this is the reference the CUDA training and inference
kernels are checked against.

Features of cell j (per variable v, cross neighbours c = W, E, S, N in 2D, L, R in 1D):
    s_v  = max_c |ubar_c - ubar_j| + sum_{n>=1} |U^j_{n,v}| + 1e-14
    (ubar_c - ubar_j) / s_v                       for every neighbour c
    U^c_{n,v} / s_v   for n >= 1                  for c in (j, neighbours)
in the order [v][mean differences, then the cells j, W, E, S, N (1D: j, L, R), modes
1..NP-1].  Neighbours follow the boundary condition (periodic wrap; outflow mirror ghost:
odd normal modes negated, same mean).  F = V (4 + 5 (NP-1)) in 2D, V (2 + 3 N) in 1D.

Network: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3 (32 hidden units).
Loss: mean weighted binary cross-entropy with logits,
    l = -[pw y log sigma(z) + (1 - y) log(1 - sigma(z))].
Adam: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr mhat / (sqrt(vhat) + eps), with
bias-corrected mhat = m / (1 - b1^t), vhat = v / (1 - b2^t).
Label of a troubled cell: flagged by the TVB indicator and the limiter changed one of its
modes n >= 1 by more than tol s_v (the relative change is harvested; tol is a training
choice).
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 32


def n_features(dim, pde, N):
    V = 1 if pde == 0 else (3 if dim == 1 else 4)
    NP = N + 1 if dim == 1 else (N + 1) * (N + 2) // 2
    return V * (2 + 3 * (NP - 1)) if dim == 1 else V * (4 + 5 * (NP - 1))


def _neighbour(mesh, u4, ix, iy, dx, dy):
    """Modes of the neighbour (ix+dx, iy+dy) with the boundary condition applied."""
    nx, ny = mesh.nx, mesh.ny
    jx, jy = ix + dx, iy + dy
    fx = fy = False
    if mesh.bc == 0:
        jx %= nx
        jy %= ny
    else:
        if jx < 0 or jx >= nx:
            jx = min(max(jx, 0), nx - 1)
            fx = True
        if jy < 0 or jy >= ny:
            jy = min(max(jy, 0), ny - 1)
            fy = True
    m = u4[jy, jx].copy()
    if fx or fy:
        from oracle import mode_ab
        for k, (a, b) in enumerate(mode_ab(mesh.dim, mesh.N)):
            s = 1.0
            if fx and a % 2:
                s = -s
            if fy and b % 2:
                s = -s
            m[:, k] *= s
    return m


def features(mesh, u):
    """[cells, F] FP64 features of every cell of the modal state u [cells, V, NP]."""
    u = np.asarray(u).reshape(mesh.shape)
    V, NP = mesh.nv, mesh.np
    nx, ny = mesh.nx, mesh.ny
    u4 = u.reshape(ny, nx, V, NP)
    c0 = 1 / math.sqrt(2) if mesh.dim == 1 else 0.5
    offs = [(-1, 0), (1, 0)] if mesh.dim == 1 else [(-1, 0), (1, 0), (0, -1), (0, 1)]
    out = np.zeros((nx * ny, n_features(mesh.dim, mesh.pde, mesh.N)))
    for iy in range(ny):
        for ix in range(nx):
            own = u4[iy, ix]
            nbs = [_neighbour(mesh, u4, ix, iy, dx, dy) for dx, dy in offs]
            row = []
            for v in range(V):
                mj = own[v, 0] * c0
                d = [nb[v, 0] * c0 - mj for nb in nbs]
                s = max(abs(x) for x in d) + np.abs(own[v, 1:]).sum() + 1e-14
                row += [x / s for x in d]
                for cell in [own] + nbs:
                    row += list(cell[v, 1:] / s)
            out[iy * nx + ix] = row
    return out


def init_params(F, rng):
    """He-uniform initial weights (FP64)."""
    def lin(fan_in, fan_out):
        b = math.sqrt(6.0 / fan_in)
        return rng.uniform(-b, b, (fan_out, fan_in)), np.zeros(fan_out)
    W1, b1 = lin(F, HIDDEN)
    W2, b2 = lin(HIDDEN, HIDDEN)
    w3, b3 = lin(HIDDEN, 1)
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "w3": w3[0], "b3": b3}


def forward(p, X):
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0)
    z = h2 @ p["w3"] + p["b3"][0]
    return z, (X, a1, h1, a2, h2)


def loss(p, X, y, pw):
    z, _ = forward(p, X)
    # log sigma(z) = -softplus(-z), log(1 - sigma(z)) = -softplus(z)
    sp_neg = np.logaddexp(0, -z)
    sp_pos = np.logaddexp(0, z)
    return float(np.mean(pw * y * sp_neg + (1 - y) * sp_pos))


def grads(p, X, y, pw):
    """Analytic gradients of the mean weighted BCE (backpropagation)."""
    z, (X, a1, h1, a2, h2) = forward(p, X)
    B = X.shape[0]
    sig = 1 / (1 + np.exp(-z))
    dz = (pw * y * (sig - 1) + (1 - y) * sig) / B
    g = {"w3": h2.T @ dz, "b3": np.array([dz.sum()])}
    dh2 = np.outer(dz, p["w3"])
    da2 = dh2 * (a2 > 0)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (a1 > 0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return g


def adam_step(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m[...] = b1 * m + (1 - b1) * g[k]
        v[...] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p


def labels(mesh, u_stage, M=0.01, tol=1e-3):
    """TVB flags of the post-stage state, the limiter's relative change of every flagged
    cell (max over v and n >= 1 of |limited - unlimited| / s_v) and the harvest label
    (change > tol)."""
    u = np.asarray(u_stage).reshape(mesh.shape)
    fl, _, _ = mesh.flag_tvb(u, M)
    lim = mesh.limit(u, fl)
    V, NP = mesh.nv, mesh.np
    nx, ny = mesh.nx, mesh.ny
    u4 = u.reshape(ny, nx, V, NP)
    c0 = 1 / math.sqrt(2) if mesh.dim == 1 else 0.5
    offs = [(-1, 0), (1, 0)] if mesh.dim == 1 else [(-1, 0), (1, 0), (0, -1), (0, 1)]
    change = np.zeros(nx * ny)
    for iy in range(ny):
        for ix in range(nx):
            c = iy * nx + ix
            if not fl[c]:
                continue
            own = u4[iy, ix]
            nbs = [_neighbour(mesh, u4, ix, iy, dx, dy) for dx, dy in offs]
            for v in range(V):
                mj = own[v, 0] * c0
                s = max(abs(nb[v, 0] * c0 - mj) for nb in nbs) + np.abs(own[v, 1:]).sum() + 1e-14
                change[c] = max(change[c], np.abs(lim[c, v, 1:] - u[c, v, 1:]).max() / s)
    return fl, (change > tol).astype(np.uint8), change
