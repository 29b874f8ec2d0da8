"""Oracle-side cases for the end-to-end parity tests, and the oracle's own sensitivity to
rounding (test helpers; no GPU needed).

The scheme's sensitivity is measured on the oracle alone: the same run is repeated from
inputs that differ by one unit in the last place (the mean of one troubled cell), and with
a relative 1-ulp perturbation of every mode after every step (the size of the rounding
differences two correct FP64 implementations make).  The largest deviation of those runs
from the unperturbed one, step by step, is the envelope a free-running comparison of two
implementations is held to.
"""
import numpy as np

import oracle
from paper_1904_11147_gb300 import workloads as W


def rel(a, b):
    """max |a-b| / max |b| per variable, largest over variables (a, b: [cell][var][mode])."""
    b = np.asarray(b)
    a = np.asarray(a).reshape(b.shape)
    scale = np.maximum(np.abs(b).max(axis=(0, 2)), 1e-300)
    return float((np.abs(a - b).max(axis=(0, 2)) / scale).max())


def rel_hi(a, b):
    """As rel, over the modes n >= 1 only and scaled by their own largest magnitude: the
    limiter rewrites only these modes, which can be orders of magnitude below U_0."""
    b = np.asarray(b)
    a = np.asarray(a).reshape(b.shape)[:, :, 1:]
    b = b[:, :, 1:]
    scale = np.maximum(np.abs(b).max(axis=(0, 2)), 1e-300)
    return float((np.abs(a - b).max(axis=(0, 2)) / scale).max())


def oracle_case(name):
    """(mesh, u0, dt) of a named free-running case."""
    if name == "burgers1d_p2_k160":
        w = W.burgers_1d(160, 2)
        o = oracle.Mesh(1, 0, 2, 160, box=w.box[0], bc=w.bc)
        u0 = o.project_ic(w.ic, w.params[0])
        dt = 0.1 * (2 / 160) / 1.5
    elif name.startswith("sod"):
        N = int(name.split("_p")[1][0])
        w = W.shock_tube("sod", 200, N)
        o = oracle.Mesh(1, 1, N, 200, box=w.box[0], bc=w.bc)
        u0 = o.project_ic(w.ic, w.params[0])
        dt = 0.1 * (1 / 200) / o.max_wavespeed(u0)[0]
    elif name.startswith("euler2d_quadrant"):
        N = 2 if "p2" in name else 3
        n = 40 if N == 2 else 24
        # without a positivity limiter some random P3 quadrant states lose positivity on
        # coarse meshes; seed 1907 stays positive for 100 steps
        w = W.euler_2d_quadrant(n, N) if N == 2 else W.euler_2d_quadrant(n, N, seed=1907)
        o = oracle.Mesh(2, 1, N, n, n, box=w.box[0], bc=w.bc)
        u0 = o.project_ic(w.ic, w.params[0])
        ws = o.max_wavespeed(u0)
        dt = 0.1 / (ws[0] * n + ws[1] * n)
    elif name == "burgers2d_p2_32":
        w = W.burgers_2d_batched(1, 2, 32, 32)
        o = oracle.Mesh(2, 0, 2, 32, 32, box=w.box[0], bc=w.bc)
        u0 = o.project_ic(w.ic, w.params[0])
        h = 4.0 / 32
        dt = 0.1 / (2 * 1.6 / h)
    else:
        raise KeyError(name)
    return o, u0, dt


def reference_run(o, u0, dt, steps):
    """The oracle's states after every step."""
    out, u = [], u0.copy()
    for _ in range(steps):
        u, _, _ = o.step(u, dt)
        out.append(u)
    return out


def perturbed_mean(o, u0, dt):
    """u0 with the mean of the first cell the first stage flags moved by one ulp."""
    fl, _, _ = o.flag_tvb(o.rk_stage(1, dt, u0, u0))
    c = int(np.argmax(fl))
    u = u0.copy()
    u[c, 0, 0] = np.nextafter(u[c, 0, 0], np.inf)
    return u


def self_deviation(o, u0, dt, ref, seeds=(0, 1, 2)):
    """Envelope of the oracle's own deviation from ref (reference_run) under 1-ulp
    perturbations: one run from perturbed_mean, and runs that multiply every mode by
    (1 +- 2^-52) with random signs after each step.  Returns (envelope, tracks)."""
    tracks = []
    u = perturbed_mean(o, u0, dt)
    tr = []
    for k in range(len(ref)):
        u, _, _ = o.step(u, dt)
        tr.append(rel(u, ref[k]))
    tracks.append(tr)
    for sd in seeds:
        rng = np.random.default_rng(sd)
        u, tr = u0.copy(), []
        for k in range(len(ref)):
            u, _, _ = o.step(u, dt)
            u = u * (1.0 + 2.0 ** -52 * rng.choice([-1.0, 1.0], size=u.shape))
            tr.append(rel(u, ref[k]))
        tracks.append(tr)
    return np.max(np.array(tracks), axis=0), tracks
