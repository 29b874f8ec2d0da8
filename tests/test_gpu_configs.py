"""The 1D workloads at their full sizes, against the oracle stage by stage (each GPU
sub-step recomputed by the oracle from the GPU's own input, see shadow_util), plus the
end states against the exact solutions."""
import math

import numpy as np
import pytest

import oracle
from oracle.exact import burgers_exact, l1_linf_1d, riemann_exact
import paper_1904_11147_gb300 as dgl
from paper_1904_11147_gb300 import workloads as W
from shadow_util import shadow_stages

pytestmark = pytest.mark.gpu


def test_burgers_1d_p2_k160_through_the_shock():
    """Workload 1: u0 = 0.5 + sin(pi x), K = 160, to t = 1.5/pi (the shock forms near
    t = 1/pi); before the shock the solution matches the characteristic solution."""
    w = W.burgers_1d(160, 2)
    o = oracle.Mesh(1, 0, 2, 160, box=w.box[0], bc=w.bc)
    g = dgl.Mesh(1, 0, 2, [160], None, w.box, bc=w.bc)
    u0 = o.project_ic(w.ic, w.params[0])
    n = int(math.ceil(w.t_end / (0.1 * (2 / 160) / 1.5)))
    dt = w.t_end / n
    ws, wl, nf, done, _ = shadow_stages(o, g, u0, dt, n)
    assert done == n and nf > 0
    print("burgers K=160: %d steps, worst stage deviation %.2e, worst limited %.2e, flagged %d" % (done, ws, wl, nf))
    # smooth phase against the exact solution
    g.set_modes(u0)
    n_s = int(0.5 / math.pi / dt)
    for _ in range(n_s):
        g.step(dt)
    m = oracle.Mesh(1, 0, 2, 160, box=w.box[0], bc=w.bc)
    l1, _ = l1_linf_1d(m, g.get_modes(), lambda x: burgers_exact(x, n_s * dt, 0.5, 1.0, math.pi))
    assert l1 < 3e-6


@pytest.mark.parametrize("N", [1, 2, 3])
def test_burgers_1d_accuracy_sweep(N):
    """Workload 1's smooth sweep: K = 20..320 at t = 0.5/pi, limiter on.  The GPU's L1
    errors equal the oracle's (same runs) and converge at about N + 1 (the TVB indicator
    flags the smooth extrema, the WENO reconstruction keeps the order there)."""
    T = 0.5 / math.pi
    errs = []
    for K in (20, 40, 80, 160, 320):
        o = oracle.Mesh(1, 0, N, K, box=(-1, 1, 0, 1))
        g = dgl.Mesh(1, 0, N, [K], None, [(-1.0, 1.0, 0.0, 1.0)])
        u = o.project_ic(W.IC_SINE, [0.5, 1.0, math.pi, 0.0])
        g.set_modes(u)
        n = int(math.ceil(T / (0.1 * (2 / K) / 1.5)))
        near = 0
        for _ in range(n):
            g.step(T / n)
            u, _, nn = o.step(u, T / n)
            near += nn
        exact = lambda x: burgers_exact(x, T, 0.5, 1.0, math.pi)
        l1_gpu, _ = l1_linf_1d(o, g.get_modes(), exact)
        l1_ref, _ = l1_linf_1d(o, u, exact)
        if near == 0:  # same runs: equal up to rounding of O(1) modes
            assert abs(l1_gpu - l1_ref) <= 1e-7 * l1_ref + 1e-12, (K, l1_gpu, l1_ref)
        errs.append(l1_gpu)
        g.close()
    orders = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    print("P%d L1 errors" % N, ["%.3e" % e for e in errs], "orders", ["%.2f" % q for q in orders])
    assert all(N + 0.5 < q < N + 1.8 for q in orders[1:])


def _cfl_dt(o, K):
    """CFL 0.1 time step from the current state's largest wave speed (over cell means)."""
    return lambda k, u: 0.1 * (1.0 / K) / o.max_wavespeed(u)[0]


@pytest.mark.parametrize("kind,t_end,l1_max", [("sod", 0.2, 2e-3), ("lax", 0.06, 4e-3)])
def test_shock_tubes_p3_k800(kind, t_end, l1_max):
    """Workload 2: Sod to t = 0.2 and Lax, P3, K = 800, outflow, CFL 0.1 from the current
    wave speed every step.  Lax stops at t = 0.06: with the TVB indicator at M = 0.01 the
    limited region keeps growing and this P3 run (oracle and GPU alike) reaches a negative
    density near t = 0.083, before the paper's t = 0.13."""
    w = W.shock_tube(kind, 800, 3)
    o = oracle.Mesh(1, 1, 3, 800, box=w.box[0], bc=w.bc)
    g = dgl.Mesh(1, 1, 3, [800], None, w.box, bc=w.bc)
    u0 = o.project_ic(w.ic, w.params[0])
    ws, wl, nf, k, t = shadow_stages(o, g, u0, _cfl_dt(o, 800), 100000, t_end=t_end, graph_check=False)
    assert abs(t - t_end) < 1e-12
    WL, WR = w.params[0][0:3], w.params[0][3:6]
    l1, _ = l1_linf_1d(o, g.get_modes(), lambda x: riemann_exact(WL, WR, 1.4, (x - 0.5) / t_end)[0])
    print("%s: %d steps, worst stage deviation %.2e, worst limited %.2e, density L1 %.2e"
          % (kind, k, ws, wl, l1))
    assert l1 < l1_max


def test_random_shock_tubes_p3_k800():
    """Workload 2: the 64 seeded random tubes, 100 steps each.  The method has no
    positivity-preserving step, and at density ratios near 10 some P3 limited polynomials
    dip below zero density at a quadrature point within the first steps; both sides must
    reach the non-finite state in the same step, and agree step by step until then."""
    nonfinite = []
    for i in range(64):
        w = W.shock_tube("random", 800, 3, index=i)
        o = oracle.Mesh(1, 1, 3, 800, box=w.box[0], bc=w.bc)
        g = dgl.Mesh(1, 1, 3, [800], None, w.box, bc=w.bc)
        u0 = o.project_ic(w.ic, w.params[0])
        _, _, _, done, _ = shadow_stages(o, g, u0, _cfl_dt(o, 800), 100, stop_on_nonfinite=True, graph_check=False)
        if done < 100:
            nonfinite.append((i, done))
        g.close()
    print("random tubes that reached a non-finite state (index, step):", nonfinite)
    assert len(nonfinite) <= 16
