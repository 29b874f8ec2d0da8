"""Example 11 (double Mach reflection) on the GPU: the DG_BC_DMR boundaries (post-shock
inflow, reflecting wall, outflow, the exact moving shock on the top side) against the oracle
stage by stage, with the positivity-preserving scaling the example adds; and a coarse run to
t = 0.2 that must stay admissible and place the shock where the exact solution has it."""
import math

import numpy as np
import pytest

import oracle
import paper_1904_11147_gb300 as dgl
from paper_1904_11147_gb300 import workloads as W
from parity_cases import rel, rel_hi

pytestmark = pytest.mark.gpu


def _pair(nx, ny, N, stream=0):
    w = W.double_mach(nx, ny, N)
    p = w.params[0]
    o = oracle.Mesh(2, 1, N, nx, ny, box=w.box[0], bc=oracle.BC_DMR, bcp=p)
    g = dgl.Mesh(2, 1, N, [nx], [ny], w.box, bc=dgl.BC_DMR, stream=stream)
    g.set_boundary_data(p)
    return w, o, g


def test_dmr_argument_errors():
    w = W.double_mach(16, 4, 2)
    g = dgl.Mesh(2, 1, 2, [16], [4], w.box, bc=dgl.BC_DMR)
    g.project_ic(dgl.IC_DMR, [w.params[0]])
    with pytest.raises(dgl.DGError):
        g.rk_stage(1, 1e-4)  # no boundary data yet
    with pytest.raises(dgl.DGError):
        g.set_boundary_data(w.params[0][:10])
    g.set_boundary_data(w.params[0])
    for bad in (lambda: g.flag_cells(dgl.IND_KXRCF, 0.0), lambda: g.set_limiter(dgl.LIM_PARENT),
                lambda: g.step(1e-4, dgl.IND_KXRCF)):
        with pytest.raises(dgl.DGError):
            bad()
    with pytest.raises(dgl.DGError):
        dgl.Mesh(1, 1, 2, [16], None, [(0.0, 1.0, 0.0, 1.0)], bc=dgl.BC_DMR)
    g.set_time(0.125)
    assert g.get_time()[0] == 0.125


@pytest.mark.parametrize("N", [2, 3])
def test_dmr_shadow(N):
    """From the initial data, every stage, its TVB flags, its limited state and its
    positivity scaling agree with the oracle from the same input (stage 1e-13, flags
    identical, limiter and scaling 1e-11, limited modes n >= 1 1e-11 of their own scale);
    the oracle evaluates the boundaries at the stage times.  The CUDA-graph step from the
    same state reproduces the stage calls bitwise, and advances the library's time."""
    import torch
    st = torch.cuda.Stream()
    nx, ny = 64, 16
    w, o, g = _pair(nx, ny, N, st.cuda_stream)
    p = w.params[0]
    # the P2/P3 projection of the oblique shock has negative density and pressure at some
    # quadrature points; the positivity-preserving scaling makes the initial data admissible
    u0 = o.project_ic(oracle.IC_DMR, p)
    g.project_ic(dgl.IC_DMR, [p])
    assert rel(g.get_modes(), u0) < 1e-13
    u0, _, bad = o.positivity_limit(u0, 1e-13)
    assert bad == 0
    g.positivity_limit(1e-13)
    assert rel(g.get_modes(), u0) < 1e-11
    ws = o.max_wavespeed(u0)
    h = 4.0 / nx
    dt = 0.1 / (ws[0] / h + ws[1] / h)
    t = 0.0
    flagged = 0
    worst = [0.0, 0.0, 0.0]
    with torch.cuda.stream(st):
        for k in range(25):
            prev = g.get_modes()
            g.set_time(t)
            us = prev
            for s, c_in, c_out in ((1, 0.0, 1.0), (2, 1.0, 0.5), (3, 0.5, 1.0)):
                g.rk_stage(s, dt)
                got = g.get_modes()
                o.t = t + c_in * dt
                ref = o.rk_stage(s, dt, prev, us)
                d = rel(got, ref)
                assert d <= 1e-13, (k, s, "stage", d)
                worst[0] = max(worst[0], d)
                o.t = t + c_out * dt
                fl, nf, _ = g.flag_cells(dgl.IND_TVB, 0.01, want=True)
                fo, nfo, _ = o.flag_tvb(got, 0.01)
                assert np.array_equal(fl, fo), (k, s, int((fl != fo).sum()))
                flagged += nf
                g.cswenolimit()
                lim = g.get_modes()
                lref = o.limit(got, fl)
                d, dh = rel(lim, lref), rel_hi(lim, lref)
                assert d <= 1e-11 and dh <= 1e-11, (k, s, "limiter", d, dh)
                worst[1] = max(worst[1], dh)
                g.positivity_limit(1e-13)
                sc = g.get_modes()
                ref_pp, _, bad = o.positivity_limit(lim, 1e-13)
                assert bad == 0
                d = rel(sc, ref_pp)
                assert d <= 1e-11, (k, s, "positivity", d)
                worst[2] = max(worst[2], d)
                us = sc
            assert abs(g.get_time()[0] - (t + dt)) <= 1e-15 * max(t, 1.0)
            # the graph step from the same state
            g.set_modes(prev)
            g.set_time(t)
            g.set_positivity(True)
            g.step(dt)
            assert np.array_equal(g.get_modes(), us), (k, "graph step differs from the stage calls")
            g.set_positivity(False)
            t += dt
    print("DMR P%d shadow: worst stage %.2e, limited modes n>=1 %.2e, scaling %.2e, flagged %d"
          % (N, worst[0], worst[1], worst[2], flagged))
    assert flagged > 0


def test_dmr_coarse_run_to_t02():
    """P2 at 240 x 60 to t = 0.2 with the positivity-preserving scaling (CFL 0.1 on the
    check-point wave speeds every step): no inadmissible mean, a finite state, and along the
    top rows the incident shock where the exact solution puts it, x_s = 1/6 + (1 + 20 t)
    / sqrt(3) (the post-shock density 8 to its left, 1.4 to its right)."""
    import torch
    st = torch.cuda.Stream()
    nx, ny, N = 240, 60, 2
    w, o, g = _pair(nx, ny, N, st.cuda_stream)
    g.project_ic(dgl.IC_DMR, [w.params[0]])
    g.positivity_limit(1e-13)  # the projected oblique shock is not admissible at every point
    g.set_positivity(True)
    h = 4.0 / nx
    t, steps = 0.0, 0
    with torch.cuda.stream(st):
        while t < 0.2 - 1e-12:
            sp = g.max_wavespeed(points=True)[0]
            dt = min(0.1 / (sp[0] / h + sp[1] / h), 0.2 - t)
            g.step(dt)
            t += dt
            steps += 1
    st.synchronize()
    changed, bad = g.positivity_counts()
    u = g.get_modes()
    assert bad == 0 and np.isfinite(u).all(), (bad, steps)
    assert abs(g.get_time()[0] - t) <= 1e-12
    rho = (u[:, 0, 0] * 0.5).reshape(ny, nx)
    xs = 1.0 / 6.0 + (1.0 + 20.0 * 0.2) / math.sqrt(3.0)
    xc = (np.arange(nx) + 0.5) * h
    top = rho[-3:].mean(axis=0)
    left = top[(xc > xs - 0.3) & (xc < xs - 0.1)]
    right = top[xc > xs + 0.1]
    print("DMR 240x60 P2: %d steps, density %.3f..%.3f, top rows left of the shock %.2f, right %.2f, "
          "scaled cells %d" % (steps, rho.min(), rho.max(), left.mean(), right.mean(), changed))
    assert abs(left.mean() - 8.0) < 0.5 and abs(right.mean() - 1.4) < 0.05
    assert rho.min() > 0 and rho.max() < 30
