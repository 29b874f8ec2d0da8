"""The learned indicator's positivity fallback against the oracle, stage by stage.

dg_step with the learned indicator limits the cells the network keeps; among the
TVB-flagged cells the network skipped, every one whose unlimited stage has a non-positive
density or pressure at a volume or face Gauss point (FP32 screen: rho > 0 and
p > 1e-6 |E|) falls back to the plain TVB decision and is limited too.  Here the network
never keeps a cell, so per instance and stage the library must produce
oracle.limit(stage, F) with F the TVB-flagged cells that fail the screen (the limiter is
a Jacobi update, so this equals the plain method's values on F and the unlimited stage
elsewhere), and its fallback count must equal the number of (instance, stage) pairs with
a non-empty F, recomputed on the host.  The states are chosen so that no screened point
lies near the decision (the FP64 host recomputation then decides exactly as the FP32
kernel).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as Lg

import oracle
import paper_1904_11147_gb300 as dgl
from parity_cases import rel, rel_hi

pytestmark = pytest.mark.gpu

G = 1.4
N = 2
# (nx, ny, low-state density): the low quadrants hold (rho, 0, 0, rho / 2) against (1, 0, 0, 1)
INSTANCES = [(20, 20, 0.01), (24, 18, 0.2), (18, 26, 0.02), (22, 22, 0.5)]


def _psi(n, x):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return math.sqrt((2 * n + 1) / 2) * Lg.legval(x, c)


def _screen_margin(u):
    """Per cell: the smallest of rho / max rho and (p - 1e-6 |E|) / |E| over the volume and
    face Gauss points the library screens; <= 0 fails."""
    g, _ = Lg.leggauss(N + 1)
    pts = [(r, s) for s in g for r in g]
    pts += [(1.0, s) for s in g] + [(-1.0, s) for s in g] + [(r, 1.0) for r in g] + [(r, -1.0) for r in g]
    ab = oracle.mode_ab(2, N)
    Phi = np.array([[_psi(a, r) * _psi(b, s) for a, b in ab] for r, s in pts])
    q = np.einsum("cvk,pk->cpv", u, Phi)
    rho, E = q[..., 0], q[..., 3]
    p = (G - 1) * (E - 0.5 * (q[..., 1] ** 2 + q[..., 2] ** 2) / rho)
    m = np.minimum(rho / np.abs(rho).max(), (p - 1e-6 * np.abs(E)) / np.maximum(np.abs(E), 1e-300))
    return m.min(axis=1)


def _oracle_learned_none_step(o, u, dt):
    """One SSP-RK3 step of the learned indicator whose network keeps no cell, with the
    per-cell positivity fallback.  Returns (state, fallbacks, failures)."""
    un = prev = u
    fb = fails = 0
    for s in (1, 2, 3):
        st = o.rk_stage(s, dt, un, prev)
        fl, _, _ = o.flag_tvb(st, 0.01)
        mg = _screen_margin(st)
        assert (fl == 0).all() or np.abs(mg[fl == 1]).min() > 1e-5, "a screened point lies near the decision"
        back = ((fl == 1) & (mg <= 0)).astype(np.uint8)
        if back.any():
            fb += 1
            prev = o.limit(st, back)
            mg2 = _screen_margin(prev)[back == 1]
            assert np.abs(mg2).min() > 1e-5
            fails += int((mg2 <= 0).any())
        else:
            prev = st
    return prev, fb, fails


def _mesh_and_state(stream):
    boxes = [(0.0, 1.0, 0.0, 1.0)] * len(INSTANCES)
    g = dgl.Mesh(2, 1, N, [i[0] for i in INSTANCES], [i[1] for i in INSTANCES], boxes, bc=1, stream=stream)
    params, os_, us = [], [], []
    for nx, ny, lo in INSTANCES:
        p = [1.0, 0.0, 0.0, 1.0, lo, 0.0, 0.0, 0.5 * lo, 1.0, 0.0, 0.0, 1.0, lo, 0.0, 0.0, 0.5 * lo, 0.5, 0.5]
        o = oracle.Mesh(2, 1, N, nx, ny, box=(0.0, 1.0, 0.0, 1.0), bc=1)
        params.append(p)
        os_.append(o)
        us.append(o.project_ic(2, p))
    g.set_modes(np.concatenate(us))
    dt = min(0.1 / (o.max_wavespeed(u)[0] * o.nx + o.max_wavespeed(u)[1] * o.ny) for o, u in zip(os_, us))
    return g, os_, us, dt


def test_fallback_stage_by_stage_matches_oracle():
    import torch
    st = torch.cuda.Stream()
    g, os_, us, dt = _mesh_and_state(st.cuda_stream)
    net = dgl.MLP(dgl.n_features(2, 1, N), seed=5)
    g.set_indicator(net, 1e30)  # keeps no cell
    sizes = [o.nx * o.ny for o in os_]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    tot_fb = tot_fail = 0
    seen_fb, seen_pass = set(), set()
    prev = np.concatenate(us)
    for k in range(4):
        with torch.cuda.stream(st):
            g.set_modes(prev)
            fb0, fail0 = g.positivity_report()
            g.step(dt, dgl.IND_MLP, 0.01)
            got = g.get_modes()
        fb1, fail1 = g.positivity_report()
        step_fb = step_fail = 0
        for i, o in enumerate(os_):
            sl = slice(offs[i], offs[i + 1])
            ref, fb, fails = _oracle_learned_none_step(o, prev[sl], dt)
            d, dh = rel(got[sl], ref), rel_hi(got[sl], ref)
            assert d <= 1e-11 and dh <= 1e-11, (k, i, fb, d, dh)
            (seen_fb if fb else seen_pass).add(i)
            step_fb += fb
            step_fail += fails
        assert fb1 - fb0 == step_fb and fail1 - fail0 == step_fail, (k, fb1 - fb0, step_fb, fail1 - fail0, step_fail)
        tot_fb += step_fb
        tot_fail += step_fail
        prev = got
    torch.cuda.synchronize()
    print("fallback instance-stages %d, failures %d, instances that fell back %s, passed %s"
          % (tot_fb, tot_fail, sorted(seen_fb), sorted(seen_pass)))
    # both branches were exercised
    assert seen_fb and seen_pass and tot_fb > 0


def test_network_keeping_every_cell_is_the_plain_method():
    """tau below every logit: the learned indicator keeps every TVB-flagged cell, so a step
    equals the plain TVB step of the oracle (no cell is skipped, no fallback)."""
    g, os_, us, dt = _mesh_and_state(0)
    net = dgl.MLP(dgl.n_features(2, 1, N), seed=5)
    g.set_indicator(net, -1e30)
    sizes = [o.nx * o.ny for o in os_]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    prev = np.concatenate(us)
    for k in range(3):
        g.set_modes(prev)
        g.step(dt, dgl.IND_MLP, 0.01)
        got = g.get_modes()
        for i, o in enumerate(os_):
            sl = slice(offs[i], offs[i + 1])
            ref, _, _ = o.step(prev[sl], dt)
            assert rel(got[sl], ref) <= 1e-11, (k, i, rel(got[sl], ref))
        prev = got
    assert g.positivity_report() == (0, 0)
