"""The learned indicator's positivity fallback against the oracle, stage by stage.

dg_step with the learned indicator limits the cells the network keeps.  When one of the
TVB-flagged cells the network skipped has a non-positive density or pressure at a volume
or face Gauss point of its unlimited stage (FP32 screen: rho > 0 and p > 1e-6 |E|), the
instance's stage is redone with all its TVB flags: the plain method's stage.  Here the
network never keeps a cell, so per instance and stage the library must produce the
unlimited stage, or oracle.limit(stage, flag_tvb(stage)) when a TVB-flagged cell fails the
screen; its fallback count must equal the number of redone (instance, stage) pairs and its
failure count the (instance, stage) pairs whose final stage still fails the screen at some
cell, both recomputed on the host.  The states are chosen so that no screened point lies near the decision (the FP64
host recomputation then decides exactly as the FP32 kernel).
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


def _oracle_fallback(o, st):
    """The learned stage with a network that keeps no cell, with the positivity fallback:
    (result, redone, failed).  Only the TVB-flagged cells the network skipped can make the
    plain stage differ, so they decide the redo; the final screen covers every cell."""
    fl, _, _ = o.flag_tvb(st, 0.01)
    res, redo = st, 0
    if fl.any():
        mg = _screen_margin(st)[fl == 1]
        assert np.abs(mg[np.isfinite(mg)]).min() > 1e-5, "a screened point lies near the decision"
        if not (mg > 0).all():
            res, redo = o.limit(st, fl), 1
    mg2 = _screen_margin(res)
    assert np.abs(mg2[np.isfinite(mg2)]).min() > 1e-5
    return res, redo, int(not (mg2 > 0).all())


def _oracle_learned_none_step(o, u, dt):
    """One SSP-RK3 step of the learned indicator whose network keeps no cell, with the
    positivity fallback.  Returns (state, stages redone, failures)."""
    prev = u
    redo = fails = 0
    for s in (1, 2, 3):
        res, r, f = _oracle_fallback(o, o.rk_stage(s, dt, u, prev))
        redo += r
        fails += f
        prev = res
    return prev, redo, fails


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
    seen_redo, seen_pass = set(), set()
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
            (seen_redo if fb else seen_pass).add(i)
            step_fb += fb
            step_fail += fails
        assert fb1 - fb0 == step_fb and fail1 - fail0 == step_fail, (k, fb1 - fb0, step_fb, fail1 - fail0, step_fail)
        tot_fb += step_fb
        tot_fail += step_fail
        prev = got
    torch.cuda.synchronize()
    print("redone instance-stages %d, failures %d, instances redone %s, never redone %s"
          % (tot_fb, tot_fail, sorted(seen_redo), sorted(seen_pass)))
    # some instances redone and others not
    assert seen_redo and seen_pass


def test_fallback_with_positivity_scaling_matches_oracle():
    """The same batch with the positivity-preserving scaling after every stage (the batched
    P3 workload's setting): per instance and stage, the fallback decision on the skipped
    cells, then the Zhang-Shu scaling of the result, against the oracle from the same input;
    with the scaling on, no failure is counted."""
    import torch
    st = torch.cuda.Stream()
    g, os_, us, dt = _mesh_and_state(st.cuda_stream)
    net = dgl.MLP(dgl.n_features(2, 1, N), seed=5)
    g.set_indicator(net, 1e30)  # keeps no cell
    g.set_positivity(True, 1e-13)
    sizes = [o.nx * o.ny for o in os_]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    prev = np.concatenate(us)
    tot = 0
    for k in range(3):
        with torch.cuda.stream(st):
            g.set_modes(prev)
            fb0, _ = g.positivity_report()
            g.step(dt, dgl.IND_MLP, 0.01)
            got = g.get_modes()
        fb1, fail1 = g.positivity_report()
        redo = 0
        for i, o in enumerate(os_):
            sl = slice(offs[i], offs[i + 1])
            u0 = prev[sl]
            a = u0
            for s in (1, 2, 3):
                stg = o.rk_stage(s, dt, u0, a)
                fl, _, _ = o.flag_tvb(stg, 0.01)
                if fl.any():
                    mg = _screen_margin(stg)[fl == 1]
                    assert np.abs(mg[np.isfinite(mg)]).min() > 1e-5, "a screened point lies near the decision"
                    if not (mg > 0).all():
                        stg = o.limit(stg, fl)
                        redo += 1
                a, _, bad = o.positivity_limit(stg, 1e-13)
                assert bad == 0
            d, dh = rel(got[sl], a), rel_hi(got[sl], a)
            assert d <= 1e-11 and dh <= 1e-11, (k, i, d, dh)
        assert fb1 - fb0 == redo and fail1 == 0, (k, fb1 - fb0, redo, fail1)
        tot += redo
        prev = got
    print("with the scaling: %d instance stages redone" % tot)
    assert tot > 0


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


def _cons(r, vx, vy, p):
    return np.array([r, r * vx, r * vy, p / (G - 1) + 0.5 * r * (vx * vx + vy * vy)])


def _hostile_state(n, seed):
    """Near-vacuum random cells with large slopes: many TVB-flagged cells fail the screen,
    and some still fail after the plain limiter (a failure)."""
    rng = np.random.default_rng(seed)
    ab = oracle.mode_ab(2, N)
    u = np.zeros((n * n, 4, len(ab)))
    for c in range(n * n):
        r, p = 10 ** rng.uniform(-2, 0), 10 ** rng.uniform(-3, 0)
        vx, vy = rng.uniform(-2, 2, 2)
        u[c, :, 0] = 2 * _cons(r, vx, vy, p)
        u[c, :, 1:] = 0.3 * rng.standard_normal((4, len(ab) - 1)) * np.abs(u[c, :, 0:1])
    return u


def test_fallback_redo_per_call():
    """dg_flag_cells(learned) + dg_cswenolimit on a state set directly, three instances: a
    near-vacuum one (redone with all its TVB flags; limited cells still fail), the stage
    output of a strong four-quadrant problem (redone), and a smooth one (nothing to do);
    each against the oracle's fallback on the same state, the counts included."""
    n0, n1, n2 = 12, 20, 16
    box = (0.0, 1.0, 0.0, 1.0)
    o0, o1, o2 = (oracle.Mesh(2, 1, N, k, k, box=box, bc=1) for k in (n0, n1, n2))
    u0 = _hostile_state(n0, 1)
    pq = [1.0, 0.0, 0.0, 1.0, 0.01, 0.0, 0.0, 0.005, 1.0, 0.0, 0.0, 1.0, 0.01, 0.0, 0.0, 0.005, 0.5, 0.5]
    q = o1.project_ic(2, pq)
    ws = o1.max_wavespeed(q)
    u1 = o1.rk_stage(1, 0.1 / (ws[0] * n1 + ws[1] * n1), q, q)
    u2 = o2.project_ic(oracle.IC_DENSITY_WAVE, [1.0, 0.2, 2 * np.pi, 2 * np.pi, 0.3, -0.2, 1.0])
    g = dgl.Mesh(2, 1, N, [n0, n1, n2], [n0, n1, n2], [box] * 3, bc=1)
    net = dgl.MLP(dgl.n_features(2, 1, N), seed=5)
    g.set_indicator(net, 1e30)  # keeps no cell
    g.set_modes(np.concatenate([u0, u1, u2]))
    fb0, fail0 = g.positivity_report()
    g.flag_cells(dgl.IND_MLP, 0.01)
    g.cswenolimit()
    got = g.get_modes()
    fb1, fail1 = g.positivity_report()
    redo, fails = [], 0
    off = 0
    for o, u in ((o0, u0), (o1, u1), (o2, u2)):
        sl = slice(off, off + o.nx * o.ny)
        ref, r, f = _oracle_fallback(o, u)
        redo.append(r)
        fails += f
        ok = np.isfinite(ref)
        assert np.array_equal(ok, np.isfinite(got[sl]))
        assert rel(np.where(ok, got[sl], 0.0), np.where(ok, ref, 0.0)) <= 1e-11
        off += o.nx * o.ny
    print("redone per instance %s, failures %d" % (redo, fails))
    assert redo == [1, 1, 0] and fails >= 1
    redo = sum(redo)
    assert fb1 - fb0 == redo and fail1 - fail0 == fails
