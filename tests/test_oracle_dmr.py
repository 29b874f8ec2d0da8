"""Pins for the oracle's double Mach reflection boundaries (Example 11, after Woodward and
Colella): the problem data satisfy the Rankine-Hugoniot conditions of a Mach 10 shock; the
reflecting wall equals the mirror-image problem on the doubled domain (no boundary there);
constant states are preserved next to the inflow side and along the wall; the top side
switches from the post- to the pre-shock state exactly at the moving shock's position."""
import math

import numpy as np
import pytest

import oracle
from paper_1904_11147_gb300 import workloads as W

G = 1.4


def _cons(w):
    rho, u, v, p = w
    return np.array([rho, rho * u, rho * v, p / (G - 1) + 0.5 * rho * (u * u + v * v)])


def _const_state(m, c):
    u = m.zeros()
    u[:, :, 0] = 2.0 * np.asarray(c)[None, :]
    return u


def test_problem_data_is_a_mach_10_shock():
    """Mass, momentum and energy fluxes through the shock, in its frame (speed 10 along the
    normal n = (cos 30, -sin 30)), are equal on both sides; the pre-shock sound speed is 1;
    the shock line's speed along x is 10 / cos 30."""
    p = W.double_mach().params[0]
    post, pre = p[0:4], p[4:8]
    n = np.array([math.sqrt(3) / 2, -0.5])
    s = 10.0
    def fluxes(w):
        rho, u, v, pr = w
        vn = u * n[0] + v * n[1] - s
        E = pr / (G - 1) + 0.5 * rho * (u * u + v * v)
        return np.array([rho * vn, rho * vn * (u * n[0] + v * n[1]) + pr, (E + pr) * vn + s * pr])
    # energy flux in the shock frame: (E + p) vn + s p accounts for the moving frame's work
    np.testing.assert_allclose(fluxes(post), fluxes(pre), rtol=1e-12, atol=1e-12)
    assert math.isclose(math.sqrt(G * pre[3] / pre[0]), 1.0, rel_tol=1e-15)
    assert math.isclose(p[10] * n[0], s, rel_tol=1e-15)
    # the velocity behind the shock is along the normal
    assert math.isclose(post[1] * n[1] - post[2] * n[0], 0.0, abs_tol=1e-14)


def _dmr_mesh(nx, ny, N, a=1.0 / 6.0, t=0.0, box=(0.0, 4.0, 0.0, 1.0)):
    p = list(W.double_mach().params[0])
    p[8] = a
    m = oracle.Mesh(2, 1, N, nx, ny, box=box, bc=oracle.BC_DMR, bcp=p)
    m.t = t
    return m, p


@pytest.mark.parametrize("N", [1, 2, 3])
def test_reflecting_wall_is_the_mirror_problem(N):
    """A random state on [0,1] x [0,1] with the wall along the whole bottom (a < 0), against
    the state mirrored into [0,1] x [-1,1] (y -> -y, rho v -> -rho v) with plain outflow
    ghosts: the operator L and the limiter (every cell troubled) agree on the two rows next
    to the wall, away from the side boundaries.  The mirror problem has no wall, so this
    fixes the reflecting rule (mirror image, normal momentum negated)."""
    nx, ny = 8, 6
    rng = np.random.default_rng(3 + N)
    m1, _ = _dmr_mesh(nx, ny, N, a=-1.0, box=(0.0, 1.0, 0.0, 1.0))
    u1 = W.random_modes(2, 1, N, nx * ny, rng, smooth=0.05)
    ab = oracle.mode_ab(2, N)
    m2 = oracle.Mesh(2, 1, N, nx, 2 * ny, box=(0.0, 1.0, -1.0, 1.0), bc=oracle.BC_OUTFLOW)
    u2 = m2.zeros().reshape(2 * ny, nx, 4, len(ab))
    v1 = u1.reshape(ny, nx, 4, len(ab))
    sgn = np.array([(-1.0) ** b for a, b in ab])
    u2[ny:] = v1
    for iy in range(ny):
        for v in range(4):
            u2[ny - 1 - iy, :, v, :] = v1[iy, :, v, :] * sgn * (-1.0 if v == 2 else 1.0)
    u2 = u2.reshape(-1, 4, len(ab))
    L1 = m1.rhs(u1).reshape(ny, nx, 4, -1)
    L2 = m2.rhs(u2).reshape(2 * ny, nx, 4, -1)
    cols = slice(1, nx - 1)
    scale = np.abs(L1[0:2, cols]).max()
    assert np.abs(L1[0:2, cols] - L2[ny:ny + 2, cols]).max() <= 1e-12 * scale
    lim1 = m1.limit(u1, np.ones(nx * ny, np.uint8)).reshape(ny, nx, 4, -1)
    lim2 = m2.limit(u2, np.ones(2 * nx * ny, np.uint8)).reshape(2 * ny, nx, 4, -1)
    scale = np.abs(lim1[0:2, cols]).max()
    assert np.abs(lim1[0:2, cols] - lim2[ny:ny + 2, cols]).max() <= 1e-12 * scale
    # and the wall makes a difference: plain outflow ghosts change the bottom row
    m3 = oracle.Mesh(2, 1, N, nx, ny, box=(0.0, 1.0, 0.0, 1.0), bc=oracle.BC_OUTFLOW)
    assert np.abs(m3.rhs(u1).reshape(ny, nx, 4, -1)[0, cols] - L1[0, cols]).max() > 1e-6 * scale


@pytest.mark.parametrize("N", [1, 2])
def test_wall_and_inflow_keep_constant_states(N):
    """Uniform flow along the wall (v = 0) keeps L = 0 in the bottom row beyond the wall's
    start; the uniform post-shock state keeps L = 0 in the left column (inflow of the same
    state), away from the top and bottom sides."""
    nx, ny = 12, 4
    m, p = _dmr_mesh(nx, ny, N)
    hx = 4.0 / nx
    u = _const_state(m, _cons([1.3, 2.0, 0.0, 0.9]))
    L = m.rhs(u).reshape(ny, nx, 4, -1)
    first = int(math.ceil((1.0 / 6.0) / hx)) + 1
    assert np.abs(L[0, first:nx - 1]).max() <= 1e-12
    u = _const_state(m, _cons(p[0:4]))
    L = m.rhs(u).reshape(ny, nx, 4, -1)
    assert np.abs(L[1:ny - 1, 0]).max() <= 1e-11 * np.abs(u).max()


@pytest.mark.parametrize("t", [0.0, 0.05, 0.13])
def test_top_side_follows_the_moving_shock(t):
    """With the post-shock state everywhere, a top-row cell changes (L != 0) exactly when
    its ghost holds the pre-shock state: when its centre lies right of the shock's position
    on the top side, x_s = 1/6 + (1 + 20 t) / sqrt(3), at the state's time t."""
    nx, ny = 48, 4
    m, p = _dmr_mesh(nx, ny, 1, t=t)
    u = _const_state(m, _cons(p[0:4]))
    L = m.rhs(u).reshape(ny, nx, 4, -1)
    xs = 1.0 / 6.0 + (1.0 + 20.0 * t) / math.sqrt(3.0)
    xc = (np.arange(nx) + 0.5) * 4.0 / nx
    changed = np.abs(L[ny - 1]).max(axis=(1, 2)) > 1e-9
    np.testing.assert_array_equal(changed[: nx - 1], (xc >= xs)[: nx - 1])
    assert changed.any() and not changed.all()


def test_step_uses_the_stage_times():
    """or_step evaluates the top boundary at the stage times t, t + dt, t + dt/2: stepping
    a state from t equals three stages with the mesh time set to those values."""
    nx, ny, N = 16, 4, 1
    dt = 1e-3
    # the shock's position on the top side passes the centre x = 1.125 of a top ghost cell
    # during the step (at t + dt/4): only stage times after t see the pre-shock ghost there
    t0 = ((1.125 - 1.0 / 6.0) * math.sqrt(3.0) - 1.0) / 20.0 - dt / 4
    m, p = _dmr_mesh(nx, ny, N, t=t0)
    rng = np.random.default_rng(1)
    u0 = _const_state(m, _cons(p[0:4])) * (1 + 0.01 * rng.standard_normal((nx * ny, 4, 3)))
    ref, _, _ = m.step(u0, dt, limit=False)
    a = u0
    for s, c in ((1, 0.0), (2, 1.0), (3, 0.5)):
        m.t = t0 + c * dt
        a = m.rk_stage(s, dt, u0, a)
    np.testing.assert_array_equal(a, ref)
    # with every stage at t the result differs
    b = u0
    m.t = t0
    for s in (1, 2, 3):
        b = m.rk_stage(s, dt, u0, b)
    assert np.abs(b - ref).max() > 1e-6
