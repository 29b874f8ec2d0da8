"""Seeded synthetic workloads.

This module only draws random numbers and states problem parameters; it holds none of
the method's arithmetic, so that the CUDA path and the CPU oracle can both take their
inputs from it.  Every workload is a closed-form initial condition of the kind the
paper's examples use (Sec. 4): a sine wave for Burgers (Examples 1, 2, 5), shock tubes
for 1D Euler (Examples 7, 8) and four-quadrant Riemann problems for 2D Euler.

Initial-condition families (``ic`` codes shared with the library's projection call):
  0 sine:          u = p0 + p1 sin(p2 x + p3 y)
  1 Riemann 1D:    (rho,u,p)_L = p0..p2 for x < p6, (rho,u,p)_R = p3..p5 otherwise
  2 four quadrant: (rho,u,v,p) for x>=p16,y>=p17 (p0..3); x<p16,y>=p17 (p4..7);
                   x<p16,y<p17 (p8..11); x>=p16,y<p17 (p12..15)
  3 density wave:  rho = p0 + p1 sin(p2 x + p3 y), u = p4, v = p5, p = p6
  4 shock/entropy: (rho,u,p) = p0..p2 for x < p3, else rho = p4 + p5 sin(p6 x), u = p7, p = p8
  5 vortex:        isentropic vortex centred at (p0 + p3, p1), strength p2, at time p3
  6 double Mach:   post-shock (rho,u,v,p) = p0..p3 where x < p8 + p9 y, pre-shock p4..p7
                   elsewhere (p10: the shock line's speed along x, for the top boundary)
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

SEED = 1904

PDE_BURGERS, PDE_EULER = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_DMR = 0, 1, 2
IC_SINE, IC_RIEMANN1D, IC_QUADRANT, IC_DENSITY_WAVE, IC_SHOCK_ENTROPY, IC_VORTEX, IC_DMR = 0, 1, 2, 3, 4, 5, 6
GAMMA = 1.4


@dataclass
class Workload:
    name: str
    dim: int
    pde: int
    N: int
    nx: list
    ny: list
    box: list            # per instance (xL, xR, yL, yR)
    bc: int
    ic: int
    params: list         # per instance parameter vector
    t_end: float
    cfl: float = 0.1
    tvb_M: float = 0.01
    gamma: float = GAMMA
    extra: dict = field(default_factory=dict)

    @property
    def n_inst(self):
        return len(self.nx)

    @property
    def nvars(self):
        return 1 if self.pde == PDE_BURGERS else (3 if self.dim == 1 else 4)

    @property
    def nmodes(self):
        return self.N + 1 if self.dim == 1 else (self.N + 1) * (self.N + 2) // 2

    @property
    def cells(self):
        return int(sum(a * b for a, b in zip(self.nx, self.ny)))

    @property
    def dofs(self):
        return self.cells * self.nvars * self.nmodes


def burgers_1d(K: int = 160, N: int = 2, t_end: float = 1.5 / math.pi) -> Workload:
    """1D Burgers on [-1,1], periodic, u0 = 0.5 + sin(pi x) (Example 1 rescaled by pi)."""
    return Workload("burgers1d_p%d_k%d" % (N, K), 1, PDE_BURGERS, N, [K], [1], [(-1.0, 1.0, 0.0, 1.0)],
                    BC_PERIODIC, IC_SINE, [[0.5, 1.0, math.pi, 0.0]], t_end)


def shock_tube(kind: str = "sod", K: int = 800, N: int = 3, index: int = 0) -> Workload:
    """1D Euler shock tubes on [0,1] split at x = 0.5: Sod (t=0.2), Lax (t=0.13), or the
    seeded random tube number ``index`` (rho,p ~ U[0.1,2], u ~ U[-1,1] per side)."""
    if kind == "sod":
        p, t = [1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 0.5], 0.2
    elif kind == "lax":
        p, t = [0.445, 0.698, 3.528, 0.5, 0.0, 0.571, 0.5], 0.13
    else:
        r = np.random.default_rng(SEED + index)
        rl, pl, rr, pr = r.uniform(0.1, 2.0, 4)
        ul, ur = r.uniform(-1.0, 1.0, 2)
        p, t = [rl, ul, pl, rr, ur, pr, 0.5], 0.1
    return Workload("%s_tube_p%d_k%d" % (kind, N, K), 1, PDE_EULER, N, [K], [1], [(0.0, 1.0, 0.0, 1.0)],
                    BC_OUTFLOW, IC_RIEMANN1D, [list(map(float, p))], t)


def shock_entropy(K: int = 200, N: int = 2) -> Workload:
    """Example 9: a Mach-3 shock running into a density wave on [0,1], outflow, to t = 0.178."""
    p = [3.857143, 2.629369, 10.333333, 0.125, 1.0, 0.2, 16.0 * math.pi, 0.0, 1.0]
    return Workload("shock_entropy_p%d_k%d" % (N, K), 1, PDE_EULER, N, [K], [1], [(0.0, 1.0, 0.0, 1.0)],
                    BC_OUTFLOW, IC_SHOCK_ENTROPY, [p], 0.178)


def isentropic_vortex(n: int = 40, N: int = 2) -> Workload:
    """Example 4: the isentropic vortex (x0 = 5, y0 = 0, beta = 5) on [0,10] x [-5,5],
    periodic, to t = 2 (the domain is our reading; the paper names only the centre)."""
    return Workload("vortex_p%d_%dx%d" % (N, n, n), 2, PDE_EULER, N, [n], [n], [(0.0, 10.0, -5.0, 5.0)],
                    BC_PERIODIC, IC_VORTEX, [[5.0, 0.0, 5.0, 0.0]], 2.0)


def double_mach(nx: int = 960, ny: int = 240, N: int = 2) -> Workload:
    """Example 11: double Mach reflection (Woodward and Colella) on [0,4] x [0,1] to t = 0.2:
    a Mach 10 shock in air (gamma = 1.4) at 60 degrees to the x axis, its foot at x = 1/6 on
    the bottom side, running right into gas at rest with rho = 1.4, p = 1.  Post-shock state
    rho = 8, p = 116.5, velocity 8.25 along the shock normal (cos 30, -sin 30).  The shock
    line x = 1/6 + y / sqrt(3) moves along x at 20 / sqrt(3) (speed 10 along its normal).
    Boundaries (BC_DMR): post-shock inflow on the left and on the bottom for x < 1/6, a
    reflecting wall on the rest of the bottom, outflow on the right, and on the top the
    post- or pre-shock state on either side of the moving shock."""
    s3 = math.sqrt(3.0)
    p = [8.0, 8.25 * s3 / 2.0, -8.25 / 2.0, 116.5, 1.4, 0.0, 0.0, 1.0, 1.0 / 6.0, 1.0 / s3, 20.0 / s3]
    return Workload("double_mach_p%d_%dx%d" % (N, nx, ny), 2, PDE_EULER, N, [nx], [ny], [(0.0, 4.0, 0.0, 1.0)],
                    BC_DMR, IC_DMR, [p], 0.2)


def quadrant_states(rng) -> list:
    """18 parameters of a four-quadrant Riemann problem split at (0.5, 0.5)."""
    p = []
    for _ in range(4):
        rho, pr = rng.uniform(0.1, 2.0, 2)
        u, v = rng.uniform(-1.0, 1.0, 2)
        p += [float(rho), float(u), float(v), float(pr)]
    return p + [0.5, 0.5]


def euler_2d_quadrant(n: int = 1024, N: int = 2, seed: int = SEED) -> Workload:
    """2D Euler four-quadrant Riemann problem on [0,1]^2, outflow, to t = 0.25."""
    rng = np.random.default_rng(seed)
    return Workload("euler2d_quadrant_p%d_%dx%d" % (N, n, n), 2, PDE_EULER, N, [n], [n], [(0.0, 1.0, 0.0, 1.0)],
                    BC_OUTFLOW, IC_QUADRANT, [quadrant_states(rng)], 0.25)


def burgers_2d_batched(n_inst: int = 64, N: int = 2, lo: int = 64, hi: int = 512, seed: int = SEED) -> Workload:
    """Batched 2D Burgers on [-2,2]^2, periodic, u0 = 0.5 + A sin(pi (x+y)/2), A ~ U[0.5,1.5],
    square meshes with sides log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    sides = [int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(n_inst)]
    amps = rng.uniform(0.5, 1.5, n_inst)
    return Workload("burgers2d_batched_p%d_x%d" % (N, n_inst), 2, PDE_BURGERS, N, sides, sides,
                    [(-2.0, 2.0, -2.0, 2.0)] * n_inst, BC_PERIODIC, IC_SINE,
                    [[0.5, float(a), math.pi / 2, math.pi / 2] for a in amps], 1.0)


def euler_2d_batched(n_inst: int = 256, N: int = 3, lo: int = 128, hi: int = 1024, seed: int = SEED) -> Workload:
    """Batched 2D Euler four-quadrant problems, sides log-uniform in [lo, hi] rounded to even
    numbers, so that the quadrant lines x = y = 0.5 fall on cell faces (a jump inside a cell
    makes the projected P3 polynomial lose positivity at quadrature points)."""
    rng = np.random.default_rng(seed)
    sides = [2 * int(round(0.5 * math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(n_inst)]
    params = [quadrant_states(rng) for _ in range(n_inst)]
    return Workload("euler2d_batched_p%d_x%d" % (N, n_inst), 2, PDE_EULER, N, sides, sides,
                    [(0.0, 1.0, 0.0, 1.0)] * n_inst, BC_OUTFLOW, IC_QUADRANT, params, 0.25)


def random_modes(dim: int, pde: int, N: int, ncell: int, rng, jump: float = 0.3, smooth: float = 0.05,
                 blocks: int = 7) -> np.ndarray:
    """Random modal states [cell][var][mode] with piecewise-constant means (jumps between
    runs of ``blocks`` cells) and small higher modes, for parity tests.  Euler states are
    drawn as positive density and internal energy well above the kinetic part."""
    nv = 1 if pde == PDE_BURGERS else (3 if dim == 1 else 4)
    npm = N + 1 if dim == 1 else (N + 1) * (N + 2) // 2
    u = np.zeros((ncell, nv, npm))
    nb = (ncell + blocks - 1) // blocks
    if pde == PDE_BURGERS:
        base = rng.uniform(-1.0, 1.0, nb).repeat(blocks)[:ncell]
        base = base + jump * rng.uniform(-1, 1, ncell) * 0.1
        u[:, 0, 0] = base
    else:
        rho = rng.uniform(0.6, 1.4, nb).repeat(blocks)[:ncell] * (1 + 0.02 * rng.uniform(-1, 1, ncell))
        vel = rng.uniform(-0.5, 0.5, (nb, dim)).repeat(blocks, axis=0)[:ncell]
        pr = rng.uniform(0.6, 1.4, nb).repeat(blocks)[:ncell]
        u[:, 0, 0] = rho
        for d in range(dim):
            u[:, 1 + d, 0] = rho * vel[:, d]
        u[:, nv - 1, 0] = pr / (GAMMA - 1) + 0.5 * rho * (vel ** 2).sum(axis=1)
    for k in range(1, npm):
        u[:, :, k] = smooth * rng.uniform(-1, 1, (ncell, nv)) * np.abs(u[:, :, 0]) / (k + 1)
    return u
