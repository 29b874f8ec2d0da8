// Shared device-side definitions of the GB300 DG library: mode ordering, mesh/instance
// descriptors, physical fluxes (Burgers and ideal-gas Euler, Eqs. (19)-(21), (23)) and the
// local Lax-Friedrichs flux (Sec. 2).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dg {

// ----------------------------------------------------------------------------- layout
// 2D total-degree modes ordered by degree d = a + b, then b ascending.
__host__ __device__ constexpr int np_of(int dim, int N) { return dim == 1 ? N + 1 : (N + 1) * (N + 2) / 2; }
__host__ __device__ constexpr int nv_of(int dim, int pde) { return pde == 0 ? 1 : (dim == 1 ? 3 : 4); }
__host__ __device__ constexpr int mode_b(int m) {
  int d = 0, start = 0;
  while (m >= start + d + 1) { start += d + 1; ++d; }
  return m - start;
}
__host__ __device__ constexpr int mode_a(int m) {
  int d = 0, start = 0;
  while (m >= start + d + 1) { start += d + 1; ++d; }
  return d - (m - start);
}
// index of mode (a, b)
__host__ __device__ constexpr int mode_idx(int a, int b) { return (a + b) * (a + b + 1) / 2 + b; }

// One mesh instance of a batch.  Cells of all instances are concatenated; the device
// state is stored as planes [var][mode][cell] of length `ctot` (total padded cells).
struct Inst {
  int nx, ny;
  long long off;  // first cell of the instance in the concatenated cell index
  double hx, hy;  // cell widths
  double xL, yL;  // lower-left corner
  double dt;      // per-instance time step (dg_set_dt)
  long long fx, fy;  // first x face / y face of the instance in the 2D face planes
};

// A tile of the 2D stage / flag kernels: instance and lower-left cell of the tile.  The
// face tiles of the split stage use `pad` for the face direction (0: x faces, 1: y faces).
struct Tile {
  int inst, x0, y0, pad;
};

// ----------------------------------------------------------------------------- arithmetic
// x with its sign flipped when f (mirror images of ghost cells): an exclusive or on the
// bit pattern, which runs on the integer pipe instead of taking an FP64 instruction.
__device__ __forceinline__ double neg_if(double x, bool f) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)((unsigned long long)f << 63));
}

// Reciprocal and square root of the 2D Euler stage fluxes and of the WENO weights, from
// the hardware's ~20-bit approximations refined by one step of Householder's third-order
// iteration: with e the relative error of the seed y, 1/x = y / (1 - e) and
// 1/sqrt(x) = y (1 - e)^(-1/2), and the first three terms of those series,
// y (1 + e + e^2) and y (1 + e/2 + 3 e^2 / 8), leave an error of order e^3 ~ 1e-18: within
// one or two ulps of the IEEE-rounded results, at about 70 % of their FP64 instruction
// cost.  Arguments whose magnitude lies outside [2^-1022, 2^1022) (zero, subnormal, huge,
// inf, NaN) take the IEEE operation, and so does a non-positive square-root argument: every
// special case gives the IEEE result.
__device__ __forceinline__ double rcp_d(double x) {
  const unsigned long long ab = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  if (ab - 0x0010000000000000ull >= 0x7fc0000000000000ull) return 1.0 / x;  // |x| outside [2^-1022, 2^1022)
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);  // x y = 1 - e
  return fma(y, fma(e, e, e), y);    // y (1 + e + e^2)
}
__device__ __forceinline__ double sqrt_d(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  if (b - 0x0010000000000000ull >= 0x7fe0000000000000ull) return sqrt(x);  // not a positive normal
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x * y, y, 1.0);               // x y^2 = 1 - e
  y = fma(y, e * fma(0.375, e, 0.5), y);              // y (1 + e/2 + 3 e^2 / 8)
  return x * y;
}

// ----------------------------------------------------------------------------- physics
// Euler helpers work on conserved variables; gm1 = gamma - 1.
template <int DIM, int PDE>
struct Phys;

template <int DIM>
struct Phys<DIM, 0> {  // Burgers, f = g = u^2 / 2
  static constexpr int V = 1;
  // flux in direction d and the largest |f'(u)|
  __device__ __forceinline__ static void flux(int, const double* u, double* f, double& a, double, double) {
    f[0] = 0.5 * u[0] * u[0];
    a = fabs(u[0]);
  }
};

template <>
struct Phys<1, 1> {  // 1D Euler (rho, m, E)
  static constexpr int V = 3;
  __device__ __forceinline__ static void flux(int, const double* u, double* f, double& a, double gam,
                                              double gm1) {
    double r = 1.0 / u[0];
    double vel = u[1] * r;
    double p = gm1 * (u[2] - 0.5 * u[1] * vel);
    f[0] = u[1];
    f[1] = fma(u[1], vel, p);
    f[2] = (u[2] + p) * vel;
    a = fabs(vel) + sqrt(gam * p * r);
  }
};

template <>
struct Phys<2, 1> {  // 2D Euler (rho, mx, my, E)
  static constexpr int V = 4;
  __device__ __forceinline__ static void flux(int dir, const double* u, double* f, double& a, double gam,
                                              double gm1) {
    double r = rcp_d(u[0]);
    double vx = u[1] * r, vy = u[2] * r;
    double p = fma(-0.5 * gm1, fma(u[1], vx, u[2] * vy), gm1 * u[3]);  // (gamma-1)(E - rho |v|^2 / 2)
    double vn = dir == 0 ? vx : vy;
    f[0] = dir == 0 ? u[1] : u[2];
    f[1] = dir == 0 ? fma(u[1], vx, p) : u[1] * vy;
    f[2] = dir == 0 ? u[2] * vx : fma(u[2], vy, p);
    f[3] = (u[3] + p) * vn;
    a = fabs(vn) + sqrt_d(gam * p * r);
  }
};

// Volume fluxes of both directions at one point, pre-scaled by sx = 2/hx and sy = 2/hy.
template <int DIM, int PDE>
__device__ __forceinline__ void vol_flux2(const double* u, double* f, double* g, double sx, double sy,
                                          double gm1) {
  if constexpr (PDE == 0) {
    double h = 0.5 * u[0] * u[0];
    f[0] = h * sx;
    g[0] = h * sy;
  } else {
    double r = 1.0 / u[0];
    double vx = u[1] * r, vy = u[2] * r;
    double p = gm1 * (u[3] - 0.5 * fma(u[1], vx, u[2] * vy));
    double vxs = vx * sx, vys = vy * sy;
    double ep = u[3] + p;
    f[0] = u[1] * sx;
    f[1] = fma(u[1], vxs, p * sx);
    f[2] = u[2] * vxs;
    f[3] = ep * vxs;
    g[0] = u[2] * sy;
    g[1] = u[1] * vys;
    g[2] = fma(u[2], vys, p * sy);
    g[3] = ep * vys;
  }
}

// Local Lax-Friedrichs flux times 2/h, written as (1/h) [(fL + fR) - alpha (uR - uL)]
// with alpha = max of the two spectral radii (Sec. 2 names Lax-Friedrichs; the local
// alpha is the reading used throughout).
template <int DIM, int PDE>
__device__ __forceinline__ void llf(int dir, const double* uL, const double* uR, double* fs, double inv_h,
                                    double gam, double gm1) {
  constexpr int V = Phys<DIM, PDE>::V;
  double fL[V], fR[V], aL, aR;
  Phys<DIM, PDE>::flux(dir, uL, fL, aL, gam, gm1);
  Phys<DIM, PDE>::flux(dir, uR, fR, aR, gam, gm1);
  // fmax drops a NaN operand; a face state without a real sound speed (negative density
  // or pressure at a quadrature point) must instead make alpha, and the step, non-finite.
  // The NaN test runs on the bit patterns (integer pipe).
  constexpr unsigned long long kAbs = 0x7fffffffffffffffull, kInf = 0x7ff0000000000000ull;
  const bool nan_lr = ((__double_as_longlong(aL) & kAbs) > kInf) | ((__double_as_longlong(aR) & kAbs) > kInf);
  const double a = nan_lr ? aL + aR : fmax(aL, aR);
#pragma unroll
  for (int v = 0; v < V; ++v) fs[v] = inv_h * fma(-a, uR[v] - uL[v], fL[v] + fR[v]);
}

// The same flux without the 1/h factor: fs = (fL + fR) - alpha (uR - uL) = 2 f*.
template <int DIM, int PDE>
__device__ __forceinline__ void llf_sum(int dir, const double* uL, const double* uR, double* fs, double gam,
                                        double gm1) {
  constexpr int V = Phys<DIM, PDE>::V;
  double fL[V], fR[V], aL, aR;
  Phys<DIM, PDE>::flux(dir, uL, fL, aL, gam, gm1);
  Phys<DIM, PDE>::flux(dir, uR, fR, aR, gam, gm1);
  constexpr unsigned long long kAbs = 0x7fffffffffffffffull, kInf = 0x7ff0000000000000ull;
  const bool nan_lr = ((__double_as_longlong(aL) & kAbs) > kInf) | ((__double_as_longlong(aR) & kAbs) > kInf);
  const double a = nan_lr ? aL + aR : fmax(aL, aR);
#pragma unroll
  for (int v = 0; v < V; ++v) fs[v] = fma(-a, uR[v] - uL[v], fL[v] + fR[v]);
}

}  // namespace dg
