// Positivity-preserving scaling of the modal Euler state (Example 11 adds it to the
// limiter, after Zhang and Shu, ref. [zs3]).  One thread per cell, grid-stride; the state
// planes are read once (coalesced across the warp) and only cells that change are
// written back, so the kernel is bound by its FP64 point evaluations.
//
// Per cell, with mean state Ubar admissible (rho > 0, p > 0):
//   eps = min(eps0, rhobar, pbar);
//   the check points S are the L-point Gauss-Lobatto rule (2L-3 >= N) in 1D and, in 2D,
//   (Gauss x Gauss-Lobatto) u (Gauss-Lobatto x Gauss) with the N+1 face Gauss points;
//   1) rho_min = min_S rho_h < eps: the density's modes n >= 1 are scaled by
//      theta1 = (rhobar - eps) / (rhobar - rho_min);
//   2) each point with p(U_q) < eps gives the t in [0,1] with p((1-t) Ubar + t U_q) = eps,
//      the root of A t^2 + B t + C = 0 (p times the positive density along the segment),
//      taken 1e-12 (relative) below the exact root so that rounding cannot leave p below
//      eps near vacuum; theta2 = min t scales the modes n >= 1 of every variable.
// A cell whose mean is not admissible is left as it is and counted.
#include "dg_shared.cuh"

namespace dg {

constexpr int kPpMaxPts = 24;  // 2D P3: 2 x 4 x 3

struct PpTab {
  double phi[kPpMaxPts][10];  // basis values [point][mode]
  double c0, gm1, eps0;
};

template <int V>
__device__ __forceinline__ double pp_pressure(const double* q, double gm1) {
  double k = q[1] * q[1];
  if (V == 4) k += q[2] * q[2];
  return gm1 * (q[V - 1] - 0.5 * k / q[0]);
}

template <int V>
__device__ __forceinline__ double pp_root(const double* ub, const double* uq, double eps, double gm1) {
  double D[V];
#pragma unroll
  for (int v = 0; v < V; ++v) D[v] = uq[v] - ub[v];
  double dm2 = D[1] * D[1], mdm = ub[1] * D[1], m2 = ub[1] * ub[1];
  if (V == 4) {
    dm2 += D[2] * D[2];
    mdm += ub[2] * D[2];
    m2 += ub[2] * ub[2];
  }
  const double A = gm1 * (D[V - 1] * D[0] - 0.5 * dm2);
  const double B = gm1 * (ub[V - 1] * D[0] + ub[0] * D[V - 1] - mdm) - eps * D[0];
  const double C = gm1 * (ub[V - 1] * ub[0] - 0.5 * m2) - eps * ub[0];
  double t;
  if (A == 0.0) {
    t = -C / B;
  } else {
    const double disc = B * B - 4.0 * A * C;
    const double sq = sqrt(disc > 0.0 ? disc : 0.0);
    const double q = -0.5 * (B + (B >= 0.0 ? sq : -sq));
    const double r1 = q / A, r2 = C / q;
    t = (r2 >= 0.0 && r2 <= 1.0) ? r2 : r1;
  }
  t *= 1.0 - 1e-12;
  return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
}

// counts[0] += cells changed, counts[1] += cells whose mean is not admissible
template <int DIM, int N>
__global__ void __launch_bounds__(128) k_positivity(double* __restrict__ U, long long ctot, long long ncell,
                                                    PpTab tb, unsigned long long* __restrict__ counts) {
  constexpr int V = DIM == 1 ? 3 : 4, NP = np_of(DIM, N);
  constexpr int L = N == 1 ? 2 : 3;
  constexpr int NPT = DIM == 1 ? L : 2 * (N + 1) * L;
  unsigned int n_changed = 0, n_bad = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    double u[V][NP];
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int k = 0; k < NP; ++k) u[v][k] = U[(long long)(v * NP + k) * ctot + c];
    double ub[V];
#pragma unroll
    for (int v = 0; v < V; ++v) ub[v] = u[v][0] * tb.c0;
    const double pb = pp_pressure<V>(ub, tb.gm1);
    if (!(ub[0] > 0.0) || !(pb > 0.0)) {
      ++n_bad;
      continue;
    }
    double eps = tb.eps0;
    if (ub[0] < eps) eps = ub[0];
    if (pb < eps) eps = pb;
    bool touched = false;
    double rmin = ub[0];
#pragma unroll 1
    for (int q = 0; q < NPT; ++q) {
      double r = 0.0;
#pragma unroll
      for (int k = 0; k < NP; ++k) r = fma(u[0][k], tb.phi[q][k], r);
      if (r < rmin) rmin = r;
    }
    if (rmin < eps) {
      const double th1 = (ub[0] - eps) / (ub[0] - rmin);
#pragma unroll
      for (int k = 1; k < NP; ++k) u[0][k] *= th1;
      touched = true;
    }
    double th2 = 1.0;
#pragma unroll 1
    for (int q = 0; q < NPT; ++q) {
      double uq[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) s = fma(u[v][k], tb.phi[q][k], s);
        uq[v] = s;
      }
      if (pp_pressure<V>(uq, tb.gm1) < eps) {
        const double t = pp_root<V>(ub, uq, eps, tb.gm1);
        if (t < th2) th2 = t;
      }
    }
    if (th2 < 1.0) {
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int k = 1; k < NP; ++k) u[v][k] *= th2;
      touched = true;
    }
    if (touched) {
      ++n_changed;
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int k = 1; k < NP; ++k) U[(long long)(v * NP + k) * ctot + c] = u[v][k];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_changed += __shfl_down_sync(0xffffffffu, n_changed, o);
    n_bad += __shfl_down_sync(0xffffffffu, n_bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (n_changed) atomicAdd(counts, (unsigned long long)n_changed);
    if (n_bad) atomicAdd(counts + 1, (unsigned long long)n_bad);
  }
}

// Largest |v_d| + c over the check points of every cell, per instance and direction:
// out[2 * inst + d] (non-negative doubles, zeroed by the caller).  Points without a real
// sound speed are skipped (a NaN never wins the comparison).
template <int DIM, int N>
__global__ void __launch_bounds__(128) k_speed_points(const double* __restrict__ U, long long ctot, long long ncell,
                                                      const int* __restrict__ cell_inst, PpTab tb, double gam,
                                                      double* __restrict__ out) {
  constexpr int V = DIM == 1 ? 3 : 4, NP = np_of(DIM, N);
  constexpr int L = N == 1 ? 2 : 3;
  constexpr int NPT = DIM == 1 ? L : 2 * (N + 1) * L;
  for (long long base = blockIdx.x * (long long)blockDim.x; base < ncell; base += (long long)gridDim.x * blockDim.x) {
    const long long c = base + threadIdx.x;
    double sm[2] = {0.0, 0.0};
    int inst = -1;
    if (c < ncell) {
      inst = cell_inst[c];
      double u[V][NP];
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int k = 0; k < NP; ++k) u[v][k] = U[(long long)(v * NP + k) * ctot + c];
#pragma unroll 1
      for (int q = 0; q < NPT; ++q) {
        double w[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < NP; ++k) s = fma(u[v][k], tb.phi[q][k], s);
          w[v] = s;
        }
        const double rho = w[0], vx = w[1] / rho, vy = DIM == 2 ? w[2] / rho : 0.0;
        const double p = tb.gm1 * (w[V - 1] - 0.5 * rho * (vx * vx + vy * vy));
        const double cs = sqrt(gam * p / rho);
        const double sx = fabs(vx) + cs, sy = fabs(vy) + cs;
        if (sx > sm[0]) sm[0] = sx;
        if (DIM == 2 && sy > sm[1]) sm[1] = sy;
      }
    }
    // one atomic per warp when the whole warp lies in one instance
    const int i0 = __shfl_sync(0xffffffffu, inst, 0);
    const bool same = __all_sync(0xffffffffu, inst == i0 || inst < 0);
    if (same) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        double m = sm[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && i0 >= 0) atomic_max_nonneg(out + 2 * i0 + d, m);
      }
    } else if (inst >= 0) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) atomic_max_nonneg(out + 2 * inst + d, sm[d]);
    }
  }
}

void launch_speed_points(int dim, int N, cudaStream_t st, const double* U, long long ctot, long long ncell,
                         const int* cell_inst, const double* phi, int npt, double gam, double* out, int nblocks) {
  PpTab tb{};
  const int NP = np_of(dim, N);
  for (int q = 0; q < npt && q < kPpMaxPts; ++q)
    for (int k = 0; k < NP; ++k) tb.phi[q][k] = phi[q * NP + k];
  tb.gm1 = gam - 1.0;
#define DG_SP(D, NN) k_speed_points<D, NN><<<nblocks, 128, 0, st>>>(U, ctot, ncell, cell_inst, tb, gam, out)
  if (dim == 1) {
    if (N == 1) DG_SP(1, 1);
    else if (N == 2) DG_SP(1, 2);
    else DG_SP(1, 3);
  } else {
    if (N == 1) DG_SP(2, 1);
    else if (N == 2) DG_SP(2, 2);
    else DG_SP(2, 3);
  }
#undef DG_SP
}

// phi: [npt][NP] basis values at the check points (host-built from the library tables)
void launch_positivity(int dim, int N, cudaStream_t st, double* U, long long ctot, long long ncell,
                       const double* phi, int npt, double c0, double gam, double eps0,
                       unsigned long long* counts, int nblocks) {
  PpTab tb{};
  const int NP = np_of(dim, N);
  for (int q = 0; q < npt && q < kPpMaxPts; ++q)
    for (int k = 0; k < NP; ++k) tb.phi[q][k] = phi[q * NP + k];
  tb.c0 = c0;
  tb.gm1 = gam - 1.0;
  tb.eps0 = eps0;
#define DG_PP(D, NN) k_positivity<D, NN><<<nblocks, 128, 0, st>>>(U, ctot, ncell, tb, counts)
  if (dim == 1) {
    if (N == 1) DG_PP(1, 1);
    else if (N == 2) DG_PP(1, 2);
    else DG_PP(1, 3);
  } else {
    if (N == 1) DG_PP(2, 1);
    else if (N == 2) DG_PP(2, 2);
    else DG_PP(2, 3);
  }
#undef DG_PP
}

}  // namespace dg
