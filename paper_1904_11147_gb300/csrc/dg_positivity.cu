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
// Most cells need no scaling: an FP32 evaluation of the check points with error margins
// (below) proves theta1 = theta2 = 1 for them, and only the others take the FP64 path.
#include "dg_convert.cuh"
#include "dg_shared.cuh"

namespace dg {

template <typename T>
struct PpTabT {
  T pg[4][4];  // psi_n at the N+1 Gauss points [i][n]
  T pl[3][4];  // psi_n at the L Gauss-Lobatto points [j][n] (-1, 0, 1; or -1, 1 for N = 1)
};
struct PpTab : PpTabT<double> {
  double c0, gm1, eps0;
  PpTabT<float> f;  // the same tables in FP32 for the screen
  float p1[4];      // psi_n(1) = max |psi_n| on [-1, 1]
};

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// Calls f(w) with the V point values of the modes u[0..V-1] at every check point: in 1D
// the Gauss-Lobatto points; in 2D (Gauss x Gauss-Lobatto) then (Gauss-Lobatto x Gauss),
// by sum factorisation over the Gauss coordinate.  Both point sets are symmetric about 0
// and psi_n has the parity of n, so even and odd parts are summed once per pair of points
// (psi_n(0) = 0 for odd n).  The order of the points is not part of the result (minima).
template <int DIM, int N, int V, typename T, class F>
__device__ __forceinline__ void for_points(const T (*u)[np_of(DIM, N)], const PpTabT<T>& tb, F&& f) {
  constexpr int L = N == 1 ? 2 : 3, NP = np_of(DIM, N);
  if constexpr (DIM == 1) {
#pragma unroll
    for (int j = 0; j < L; ++j) {
      T w[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        T s = 0;
#pragma unroll
        for (int k = 0; k < NP; ++k) s = fma_t(u[v][k], tb.pl[j][k], s);
        w[v] = s;
      }
      f(w);
    }
  } else {
    // values of sum_c t_c psi_c(l) at the Gauss-Lobatto points l = -1, (0,) 1
    auto lobatto = [&](const T (&t)[V][N + 1]) {
      T wp[V], wm[V], w0[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        T ev = t[v][0] * tb.pl[L - 1][0], od = t[v][1] * tb.pl[L - 1][1];
#pragma unroll
        for (int c = 2; c <= N; ++c) {
          if (c & 1) od = fma_t(t[v][c], tb.pl[L - 1][c], od);
          else ev = fma_t(t[v][c], tb.pl[L - 1][c], ev);
        }
        wp[v] = ev + od;
        wm[v] = ev - od;
        if (L == 3) {
          T z = t[v][0] * tb.pl[1][0];
#pragma unroll
          for (int c = 2; c <= N; c += 2) z = fma_t(t[v][c], tb.pl[1][c], z);
          w0[v] = z;
        }
      }
      f(wm);
      if (L == 3) f(w0);
      f(wp);
    };
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      // pass 0: t_b = sum_a U_ab psi_a(g_i), point (g_i, l_j) = sum_b t_b psi_b(l_j)
      // pass 1: t_a = sum_b U_ab psi_b(g_i), point (l_j, g_i) = sum_a t_a psi_a(l_j)
      // Gauss points in symmetric pairs; for N = 3 one at a time (fewer registers)
      constexpr bool kPair = N < 3;
#pragma unroll 1
      for (int i = 0; i < (kPair ? (N + 2) / 2 : N + 1); ++i) {
        const bool mid = !kPair || ((N % 2 == 0) && i == N / 2);  // one point (0 for N even)
        T tp[V][N + 1], tm[V][N + 1];
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int c = 0; c <= N; ++c) {
            T ev = 0, od = 0;
#pragma unroll
            for (int d = 0; d <= N - c; ++d) {
              const int m = pass == 0 ? mode_idx(d, c) : mode_idx(c, d);
              if (d & 1) {
                if (!kPair) ev = fma_t(u[v][m], tb.pg[i][d], ev);
                else if (!mid) od = d == 1 ? u[v][m] * tb.pg[i][d] : fma_t(u[v][m], tb.pg[i][d], od);
              } else {
                ev = d == 0 ? u[v][m] * tb.pg[i][d] : fma_t(u[v][m], tb.pg[i][d], ev);
              }
            }
            const bool has_od = !mid && c < N;
            tp[v][c] = has_od ? ev + od : ev;  // at g_i
            tm[v][c] = has_od ? ev - od : ev;  // at g_{N-i} = -g_i
          }
        lobatto(tp);
        if (!mid) lobatto(tm);
      }
    }
  }
}

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

// True when FP32 arithmetic with error margins proves that no check point of cell c needs
// scaling: rho > eps and rho p > eps rho at every point, i.e. theta1 = theta2 = 1 and the
// FP64 decisions below cannot fire.  With S_v = sum_k |U_vk| max|phi_k| (a bound on |u_v| at
// every point) and delta = 2^-16 (over 16 times the error of truncating the modes to FP32
// and of the FP32 sums), each point value is within delta S_v of the exact one, rho p
// (times gamma - 1, minus eps rho) within 4 delta B, B = (gamma-1)(S_E S_rho + |S_m|^2) +
// eps S_rho.  The caller requires rhobar, pbar >= 1e-10 and the bounds stay below 1e15, so
// the margins are normal FP32 numbers; a NaN or infinity anywhere fails the test.
template <int DIM, int N>
__device__ __forceinline__ bool screen_unchanged(const double* __restrict__ U, long long ctot, long long c,
                                                 const PpTab& tb, float eps) {
  constexpr int V = DIM == 1 ? 3 : 4, NP = np_of(DIM, N);
  constexpr float kDelta = 1.0f / 65536.0f;
  float u[V][NP], S[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      u[v][k] = d2f_trunc(U[(long long)(v * NP + k) * ctot + c]);
      const float phi = DIM == 1 ? tb.p1[k] : tb.p1[mode_a(k)] * tb.p1[mode_b(k)];
      s = fmaf(fabsf(u[v][k]), phi, s);
    }
    S[v] = s;
  }
  float sm2 = S[1] * S[1];
  if (V == 4) sm2 = fmaf(S[2], S[2], sm2);
  const float gm1 = (float)tb.gm1;
  const float B = fmaf(gm1, fmaf(S[V - 1], S[0], sm2), eps * S[0]);
  if (!(B < 1e30f) || !(S[0] < 1e15f)) return false;
  const float rho_min = fmaf(kDelta, S[0], eps), q_min = 4.0f * kDelta * B;
  bool ok = true;
  for_points<DIM, N, V>(u, tb.f, [&](const float* w) {
    float k2 = w[1] * w[1];
    if (V == 4) k2 = fmaf(w[2], w[2], k2);
    const float q = fmaf(gm1, fmaf(w[V - 1], w[0], -0.5f * k2), -eps * w[0]);
    ok &= (w[0] > rho_min) & (q > q_min);
  });
  return ok;
}

// First pass: lists the cells that the FP32 screen cannot prove unchanged (and those with
// an inadmissible mean, which the second pass counts); warp ballot, one atomic per warp.
template <int DIM, int N>
__global__ void __launch_bounds__(256) k_pp_screen(const double* __restrict__ U, long long ctot, long long ncell,
                                                   PpTab tb, int* __restrict__ list, unsigned int* __restrict__ n_list) {
  constexpr int V = DIM == 1 ? 3 : 4, NP = np_of(DIM, N);
  const int lane = threadIdx.x & 31;
  for (long long base = blockIdx.x * (long long)blockDim.x; base < ncell; base += (long long)gridDim.x * blockDim.x) {
    const long long c = base + threadIdx.x;
    bool keep = false;
    if (c < ncell) {
      double ub[V];
#pragma unroll
      for (int v = 0; v < V; ++v) ub[v] = U[(long long)(v * NP) * ctot + c] * tb.c0;
      const double pb = pp_pressure<V>(ub, tb.gm1);
      if (!(ub[0] > 0.0) || !(pb > 0.0)) {
        keep = true;
      } else {
        double eps = tb.eps0;
        if (ub[0] < eps) eps = ub[0];
        if (pb < eps) eps = pb;
        keep = !(ub[0] >= 1e-10 && pb >= 1e-10 && screen_unchanged<DIM, N>(U, ctot, c, tb, (float)eps));
      }
    }
    const unsigned int bal = __ballot_sync(0xffffffffu, keep);
    unsigned int pos0 = 0;
    if (lane == 0 && bal) pos0 = atomicAdd(n_list, (unsigned)__popc(bal));
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    if (keep) list[pos0 + __popc(bal & ((1u << lane) - 1u))] = (int)c;
  }
}

// Second pass, FP64, over the listed cells.  counts[0] += cells changed, counts[1] += cells
// whose mean is not admissible.  The density pass gives rho_min; the pressure pass
// evaluates every variable of the unscaled state and applies the density factor to the
// density point values (rho' = rhobar + theta1 (rho - rhobar), the point values of the
// scaled modes).
template <int DIM, int N>
__global__ void __launch_bounds__(128) k_positivity(double* __restrict__ U, long long ctot,
                                                    const int* __restrict__ list,
                                                    const unsigned int* __restrict__ n_list, PpTab tb,
                                                    unsigned long long* __restrict__ counts) {
  constexpr int V = DIM == 1 ? 3 : 4, NP = np_of(DIM, N);
  unsigned int n_changed = 0, n_bad = 0;
  const unsigned int nl = *n_list;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
    const long long c = list[i];
    double ub[V];
#pragma unroll
    for (int v = 0; v < V; ++v) ub[v] = U[(long long)(v * NP) * ctot + c] * tb.c0;
    const double pb = pp_pressure<V>(ub, tb.gm1);
    if (!(ub[0] > 0.0) || !(pb > 0.0)) {
      ++n_bad;
      continue;
    }
    double eps = tb.eps0;
    if (ub[0] < eps) eps = ub[0];
    if (pb < eps) eps = pb;
    double u[V][NP];
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int k = 0; k < NP; ++k) u[v][k] = U[(long long)(v * NP + k) * ctot + c];
    // one pass for the density minimum and, assuming theta1 = 1 (the density needs no
    // scaling: the usual case), the pressure factor; with theta1 < 1 a second pass redoes
    // the pressure factor on the scaled density
    double rmin = ub[0], th1 = 1.0, th2 = 1.0;
    auto pressure_point = [&](const double* w) {
      double q[V];
#pragma unroll
      for (int v = 0; v < V; ++v) q[v] = w[v];
      if (th1 < 1.0) q[0] = fma(th1, w[0] - ub[0], ub[0]);
      // p < eps tested as rho p < eps rho (rho >= eps > 0 here): no division per point
      double k2 = q[1] * q[1];
      if (V == 4) k2 = fma(q[2], q[2], k2);
      const double rp = tb.gm1 * fma(q[V - 1], q[0], -0.5 * k2);
      if (rp < eps * q[0]) {
        const double t = pp_root<V>(ub, q, eps, tb.gm1);
        if (t < th2) th2 = t;
      }
    };
    for_points<DIM, N, V>(u, tb, [&](const double* w) {
      if (w[0] < rmin) rmin = w[0];
      pressure_point(w);
    });
    if (rmin < eps) {
      th1 = (ub[0] - eps) / (ub[0] - rmin);
      th2 = 1.0;
      for_points<DIM, N, V>(u, tb, pressure_point);
    }
    if (th1 < 1.0 || th2 < 1.0) {
      ++n_changed;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const double f = v == 0 ? th1 * th2 : th2;
#pragma unroll
        for (int k = 1; k < NP; ++k) U[(long long)(v * NP + k) * ctot + c] = u[v][k] * f;
      }
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

// FP32 bounds of a cell's wave-speed bound max |v_d| + max c over its check points (the
// FP64 value of k_speed_points): lo[d] <= it <= hi[d].  Point values carry the margins of
// screen_unchanged (delta S_v); a point enters hi when its pressure may be >= 0 and lo only
// when it surely is (the FP64 pass skips points without a real sound speed); a point whose
// density may be <= 0 leaves hi unbounded.  The results are widened by 2^-12 (relative),
// far more than the FP32 rounding of the bound formulas.
template <int DIM, int N>
__device__ __forceinline__ void speed_bounds32(const double* __restrict__ U, long long ctot, long long c,
                                               const PpTab& tb, float gam, float (&lo)[2], float (&hi)[2]) {
  constexpr int V = DIM == 1 ? 3 : 4, NP = np_of(DIM, N);
  constexpr float kDelta = 1.0f / 65536.0f;
  const float kInf = __int_as_float(0x7f800000);
  float u[V][NP], S[V];
  bool unbounded = false;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    float sv = 0.f;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      u[v][k] = d2f_trunc(U[(long long)(v * NP + k) * ctot + c]);
      const float phi = DIM == 1 ? tb.p1[k] : tb.p1[mode_a(k)] * tb.p1[mode_b(k)];
      sv = fmaf(fabsf(u[v][k]), phi, sv);
    }
    S[v] = kDelta * sv;
    unbounded |= !(sv < 1e15f);
  }
  const float gm1 = gam - 1.0f;
  float vlo[2] = {0.f, 0.f}, vhi[2] = {0.f, 0.f}, c2lo = 0.f, c2hi = 0.f;
  for_points<DIM, N, V>(u, tb.f, [&](const float* w) {
    const float rl = w[0] - S[0], ru = w[0] + S[0];
    if (!(rl > 0.f)) {
      unbounded = true;
      return;
    }
    float ml[2] = {0.f, 0.f}, mu[2] = {0.f, 0.f};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      mu[d] = fabsf(w[1 + d]) + S[1 + d];
      ml[d] = fmaxf(fabsf(w[1 + d]) - S[1 + d], 0.f);
    }
    const float m2l = fmaf(ml[1], ml[1], ml[0] * ml[0]), m2u = fmaf(mu[1], mu[1], mu[0] * mu[0]);
    const float pu = gm1 * ((w[V - 1] + S[V - 1]) - 0.5f * m2l / ru);
    const float pl = gm1 * ((w[V - 1] - S[V - 1]) - 0.5f * m2u / rl);
    if (pu >= 0.f) {
      c2hi = fmaxf(c2hi, gam * pu / rl);
#pragma unroll
      for (int d = 0; d < DIM; ++d) vhi[d] = fmaxf(vhi[d], mu[d] / rl);
    }
    if (pl > 0.f) {
      c2lo = fmaxf(c2lo, gam * pl / ru);
#pragma unroll
      for (int d = 0; d < DIM; ++d) vlo[d] = fmaxf(vlo[d], ml[d] / ru);
    }
  });
  const float cl = sqrtf(c2lo), ch = sqrtf(c2hi);
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    lo[d] = (vlo[d] + cl) * (1.0f - 1.0f / 4096.0f);
    hi[d] = unbounded ? kInf : (vhi[d] + ch) * (1.0f + 1.0f / 4096.0f);
  }
}

// Pass 1: per instance and direction the largest lower bound over its cells (the float
// bits of non-negative values order like unsigned integers); lb zeroed by the caller.
template <int DIM, int N>
__global__ void __launch_bounds__(256) k_speed_lb(const double* __restrict__ U, long long ctot, long long ncell,
                                                  const int* __restrict__ cell_inst, PpTab tb, float gam,
                                                  unsigned int* __restrict__ lb) {
  for (long long base = blockIdx.x * (long long)blockDim.x; base < ncell; base += (long long)gridDim.x * blockDim.x) {
    const long long c = base + threadIdx.x;
    float lo[2] = {0.f, 0.f}, hi[2];
    int inst = -1;
    if (c < ncell) {
      inst = cell_inst[c];
      speed_bounds32<DIM, N>(U, ctot, c, tb, gam, lo, hi);
    }
    const int i0 = __shfl_sync(0xffffffffu, inst, 0);
    const bool same = __all_sync(0xffffffffu, inst == i0 || inst < 0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      if (same) {
        float m = lo[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && i0 >= 0) atomicMax(lb + 2 * i0 + d, __float_as_uint(m));
      } else if (inst >= 0) {
        atomicMax(lb + 2 * inst + d, __float_as_uint(lo[d]));
      }
    }
  }
}

// Pass 2: lists the cells whose upper bound reaches their instance's largest lower bound in
// some direction -- only these can hold the instance's maximum.
template <int DIM, int N>
__global__ void __launch_bounds__(256) k_speed_screen(const double* __restrict__ U, long long ctot, long long ncell,
                                                      const int* __restrict__ cell_inst, PpTab tb, float gam,
                                                      const unsigned int* __restrict__ lb, int* __restrict__ list,
                                                      unsigned int* __restrict__ n_list) {
  const int lane = threadIdx.x & 31;
  for (long long base = blockIdx.x * (long long)blockDim.x; base < ncell; base += (long long)gridDim.x * blockDim.x) {
    const long long c = base + threadIdx.x;
    bool keep = false;
    if (c < ncell) {
      const int inst = cell_inst[c];
      float lo[2], hi[2];
      speed_bounds32<DIM, N>(U, ctot, c, tb, gam, lo, hi);
#pragma unroll
      for (int d = 0; d < DIM; ++d) keep |= !(hi[d] < __uint_as_float(lb[2 * inst + d]));
    }
    const unsigned int bal = __ballot_sync(0xffffffffu, keep);
    unsigned int pos0 = 0;
    if (lane == 0 && bal) pos0 = atomicAdd(n_list, (unsigned)__popc(bal));
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    if (keep) list[pos0 + __popc(bal & ((1u << lane) - 1u))] = (int)c;
  }
}

// Pass 3, FP64, over the listed cells: out[2 * inst + d] = max of max |v_d| + max c over the
// check points (one square root per cell), the non-negative doubles zeroed by the caller.
// Points without a real sound speed are skipped (a NaN never wins the comparison).
template <int DIM, int N>
__global__ void __launch_bounds__(128) k_speed_points(const double* __restrict__ U, long long ctot,
                                                      const int* __restrict__ list,
                                                      const unsigned int* __restrict__ n_list,
                                                      const int* __restrict__ cell_inst, PpTab tb, double gam,
                                                      double* __restrict__ out) {
  constexpr int V = DIM == 1 ? 3 : 4, NP = np_of(DIM, N);
  const unsigned int nl = *n_list;
  for (unsigned int base = blockIdx.x * blockDim.x; base < nl; base += gridDim.x * blockDim.x) {
    const unsigned int i = base + threadIdx.x;
    double sm[2] = {0.0, 0.0};
    int inst = -1;
    if (i < nl) {
      const long long c = list[i];
      inst = cell_inst[c];
      double u[V][NP];
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int k = 0; k < NP; ++k) u[v][k] = U[(long long)(v * NP + k) * ctot + c];
      double vmax[2] = {0.0, 0.0}, c2max = 0.0;
      for_points<DIM, N, V>(u, tb, [&](const double* w) {
        const double r = rcp_d(w[0]), vx = w[1] * r, vy = DIM == 2 ? w[2] * r : 0.0;
        const double p = tb.gm1 * (w[V - 1] - 0.5 * w[0] * (vx * vx + vy * vy));
        const double c2 = gam * p * r;
        if (c2 >= 0.0) {  // a real sound speed (false for NaN)
          if (c2 > c2max) c2max = c2;
          if (fabs(vx) > vmax[0]) vmax[0] = fabs(vx);
          if (DIM == 2 && fabs(vy) > vmax[1]) vmax[1] = fabs(vy);
        }
      });
      const double cs = sqrt(c2max);
      sm[0] = vmax[0] + cs;
      if (DIM == 2) sm[1] = vmax[1] + cs;
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

static PpTab make_tab(int N, const double* pg, const double* pl, double c0, double gam, double eps0) {
  PpTab tb{};
  const int L = N == 1 ? 2 : 3;
  for (int i = 0; i <= N; ++i)
    for (int k = 0; k <= N; ++k) {
      tb.pg[i][k] = pg[i * (N + 1) + k];
      tb.f.pg[i][k] = (float)tb.pg[i][k];
    }
  for (int j = 0; j < L; ++j)
    for (int k = 0; k <= N; ++k) {
      tb.pl[j][k] = pl[j * (N + 1) + k];
      tb.f.pl[j][k] = (float)tb.pl[j][k];
    }
  // psi_n(1) (the last Gauss-Lobatto point), rounded up so that S_v stays a bound
  for (int k = 0; k <= N; ++k) tb.p1[k] = nextafterf((float)std::fabs(tb.pl[L - 1][k]), 1e30f);
  tb.c0 = c0;
  tb.gm1 = gam - 1.0;
  tb.eps0 = eps0;
  return tb;
}

// pg: psi_n at the Gauss points [(N+1)][(N+1)], pl: at the Gauss-Lobatto points [L][(N+1)];
// lb: [2 n_inst] scratch, list: int[ncell] scratch, n_list: its length (both zeroed here);
// out [2 n_inst] zeroed by the caller
void launch_speed_points(int dim, int N, cudaStream_t st, const double* U, long long ctot, long long ncell,
                         const int* cell_inst, const double* pg, const double* pl, double gam, double* out,
                         unsigned int* lb, int n_inst, int* list, unsigned int* n_list, int nblocks) {
  const PpTab tb = make_tab(N, pg, pl, 0.0, gam, 0.0);
  cudaMemsetAsync(lb, 0, sizeof(unsigned int) * 2 * n_inst, st);
  cudaMemsetAsync(n_list, 0, sizeof(unsigned int), st);
  const long long want = (ncell + 255) / 256;
  const int nb1 = (int)(want < 4LL * nblocks ? want : 4LL * nblocks);
  const float g32 = (float)gam;
#define DG_SP(D, NN)                                                                                        \
  do {                                                                                                      \
    k_speed_lb<D, NN><<<nb1, 256, 0, st>>>(U, ctot, ncell, cell_inst, tb, g32, lb);                        \
    k_speed_screen<D, NN><<<nb1, 256, 0, st>>>(U, ctot, ncell, cell_inst, tb, g32, lb, list, n_list);      \
    k_speed_points<D, NN><<<nblocks, 128, 0, st>>>(U, ctot, list, n_list, cell_inst, tb, gam, out);        \
  } while (0)
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

// list: int[ncell] scratch, n_list: its length (zeroed here)
void launch_positivity(int dim, int N, cudaStream_t st, double* U, long long ctot, long long ncell,
                       const double* pg, const double* pl, double c0, double gam, double eps0,
                       int* list, unsigned int* n_list, unsigned long long* counts, int nblocks) {
  const PpTab tb = make_tab(N, pg, pl, c0, gam, eps0);
  cudaMemsetAsync(n_list, 0, sizeof(unsigned int), st);
  const long long want = (ncell + 255) / 256;
  const int nb1 = (int)(want < 4LL * nblocks ? want : 4LL * nblocks);
#define DG_PP(D, NN)                                                                                  \
  do {                                                                                                \
    k_pp_screen<D, NN><<<nb1, 256, 0, st>>>(U, ctot, ncell, tb, list, n_list);                        \
    k_positivity<D, NN><<<nblocks, 128, 0, st>>>(U, ctot, list, n_list, tb, counts);                  \
  } while (0)
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
