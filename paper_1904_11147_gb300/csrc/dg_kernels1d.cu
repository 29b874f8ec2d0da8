// 1D kernels (P^N, N = 1..3; Burgers V = 1, Euler V = 3).  The 1D workloads are small
// (hundreds to thousands of cells), so these kernels favour simplicity: one thread per
// cell, the two face fluxes of a cell evaluated by that cell.
#include "dg_ic.cuh"
#include "dg_shared.cuh"
#include "tables.h"

namespace dg {
namespace k1 {

constexpr int kBlock = 256;  // cells per tile

template <int N>
struct Lay {
  static constexpr int Q = N + 1, N1 = N + 1, NS = 2 * N + 1, NG = (N == 1 ? 2 : 4);
  static constexpr int SIZE = 2 * Q * N1 + 3 * N1 + NS * N1 + N1 * NG * N1 + NG * N1 + N1 * N1 * N1 + NG * N1 +
                              NG + 2 * NG * N1 + 3 * NG + 3 * 8 + 8 * N1;
};
__host__ __device__ constexpr int base_of(int N) {
  return N == 1 ? 0 : (N == 2 ? Lay<1>::SIZE : Lay<1>::SIZE + Lay<2>::SIZE);
}
template <int N>
struct Off {
  using L = Lay<N>;
  static constexpr int Q = L::Q, N1 = L::N1, NS = L::NS, NG = L::NG;
  static constexpr int P = base_of(N);          // [Q][N1] psi_n(x_q)
  static constexpr int D = P + Q * N1;          // [Q][N1] w_q psi_n'(x_q)
  static constexpr int P1 = D + Q * N1;         // psi_n(1)
  static constexpr int M1 = P1 + N1;            // psi_n(-1)
  static constexpr int P0 = M1 + N1;            // psi_n(0)
  static constexpr int SA = P0 + N1;            // [NS][N1]
  static constexpr int WC = SA + NS * N1;       // [N1][NG][N1]
  static constexpr int GAM = WC + N1 * NG * N1; // [NG][N1]
  static constexpr int BB = GAM + NG * N1;      // [N1][N1][N1]
  static constexpr int PG = BB + N1 * N1 * N1;  // [NG][N1]
  static constexpr int WG = PG + NG * N1;       // [NG]
  static constexpr int GPN = WG + NG;
  static constexpr int GMN = GPN + NG * N1;
  static constexpr int SGP = GMN + NG * N1;
  static constexpr int SGM = SGP + NG;
  static constexpr int NEG = SGM + NG;
  static constexpr int PX = NEG + NG;
  static constexpr int PW = PX + 8;
  static constexpr int PQP = PW + 8;
  static constexpr int PP = PQP + 8;
  static constexpr int END = PP + 8 * N1;
};
static_assert(Off<3>::END == Lay<1>::SIZE + Lay<2>::SIZE + Lay<3>::SIZE, "table layout");
constexpr int kTabSize = Off<3>::END;

__constant__ double c_tab[kTabSize];
#define T(x) c_tab[(x)]

template <int N>
void pack(const dgt::Tabs& t, double* h) {
  using O = Off<N>;
  constexpr int Q = O::Q, N1 = O::N1, NS = O::NS, NG = O::NG;
  for (int q = 0; q < Q; ++q)
    for (int n = 0; n < N1; ++n) {
      h[O::P + q * N1 + n] = t.psi_q[q][n];
      h[O::D + q * N1 + n] = t.gw[q] * t.dpsi_q[q][n];
    }
  for (int n = 0; n < N1; ++n) {
    h[O::P1 + n] = t.psi_p1[n];
    h[O::M1 + n] = t.psi_m1[n];
    h[O::P0 + n] = t.psi_0[n];
  }
  for (int k = 0; k < NS; ++k)
    for (int n = 0; n < N1; ++n) h[O::SA + k * N1 + n] = t.SA[k][n];
  for (int i = 0; i < N1; ++i)
    for (int g = 0; g < NG; ++g)
      for (int k = 0; k < N1; ++k) h[O::WC + (i * NG + g) * N1 + k] = t.C[i][g][k];
  for (int g = 0; g < NG; ++g)
    for (int i = 0; i < N1; ++i) {
      h[O::GAM + g * N1 + i] = t.gam[g][i];
      h[O::GPN + g * N1 + i] = t.gpn[g][i];
      h[O::GMN + g * N1 + i] = t.gmn[g][i];
    }
  for (int i = 0; i < N1; ++i)
    for (int k = 0; k < N1; ++k)
      for (int l = 0; l < N1; ++l) h[O::BB + (i * N1 + k) * N1 + l] = t.B[i][k][l];
  for (int g = 0; g < NG; ++g) {
    for (int n = 0; n < N1; ++n) h[O::PG + g * N1 + n] = t.psiG[g][n];
    h[O::WG + g] = t.rw[g];
    h[O::SGP + g] = t.sgp[g];
    h[O::SGM + g] = t.sgm[g];
    h[O::NEG + g] = t.neg[g] ? 1.0 : 0.0;
  }
  for (int q = 0; q < t.QP; ++q) {
    h[O::PX + q] = t.px[q];
    h[O::PW + q] = t.pw[q];
    for (int n = 0; n < N1; ++n) h[O::PP + q * N1 + n] = t.ppsi[q][n];
  }
  h[O::PQP] = t.QP;
}

// modes of cell ix with the boundary condition (periodic wrap / outflow mirror)
template <int V, int N1>
__device__ __forceinline__ void load_cell(const double* __restrict__ U, long long ctot, const Inst& I, int ix, int bc,
                                          double (&u)[V][N1]) {
  bool flip = false;
  if (bc == 0) {
    ix = ix < 0 ? ix + I.nx : (ix >= I.nx ? ix - I.nx : ix);
  } else {
    if (ix < 0) { ix = 0; flip = true; }
    if (ix >= I.nx) { ix = I.nx - 1; flip = true; }
  }
  const long long g = I.off + ix;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int n = 0; n < N1; ++n) {
      const double x = __ldg(U + (long long)(v * N1 + n) * ctot + g);
      u[v][n] = neg_if(x, flip && (n & 1));
    }
}

template <int PDE, int N>
__global__ void __launch_bounds__(kBlock)
    k_stage1(const double* __restrict__ un, const double* __restrict__ us, double* __restrict__ out,
             const Inst* __restrict__ insts, const Tile* __restrict__ tiles, long long ctot, int bc, int stage,
             double dt_all, double gam) {
  using O = Off<N>;
  constexpr int V = nv_of(1, PDE), N1 = N + 1, Q = N + 1;
  const Tile tile = tiles[blockIdx.x];
  const Inst I = insts[tile.inst];
  const int ix = tile.x0 + threadIdx.x;
  if (ix >= I.nx) return;
  const double gm1 = gam - 1.0, s = 2.0 / I.hx, ih = 1.0 / I.hx;
  double u[V][N1], ul[V][N1], ur[V][N1];
  load_cell<V, N1>(us, ctot, I, ix, bc, u);
  load_cell<V, N1>(us, ctot, I, ix - 1, bc, ul);
  load_cell<V, N1>(us, ctot, I, ix + 1, bc, ur);
  double acc[V][N1];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int n = 0; n < N1; ++n) acc[v][n] = 0.0;
  // volume term (2/h) sum_q w_q f(u(x_q)) psi_n'(x_q)
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    double uq[V], f[V], a;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      double t = u[v][0] * T(O::P + q * N1);
#pragma unroll
      for (int n = 1; n < N1; ++n) t = fma(u[v][n], T(O::P + q * N1 + n), t);
      uq[v] = t;
    }
    Phys<1, PDE>::flux(0, uq, f, a, gam, gm1);
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int n = 1; n < N1; ++n) acc[v][n] = fma(s * f[v], T(O::D + q * N1 + n), acc[v][n]);
  }
  // traces and the two face fluxes (times 2/h)
  double aL[V], aR[V], bL[V], bR[V], fl[V], fr[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double x0 = 0, x1 = 0, x2 = 0, x3 = 0;
#pragma unroll
    for (int n = 0; n < N1; ++n) {
      x0 = fma(ul[v][n], T(O::P1 + n), x0);
      x1 = fma(u[v][n], T(O::M1 + n), x1);
      x2 = fma(u[v][n], T(O::P1 + n), x2);
      x3 = fma(ur[v][n], T(O::M1 + n), x3);
    }
    aL[v] = x0; aR[v] = x1; bL[v] = x2; bR[v] = x3;
  }
  llf<1, PDE>(0, aL, aR, fl, ih, gam, gm1);
  llf<1, PDE>(0, bL, bR, fr, ih, gam, gm1);
  const long long g = I.off + ix;
  const double dt = dt_all > 0.0 ? dt_all : I.dt;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int n = 0; n < N1; ++n) {
      const double L = acc[v][n] - (fr[v] * T(O::P1 + n) - fl[v] * T(O::M1 + n));
      const long long idx = (long long)(v * N1 + n) * ctot + g;
      const double e = fma(dt, L, us[idx]);
      double r;
      if (stage == 1) r = e;
      else if (stage == 2) r = fma(0.75, un[idx], 0.25 * e);
      else r = fma(1.0 / 3.0, un[idx], (2.0 / 3.0) * e);
      out[idx] = r;
    }
}

// TVB minmod flags (see the 2D kernel); mean = U_0 psi_0, face values by a plain
// serial sum without fused multiply-adds.
template <int PDE, int N>
__global__ void __launch_bounds__(kBlock)
    k_flag1(const double* __restrict__ U, const Inst* __restrict__ insts, const Tile* __restrict__ tiles,
            long long ctot, int bc, double M, unsigned char* __restrict__ flags, Counters* cnt,
            int* __restrict__ list_cell, int* __restrict__ list_inst) {
  using O = Off<N>;
  constexpr int V = nv_of(1, PDE), N1 = N + 1;
  const Tile tile = tiles[blockIdx.x];
  const Inst I = insts[tile.inst];
  const int ix = tile.x0 + threadIdx.x;
  int fl = 0;
  bool near = false;
  long long g = 0;
  if (ix < I.nx) {
    g = I.off + ix;
    int jl = ix - 1, jr = ix + 1;
    if (bc == 0) {
      jl = jl < 0 ? jl + I.nx : jl;
      jr = jr >= I.nx ? jr - I.nx : jr;
    } else {
      jl = jl < 0 ? 0 : jl;
      jr = jr >= I.nx ? I.nx - 1 : jr;
    }
    const long long mh2 = __double_as_longlong(M * I.hx * I.hx);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const double* P = U + (long long)(v * N1) * ctot;
      const double p0 = T(O::P0);
      const double mean = __dmul_rn(__ldg(P + g), p0);
      const double mL = __dmul_rn(__ldg(P + I.off + jl), p0), mR = __dmul_rn(__ldg(P + I.off + jr), p0);
      double up = 0.0, um = 0.0;
#pragma unroll
      for (int n = 0; n < N1; ++n) {  // psi_n(-1) = (-1)^n psi_n(1): one product per mode
        const double pc = __dmul_rn(__ldg(P + (long long)n * ctot + g), T(O::P1 + n));
        up = __dadd_rn(up, pc);
        um = (n & 1) ? __dsub_rn(um, pc) : __dadd_rn(um, pc);
      }
      const double dp = __dsub_rn(mR, mean), dm = __dsub_rn(mean, mL);
      fl |= tvb_changes_bits(__dsub_rn(up, mean), dp, dm, mh2, near);
      fl |= tvb_changes_bits(__dsub_rn(mean, um), dp, dm, mh2, near);
    }
    flags[g] = (unsigned char)(fl | (near ? 2 : 0));  // bit 0 troubled, bit 1 near threshold
  }
  block_compact(fl, near ? 1 : 0, g, tile.inst, cnt, list_cell, list_inst);
}

template <int N>
__device__ __forceinline__ void weno(const double* avg, double* out) {
  using O = Off<N>;
  constexpr int N1 = N + 1, NG = O::NG;
  const double eps = 1e-6;
  // beta_i and p_i - c do not change when a constant c is removed from all averages
  // (constants are reproduced; Eq. (13) holds only derivatives): work on averages
  // centred at the troubled cell's own, which avoids cancellation in beta.
  const double c = avg[N];
  double dv[2 * N + 1];
#pragma unroll
  for (int k = 0; k < 2 * N + 1; ++k) dv[k] = avg[k] - c;
  double inv[N1];
#pragma unroll
  for (int i = 0; i < N1; ++i) {
    double beta = 0.0;
#pragma unroll
    for (int k = 0; k < N1; ++k) {
      double r = 0.0;
#pragma unroll
      for (int l = 0; l < N1; ++l) r = fma(T(O::BB + (i * N1 + k) * N1 + l), dv[i + l], r);
      beta = fma(dv[i + k], r, beta);
    }
    const double d = eps + beta;
    inv[i] = 1.0 / (d * d);
  }
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    double p[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < N1; ++k) s = fma(T(O::WC + (i * NG + g) * N1 + k), dv[i + k], s);
      p[i] = c + s;
    }
    if (T(O::NEG + g) == 0.0) {
      double sw = 0.0, su = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        const double wb = T(O::GAM + g * N1 + i) * inv[i];
        sw += wb;
        su = fma(wb, p[i], su);
      }
      out[g] = su / sw;
    } else {
      double swp = 0.0, sup = 0.0, swm = 0.0, sum = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        const double wp = T(O::GPN + g * N1 + i) * inv[i];
        const double wm = T(O::GMN + g * N1 + i) * inv[i];
        swp += wp;
        sup = fma(wp, p[i], sup);
        swm += wm;
        sum = fma(wm, p[i], sum);
      }
      out[g] = T(O::SGP + g) * (sup / swp) - T(O::SGM + g) * (sum / swm);
    }
  }
}

// CSWENO in 1D (Sec. 3): subcell averages of the neighbours (Fig. 1), characteristic
// fields at the troubled cell's mean for Euler, WENO at the Step 1 points, Eq. (16).
template <int PDE, int N>
__global__ void __launch_bounds__(128)
    k_limit1(const double* __restrict__ U, const Inst* __restrict__ insts, long long ctot, int bc,
             const int* __restrict__ list_cell, const int* __restrict__ list_inst, const Counters* __restrict__ cnt,
             double* __restrict__ lim, long long cap, double gam) {
  using O = Off<N>;
  constexpr int V = nv_of(1, PDE), N1 = N + 1, NS = O::NS, NG = O::NG;
  const unsigned int n = cnt->n_flag;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long g = list_cell[i];
    const Inst I = insts[list_inst[i]];
    const int ix = (int)(g - I.off);
    double avg[V][NS];
#pragma unroll
    for (int d = -1; d <= 1; ++d) {
      double u[V][N1];
      load_cell<V, N1>(U, ctot, I, ix + d, bc, u);
      const int k0 = d < 0 ? 0 : (d == 0 ? N : N + 1), kn = d == 0 ? 1 : N;
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int k = k0; k < k0 + kn; ++k) {
          double s = 0.0;
#pragma unroll
          for (int m = 0; m < N1; ++m) s = fma(u[v][m], T(O::SA + k * N1 + m), s);
          avg[v][k] = s;
        }
    }
    double val[V][NG];
    if constexpr (PDE == 1) {
      double mean[3];
#pragma unroll
      for (int v = 0; v < 3; ++v) mean[v] = __ldg(U + (long long)(v * N1) * ctot + g) * T(O::SA + N * N1);
      const double rho = mean[0], r = 1.0 / rho, vel = mean[1] * r;
      const double p = (gam - 1.0) * (mean[2] - 0.5 * rho * vel * vel);
      const double c = sqrt(gam * p * r), ic = 1.0 / c, H = (mean[2] + p) * r;
      const double b1 = (gam - 1.0) * ic * ic, b2 = 0.5 * b1 * vel * vel;
      const double R[3][3] = {{1.0, 1.0, 1.0}, {vel - c, vel, vel + c}, {H - vel * c, 0.5 * vel * vel, H + vel * c}};
      const double L[3][3] = {{0.5 * (b2 + vel * ic), -0.5 * (b1 * vel + ic), 0.5 * b1},
                              {1.0 - b2, b1 * vel, -b1},
                              {0.5 * (b2 - vel * ic), 0.5 * (ic - b1 * vel), 0.5 * b1}};
      double wv[3][NG];
#pragma unroll
      for (int f = 0; f < 3; ++f) {
        double wc[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) wc[k] = fma(L[f][0], avg[0][k], fma(L[f][1], avg[1][k], L[f][2] * avg[2][k]));
        weno<N>(wc, wv[f]);
      }
#pragma unroll
      for (int v = 0; v < 3; ++v)
#pragma unroll
        for (int q = 0; q < NG; ++q) val[v][q] = fma(R[v][0], wv[0][q], fma(R[v][1], wv[1][q], R[v][2] * wv[2][q]));
    } else {
      weno<N>(avg[0], val[0]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int m = 1; m < N1; ++m) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NG; ++q) s = fma(T(O::WG + q) * val[v][q], T(O::PG + q * N1 + m), s);
        lim[(long long)(v * N1 + m) * cap + i] = s;
      }
  }
}


template <int PDE, int N>
__global__ void k_project1(double* __restrict__ U, const Inst* __restrict__ insts, const int* __restrict__ cell_inst,
                           long long ncell, long long ctot, int kind, const double* __restrict__ params, int np,
                           double gam) {
  using O = Off<N>;
  constexpr int V = nv_of(1, PDE), N1 = N + 1;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const int ii = cell_inst[g];
  const Inst I = insts[ii];
  const int ix = (int)(g - I.off);
  const double* p = params + (long long)ii * np;
  const int QP = (int)T(O::PQP);
  double acc[V][N1];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int n = 0; n < N1; ++n) acc[v][n] = 0.0;
  for (int q = 0; q < QP; ++q) {
    const double x = I.xL + I.hx * (ix + 0.5 * (1.0 + T(O::PX + q)));
    double u[V];
    ic_eval1(kind, p, x, gam, u);
#pragma unroll
    for (int n = 0; n < N1; ++n) {
      const double c = T(O::PW + q) * T(O::PP + q * N1 + n);
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v][n] = fma(c, u[v], acc[v][n]);
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int n = 0; n < N1; ++n) U[(long long)(v * N1 + n) * ctot + g] = acc[v][n];
}

template <int PDE, int N>
__global__ void k_speed1(const double* __restrict__ U, const Inst* __restrict__ insts, const int* __restrict__ cell_inst,
                         long long ncell, long long ctot, double gam, double* out) {
  using O = Off<N>;
  constexpr int V = nv_of(1, PDE), N1 = N + 1;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  double u[V];
  for (int v = 0; v < V; ++v) u[v] = U[(long long)(v * N1) * ctot + g] * T(O::P0);
  double s;
  if constexpr (PDE == 0) {
    s = fabs(u[0]);
  } else {
    const double r = 1.0 / u[0], vel = u[1] * r;
    const double p = (gam - 1.0) * (u[2] - 0.5 * u[0] * vel * vel);
    s = fabs(vel) + sqrt(gam * p * r);
  }
  atomic_max_nonneg(out + 2 * cell_inst[g], s);
}

#undef T
}  // namespace k1


cudaError_t upload_tables1(const dgt::Tabs* tabs) {
  static double h[k1::kTabSize];
  for (int i = 0; i < k1::kTabSize; ++i) h[i] = 0.0;
  k1::pack<1>(tabs[0], h);
  k1::pack<2>(tabs[1], h);
  k1::pack<3>(tabs[2], h);
  return cudaMemcpyToSymbol(k1::c_tab, h, sizeof(h));
}

#define DG_DISPATCH1(PDE, N, CALL) \
  do {                                                   \
    if ((PDE) == 0 && (N) == 1) { constexpr int P_ = 0, N_ = 1; CALL; } \
    else if ((PDE) == 0 && (N) == 2) { constexpr int P_ = 0, N_ = 2; CALL; } \
    else if ((PDE) == 0 && (N) == 3) { constexpr int P_ = 0, N_ = 3; CALL; } \
    else if ((PDE) == 1 && (N) == 1) { constexpr int P_ = 1, N_ = 1; CALL; } \
    else if ((PDE) == 1 && (N) == 2) { constexpr int P_ = 1, N_ = 2; CALL; } \
    else { constexpr int P_ = 1, N_ = 3; CALL; } \
  } while (0)

int tile_w1() { return k1::kBlock; }

void launch_stage1(int pde, int N, const LaunchArgs& a, int stage, double dt_all) {
  DG_DISPATCH1(pde, N, (k1::k_stage1<P_, N_><<<a.ntiles, k1::kBlock, 0, a.st>>>(a.un, a.us, a.out, a.inst, a.tiles,
                                                                                 a.ctot, a.bc, stage, dt_all, a.gam)));
}

void launch_flag1(int pde, int N, const LaunchArgs& a, double M, unsigned char* flags, Counters* cnt, int* lc,
                  int* li) {
  DG_DISPATCH1(pde, N, (k1::k_flag1<P_, N_><<<a.ntiles, k1::kBlock, 0, a.st>>>(a.us, a.inst, a.tiles, a.ctot, a.bc,
                                                                                M, flags, cnt, lc, li)));
}

void launch_limit1(int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt,
                   double* lim, int nblocks) {
  DG_DISPATCH1(pde, N, (k1::k_limit1<P_, N_><<<nblocks, 128, 0, a.st>>>(a.us, a.inst, a.ctot, a.bc, lc, li, cnt,
                                                                          lim, a.cap, a.gam)));
}

void launch_scatter1(int pde, int N, const LaunchArgs& a, const double* lim, const int* lc, const Counters* cnt,
                     int nblocks) {
  DG_DISPATCH1(pde, N, (k_scatter<nv_of(1, P_), np_of(1, N_)><<<nblocks, 256, 0, a.st>>>(a.out, a.ctot, lim, a.cap,
                                                                                          lc, cnt)));
}

void launch_project1(int pde, int N, const LaunchArgs& a, const int* cell_inst, int kind, const double* params,
                     int np) {
  const int nb = (int)((a.ncell + 127) / 128);
  DG_DISPATCH1(pde, N, (k1::k_project1<P_, N_><<<nb, 128, 0, a.st>>>(a.out, a.inst, cell_inst, a.ncell, a.ctot,
                                                                       kind, params, np, a.gam)));
}

void launch_speed1(int pde, int N, const LaunchArgs& a, const int* cell_inst, double* out) {
  const int nb = (int)((a.ncell + 255) / 256);
  DG_DISPATCH1(pde, N, (k1::k_speed1<P_, N_><<<nb, 256, 0, a.st>>>(a.us, a.inst, cell_inst, a.ncell, a.ctot,
                                                                     a.gam, out)));
}

}  // namespace dg
