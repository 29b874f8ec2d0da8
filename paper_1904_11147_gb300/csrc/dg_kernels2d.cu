// 2D kernels (Cartesian cells, total-degree P^N, N = 1..3; Burgers V = 1, Euler V = 4).
//
//   k_face2     split stage, face pass: traces of the two cells, local Lax-Friedrichs
//               flux at the face points, projection on the transverse modes (per face)
//   k_cell2     split stage, cell pass: volume quadrature, lifting of the four faces,
//               stage combination (per cell); the default form of one stage of Eq. (5)
//   k_stage2    the same stage fused in one kernel per tile (halo warps, shared faces),
//               an autotuner alternative
//   k_flag2     TVB minmod indicator + ballot/scan compaction of troubled cells
//   k_limit2    CSWENO limiter (Sec. 3): Burgers one thread per troubled cell, Euler
//               four lanes per troubled cell (k_limit2_euler_quad)
//   k_project2  initial L2 projection (Eq. (2))
//   k_speed2    largest characteristic speed over the cell means
//
// FP64 arithmetic is the bound on GB300 (the FP64 pipe runs at 1/64 of FP32), so the
// kernels are laid out to keep every lane of every FP64 warp instruction useful and to
// avoid recomputing traces or face fluxes.
#include "dg_ic.cuh"
#include "dg_shared.cuh"
#include "tables.h"

namespace dg {
namespace k2 {

constexpr int TX = 32;  // tile width = one warp
constexpr int TY = 8;   // rows per tile of the indicator and projection kernels

// ----------------------------------------------------------------------------- tables
template <int N>
struct Lay {
  static constexpr int Q = N + 1, NP = (N + 1) * (N + 2) / 2, NS = 2 * N + 1, NG = (N == 1 ? 2 : 4);
  static constexpr int N1 = N + 1;
  static constexpr int SIZE_DG = 3 * Q * Q * NP + N1 + 2 * Q * N1;
  static constexpr int SIZE_FLAG = 4 * NP + 1;
  static constexpr int SIZE_LIM = NS * N1 + N1 * NG * N1 + NG * N1 + N1 * N1 * N1 + NG * N1 + NG +
                                  2 * NG * N1 + 3 * NG;
  static constexpr int SIZE_PROJ = 3 * 8 + 8 * N1;
  static constexpr int SIZE_SPLIT = Q * N1;
  static constexpr int SIZE_LIM2 = N1 * (N * N1 / 2) + NG * N1;
  static constexpr int SIZE_K = Q * N1 + N1;
  static constexpr int SIZE_LIM3 = N1 * NG * N1;
  static constexpr int SIZE = SIZE_DG + SIZE_FLAG + SIZE_LIM + SIZE_PROJ + SIZE_SPLIT + SIZE_LIM2 + SIZE_K + SIZE_LIM3;
};
__host__ __device__ constexpr int base_of(int N) {
  return N == 1 ? 0 : (N == 2 ? Lay<1>::SIZE : Lay<1>::SIZE + Lay<2>::SIZE);
}
template <int N>
struct Off {
  using L = Lay<N>;
  static constexpr int Q = L::Q, NP = L::NP, NS = L::NS, NG = L::NG, N1 = L::N1;
  static constexpr int VP = base_of(N);          // [Q*Q][NP] psi_a(x_qx) psi_b(x_qy)
  static constexpr int VDX = VP + Q * Q * NP;    // w w psi_a'(x_qx) psi_b(x_qy)
  static constexpr int VDY = VDX + Q * Q * NP;   // w w psi_a(x_qx) psi_b'(x_qy)
  static constexpr int P1 = VDY + Q * Q * NP;    // psi_n(1)
  static constexpr int PQ = P1 + N1;             // [Q][N1] psi_n(x_q)
  static constexpr int WPQ = PQ + Q * N1;        // [Q][N1] w_q psi_n(x_q)
  static constexpr int TE = WPQ + Q * N1;        // [NP] psi_a(1) psi_b(0)
  static constexpr int TW = TE + NP;             // psi_a(-1) psi_b(0)
  static constexpr int TN = TW + NP;             // psi_a(0) psi_b(1)
  static constexpr int TS = TN + NP;             // psi_a(0) psi_b(-1)
  static constexpr int C00 = TS + NP;            // psi_0(0)^2
  static constexpr int SA = C00 + 1;             // [NS][N1]
  static constexpr int WC = SA + NS * N1;        // [N1 stencil][NG][N1]
  static constexpr int GAM = WC + N1 * NG * N1;  // [NG][N1]
  static constexpr int BB = GAM + NG * N1;       // [N1][N1][N1]
  static constexpr int PG = BB + N1 * N1 * N1;   // [NG][N1] psi_n(r_g)
  static constexpr int WG = PG + NG * N1;        // [NG]
  static constexpr int GPN = WG + NG;            // [NG][N1]
  static constexpr int GMN = GPN + NG * N1;      // [NG][N1]
  static constexpr int SGP = GMN + NG * N1;      // [NG]
  static constexpr int SGM = SGP + NG;           // [NG]
  static constexpr int NEG = SGM + NG;           // [NG] 1.0 where a weight is negative
  static constexpr int PX = NEG + NG;            // [8]
  static constexpr int PW = PX + 8;              // [8]
  static constexpr int PQP = PW + 8;             // [8] (count in slot 0)
  static constexpr int PP = PQP + 8;             // [8][N1]
  static constexpr int WDQ = PP + 8 * N1;        // [Q][N1] w_q psi_n'(x_q)
  static constexpr int BD = WDQ + Q * N1;        // [N1][j <= j'] Eq. (13) on differences (see pack)
  static constexpr int WPG = BD + N1 * (N * N1 / 2);  // [NG][N1] w_g psi_n(r_g)
  static constexpr int KQ = WPG + NG * N1;       // [Q][N1] sqrt(2) psi_n(x_q) = psi_n(x_q) / psi_0
  static constexpr int KP1 = KQ + Q * N1;        // [N1] sqrt(2) psi_n(1)
  static constexpr int WCG = KP1 + N1;           // [N1 stencil][NG][N1] gamma_gi C_igk
  static constexpr int END = WCG + N1 * NG * N1;
};
static_assert(Off<3>::END == Lay<1>::SIZE + Lay<2>::SIZE + Lay<3>::SIZE, "table layout");
constexpr int kTabSize = Off<3>::END;

__constant__ double c_tab[kTabSize];

#define T(x) c_tab[(x)]

template <int N>
void pack(const dgt::Tabs& t, double* h) {
  using O = Off<N>;
  constexpr int Q = O::Q, NP = O::NP, NS = O::NS, NG = O::NG, N1 = O::N1;
  for (int qy = 0; qy < Q; ++qy)
    for (int qx = 0; qx < Q; ++qx)
      for (int m = 0; m < NP; ++m) {
        int a = mode_a(m), b = mode_b(m), q = qy * Q + qx;
        double ww = t.gw[qx] * t.gw[qy];
        h[O::VP + q * NP + m] = t.psi_q[qx][a] * t.psi_q[qy][b];
        h[O::VDX + q * NP + m] = ww * t.dpsi_q[qx][a] * t.psi_q[qy][b];
        h[O::VDY + q * NP + m] = ww * t.psi_q[qx][a] * t.dpsi_q[qy][b];
      }
  for (int n = 0; n < N1; ++n) h[O::P1 + n] = t.psi_p1[n];
  for (int q = 0; q < Q; ++q)
    for (int n = 0; n < N1; ++n) {
      h[O::PQ + q * N1 + n] = t.psi_q[q][n];
      h[O::WPQ + q * N1 + n] = t.gw[q] * t.psi_q[q][n];
    }
  for (int m = 0; m < NP; ++m) {
    int a = mode_a(m), b = mode_b(m);
    h[O::TE + m] = t.psi_p1[a] * t.psi_0[b];
    h[O::TW + m] = t.psi_m1[a] * t.psi_0[b];
    h[O::TN + m] = t.psi_0[a] * t.psi_p1[b];
    h[O::TS + m] = t.psi_0[a] * t.psi_m1[b];
  }
  h[O::C00] = t.psi_0[0] * t.psi_0[0];
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
  for (int q = 0; q < Q; ++q)
    for (int n = 0; n < N1; ++n) h[O::WDQ + q * N1 + n] = t.gw[q] * t.dpsi_q[q][n];
  for (int g = 0; g < NG; ++g)
    for (int n = 0; n < N1; ++n) h[O::WPG + g * N1 + n] = t.rw[g] * t.psiG[g][n];
  for (int q = 0; q < Q; ++q)
    for (int n = 0; n < N1; ++n) h[O::KQ + q * N1 + n] = t.kq[q][n];
  for (int n = 0; n < N1; ++n) h[O::KP1 + n] = t.kp1[n];
  // beta_i as a quadratic form in the N differences d_j = x_{i+j+1} - x_{i+j} of the
  // stencil's averages x (beta ignores constants): with x_{i+k} - x_i = sum_{j<k} d_j,
  // M_jj' = sum_{k > j, l > j'} B_ikl; packed as M_jj and M_jj' + M_j'j (j < j')
  for (int i = 0; i < N1; ++i) {
    int j = 0;
    for (int a = 0; a < N; ++a)
      for (int b = a; b < N; ++b, ++j) {
        double mab = 0.0, mba = 0.0;
        for (int k = a + 1; k < N1; ++k)
          for (int l = b + 1; l < N1; ++l) {
            mab += t.B[i][k][l];
            mba += t.B[i][l][k];
          }
        h[O::BD + i * (N * N1 / 2) + j] = a == b ? mab : mab + mba;
      }
  }
  for (int i = 0; i < N1; ++i)
    for (int g = 0; g < NG; ++g)
      for (int k = 0; k < N1; ++k) h[O::WCG + (i * NG + g) * N1 + k] = t.gam[g][i] * t.C[i][g][k];
}

// ----------------------------------------------------------------------------- loads
// Loads the modes of cell (ix, iy) of instance I, applying the boundary condition for
// ghost cells: periodic wraps; outflow mirrors the boundary cell (modes odd in the
// normal direction change sign).
template <int V, int NP>
__device__ __forceinline__ void load_cell(const double* __restrict__ U, long long ctot, const Inst& I, int ix,
                                          int iy, int bc, double (&u)[V][NP]) {
  bool fx = false, fy = false;
  if (bc == 0) {
    ix = ix < 0 ? ix + I.nx : (ix >= I.nx ? ix - I.nx : ix);
    iy = iy < 0 ? iy + I.ny : (iy >= I.ny ? iy - I.ny : iy);
  } else {
    if (ix < 0) { ix = 0; fx = true; }
    if (ix >= I.nx) { ix = I.nx - 1; fx = true; }
    if (iy < 0) { iy = 0; fy = true; }
    if (iy >= I.ny) { iy = I.ny - 1; fy = true; }
  }
  const long long g = I.off + (long long)iy * I.nx + ix;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      double x = __ldg(U + (long long)(v * NP + m) * ctot + g);
      bool flip = (fx && (mode_a(m) & 1)) != (fy && (mode_b(m) & 1));
      u[v][m] = neg_if(x, flip);
    }
}

// load_cell with the kBcDmr ghosts (dmr_ghost) for cells outside instance `inst`.
// t: the time of the state U.
template <int V, int NP>
__device__ __forceinline__ void load_cell_bc(const double* __restrict__ U, long long ctot, const Inst& I, int inst,
                                             int ix, int iy, int bc, const double* __restrict__ bcd, double t,
                                             double (&u)[V][NP]) {
  if (bc != kBcDmr || (ix >= 0 && ix < I.nx && iy >= 0 && iy < I.ny)) {
    load_cell<V, NP>(U, ctot, I, ix, iy, bc, u);
    return;
  }
  const Ghost gh = dmr_ghost(I, inst, ix, iy, bcd, t);
  if (gh.c) {  // constant state: U_00 = mean / psi_0^2 = 2 mean, no other mode
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int m = 0; m < NP; ++m) u[v][m] = m == 0 ? 2.0 * gh.c[v] : 0.0;
    return;
  }
  const long long g = I.off + (long long)gh.jy * I.nx + gh.jx;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      const double x = __ldg(U + (long long)(v * NP + m) * ctot + g);
      const bool flip = ((gh.fx && (mode_a(m) & 1)) != (gh.fy && (mode_b(m) & 1))) != (gh.fv && v == 2);
      u[v][m] = neg_if(x, flip);
    }
}

// Traces on the east (r = +1) and west (r = -1) faces at the Q face points:
// u(+-1, s_q) = sum_b psi_b(s_q) sum_a (+-1)^a U_ab psi_a(1).
template <int N, int V, int NP>
__device__ __forceinline__ void traces_x(const double (&u)[V][NP], double (&tE)[N + 1][V], double (&tW)[N + 1][V]) {
  using O = Off<N>;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double ev[N + 1], od[N + 1];
#pragma unroll
    for (int b = 0; b <= N; ++b) {
      ev[b] = 0.0;
      od[b] = 0.0;
#pragma unroll
      for (int a = 0; a <= N - b; ++a) {
        double c = u[v][mode_idx(a, b)] * T(O::P1 + a);
        if (a & 1) od[b] += c; else ev[b] += c;
      }
    }
#pragma unroll
    for (int q = 0; q <= N; ++q) {
      double e = 0.0, w = 0.0;
#pragma unroll
      for (int b = 0; b <= N; ++b) {
        e = fma(ev[b] + od[b], T(O::PQ + q * (N + 1) + b), e);
        w = fma(ev[b] - od[b], T(O::PQ + q * (N + 1) + b), w);
      }
      tE[q][v] = e;
      tW[q][v] = w;
    }
  }
}

// Traces on the north (s = +1) and south (s = -1) faces.
template <int N, int V, int NP>
__device__ __forceinline__ void traces_y(const double (&u)[V][NP], double (&tN)[N + 1][V], double (&tS)[N + 1][V]) {
  using O = Off<N>;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double ev[N + 1], od[N + 1];
#pragma unroll
    for (int a = 0; a <= N; ++a) {
      ev[a] = 0.0;
      od[a] = 0.0;
#pragma unroll
      for (int b = 0; b <= N - a; ++b) {
        double c = u[v][mode_idx(a, b)] * T(O::P1 + b);
        if (b & 1) od[a] += c; else ev[a] += c;
      }
    }
#pragma unroll
    for (int q = 0; q <= N; ++q) {
      double n = 0.0, s = 0.0;
#pragma unroll
      for (int a = 0; a <= N; ++a) {
        n = fma(ev[a] + od[a], T(O::PQ + q * (N + 1) + a), n);
        s = fma(ev[a] - od[a], T(O::PQ + q * (N + 1) + a), s);
      }
      tN[q][v] = n;
      tS[q][v] = s;
    }
  }
}

// Trace on one face at the Q face points for halo cells, which need a single side:
// dir 0: east face (r = +1); dir 1: north face (s = +1).  A halo cell that needs the west
// (south) trace passes its modes with the odd normal degrees negated (mirror image).
template <int N, int V, int NP>
__device__ __forceinline__ void trace_one(const double (&u)[V][NP], int dir, double (&tr)[N + 1][V]) {
  using O = Off<N>;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double e[N + 1];
#pragma unroll
    for (int t = 0; t <= N; ++t) {  // t: transverse degree
      double s = 0.0;
#pragma unroll
      for (int n = 0; n <= N - t; ++n) {  // n: normal degree
        const int m = dir == 0 ? mode_idx(n, t) : mode_idx(t, n);
        s = fma(u[v][m], T(O::P1 + n), s);
      }
      e[t] = s;
    }
#pragma unroll
    for (int q = 0; q <= N; ++q) {
      double r = 0.0;
#pragma unroll
      for (int t = 0; t <= N; ++t) r = fma(e[t], T(O::PQ + q * (N + 1) + t), r);
      tr[q][v] = r;
    }
  }
}

// ----------------------------------------------------------------------------- stage
// One tile of TX x TYS cells per block (TYS = 4 or 8, chosen by the autotuner).  Warps
// 0..TYS-1 hold the interior rows, warp TYS the row below the tile, warp TYS+1 the row
// above it, warp TYS+2 the west (lanes 0..15) and
// east (lanes 16..31) halo cells, so that every trace and every face flux is computed
// exactly once per tile by a full warp.
template <int PDE, int N, int TYS>
__global__ void __launch_bounds__((TYS + 3) * 32, 1)
    k_stage2(const double* __restrict__ un, const double* __restrict__ us, double* __restrict__ out,
             const Inst* __restrict__ insts, const Tile* __restrict__ tiles, long long ctot, int bc, int stage,
             double dt_all, double gam, int ntiles, int* __restrict__ queue) {
  using O = Off<N>;
  constexpr int V = nv_of(2, PDE), NP = np_of(2, N), Q = N + 1, QV = Q * V;
  // east traces, then x-face fluxes: [QV][TYS][TX+1]; north traces, then y-face fluxes:
  // [QV][TYS+1][TX] (dynamic shared memory, above the 48 KB static limit for Euler P2/P3)
  extern __shared__ double smem[];
  double* const sEb = smem;
  double* const sNb = smem + QV * TYS * (TX + 1);
#define sE(qv, r, c) sEb[((qv) * TYS + (r)) * (TX + 1) + (c)]
#define sN(qv, r, c) sNb[((qv) * (TYS + 1) + (r)) * TX + (c)]
  // one tile per block, or (queue != null) a persistent block taking tiles from the queue
  __shared__ int s_tile;
  int tix = blockIdx.x;
  if (queue) {
    if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
    __syncthreads();
    tix = s_tile;
  }
  while (tix < ntiles) {
  const Tile tile = tiles[tix];
  const Inst I = insts[tile.inst];
  const int ncols = min(TX, I.nx - tile.x0), nrows = min(TYS, I.ny - tile.y0);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double gm1 = gam - 1.0;
  const double sx = 2.0 / I.hx, sy = 2.0 / I.hy, ihx = 1.0 / I.hx, ihy = 1.0 / I.hy;

  const bool interior = w < TYS && w < nrows && lane < ncols;
  double acc[V][NP];
  double trW[Q][V], trS[Q][V];
  // ---------------------------------------------------------------- phase 1
  if (interior) {
    double u[V][NP];
    load_cell<V, NP>(us, ctot, I, tile.x0 + lane, tile.y0 + w, bc, u);
    double tE[Q][V], tN[Q][V];
    traces_x<N>(u, tE, trW);
    traces_y<N>(u, tN, trS);
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        sE(q * V + v, w, lane + 1) = tE[q][v];
        sN(q * V + v, w + 1, lane) = tN[q][v];
      }
    // volume term: (2/hx) sum_q w w f psi_a' psi_b + (2/hy) sum_q w w g psi_a psi_b'
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int m = 0; m < NP; ++m) acc[v][m] = 0.0;
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) {
      // sum factorisation: t_b(x_qx) = sum_a U_ab psi_a(x_qx), then u = sum_b t_b psi_b(y_qy)
      double tb[V][N + 1];
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int b = 0; b <= N; ++b) {
          double t = u[v][mode_idx(0, b)] * T(O::PQ + qx * (N + 1));
#pragma unroll
          for (int a = 1; a <= N - b; ++a) t = fma(u[v][mode_idx(a, b)], T(O::PQ + qx * (N + 1) + a), t);
          tb[v][b] = t;
        }
#pragma unroll
      for (int qy = 0; qy < Q; ++qy) {
        const int q = qy * Q + qx;
        double uq[V], f[V], g[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          double t = tb[v][0] * T(O::PQ + qy * (N + 1));
#pragma unroll
          for (int b = 1; b <= N; ++b) t = fma(tb[v][b], T(O::PQ + qy * (N + 1) + b), t);
          uq[v] = t;
        }
        vol_flux2<2, PDE>(uq, f, g, sx, sy, gm1);
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int m = 1; m < NP; ++m) {
            if (mode_a(m) >= 1) acc[v][m] = fma(f[v], T(O::VDX + q * NP + m), acc[v][m]);
            if (mode_b(m) >= 1) acc[v][m] = fma(g[v], T(O::VDY + q * NP + m), acc[v][m]);
          }
      }
    }
  } else if (w == TYS) {  // row below the tile: its north traces
    if (lane < ncols) {
      double u[V][NP], tN[Q][V];
      load_cell<V, NP>(us, ctot, I, tile.x0 + lane, tile.y0 - 1, bc, u);
      trace_one<N>(u, 1, tN);
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) sN(q * V + v, 0, lane) = tN[q][v];
    }
  } else if (w == TYS + 1) {  // row above the tile: its south traces (kept for phase 2)
    if (lane < ncols) {
      double u[V][NP];
      load_cell<V, NP>(us, ctot, I, tile.x0 + lane, tile.y0 + nrows, bc, u);
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int m = 0; m < NP; ++m)
          if (mode_b(m) & 1) u[v][m] = neg_if(u[v][m], true);
      trace_one<N>(u, 1, trS);
    }
  } else if (w == TYS + 2) {  // west halo (lanes < 16) east traces, east halo west traces
    const bool east = lane >= 16;
    const int row = east ? lane - 16 : lane;
    if (row < nrows) {
      double u[V][NP], tA[Q][V];
      load_cell<V, NP>(us, ctot, I, east ? tile.x0 + ncols : tile.x0 - 1, tile.y0 + row, bc, u);
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int m = 0; m < NP; ++m)
          u[v][m] = neg_if(u[v][m], east && (mode_a(m) & 1));
      trace_one<N>(u, 0, tA);
#pragma unroll
      for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if (!east) sE(q * V + v, row, 0) = tA[q][v];
          trW[q][v] = tA[q][v];
        }
    }
  }
  __syncthreads();
  // ---------------------------------------------------------------- phase 2: face fluxes
  if (interior) {
    double uL[V], uR[V], fs[V];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        uL[v] = sE(q * V + v, w, lane);
        uR[v] = trW[q][v];
      }
      llf<2, PDE>(0, uL, uR, fs, ihx, gam, gm1);
#pragma unroll
      for (int v = 0; v < V; ++v) sE(q * V + v, w, lane) = fs[v];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        uL[v] = sN(q * V + v, w, lane);
        uR[v] = trS[q][v];
      }
      llf<2, PDE>(1, uL, uR, fs, ihy, gam, gm1);
#pragma unroll
      for (int v = 0; v < V; ++v) sN(q * V + v, w, lane) = fs[v];
    }
  } else if (w == TYS + 1) {
    if (lane < ncols) {
      double uL[V], fs[V];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
#pragma unroll
        for (int v = 0; v < V; ++v) uL[v] = sN(q * V + v, nrows, lane);
        llf<2, PDE>(1, uL, trS[q], fs, ihy, gam, gm1);
#pragma unroll
        for (int v = 0; v < V; ++v) sN(q * V + v, nrows, lane) = fs[v];
      }
    }
  } else if (w == TYS + 2) {
    const int row = lane - 16;
    if (lane >= 16 && row < nrows) {
      double uL[V], fs[V];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
#pragma unroll
        for (int v = 0; v < V; ++v) uL[v] = sE(q * V + v, row, ncols);
        llf<2, PDE>(0, uL, trW[q], fs, ihx, gam, gm1);
#pragma unroll
        for (int v = 0; v < V; ++v) sE(q * V + v, row, ncols) = fs[v];
      }
    }
  }
  __syncthreads();
  // ---------------------------------------------------------------- phase 3: lift + RK
  if (interior) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    // x faces: acc_ab -= psi_a(1) sum_q w_q psi_b(s_q) [F_E(q) - (-1)^a F_W(q)]
    double dxs[Q], sxs[Q], dys[Q], sys[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      double fe = sE(q * V + v, w, lane + 1), fw = sE(q * V + v, w, lane);
      double fn = sN(q * V + v, w + 1, lane), fsv = sN(q * V + v, w, lane);
      dxs[q] = fe - fw;
      sxs[q] = fe + fw;
      dys[q] = fn - fsv;
      sys[q] = fn + fsv;
    }
#pragma unroll
    for (int b = 0; b <= N; ++b) {
      double Sp = 0.0, Sm = 0.0, Tp = 0.0, Tm = 0.0;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const double c = T(O::WPQ + q * (N + 1) + b);
        Sp = fma(c, dxs[q], Sp);
        Sm = fma(c, sxs[q], Sm);
        Tp = fma(c, dys[q], Tp);
        Tm = fma(c, sys[q], Tm);
      }
      // here b plays the transverse index: x faces use psi_b(s), y faces psi_a(r)
#pragma unroll
      for (int a = 0; a <= N - b; ++a) {
        const int mx = mode_idx(a, b);  // x faces: transverse degree b, normal degree a
        acc[v][mx] = fma(-T(O::P1 + a), (a & 1) ? Sm : Sp, acc[v][mx]);
        const int my = mode_idx(b, a);  // y faces: transverse degree b (in x), normal a
        acc[v][my] = fma(-T(O::P1 + a), (a & 1) ? Tm : Tp, acc[v][my]);
      }
    }
  }
  const long long g = I.off + (long long)(tile.y0 + w) * I.nx + tile.x0 + lane;
  const double dt = dt_all > 0.0 ? dt_all : I.dt;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      const long long idx = (long long)(v * NP + m) * ctot + g;
      double e = fma(dt, acc[v][m], us[idx]);
      double r;
      if (stage == 1) r = e;
      else if (stage == 2) r = fma(0.75, un[idx], 0.25 * e);
      else r = fma(1.0 / 3.0, un[idx], (2.0 / 3.0) * e);
      out[idx] = r;
    }
  }  // interior
  if (!queue) break;
  __syncthreads();  // shared memory and s_tile are reused by the next tile
  if (threadIdx.x == 0) s_tile = atomicAdd(queue, 1);
  __syncthreads();
  tix = s_tile;
  }  // tiles
}

#undef sE
#undef sN

// ----------------------------------------------------------------------------- split stage
// The same stage of Eq. (5) as two passes without block barriers or halo work:
//   k_face2  one thread per face: the traces of the two cells at the Q face points, the
//            local Lax-Friedrichs flux there, and its projection onto the transverse modes
//              P_b = sum_q w_q psi_b(s_q) [f(uL) + f(uR) - alpha (uR - uL)],  b = 0..N,
//            stored in planes [v*(N+1) + b][face] (x faces and y faces apart); the traces
//            are formed doubled (face_trace2), so the planes hold 2^d P_b, d the degree
//            of homogeneity of the flux (1 Euler, 2 Burgers);
//   k_cell2  one thread per cell: the volume term (at doubled point values, likewise),
//            the lifting of the four faces' P_b and the stage combination, with 2^-d
//            folded into the scalings 2/h and 1/h.
// Every face flux is computed once; all lanes of every warp do the same work.

// Values at the Q Gauss points of sum_t e_t psi_t(s).  The points are symmetric
// (s_{Q-1-q} = -s_q) and psi_t has the parity of t, so the even and odd sums are formed
// once per pair of points; psi_0 is constant.
template <int N>
__device__ __forceinline__ void eval_gauss(const double (&e)[N + 1], double (&out)[N + 1]) {
  using O = Off<N>;
  constexpr int Q = N + 1;
  const double p0 = e[0] * T(O::PQ);
#pragma unroll
  for (int q = 0; q < Q / 2; ++q) {
    double ev = p0, od = e[1] * T(O::PQ + q * (N + 1) + 1);
#pragma unroll
    for (int t = 2; t <= N; ++t) {
      if (t & 1) od = fma(e[t], T(O::PQ + q * (N + 1) + t), od);
      else ev = fma(e[t], T(O::PQ + q * (N + 1) + t), ev);
    }
    out[q] = ev + od;
    out[Q - 1 - q] = ev - od;
  }
  if constexpr (Q & 1) {
    double ev = p0;
#pragma unroll
    for (int t = 2; t <= N; t += 2) ev = fma(e[t], T(O::PQ + (Q / 2) * (N + 1) + t), ev);
    out[Q / 2] = ev;
  }
}

// Twice the values at the Q Gauss points of sum_t e_t psi_t(s) / psi_0 (e given over
// psi_0): 2 sum_t (e_t / psi_0) psi_t(s) psi_0 = e_0 + sum_{t>=1} e_t sqrt(2) psi_t(s), so the
// constant term enters without a multiplication.  Symmetric pairs as in eval_gauss.
template <int N>
__device__ __forceinline__ void eval_gauss2(const double (&e)[N + 1], double (&out)[N + 1]) {
  using O = Off<N>;
  constexpr int Q = N + 1;
#pragma unroll
  for (int q = 0; q < Q / 2; ++q) {
    double ev = e[0], od = e[1] * T(O::KQ + q * (N + 1) + 1);
#pragma unroll
    for (int t = 2; t <= N; ++t) {
      if (t & 1) od = fma(e[t], T(O::KQ + q * (N + 1) + t), od);
      else ev = fma(e[t], T(O::KQ + q * (N + 1) + t), ev);
    }
    out[q] = ev + od;
    out[Q - 1 - q] = ev - od;
  }
  if constexpr (Q & 1) {
    double ev = e[0];
#pragma unroll
    for (int t = 2; t <= N; t += 2) ev = fma(e[t], T(O::KQ + (Q / 2) * (N + 1) + t), ev);
    out[Q / 2] = ev;
  }
}

// Twice the trace of a cell on its face normal to `dir` at the Q face points, the +1 side
// (east / north) or, with minus = true, the -1 side (west / south), whose normal modes of
// odd degree enter with the opposite sign.  With psi_n(1) = psi_0 sqrt(2 n + 1), the sum
// over the normal degree is formed over psi_0 (its constant term needs no multiplication)
// and eval_gauss2 doubles the result; the fluxes of the split stage are homogeneous in the
// state (Euler of degree 1, Burgers of degree 2), so the passes carry the factor 2 and
// remove it, exactly, in the final scalings.  The mirror image of a cell (outflow ghost)
// gives a bitwise identical trace on the shared face.
template <int N, int V, int NP>
__device__ __forceinline__ void face_trace2(const double (&u)[V][NP], int dir, bool minus, double (&tr)[N + 1][V]) {
  using O = Off<N>;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double e[N + 1], val[N + 1];
#pragma unroll
    for (int t = 0; t <= N; ++t) {  // transverse degree t, normal degree n
      double s = u[v][dir == 0 ? mode_idx(0, t) : mode_idx(t, 0)];
#pragma unroll
      for (int n = 1; n <= N - t; ++n) {
        const double x = u[v][dir == 0 ? mode_idx(n, t) : mode_idx(t, n)];
        s = fma(neg_if(x, minus && (n & 1)), T(O::KP1 + n), s);
      }
      e[t] = s;
    }
    eval_gauss2<N>(e, val);
#pragma unroll
    for (int q = 0; q <= N; ++q) tr[q][v] = val[q];
  }
}

// Trace of a cell on its face normal to `dir` at the Q face points: the +1 side
// (east / north) or, with minus = true, the -1 side (west / south), whose normal modes of
// odd degree enter with the opposite sign.  The mirror image of a cell (outflow ghost)
// therefore gives a bitwise identical trace on the shared face.
template <int N, int V, int NP>
__device__ __forceinline__ void face_trace(const double (&u)[V][NP], int dir, bool minus, double (&tr)[N + 1][V]) {
  using O = Off<N>;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double e[N + 1], val[N + 1];
#pragma unroll
    for (int t = 0; t <= N; ++t) {  // transverse degree t, normal degree n
      double s = u[v][dir == 0 ? mode_idx(0, t) : mode_idx(t, 0)] * T(O::P1);
#pragma unroll
      for (int n = 1; n <= N - t; ++n) {
        const double x = u[v][dir == 0 ? mode_idx(n, t) : mode_idx(t, n)];
        s = fma(neg_if(x, minus && (n & 1)), T(O::P1 + n), s);
      }
      e[t] = s;
    }
    eval_gauss<N>(e, val);
#pragma unroll
    for (int q = 0; q <= N; ++q) tr[q][v] = val[q];
  }
}

// Face tiles: 32 faces along x by 4 rows; Tile::pad = 0 for x faces (k = 0..nx, j < ny),
// 1 for y faces (k < nx, j = 0..ny).  Face k of a row lies between cells k-1 and k.
template <int PDE, int N>
__global__ void __launch_bounds__(128) k_face2(const double* __restrict__ us, const Inst* __restrict__ insts,
                                               const Tile* __restrict__ tiles, long long ctot, int bc, double gam,
                                               double* __restrict__ fx, long long fxt, double* __restrict__ fy,
                                               long long fyt, const double* __restrict__ bcd, int stage,
                                               double dt_all) {
  using O = Off<N>;
  constexpr int V = nv_of(2, PDE), NP = np_of(2, N), Q = N + 1;
  const Tile tile = tiles[blockIdx.x];
  const Inst I = insts[tile.inst];
  const int dir = tile.pad;
  const int k = tile.x0 + (threadIdx.x & 31), j = tile.y0 + (threadIdx.x >> 5);
  if (dir == 0 ? (k > I.nx || j >= I.ny) : (k >= I.nx || j > I.ny)) return;
  const double gm1 = gam - 1.0;
  // kBcDmr: the stage's input holds at t^n, t^n + dt, t^n + dt/2 for stages 1, 2, 3
  double t_in = 0.0;
  if (bc == kBcDmr) t_in = dmr_time(bcd, tile.inst, 2) + (stage == 1 ? 0.0 : (stage == 2 ? 1.0 : 0.5)) * (dt_all > 0.0 ? dt_all : I.dt);
  double tL[Q][V], tR[Q][V];
  {
    double u[V][NP];
    load_cell_bc<V, NP>(us, ctot, I, tile.inst, dir == 0 ? k - 1 : k, dir == 0 ? j : j - 1, bc, bcd, t_in, u);
    face_trace2<N>(u, dir, false, tL);
  }
  {
    double u[V][NP];
    load_cell_bc<V, NP>(us, ctot, I, tile.inst, k, j, bc, bcd, t_in, u);
    face_trace2<N>(u, dir, true, tR);
  }
  double G[Q][V];
#pragma unroll
  for (int q = 0; q < Q; ++q) llf_sum<2, PDE>(dir, tL[q], tR[q], G[q], gam, gm1);
  // P_b = sum_q w_q psi_b(s_q) G(q), summed over symmetric pairs of points
  double* const base = dir == 0 ? fx + I.fx + (long long)j * (I.nx + 1) + k : fy + I.fy + (long long)j * I.nx + k;
  const long long stride = dir == 0 ? fxt : fyt;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double S[Q / 2 + 1], D[Q / 2 + 1];
#pragma unroll
    for (int q = 0; q < Q / 2; ++q) {
      S[q] = G[q][v] + G[Q - 1 - q][v];
      D[q] = G[q][v] - G[Q - 1 - q][v];
    }
#pragma unroll
    for (int b = 0; b <= N; ++b) {
      double P = 0.0;
      bool first = true;
#pragma unroll
      for (int q = 0; q < Q / 2; ++q) {
        const double x = (b & 1) ? D[q] : S[q];
        P = first ? x * T(O::WPQ + q * (N + 1) + b) : fma(x, T(O::WPQ + q * (N + 1) + b), P);
        first = false;
      }
      if ((Q & 1) && !(b & 1)) P = fma(G[Q / 2][v], T(O::WPQ + (Q / 2) * (N + 1) + b), P);
      base[(long long)(v * (N + 1) + b) * stride] = P;
    }
  }
}

// One thread per cell over the 32 x 8 cell tiles (lane = column, warp = row).
// Two blocks per SM (at most 128 registers) except for Euler P3, which needs more registers.
template <int PDE, int N>
__global__ void __launch_bounds__(256, (PDE == 1 && N == 3) ? 1 : 2) k_cell2(const double* __restrict__ un, const double* __restrict__ us,
                                               double* __restrict__ out, const Inst* __restrict__ insts,
                                               const Tile* __restrict__ tiles, long long ctot, int stage,
                                               double dt_all, const double* __restrict__ fx, long long fxt,
                                               const double* __restrict__ fy, long long fyt, double gam) {
  using O = Off<N>;
  constexpr int V = nv_of(2, PDE), NP = np_of(2, N), Q = N + 1;
  const Tile tile = tiles[blockIdx.x];
  const Inst I = insts[tile.inst];
  const int ix = tile.x0 + (threadIdx.x & 31), iy = tile.y0 + (threadIdx.x >> 5);
  if (ix >= I.nx || iy >= I.ny) return;
  const long long g = I.off + (long long)iy * I.nx + ix;
  const double gm1 = gam - 1.0, hgm1 = -0.5 * gm1;
  // Euler P3 keeps the cell's modes in shared memory (one slot per thread and mode: no
  // sharing, no barrier), which leaves the registers to the sum factorisation
  constexpr bool kSmemU = PDE == 1 && N == 3;
  extern __shared__ double s_u[];
  double u[V][NP];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      const double x = __ldg(us + (long long)(v * NP + m) * ctot + g);
      if constexpr (kSmemU) s_u[(v * NP + m) * 256 + threadIdx.x] = x;
      else u[v][m] = x;
    }
  // volume term, unscaled: X_ab = sum_q w w f psi_a' psi_b (a >= 1), Y_ab likewise with g (b >= 1),
  // sum-factorised: for every x point the column sums over y, then the x weights
  double X[V][NP], Y[V][NP];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) X[v][m] = Y[v][m] = 0.0;
  if constexpr (kSmemU) {
#pragma unroll
    for (int qx = 0; qx < Q; ++qx) {
      double tb[V][N + 1];
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int b = 0; b <= N; ++b) {
          // t_b over psi_0 (see eval_gauss2): the constant term needs no multiplication
          double t = s_u[(v * NP + mode_idx(0, b)) * 256 + threadIdx.x];
#pragma unroll
          for (int a = 1; a <= N - b; ++a)
            t = fma(s_u[(v * NP + mode_idx(a, b)) * 256 + threadIdx.x], T(O::KQ + qx * (N + 1) + a), t);
          tb[v][b] = t;
        }
      double col[V][Q];  // twice u at (x_qx, y_qy)
#pragma unroll
      for (int v = 0; v < V; ++v) {
        double val[Q];
        eval_gauss2<N>(tb[v], val);
#pragma unroll
        for (int qy = 0; qy < Q; ++qy) col[v][qy] = val[qy];
      }
      // column sums over symmetric pairs of y points: G_b = sum_y w psi_b(y) f (b < N),
      // H_b = sum_y w psi_b'(y) g (b >= 1), stored at H[b - 1]; Q = N + 1 is even here
      static_assert((Q & 1) == 0, "P3: no middle point");
      double G[V][N], H[V][N];
#pragma unroll
      for (int qp = 0; qp < Q / 2; ++qp) {
        double fA[V], gA[V], fB[V], gB[V];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const int qy = side == 0 ? qp : Q - 1 - qp;
          const double rho = col[0][qy], mx = col[1][qy], my = col[2][qy], E = col[3][qy];
          const double r = rcp_d(rho);
          const double vx = mx * r, vy = my * r;
          const double p = fma(hgm1, fma(mx, vx, my * vy), gm1 * E);  // (gamma-1)(E - rho |v|^2 / 2)
          const double ep = E + p;
          double* f = side == 0 ? fA : fB;
          double* gg = side == 0 ? gA : gB;
          f[0] = mx;
          f[1] = fma(mx, vx, p);
          f[2] = my * vx;
          f[3] = ep * vx;
          gg[0] = my;
          gg[1] = f[2];
          gg[2] = fma(my, vy, p);
          gg[3] = ep * vy;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const double fS = fA[v] + fB[v], fD = fA[v] - fB[v], gS = gA[v] + gB[v], gD = gA[v] - gB[v];
#pragma unroll
          for (int b = 0; b < N; ++b) {
            const double x = (b & 1) ? fD : fS;
            G[v][b] = qp == 0 ? x * T(O::WPQ + b) : fma(x, T(O::WPQ + qp * (N + 1) + b), G[v][b]);
          }
#pragma unroll
          for (int b = 1; b <= N; ++b) {
            const double x = (b & 1) ? gS : gD;
            H[v][b - 1] = qp == 0 ? x * T(O::WDQ + b) : fma(x, T(O::WDQ + qp * (N + 1) + b), H[v][b - 1]);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
#pragma unroll
        for (int b = 0; b < N; ++b)
#pragma unroll
          for (int a = 1; a <= N - b; ++a)
            X[v][mode_idx(a, b)] = fma(T(O::WDQ + qx * (N + 1) + a), G[v][b], X[v][mode_idx(a, b)]);
#pragma unroll
        for (int b = 1; b <= N; ++b)
#pragma unroll
          for (int a = 0; a <= N - b; ++a)
            Y[v][mode_idx(a, b)] = fma(T(O::WPQ + qx * (N + 1) + a), H[v][b - 1], Y[v][mode_idx(a, b)]);
      }
    }
  } else {
    // x points in symmetric pairs (t_b formed once per pair).  Euler P3 takes the direct
    // form (one quadrature point at a time), which needs fewer registers.
    constexpr bool kPair = true;
    constexpr int NX = (Q + 1) / 2;
  #pragma unroll
    for (int qp = 0; qp < NX; ++qp) {
      // t_b(x) = sum_a U_ab psi_a(x) at the pair of points x_qp and x_{Q-1-qp} = -x_qp (parts
      // even and odd in a), or at one point (for the middle point 0, psi_a vanishes for odd a)
      const bool single = !kPair || ((Q & 1) && qp == Q / 2);
      const bool zero = (Q & 1) && qp == Q / 2;
      double tb[2][V][N + 1];
  #pragma unroll
      for (int v = 0; v < V; ++v)
  #pragma unroll
        for (int b = 0; b <= N; ++b) {
          // over psi_0 (see eval_gauss2): the constant term needs no multiplication
          double ev = u[v][mode_idx(0, b)], od = 0.0;
  #pragma unroll
          for (int a = 1; a <= N - b; ++a) {
            if (a & 1) {
              if (zero) continue;
              if (single) ev = fma(u[v][mode_idx(a, b)], T(O::KQ + qp * (N + 1) + a), ev);
              else od = a == 1 ? u[v][mode_idx(a, b)] * T(O::KQ + qp * (N + 1) + a)
                               : fma(u[v][mode_idx(a, b)], T(O::KQ + qp * (N + 1) + a), od);
            } else {
              ev = fma(u[v][mode_idx(a, b)], T(O::KQ + qp * (N + 1) + a), ev);
            }
          }
          const bool has_od = !single && b < N;
          tb[0][v][b] = has_od ? ev + od : ev;
          tb[1][v][b] = has_od ? ev - od : ev;
        }
  #pragma unroll
      for (int side = 0; side < 2; ++side) {
        if (single && side == 1) break;
        const int qx = side == 0 ? qp : Q - 1 - qp;
        const bool mid = (Q & 1) && qx == Q / 2;
        double col[V][Q];  // twice u at (x_qx, y_qy) for every qy
  #pragma unroll
        for (int v = 0; v < V; ++v) {
          double val[Q];
          eval_gauss2<N>(tb[side][v], val);
  #pragma unroll
          for (int qy = 0; qy < Q; ++qy) col[v][qy] = val[qy];
        }
        double F[Q][V], Gq[Q][V];
  #pragma unroll
        for (int qy = 0; qy < Q; ++qy) {
          if constexpr (PDE == 0) {
            const double h = 0.5 * col[0][qy] * col[0][qy];
            F[qy][0] = h;
            Gq[qy][0] = h;
          } else {
            const double rho = col[0][qy], mx = col[1][qy], my = col[2][qy], E = col[3][qy];
            const double r = rcp_d(rho);
            const double vx = mx * r, vy = my * r;
            const double p = fma(hgm1, fma(mx, vx, my * vy), gm1 * E);  // (gamma-1)(E - rho |v|^2 / 2)
            const double ep = E + p;
            F[qy][0] = mx;
            F[qy][1] = fma(mx, vx, p);
            F[qy][2] = my * vx;
            F[qy][3] = ep * vx;
            Gq[qy][0] = my;
            Gq[qy][1] = F[qy][2];
            Gq[qy][2] = fma(my, vy, p);
            Gq[qy][3] = ep * vy;
          }
        }
  #pragma unroll
        for (int v = 0; v < V; ++v) {
          // sums and differences over the symmetric pairs of y points
          double fS[Q / 2 + 1], fD[Q / 2 + 1], gS[Q / 2 + 1], gD[Q / 2 + 1];
  #pragma unroll
          for (int q = 0; q < Q / 2; ++q) {
            fS[q] = F[q][v] + F[Q - 1 - q][v];
            fD[q] = F[q][v] - F[Q - 1 - q][v];
            gS[q] = Gq[q][v] + Gq[Q - 1 - q][v];
            gD[q] = Gq[q][v] - Gq[Q - 1 - q][v];
          }
          // x derivative part: G_b = sum_y w psi_b(y) f (psi_b has the parity of b)
  #pragma unroll
          for (int b = 0; b < N; ++b) {
            double G = 0.0;
  #pragma unroll
            for (int q = 0; q < Q / 2; ++q)
              G = q == 0 ? ((b & 1) ? fD[0] : fS[0]) * T(O::WPQ + b)
                         : fma((b & 1) ? fD[q] : fS[q], T(O::WPQ + q * (N + 1) + b), G);
            if ((Q & 1) && !(b & 1)) G = fma(F[Q / 2][v], T(O::WPQ + (Q / 2) * (N + 1) + b), G);
  #pragma unroll
            for (int a = 1; a <= N - b; ++a) {
              if (mid && !(a & 1)) continue;  // psi_a'(0) = 0 for even a
              X[v][mode_idx(a, b)] = fma(T(O::WDQ + qx * (N + 1) + a), G, X[v][mode_idx(a, b)]);
            }
          }
          // y derivative part: H_b = sum_y w psi_b'(y) g (psi_b' has the parity of b + 1)
  #pragma unroll
          for (int b = 1; b <= N; ++b) {
            double H = 0.0;
  #pragma unroll
            for (int q = 0; q < Q / 2; ++q)
              H = q == 0 ? ((b & 1) ? gS[0] : gD[0]) * T(O::WDQ + b)
                         : fma((b & 1) ? gS[q] : gD[q], T(O::WDQ + q * (N + 1) + b), H);
            if ((Q & 1) && (b & 1)) H = fma(Gq[Q / 2][v], T(O::WDQ + (Q / 2) * (N + 1) + b), H);
  #pragma unroll
            for (int a = 0; a <= N - b; ++a) {
              if (mid && (a & 1)) continue;  // psi_a(0) = 0 for odd a
              Y[v][mode_idx(a, b)] = fma(T(O::WPQ + qx * (N + 1) + a), H, Y[v][mode_idx(a, b)]);
            }
          }
        }
      }
    }
  }
  // acc = (2/hx) X + (2/hy) Y - (1/hx) psi_a(1) [P_b(E) -+ P_b(W)] - (1/hy) psi_b(1) [P_a(N) -+ P_a(S)],
  // where X, Y and the P_b were formed from doubled states: the scalings take 2^-d (exact)
  constexpr double kHom = PDE == 1 ? 0.5 : 0.25;
  const double sx = (2.0 / I.hx) * kHom, sy = (2.0 / I.hy) * kHom, ihx = 0.5 * sx, ihy = 0.5 * sy;
  double cx[N + 1], cy[N + 1];
#pragma unroll
  for (int n = 0; n <= N; ++n) {
    cx[n] = -ihx * T(O::P1 + n);
    cy[n] = -ihy * T(O::P1 + n);
  }
  const double* const pw = fx + I.fx + (long long)iy * (I.nx + 1) + ix;  // west face; east = pw + 1
  const double* const ps = fy + I.fy + (long long)iy * I.nx + ix;        // south face; north = ps + nx
  const double dt = dt_all > 0.0 ? dt_all : I.dt;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    double acc[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      const bool hx_ = mode_a(m) >= 1, hy_ = mode_b(m) >= 1;
      acc[m] = hx_ ? (hy_ ? fma(sx, X[v][m], sy * Y[v][m]) : sx * X[v][m]) : (hy_ ? sy * Y[v][m] : 0.0);
    }
#pragma unroll
    for (int b = 0; b <= N; ++b) {
      const long long pl = (long long)(v * (N + 1) + b);
      const double PW = __ldg(pw + pl * fxt), PE = __ldg(pw + pl * fxt + 1);
      const double PS = __ldg(ps + pl * fyt), PN = __ldg(ps + pl * fyt + I.nx);
      const double Dx = PE - PW, Sx = PE + PW, Dy = PN - PS, Sy = PN + PS;
#pragma unroll
      for (int a = 0; a <= N - b; ++a) {
        const int mx = mode_idx(a, b);  // x faces: normal degree a, transverse degree b
        acc[mx] = fma(cx[a], (a & 1) ? Sx : Dx, acc[mx]);
        const int my = mode_idx(b, a);  // y faces: transverse degree b (in x), normal a
        acc[my] = fma(cy[a], (a & 1) ? Sy : Dy, acc[my]);
      }
    }
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      const long long idx = (long long)(v * NP + m) * ctot + g;
      const double e = fma(dt, acc[m], us[idx]);
      double r;
      if (stage == 1) r = e;
      else if (stage == 2) r = fma(0.75, un[idx], 0.25 * e);
      else r = fma(1.0 / 3.0, un[idx], (2.0 / 3.0) * e);
      out[idx] = r;
    }
  }
}

// ----------------------------------------------------------------------------- indicator
// TVB modified minmod (Cockburn-Shu) on conserved variables, x test on the east/west
// edge midpoints and y test on the north/south ones.  The face values and means are
// formed without fused multiply-adds and in the order of a plain serial sum over the
// modes, so the decision is reproducible bit for bit; products whose table factor is
// exactly zero (psi_b(0) for odd b) are skipped, which leaves every partial sum unchanged.

template <int PDE, int N>
__global__ void __launch_bounds__(256)
    k_flag2(const double* __restrict__ U, const Inst* __restrict__ insts, const Tile* __restrict__ tiles,
            long long ctot, int bc, double M, unsigned char* __restrict__ flags, Counters* cnt,
            int* __restrict__ list_cell, int* __restrict__ list_inst, const double* __restrict__ bcd) {
  using O = Off<N>;
  constexpr int V = nv_of(2, PDE), NP = np_of(2, N);
  const Tile tile = tiles[blockIdx.x];
  const Inst I = insts[tile.inst];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ix = tile.x0 + lane, iy = tile.y0 + w;
  const bool active = ix < I.nx && iy < I.ny;
  const double c00 = T(O::C00);
  int fl = 0;
  bool near = false;
  long long g = active ? I.off + (long long)iy * I.nx + ix : 0;
  // every cell's means go to shared memory once; the neighbours inside the tile read them
  // there, those outside it (and ghosts) form them from their U_00 as before
  __shared__ double s_mean[V][TY][TX];
  if (active) {
#pragma unroll
    for (int v = 0; v < V; ++v) s_mean[v][w][lane] = __dmul_rn(__ldg(U + (long long)(v * NP) * ctot + g), c00);
  }
  __syncthreads();
  if (active) {
    // neighbour cells (outflow ghosts have the boundary cell's mean)
    auto nb = [&](int jx, int jy) -> long long {
      if (bc == 0) {
        jx = jx < 0 ? jx + I.nx : (jx >= I.nx ? jx - I.nx : jx);
        jy = jy < 0 ? jy + I.ny : (jy >= I.ny ? jy - I.ny : jy);
      } else {
        jx = jx < 0 ? 0 : (jx >= I.nx ? I.nx - 1 : jx);
        jy = jy < 0 ? 0 : (jy >= I.ny ? I.ny - 1 : jy);
      }
      return I.off + (long long)jy * I.nx + jx;
    };
    const long long gW = nb(ix - 1, iy), gE = nb(ix + 1, iy), gS = nb(ix, iy - 1), gN = nb(ix, iy + 1);
    const bool inW = lane > 0, inE = lane < TX - 1 && ix + 1 < I.nx;
    const bool inS = w > 0, inN = w < TY - 1 && iy + 1 < I.ny;
    // kBcDmr: the neighbours' U_00 (W, E, S, N) follow dmr_ghost where they lie outside
    // (decided again per variable: only boundary cells of such meshes take this path)
    const bool dmr = bc == kBcDmr && (ix == 0 || iy == 0 || ix == I.nx - 1 || iy == I.ny - 1);
    auto nb_u00 = [&](int k, const double* P, long long gk, int v) -> double {
      if (!dmr) return __ldg(P + gk);
      const int jx = ix + (k == 0 ? -1 : (k == 1 ? 1 : 0)), jy = iy + (k == 2 ? -1 : (k == 3 ? 1 : 0));
      if (jx >= 0 && jx < I.nx && jy >= 0 && jy < I.ny) return __ldg(P + gk);
      const Ghost gh = dmr_ghost(I, tile.inst, jx, jy, bcd, dmr_time(bcd, tile.inst, 0));
      if (gh.c) return 2.0 * gh.c[v];
      return neg_if(__ldg(P + I.off + (long long)gh.jy * I.nx + gh.jx), gh.fv && v == 2);
    };
    const long long mx2 = __double_as_longlong(M * I.hx * I.hx), my2 = __double_as_longlong(M * I.hy * I.hy);
#pragma unroll 1
    for (int v = 0; v < V; ++v) {  // one variable at a time keeps the kernel at 4 blocks per SM
      const double* P = U + (long long)(v * NP) * ctot;
      const double mean = s_mean[v][w][lane];
      const double mW = inW ? s_mean[v][w][lane - 1] : __dmul_rn(nb_u00(0, P, gW, v), c00);
      const double mE = inE ? s_mean[v][w][lane + 1] : __dmul_rn(nb_u00(1, P, gE, v), c00);
      const double mS = inS ? s_mean[v][w - 1][lane] : __dmul_rn(nb_u00(2, P, gS, v), c00);
      const double mN = inN ? s_mean[v][w + 1][lane] : __dmul_rn(nb_u00(3, P, gN, v), c00);
      // the serial sums start from their first term (0 + x = x up to the sign of a zero,
      // which no decision below depends on)
      double uE = 0.0, uW = 0.0, uN = 0.0, uS = 0.0;
      bool firstE = true, firstN = true;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const int a = mode_a(m), b = mode_b(m);
        const double ck = __ldg(P + (long long)m * ctot + g);
        if (!(b & 1)) {  // psi_b(0) != 0: east/west products (west = (-1)^a east)
          const double pe = __dmul_rn(ck, T(O::TE + m));
          uE = firstE ? pe : __dadd_rn(uE, pe);
          uW = firstE ? ((a & 1) ? -pe : pe) : ((a & 1) ? __dsub_rn(uW, pe) : __dadd_rn(uW, pe));
          firstE = false;
        }
        if (!(a & 1)) {  // psi_a(0) != 0: north/south products (south = (-1)^b north)
          const double pn = __dmul_rn(ck, T(O::TN + m));
          uN = firstN ? pn : __dadd_rn(uN, pn);
          uS = firstN ? ((b & 1) ? -pn : pn) : ((b & 1) ? __dsub_rn(uS, pn) : __dadd_rn(uS, pn));
          firstN = false;
        }
      }
      const double dpx = __dsub_rn(mE, mean), dmx = __dsub_rn(mean, mW);
      const double dpy = __dsub_rn(mN, mean), dmy = __dsub_rn(mean, mS);
      fl |= tvb_changes_bits(__dsub_rn(uE, mean), dpx, dmx, mx2, near);
      fl |= tvb_changes_bits(__dsub_rn(mean, uW), dpx, dmx, mx2, near);
      fl |= tvb_changes_bits(__dsub_rn(uN, mean), dpy, dmy, my2, near);
      fl |= tvb_changes_bits(__dsub_rn(mean, uS), dpy, dmy, my2, near);
    }
    flags[g] = (unsigned char)(fl | (near ? 2 : 0));  // bit 0 troubled, bit 1 near threshold
  }
  block_compact(fl, near ? 1 : 0, g, tile.inst, cnt, list_cell, list_inst);
}

// ----------------------------------------------------------------------------- limiter
// One WENO reconstruction (Sec. 3, Steps 2-5) from the 2N+1 stencil averages to the NG
// Step 1 points.  Eq. (14) read as wbar_i = gamma_i / (eps + beta_i)^2; where a linear
// weight is negative (P3) the split gamma = sigma+ gamma~+ - sigma- gamma~- of Shi, Hu and
// Shu is used, each part normalised separately.
template <int N>
__device__ __forceinline__ void weno(const double* avg, double* out) {
  using O = Off<N>;
  constexpr int N1 = N + 1, NG = O::NG;
  const double eps = 1e-6;
  // p_i - c does not change when a constant c is removed from all averages (constants are
  // reproduced): work on averages centred at the troubled cell's own
  const double c = avg[N];
  double dv[2 * N + 1];
#pragma unroll
  for (int k = 0; k < 2 * N + 1; ++k) dv[k] = avg[k] - c;
  // Eq. (13) holds only derivatives, so beta_i is a quadratic form in the differences of
  // the stencil's averages: beta_i = sum_j df_{i+j} sum_{j' >= j} Md_jj' df_{i+j'};
  // inv_i = 1 / (eps + beta_i)^2
  constexpr int ND = N * N1 / 2;
  double df[2 * N];
#pragma unroll
  for (int k = 0; k < 2 * N; ++k) df[k] = avg[k + 1] - avg[k];
  double inv[N1];
#pragma unroll
  for (int i = 0; i < N1; ++i) {
    double beta = 0.0;
    int j = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double r = T(O::BD + i * ND + j) * df[i + k];
      ++j;
#pragma unroll
      for (int l = k + 1; l < N; ++l, ++j) r = fma(T(O::BD + i * ND + j), df[i + l], r);
      beta = k == 0 ? df[i] * r : fma(df[i + k], r, beta);
    }
    const double d = eps + beta;
    inv[i] = rcp_d(d * d);
  }
  // Eqs. (14)-(15): u_g = c + sum_i wbar_i (p_i - c) / sum_i wbar_i, wbar_i = gamma_gi inv_i;
  // with the linear weights folded into the reconstruction tables (WCG = gamma_gi C_igk)
  // the numerator is sum_i inv_i (gamma_gi (p_i - c))
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    if (T(O::NEG + g) == 0.0) {
      double sw = 0.0, su = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        double s = T(O::WCG + (i * NG + g) * N1) * dv[i];
#pragma unroll
        for (int k = 1; k < N1; ++k) s = fma(T(O::WCG + (i * NG + g) * N1 + k), dv[i + k], s);
        sw = i == 0 ? T(O::GAM + g * N1) * inv[0] : fma(T(O::GAM + g * N1 + i), inv[i], sw);
        su = i == 0 ? inv[0] * s : fma(inv[i], s, su);
      }
      out[g] = fma(su, rcp_d(sw), c);
    } else {
      double p[N1];
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        double s = T(O::WC + (i * NG + g) * N1) * dv[i];
#pragma unroll
        for (int k = 1; k < N1; ++k) s = fma(T(O::WC + (i * NG + g) * N1 + k), dv[i + k], s);
        p[i] = s;
      }
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
      // sigma+ - sigma- = 1: the constant c passes through the split unchanged
      out[g] = c + (T(O::SGP + g) * (sup * rcp_d(swp)) - T(O::SGM + g) * (sum * rcp_d(swm)));
    }
  }
}

// Right/left eigenvectors of the 2D Euler flux Jacobian in direction dir at state u.
__device__ __forceinline__ void euler_eig2(const double* u, int dir, double gam, double (&R)[4][4],
                                           double (&L)[4][4]) {
  const double rho = u[0], r = rcp_d(rho);
  const double vx = u[1] * r, vy = u[2] * r, q2 = vx * vx + vy * vy;
  const double p = (gam - 1.0) * (u[3] - 0.5 * rho * q2);
  const double c = sqrt_d(gam * p * r), ic = rcp_d(c);
  const double H = (u[3] + p) * r;
  const double b1 = (gam - 1.0) * ic * ic, b2 = 0.5 * b1 * q2;
  const double vn = dir == 0 ? vx : vy, vt = dir == 0 ? vy : vx;
  const int in = dir == 0 ? 1 : 2, it = dir == 0 ? 2 : 1;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { R[i][j] = 0.0; L[i][j] = 0.0; }
  R[0][0] = 1.0; R[in][0] = vn - c; R[it][0] = vt; R[3][0] = H - vn * c;
  R[0][1] = 1.0; R[in][1] = vn;     R[it][1] = vt; R[3][1] = 0.5 * q2;
  R[it][2] = 1.0; R[3][2] = vt;
  R[0][3] = 1.0; R[in][3] = vn + c; R[it][3] = vt; R[3][3] = H + vn * c;
  L[0][0] = 0.5 * (b2 + vn * ic); L[0][in] = -0.5 * (b1 * vn + ic); L[0][it] = -0.5 * b1 * vt; L[0][3] = 0.5 * b1;
  L[1][0] = 1.0 - b2;             L[1][in] = b1 * vn;               L[1][it] = b1 * vt;        L[1][3] = -b1;
  L[2][0] = -vt;                  L[2][it] = 1.0;
  L[3][0] = 0.5 * (b2 - vn * ic); L[3][in] = 0.5 * (ic - b1 * vn);  L[3][it] = -0.5 * b1 * vt; L[3][3] = 0.5 * b1;
}

// CSWENO on the listed cells; thread i handles list entry i.  Output: the limited modes
// 1..NP-1 in list order (lim[(v*NP + m) * cap + i]).
template <int PDE, int N>
__global__ void __launch_bounds__(128)
    k_limit2(const double* __restrict__ U, const Inst* __restrict__ insts, long long ctot, int bc,
             const int* __restrict__ list_cell, const int* __restrict__ list_inst, const Counters* __restrict__ cnt,
             double* __restrict__ lim, long long cap, double gam) {
  using O = Off<N>;
  constexpr int V = nv_of(2, PDE), NP = np_of(2, N), NS = O::NS, NG = O::NG, N1 = N + 1;
  const unsigned int n = cnt->n_flag;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long g = list_cell[i];
    const Inst I = insts[list_inst[i]];
    const int loc = (int)(g - I.off);
    const int ix = loc % I.nx, iy = loc / I.nx;
    // (2N+1)^2 sub-rectangle averages of the 3x3 neighbourhood (Fig. 1 in each direction)
    double avg[V][NS][NS];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        double u[V][NP];
        load_cell<V, NP>(U, ctot, I, ix + dx, iy + dy, bc, u);
        constexpr int k0[3] = {0, N, N + 1};
        constexpr int kn[3] = {N, 1, N};
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int kx = k0[dx + 1]; kx < k0[dx + 1] + kn[dx + 1]; ++kx) {
            double t[N1];  // t_b = sum_a U_ab SA[kx][a]
#pragma unroll
            for (int b = 0; b <= N; ++b) {
              double s = 0.0;
#pragma unroll
              for (int a = 0; a <= N - b; ++a) s = fma(u[v][mode_idx(a, b)], T(O::SA + kx * N1 + a), s);
              t[b] = s;
            }
#pragma unroll
            for (int ky = k0[dy + 1]; ky < k0[dy + 1] + kn[dy + 1]; ++ky) {
              double s = 0.0;
#pragma unroll
              for (int b = 0; b <= N; ++b) s = fma(t[b], T(O::SA + ky * N1 + b), s);
              avg[v][ky][kx] = s;
            }
          }
      }
    // x sweep: rowval[v][ky][g] = average over row ky of u(x_g, y)
    double rowv[V][NS][NG];
    double pv[V][NG][NG];  // [v][gy][gx]
    if constexpr (PDE == 1) {
      double mean[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) mean[v] = __ldg(U + (long long)(v * NP) * ctot + g) * T(O::C00);
      double R[4][4], L[4][4];
      euler_eig2(mean, 0, gam, R, L);
#pragma unroll
      for (int ky = 0; ky < NS; ++ky) {
        double wv[4][NG];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          double wc[NS];
#pragma unroll
          for (int kx = 0; kx < NS; ++kx) {
            double s = 0.0;
#pragma unroll
            for (int v = 0; v < 4; ++v)
              s = fma(L[f][v], avg[v][ky][kx], s);
            wc[kx] = s;
          }
          weno<N>(wc, wv[f]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
          for (int q = 0; q < NG; ++q) {
            double s = 0.0;
#pragma unroll
            for (int f = 0; f < 4; ++f) s = fma(R[v][f], wv[f][q], s);
            rowv[v][ky][q] = s;
          }
      }
      euler_eig2(mean, 1, gam, R, L);
#pragma unroll
      for (int gx = 0; gx < NG; ++gx) {
        double wv[4][NG];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          double wc[NS];
#pragma unroll
          for (int ky = 0; ky < NS; ++ky) {
            double s = 0.0;
#pragma unroll
            for (int v = 0; v < 4; ++v) s = fma(L[f][v], rowv[v][ky][gx], s);
            wc[ky] = s;
          }
          weno<N>(wc, wv[f]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
          for (int gy = 0; gy < NG; ++gy) {
            double s = 0.0;
#pragma unroll
            for (int f = 0; f < 4; ++f) s = fma(R[v][f], wv[f][gy], s);
            pv[v][gy][gx] = s;
          }
      }
    } else {
#pragma unroll
      for (int ky = 0; ky < NS; ++ky) weno<N>(avg[0][ky], rowv[0][ky]);
#pragma unroll
      for (int gx = 0; gx < NG; ++gx) {
        double col[NS], r[NG];
#pragma unroll
        for (int ky = 0; ky < NS; ++ky) col[ky] = rowv[0][ky][gx];
        weno<N>(col, r);
#pragma unroll
        for (int gy = 0; gy < NG; ++gy) pv[0][gy][gx] = r[gy];
      }
    }
    // Step 6 (Eq. (16)) with the tensor rule: U_ab = sum w_gx w_gy u psi_a(x_gx) psi_b(y_gy)
#pragma unroll
    for (int v = 0; v < V; ++v) {
      double tq[NG][N1];  // tq[gy][a] = sum_gx w_gx psi_a(x_gx) pv[gy][gx]
#pragma unroll
      for (int gy = 0; gy < NG; ++gy)
#pragma unroll
        for (int a = 0; a <= N; ++a) {
          double s = 0.0;
#pragma unroll
          for (int gx = 0; gx < NG; ++gx) s = fma(T(O::WPG + gx * N1 + a), pv[v][gy][gx], s);
          tq[gy][a] = s;
        }
#pragma unroll
      for (int m = 1; m < NP; ++m) {
        const int a = mode_a(m), b = mode_b(m);
        double s = 0.0;
#pragma unroll
        for (int gy = 0; gy < NG; ++gy) s = fma(T(O::WPG + gy * N1 + b), tq[gy][a], s);
        lim[(long long)(v * NP + m) * cap + i] = s;
      }
    }
  }
}


// CSWENO for 2D Euler with four lanes per troubled cell (8 cells per warp).  Lane q of a
// quad owns conserved variable q for the subcell averages and the projection, and
// characteristic field q in the two sweeps; the quad exchanges values with shuffles, so
// all lanes run the same FP64 instruction stream (the FP64 pipe is the bottleneck) while
// each thread holds a quarter of the per-cell state.  With a work counter (lq, zero at
// launch) every warp takes its next 8 cells from it, so the work spreads evenly over the
// resident warps whatever the grid; without one the warps stride over the list.
template <int N>
__global__ void __launch_bounds__(128)
    k_limit2_euler_quad(const double* __restrict__ U, const Inst* __restrict__ insts, long long ctot, int bc,
                        const int* __restrict__ list_cell, const int* __restrict__ list_inst,
                        const Counters* __restrict__ cnt, double* __restrict__ lim, long long cap, double gam,
                        unsigned int* __restrict__ lq, const double* __restrict__ bcd) {
  using O = Off<N>;
  constexpr int NP = np_of(2, N), NS = O::NS, NG = O::NG, N1 = N + 1;
  const unsigned int n = cnt->n_flag;
  const int lane = threadIdx.x & 31, q = lane & 3, qb = lane & ~3;
  const unsigned int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (unsigned int it = 0;; ++it) {
    unsigned int base;
    if (lq) {
      unsigned int b0 = 0;
      if (lane == 0) b0 = atomicAdd(lq, 8u);
      base = __shfl_sync(0xffffffffu, b0, 0);
    } else {
      base = (warp + it * nwarps) * 8u;
    }
    if (base >= n) break;
    const unsigned int i0 = base + (lane >> 2);
    const bool active = i0 < n;
    const unsigned int i = active ? i0 : n - 1;  // idle quads repeat a valid entry
    const long long g = list_cell[i];
    const int inst = list_inst[i];
    const Inst I = insts[inst];
    const int loc = (int)(g - I.off);
    const int ix = loc % I.nx, iy = loc / I.nx;
    // subcell averages of variable q
    double avg[NS][NS];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        int jx = ix + dx, jy = iy + dy;
        bool fx = false, fy = false, fv = false;
        const double* cst = nullptr;  // kBcDmr constant ghost
        if (bc == 0) {
          jx = jx < 0 ? jx + I.nx : (jx >= I.nx ? jx - I.nx : jx);
          jy = jy < 0 ? jy + I.ny : (jy >= I.ny ? jy - I.ny : jy);
        } else if (bc == kBcDmr && (jx < 0 || jx >= I.nx || jy < 0 || jy >= I.ny)) {
          const Ghost gh = dmr_ghost(I, inst, jx, jy, bcd, dmr_time(bcd, inst, 0));
          cst = gh.c;
          jx = gh.jx;
          jy = gh.jy;
          fx = gh.fx;
          fy = gh.fy;
          fv = gh.fv && q == 2;
          if (cst) { jx = 0; jy = 0; }
        } else {
          if (jx < 0) { jx = 0; fx = true; }
          if (jx >= I.nx) { jx = I.nx - 1; fx = true; }
          if (jy < 0) { jy = 0; fy = true; }
          if (jy >= I.ny) { jy = I.ny - 1; fy = true; }
        }
        const long long gj = I.off + (long long)jy * I.nx + jx;
        double u[NP];
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const double x = __ldg(U + (long long)(q * NP + m) * ctot + gj);
          const bool flip = ((fx && (mode_a(m) & 1)) != (fy && (mode_b(m) & 1))) != fv;
          u[m] = neg_if(x, flip);
          if (cst) u[m] = m == 0 ? 2.0 * cst[q] : 0.0;
        }
        constexpr int k0[3] = {0, N, N + 1};
        constexpr int kn[3] = {N, 1, N};
#pragma unroll
        for (int kx = k0[dx + 1]; kx < k0[dx + 1] + kn[dx + 1]; ++kx) {
          double t[N1];
#pragma unroll
          for (int b = 0; b <= N; ++b) {
            double sum = 0.0;
#pragma unroll
            for (int a = 0; a <= N - b; ++a) sum = fma(u[mode_idx(a, b)], T(O::SA + kx * N1 + a), sum);
            t[b] = sum;
          }
#pragma unroll
          for (int ky = k0[dy + 1]; ky < k0[dy + 1] + kn[dy + 1]; ++ky) {
            double sum = 0.0;
#pragma unroll
            for (int b = 0; b <= N; ++b) sum = fma(t[b], T(O::SA + ky * N1 + b), sum);
            avg[ky][kx] = sum;
          }
        }
      }
    // mean state of the troubled cell, gathered over the quad
    const double mq = __ldg(U + (long long)(q * NP) * ctot + g) * T(O::C00);
    double mean[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) mean[v] = __shfl_sync(0xffffffffu, mq, qb | v);
    double Lq[4], Rq[4];  // row q of the left and right eigenvector matrices
    auto rows_of = [&](int dir) {
      double R[4][4], L[4][4];
      euler_eig2(mean, dir, gam, R, L);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Lq[v] = q == 0 ? L[0][v] : (q == 1 ? L[1][v] : (q == 2 ? L[2][v] : L[3][v]));
        Rq[v] = q == 0 ? R[0][v] : (q == 1 ? R[1][v] : (q == 2 ? R[2][v] : R[3][v]));
      }
    };
    // x sweep: field q of each row, back to variable q at the NG x points
    rows_of(0);
    double rowv[NS][NG];
#pragma unroll
    for (int ky = 0; ky < NS; ++ky) {
      double w[NS], r[NG];
#pragma unroll
      for (int kx = 0; kx < NS; ++kx) {
        double s = 0.0;
#pragma unroll
        for (int v = 0; v < 4; ++v) s = fma(Lq[v], __shfl_sync(0xffffffffu, avg[ky][kx], qb | v), s);
        w[kx] = s;
      }
      weno<N>(w, r);
#pragma unroll
      for (int gx = 0; gx < NG; ++gx) {
        double s = 0.0;
#pragma unroll
        for (int f = 0; f < 4; ++f) s = fma(Rq[f], __shfl_sync(0xffffffffu, r[gx], qb | f), s);
        rowv[ky][gx] = s;
      }
    }
    // y sweep: field q of each x point's column, back to variable q at the NG y points
    rows_of(1);
    double pv[NG][NG];  // [gy][gx]
#pragma unroll
    for (int gx = 0; gx < NG; ++gx) {
      double w[NS], r[NG];
#pragma unroll
      for (int ky = 0; ky < NS; ++ky) {
        double s = 0.0;
#pragma unroll
        for (int v = 0; v < 4; ++v) s = fma(Lq[v], __shfl_sync(0xffffffffu, rowv[ky][gx], qb | v), s);
        w[ky] = s;
      }
      weno<N>(w, r);
#pragma unroll
      for (int gy = 0; gy < NG; ++gy) {
        double s = 0.0;
#pragma unroll
        for (int f = 0; f < 4; ++f) s = fma(Rq[f], __shfl_sync(0xffffffffu, r[gy], qb | f), s);
        pv[gy][gx] = s;
      }
    }
    // Step 6 for variable q (tensor Gauss / Gauss-Lobatto rule)
    double tq[NG][N1];
#pragma unroll
    for (int gy = 0; gy < NG; ++gy)
#pragma unroll
      for (int a = 0; a <= N; ++a) {
        double s = 0.0;
#pragma unroll
        for (int gx = 0; gx < NG; ++gx) s = fma(T(O::WPG + gx * N1 + a), pv[gy][gx], s);
        tq[gy][a] = s;
      }
    if (active) {
#pragma unroll
      for (int m = 1; m < NP; ++m) {
        const int a = mode_a(m), b = mode_b(m);
        double s = 0.0;
#pragma unroll
        for (int gy = 0; gy < NG; ++gy) s = fma(T(O::WPG + gy * N1 + b), tq[gy][a], s);
        lim[(long long)(q * NP + m) * cap + i] = s;
      }
    }
  }
}

// ----------------------------------------------------------------------------- projection
// Eq. (2) for the initial data: U_ab = sum_{qx,qy} w w u0(x, y) psi_a psi_b with N+4 Gauss
// points per direction.  Parameters per instance (see dg.h for the families).

template <int PDE, int N>
__global__ void k_project2(double* __restrict__ U, const Inst* __restrict__ insts, const int* __restrict__ cell_inst,
                           long long ncell, long long ctot, int kind, const double* __restrict__ params, int np,
                           double gam) {
  using O = Off<N>;
  constexpr int V = nv_of(2, PDE), NP = np_of(2, N), N1 = N + 1;
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const int ii = cell_inst[g];
  const Inst I = insts[ii];
  const int loc = (int)(g - I.off), ix = loc % I.nx, iy = loc / I.nx;
  const double* p = params + (long long)ii * np;
  const int QP = (int)T(O::PQP);
  double acc[V][NP];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) acc[v][m] = 0.0;
  for (int qy = 0; qy < QP; ++qy)
    for (int qx = 0; qx < QP; ++qx) {
      const double x = I.xL + I.hx * (ix + 0.5 * (1.0 + T(O::PX + qx)));
      const double y = I.yL + I.hy * (iy + 0.5 * (1.0 + T(O::PX + qy)));
      double u[V];
      ic_eval2(kind, p, x, y, gam, u);
      const double ww = T(O::PW + qx) * T(O::PW + qy);
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const double c = ww * T(O::PP + qx * N1 + mode_a(m)) * T(O::PP + qy * N1 + mode_b(m));
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v][m] = fma(c, u[v], acc[v][m]);
      }
    }
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) U[(long long)(v * NP + m) * ctot + g] = acc[v][m];
}

template <int PDE, int N>
__global__ void k_speed2(const double* __restrict__ U, const Inst* __restrict__ insts, const int* __restrict__ cell_inst,
                         long long ncell, long long ctot, double gam, double* out) {
  using O = Off<N>;
  constexpr int V = nv_of(2, PDE), NP = np_of(2, N);
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  double u[V];
  for (int v = 0; v < V; ++v) u[v] = U[(long long)(v * NP) * ctot + g] * T(O::C00);
  double sx, sy;
  if constexpr (PDE == 0) {
    sx = sy = fabs(u[0]);
  } else {
    const double r = 1.0 / u[0], vx = u[1] * r, vy = u[2] * r;
    const double p = (gam - 1.0) * (u[3] - 0.5 * u[0] * (vx * vx + vy * vy));
    const double c = sqrt(gam * p * r);
    sx = fabs(vx) + c;
    sy = fabs(vy) + c;
  }
  const int ii = cell_inst[g];
  atomic_max_nonneg(out + 2 * ii, sx);
  atomic_max_nonneg(out + 2 * ii + 1, sy);
}

#undef T

}  // namespace k2

// ----------------------------------------------------------------------------- host side

cudaError_t upload_tables2(const dgt::Tabs* tabs /* [3] for N = 1..3 */) {
  static double h[k2::kTabSize];
  for (int i = 0; i < k2::kTabSize; ++i) h[i] = 0.0;
  k2::pack<1>(tabs[0], h);
  k2::pack<2>(tabs[1], h);
  k2::pack<3>(tabs[2], h);
  return cudaMemcpyToSymbol(k2::c_tab, h, sizeof(h));
}

#define DG_DISPATCH2(PDE, N, CALL) \
  do {                                                   \
    if ((PDE) == 0 && (N) == 1) { constexpr int P_ = 0, N_ = 1; CALL; } \
    else if ((PDE) == 0 && (N) == 2) { constexpr int P_ = 0, N_ = 2; CALL; } \
    else if ((PDE) == 0 && (N) == 3) { constexpr int P_ = 0, N_ = 3; CALL; } \
    else if ((PDE) == 1 && (N) == 1) { constexpr int P_ = 1, N_ = 1; CALL; } \
    else if ((PDE) == 1 && (N) == 2) { constexpr int P_ = 1, N_ = 2; CALL; } \
    else { constexpr int P_ = 1, N_ = 3; CALL; } \
  } while (0)

int stage_threads2(int tys) { return (tys + 3) * 32; }

template <int PDE, int N, int TYS>
static size_t stage_smem2() {
  constexpr int QV = (N + 1) * nv_of(2, PDE);
  return sizeof(double) * (size_t)(QV * TYS * (k2::TX + 1) + QV * (TYS + 1) * k2::TX);
}

template <int PDE, int N>
static cudaError_t prep_stage2() {
  // opt in to more than 48 KB of dynamic shared memory (set per device, outside captures)
  cudaError_t e = cudaFuncSetAttribute(k2::k_stage2<PDE, N, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)stage_smem2<PDE, N, 8>());
  if (e != cudaSuccess) return e;
  if (PDE == 1 && N == 3) {
    e = cudaFuncSetAttribute(k2::k_cell2<PDE, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * 4 * 10 * 256));
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k2::k_stage2<PDE, N, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)stage_smem2<PDE, N, 4>());
}

cudaError_t prepare2(int pde, int N) {
  cudaError_t e = cudaSuccess;
  DG_DISPATCH2(pde, N, (e = prep_stage2<P_, N_>()));
  return e;
}

template <int PDE, int N, int TYS>
static void run_stage2(const LaunchArgs& a, int stage, double dt_all, int* queue, int grid) {
  const size_t bytes = stage_smem2<PDE, N, TYS>();
  k2::k_stage2<PDE, N, TYS><<<queue ? grid : a.ntiles, (TYS + 3) * 32, bytes, a.st>>>(
      a.un, a.us, a.out, a.inst, a.tiles, a.ctot, a.bc, stage, dt_all, a.gam, a.ntiles, queue);
}
// dynamic shared memory of the cell pass: the modes of its 256 cells for Euler P3
static constexpr size_t cell_smem2(int pde, int N) {
  return pde == 1 && N == 3 ? sizeof(double) * 4 * 10 * 256 : 0;
}

// split form: the face pass over the face tiles, then the cell pass over the 32 x 8 cell tiles
void launch_stage2_split(int pde, int N, const LaunchArgs& a, int stage, double dt_all, const Tile* face_tiles,
                         int nface_tiles, double* fx, long long fxt, double* fy, long long fyt) {
  DG_DISPATCH2(pde, N, (k2::k_face2<P_, N_><<<nface_tiles, 128, 0, a.st>>>(a.us, a.inst, face_tiles, a.ctot, a.bc,
                                                                            a.gam, fx, fxt, fy, fyt, a.bcd, stage,
                                                                            dt_all)));
  DG_DISPATCH2(pde, N, (k2::k_cell2<P_, N_><<<a.ntiles, 256, cell_smem2(P_, N_), a.st>>>(a.un, a.us, a.out, a.inst, a.tiles, a.ctot,
                                                                         stage, dt_all, fx, fxt, fy, fyt, a.gam)));
}
int tile_w2() { return k2::TX; }
int tile_h2() { return k2::TY; }

// queue != null: persistent launch of `grid` blocks popping tiles from *queue (zeroed by the
// caller before the launch); otherwise one block per tile
void launch_stage2(int pde, int N, const LaunchArgs& a, int stage, double dt_all, int tys, int* queue, int grid) {
  if (tys == 4) DG_DISPATCH2(pde, N, (run_stage2<P_, N_, 4>(a, stage, dt_all, queue, grid)));
  else DG_DISPATCH2(pde, N, (run_stage2<P_, N_, 8>(a, stage, dt_all, queue, grid)));
}

void launch_flag2(int pde, int N, const LaunchArgs& a, double M, unsigned char* flags, Counters* cnt, int* lc,
                  int* li) {
  DG_DISPATCH2(pde, N, (k2::k_flag2<P_, N_><<<a.ntiles, 256, 0, a.st>>>(a.us, a.inst, a.tiles, a.ctot, a.bc, M,
                                                                          flags, cnt, lc, li, a.bcd)));
}

void launch_limit2(int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt,
                   double* lim, int nblocks) {
  if (pde == 1) {  // Euler: four lanes per troubled cell
    if (a.lq) cudaMemsetAsync(a.lq, 0, sizeof(unsigned int), a.st);
    if (N == 1) k2::k_limit2_euler_quad<1><<<nblocks, 128, 0, a.st>>>(a.us, a.inst, a.ctot, a.bc, lc, li, cnt, lim, a.cap, a.gam, a.lq, a.bcd);
    else if (N == 2) k2::k_limit2_euler_quad<2><<<nblocks, 128, 0, a.st>>>(a.us, a.inst, a.ctot, a.bc, lc, li, cnt, lim, a.cap, a.gam, a.lq, a.bcd);
    else k2::k_limit2_euler_quad<3><<<nblocks, 128, 0, a.st>>>(a.us, a.inst, a.ctot, a.bc, lc, li, cnt, lim, a.cap, a.gam, a.lq, a.bcd);
    return;
  }
  DG_DISPATCH2(pde, N, (k2::k_limit2<P_, N_><<<nblocks, 128, 0, a.st>>>(a.us, a.inst, a.ctot, a.bc, lc, li, cnt,
                                                                          lim, a.cap, a.gam)));
}

void launch_scatter2(int pde, int N, const LaunchArgs& a, const double* lim, const int* lc, const Counters* cnt,
                     int nblocks) {
  DG_DISPATCH2(pde, N, (k_scatter<nv_of(2, P_), np_of(2, N_)><<<nblocks, 256, 0, a.st>>>(
                           a.out, a.ctot, lim, a.cap, lc, cnt)));
}

void launch_project2(int pde, int N, const LaunchArgs& a, const int* cell_inst, int kind, const double* params,
                     int np) {
  const int nb = (int)((a.ncell + 127) / 128);
  DG_DISPATCH2(pde, N, (k2::k_project2<P_, N_><<<nb, 128, 0, a.st>>>(a.out, a.inst, cell_inst, a.ncell, a.ctot,
                                                                       kind, params, np, a.gam)));
}

void launch_speed2(int pde, int N, const LaunchArgs& a, const int* cell_inst, double* out) {
  const int nb = (int)((a.ncell + 255) / 256);
  DG_DISPATCH2(pde, N, (k2::k_speed2<P_, N_><<<nb, 256, 0, a.st>>>(a.us, a.inst, cell_inst, a.ncell, a.ctot,
                                                                     a.gam, out)));
}

}  // namespace dg
