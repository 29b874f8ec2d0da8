// Parent WENO limiter (Qiu and Shu, ref. [qs1]; the limiter the paper compares CSWENO
// with in Sec. 4): the reconstruction of Sec. 3, Steps 2-6, on the averages of the whole
// cells j-N .. j+N instead of subcells of the immediate neighbours.  In 2D: dimension by
// dimension on the (2N+1)^2 cell averages around the troubled cell (x sweep, then y sweep,
// tensor projection), characteristic fields with the x (y) Jacobian eigenvectors at the
// troubled cell's mean for Euler.  Outflow ghosts mirror the interior cell at the
// reflected position (ghost -1-k <-> cell k; a mirror image keeps the mean).
//
// One thread per listed (troubled) cell, the same compacted list and compact output
// buffer as the CSWENO kernels; the scatter kernel writes the result back (Jacobi).
// Only cell means are read from the neighbourhood: (2N+1)^dim cells x V values.
#include "dg_shared.cuh"
#include "tables.h"

namespace dg {
namespace pw {

struct PTab {
  double C[4][4][4];    // [stencil i][point g][k]: p_i(x_g) = sum_k C avg[i + k]
  double gam[4][4];     // [g][i] linear weights
  double B[4][4][4];    // [i][k][l]: beta_i = sum_kl avg[i+k] B avg[i+l]
  double gpn[4][4], gmn[4][4], sgp[4], sgm[4], neg[4];  // split of negative weights
  double pg[4][4];      // psi_n at the reconstruction points [g][n]
  double wg[4];         // their quadrature weights
  double psi0;          // psi_0 (cell mean = U_0 psi_0 in 1D, U_00 psi_0^2 in 2D)
};

__constant__ PTab c_pt[3];

__device__ __forceinline__ int reflect(int j, int n, int bc) {
  if (bc == 0) {
    j %= n;
    return j < 0 ? j + n : j;
  }
  if (j < 0) j = -1 - j;
  if (j >= n) j = 2 * n - 1 - j;
  return j < 0 ? 0 : (j >= n ? n - 1 : j);
}

// WENO at the reconstruction points from 2N+1 averages (Steps 2-5, Eq. (14)-(15); the
// Shi-Hu-Shu split where a linear weight is negative).  beta and p_i are evaluated on the
// averages centred at the troubled cell's own (exact: constants are reproduced and
// Eq. (13) holds only derivatives).
template <int N>
__device__ __forceinline__ void weno_p(const PTab& t, const double* avg, double* out) {
  constexpr int N1 = N + 1, NG = N == 1 ? 2 : 4;
  const double eps = 1e-6;
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
      for (int l = 0; l < N1; ++l) r = fma(t.B[i][k][l], dv[i + l], r);
      beta = fma(dv[i + k], r, beta);
    }
    const double d = eps + beta;
    inv[i] = rcp_d(d * d);
  }
  // u_g = c + sum_i wbar_i (p_i - c) / sum_i wbar_i
#pragma unroll
  for (int g = 0; g < NG; ++g) {
    double p[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < N1; ++k) s = fma(t.C[i][g][k], dv[i + k], s);
      p[i] = s;
    }
    if (t.neg[g] == 0.0) {
      double sw = 0.0, su = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        const double wb = t.gam[g][i] * inv[i];
        sw += wb;
        su = fma(wb, p[i], su);
      }
      out[g] = fma(su, rcp_d(sw), c);
    } else {
      double swp = 0.0, sup = 0.0, swm = 0.0, sum = 0.0;
#pragma unroll
      for (int i = 0; i < N1; ++i) {
        const double wp = t.gpn[g][i] * inv[i], wm = t.gmn[g][i] * inv[i];
        swp += wp;
        sup = fma(wp, p[i], sup);
        swm += wm;
        sum = fma(wm, p[i], sum);
      }
      // sigma+ - sigma- = 1: the constant c passes through the split unchanged
      out[g] = c + (t.sgp[g] * (sup * rcp_d(swp)) - t.sgm[g] * (sum * rcp_d(swm)));
    }
  }
}

// right (R) and left (L) eigenvectors of the Euler flux Jacobian at the mean state u:
// 1D (V = 3), or 2D (V = 4) in direction dir
template <int V>
__device__ __forceinline__ void eig(const double* u, int dir, double gam, double (&R)[V][V], double (&L)[V][V]) {
  const double rho = u[0], r = 1.0 / rho;
  const double vx = u[1] * r, vy = V == 4 ? u[2] * r : 0.0, q2 = vx * vx + vy * vy;
  const double p = (gam - 1.0) * (u[V - 1] - 0.5 * rho * q2);
  const double c = sqrt(gam * p * r), ic = 1.0 / c;
  const double H = (u[V - 1] + p) * r;
  const double b1 = (gam - 1.0) * ic * ic, b2 = 0.5 * b1 * q2;
#pragma unroll
  for (int i = 0; i < V; ++i)
#pragma unroll
    for (int j = 0; j < V; ++j) { R[i][j] = 0.0; L[i][j] = 0.0; }
  if constexpr (V == 3) {
    R[0][0] = 1.0; R[1][0] = vx - c; R[2][0] = H - vx * c;
    R[0][1] = 1.0; R[1][1] = vx;     R[2][1] = 0.5 * q2;
    R[0][2] = 1.0; R[1][2] = vx + c; R[2][2] = H + vx * c;
    L[0][0] = 0.5 * (b2 + vx * ic); L[0][1] = -0.5 * (b1 * vx + ic); L[0][2] = 0.5 * b1;
    L[1][0] = 1.0 - b2;             L[1][1] = b1 * vx;               L[1][2] = -b1;
    L[2][0] = 0.5 * (b2 - vx * ic); L[2][1] = 0.5 * (ic - b1 * vx);  L[2][2] = 0.5 * b1;
  } else {
    const double vn = dir == 0 ? vx : vy, vt = dir == 0 ? vy : vx;
    const int in = dir == 0 ? 1 : 2, it = dir == 0 ? 2 : 1;
    R[0][0] = 1.0; R[in][0] = vn - c; R[it][0] = vt; R[3][0] = H - vn * c;
    R[0][1] = 1.0; R[in][1] = vn;     R[it][1] = vt; R[3][1] = 0.5 * q2;
    R[it][2] = 1.0; R[3][2] = vt;
    R[0][3] = 1.0; R[in][3] = vn + c; R[it][3] = vt; R[3][3] = H + vn * c;
    L[0][0] = 0.5 * (b2 + vn * ic); L[0][in] = -0.5 * (b1 * vn + ic); L[0][it] = -0.5 * b1 * vt; L[0][3] = 0.5 * b1;
    L[1][0] = 1.0 - b2;             L[1][in] = b1 * vn;               L[1][it] = b1 * vt;        L[1][3] = -b1;
    L[2][0] = -vt;                  L[2][it] = 1.0;
    L[3][0] = 0.5 * (b2 - vn * ic); L[3][in] = 0.5 * (ic - b1 * vn);  L[3][it] = -0.5 * b1 * vt; L[3][3] = 0.5 * b1;
  }
}

// one sweep: averages a[v][k] (k over the 2N+1 stencil cells) -> point values o[v][g],
// in characteristic fields for Euler
template <int PDE, int V, int N>
__device__ __forceinline__ void sweep(const PTab& t, const double (&a)[V][2 * N + 1], const double (&R)[V][V],
                                      const double (&L)[V][V], double (&o)[V][N == 1 ? 2 : 4]) {
  constexpr int NS = 2 * N + 1, NG = N == 1 ? 2 : 4;
  if constexpr (PDE == 0) {
    weno_p<N>(t, a[0], o[0]);
  } else {
    double wv[V][NG];
#pragma unroll
    for (int f = 0; f < V; ++f) {
      double wc[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        double s = 0.0;
#pragma unroll
        for (int v = 0; v < V; ++v) s = fma(L[f][v], a[v][k], s);
        wc[k] = s;
      }
      weno_p<N>(t, wc, wv[f]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        double s = 0.0;
#pragma unroll
        for (int f = 0; f < V; ++f) s = fma(R[v][f], wv[f][g], s);
        o[v][g] = s;
      }
  }
}

template <int PDE, int N>
__global__ void __launch_bounds__(128)
    k_parent1(const double* __restrict__ U, const Inst* __restrict__ insts, long long ctot, int bc,
              const int* __restrict__ list_cell, const int* __restrict__ list_inst, const Counters* __restrict__ cnt,
              double* __restrict__ lim, long long cap, double gam) {
  constexpr int V = nv_of(1, PDE), N1 = N + 1, NS = 2 * N + 1, NG = N == 1 ? 2 : 4;
  const PTab& t = c_pt[N - 1];
  const unsigned int n = cnt->n_flag;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long g = list_cell[i];
    const Inst I = insts[list_inst[i]];
    const int ix = (int)(g - I.off);
    double a[V][NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      const long long c = I.off + reflect(ix + k - N, I.nx, bc);
#pragma unroll
      for (int v = 0; v < V; ++v) a[v][k] = U[(long long)(v * N1) * ctot + c] * t.psi0;
    }
    double R[V][V], L[V][V];
    if constexpr (PDE == 1) {
      double mean[V];
#pragma unroll
      for (int v = 0; v < V; ++v) mean[v] = a[v][N];
      eig<V>(mean, 0, gam, R, L);
    }
    double val[V][NG];
    sweep<PDE, V, N>(t, a, R, L, val);
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int m = 1; m < N1; ++m) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NG; ++q) s = fma(t.wg[q] * val[v][q], t.pg[q][m], s);
        lim[(long long)(v * N1 + m) * cap + i] = s;
      }
  }
}

template <int PDE, int N>
__global__ void __launch_bounds__(128)
    k_parent2(const double* __restrict__ U, const Inst* __restrict__ insts, long long ctot, int bc,
              const int* __restrict__ list_cell, const int* __restrict__ list_inst, const Counters* __restrict__ cnt,
              double* __restrict__ lim, long long cap, double gam) {
  constexpr int V = nv_of(2, PDE), NP = np_of(2, N), NS = 2 * N + 1, NG = N == 1 ? 2 : 4;
  const PTab& t = c_pt[N - 1];
  const unsigned int n = cnt->n_flag;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long g = list_cell[i];
    const Inst I = insts[list_inst[i]];
    const int loc = (int)(g - I.off);
    const int ix = loc % I.nx, iy = loc / I.nx;
    double Rx[V][V], Lx[V][V], Ry[V][V], Ly[V][V];
    if constexpr (PDE == 1) {
      double mean[V];
#pragma unroll
      for (int v = 0; v < V; ++v) mean[v] = U[(long long)(v * NP) * ctot + g] * t.psi0 * t.psi0;
      eig<V>(mean, 0, gam, Rx, Lx);
      eig<V>(mean, 1, gam, Ry, Ly);
    }
    // x sweep, row by row: rowv[v][ky][gx] = average over row ky of u(x_gx, y)
    double rowv[V][NS][NG];
#pragma unroll
    for (int ky = 0; ky < NS; ++ky) {
      const long long row = I.off + (long long)reflect(iy + ky - N, I.ny, bc) * I.nx;
      double a[V][NS];
#pragma unroll
      for (int kx = 0; kx < NS; ++kx) {
        const long long c = row + reflect(ix + kx - N, I.nx, bc);
#pragma unroll
        for (int v = 0; v < V; ++v) a[v][kx] = U[(long long)(v * NP) * ctot + c] * t.psi0 * t.psi0;
      }
      double o[V][NG];
      sweep<PDE, V, N>(t, a, Rx, Lx, o);
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int q = 0; q < NG; ++q) rowv[v][ky][q] = o[v][q];
    }
    // y sweep per x point, then the tensor projection onto the modes 1 <= a+b <= N
    double acc[V][NP];
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int m = 0; m < NP; ++m) acc[v][m] = 0.0;
#pragma unroll
    for (int gx = 0; gx < NG; ++gx) {
      double a[V][NS];
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int ky = 0; ky < NS; ++ky) a[v][ky] = rowv[v][ky][gx];
      double o[V][NG];
      sweep<PDE, V, N>(t, a, Ry, Ly, o);
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int gy = 0; gy < NG; ++gy) {
          const double w = t.wg[gx] * t.wg[gy] * o[v][gy];
#pragma unroll
          for (int m = 1; m < NP; ++m) acc[v][m] = fma(w * t.pg[gx][mode_a(m)], t.pg[gy][mode_b(m)], acc[v][m]);
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int m = 1; m < NP; ++m) lim[(long long)(v * NP + m) * cap + i] = acc[v][m];
  }
}

}  // namespace pw

cudaError_t upload_tables_parent(const dgt::Tabs* tabs /* [3], built with parent = true */) {
  pw::PTab h[3] = {};
  for (int n = 1; n <= 3; ++n) {
    const dgt::Tabs& t = tabs[n - 1];
    pw::PTab& p = h[n - 1];
    for (int i = 0; i <= n; ++i)
      for (int g = 0; g < t.NG; ++g)
        for (int k = 0; k <= n; ++k) p.C[i][g][k] = t.C[i][g][k];
    for (int g = 0; g < t.NG; ++g) {
      for (int i = 0; i <= n; ++i) {
        p.gam[g][i] = t.gam[g][i];
        p.gpn[g][i] = t.gpn[g][i];
        p.gmn[g][i] = t.gmn[g][i];
      }
      p.sgp[g] = t.sgp[g];
      p.sgm[g] = t.sgm[g];
      p.neg[g] = t.neg[g] ? 1.0 : 0.0;
      p.wg[g] = t.rw[g];
      for (int k = 0; k <= n; ++k) p.pg[g][k] = t.psiG[g][k];
    }
    for (int i = 0; i <= n; ++i)
      for (int k = 0; k <= n; ++k)
        for (int l = 0; l <= n; ++l) p.B[i][k][l] = t.B[i][k][l];
    p.psi0 = t.psi_0[0];
  }
  return cudaMemcpyToSymbol(pw::c_pt, h, sizeof(h));
}

void launch_parent(int dim, int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt,
                   double* lim, int nblocks) {
  // one warp per block, four times the usual grid: the troubled-cell count is known only on
  // the device, and small lists then still spread over all SMs
#define DG_PW(K, P, NN) pw::K<P, NN><<<4 * nblocks, 32, 0, a.st>>>(a.us, a.inst, a.ctot, a.bc, lc, li, cnt, lim, a.cap, a.gam)
#define DG_PW_N(K, P)  \
  do {                 \
    if (N == 1) DG_PW(K, P, 1); \
    else if (N == 2) DG_PW(K, P, 2); \
    else DG_PW(K, P, 3); \
  } while (0)
  if (dim == 1) {
    if (pde == 0) DG_PW_N(k_parent1, 0);
    else DG_PW_N(k_parent1, 1);
  } else {
    if (pde == 0) DG_PW_N(k_parent2, 0);
    else DG_PW_N(k_parent2, 1);
  }
#undef DG_PW_N
#undef DG_PW
}

}  // namespace dg
