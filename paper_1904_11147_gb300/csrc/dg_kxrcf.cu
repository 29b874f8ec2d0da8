// KXRCF troubled-cell indicator (Sec. 3, step 1: the paper's own choice, after
// Krivodonova et al., ref. [kxrcf]) with the ballot/scan compaction of the troubled cells.
//
// For an indicator variable w of cell j (u for Burgers; density and total energy for
// Euler, either one flags the cell):
//   I_j = | int over the inflow faces of (w_j - w_nb) ds | / ( r^((N+1)/2) |inflow| max|w_j| ),
// r the radius of the circle circumscribing the cell (per instance, computed on the host),
// max|w_j| over the cell's (N+1)^dim Gauss points; troubled when I_j > 1, decided as
// num > den.  A face is inflow when its outward normal has a negative product with the
// mean velocity (sign of the mean momentum for Euler, of ubar for Burgers in every
// direction); face integrals use the (N+1)-point Gauss rule along the face.  Neighbours
// follow the boundary condition (periodic, or the mirrored boundary cell at outflow).
//
// A face trace has degree N along the face and the (N+1)-point Gauss rule integrates it
// exactly, so by orthonormality the face integral keeps only the transverse-degree-0
// part: int_face w ds = |face| / sqrt(2) * sum_a U_a0 psi_a(+-1).  The Gauss-point maximum
// uses sum factorisation.  This is the oracle's definition evaluated in fewer operations:
// the decisions agree except where num and den are within rounding of each other (the
// near-threshold cells, counted).  One thread per cell on the tiles of the TVB indicator.
#include "dg_shared.cuh"

namespace dg {

struct KxTab {
  double pm[4], pp[4];  // psi_n(-1), psi_n(+1)
  double pq[4][4];      // psi_n at the (N+1) Gauss points [q][n]
  double w[4];          // Gauss weights
};

// near (reporting only): within kNearUlp units in the last place, a window that contains
// the 1e-12 relative one (see tvb_changes_bits)
__device__ __forceinline__ bool kx_near(double a, double b) {
  const long long d = __double_as_longlong(a) - __double_as_longlong(b);
  return d <= kNearUlp && d >= -kNearUlp;
}

template <int DIM, int PDE, int N>
__global__ void __launch_bounds__(256) k_kxrcf(const double* __restrict__ U, const Inst* __restrict__ insts,
                                               const Tile* __restrict__ tiles, long long ctot, int bc,
                                               const double* __restrict__ hpow, KxTab tb,
                                               unsigned char* __restrict__ flags, Counters* cnt,
                                               int* __restrict__ list_cell, int* __restrict__ list_inst) {
  constexpr int V = nv_of(DIM, PDE), NP = np_of(DIM, N), Q = N + 1;
  constexpr int NW = PDE == 0 ? 1 : 2;
  const Tile tile = tiles[blockIdx.x];
  const Inst I = insts[tile.inst];
  const int ix = DIM == 1 ? tile.x0 + (int)threadIdx.x : tile.x0 + (int)(threadIdx.x & 31);
  const int iy = DIM == 1 ? 0 : tile.y0 + (int)(threadIdx.x >> 5);
  const bool active = ix < I.nx && iy < I.ny;
  int fl = 0;
  bool near = false;
  long long g = 0;
  if (active) {
    g = I.off + (long long)iy * I.nx + ix;
    const double hp = hpow[tile.inst];
    const double vx = U[(long long)(PDE == 0 ? 0 : NP) * ctot + g];
    const double vy = DIM == 2 ? U[(long long)(PDE == 0 ? 0 : 2 * NP) * ctot + g] : 0.0;
    // faces: 1D L, R; 2D W, E, S, N
    constexpr int NF = 2 * DIM;
    bool in[NF];
    in[0] = vx > 0.0;
    in[1] = vx < 0.0;
    if (DIM == 2) {
      in[2 % NF] = vy > 0.0;
      in[3 % NF] = vy < 0.0;
    }
    // neighbour cell of face f and whether it is the mirrored boundary cell
    auto neighbour = [&](int f, bool& mirror) -> long long {
      int jx = ix + (f == 0 ? -1 : (f == 1 ? 1 : 0));
      int jy = iy + (f == 2 ? -1 : (f == 3 ? 1 : 0));
      mirror = false;
      if (bc == 0) {
        jx = jx < 0 ? jx + I.nx : (jx >= I.nx ? jx - I.nx : jx);
        jy = jy < 0 ? jy + I.ny : (jy >= I.ny ? jy - I.ny : jy);
      } else if (jx < 0 || jx >= I.nx || jy < 0 || jy >= I.ny) {
        mirror = true;
        jx = ix;
        jy = iy;
      }
      return I.off + (long long)jy * I.nx + jx;
    };
    constexpr double kInvSqrt2 = 0.70710678118654752440;
#pragma unroll
    for (int iw = 0; iw < NW; ++iw) {
      const int v = iw == 0 ? 0 : V - 1;
      const double* P = U + (long long)(v * NP) * ctot;
      double uc[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) uc[k] = P[(long long)k * ctot + g];
      double num = 0.0, len = 0.0;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (!in[f]) continue;
        bool mirror;
        const long long gn = neighbour(f, mirror);
        // own trace at the face (normal degree n, transverse degree 0) and the
        // neighbour's trace at the same face (its opposite side)
        const bool low = (f & 1) == 0;  // W or S face: own side r = -1, neighbour's r = +1
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int n = 0; n <= N; ++n) {
          const int k = DIM == 1 ? n : (f < 2 ? mode_idx(n, 0) : mode_idx(0, n));
          const double x = P[(long long)k * ctot + gn];
          const double xn = neg_if(x, mirror && (n & 1));
          a = fma(uc[k], low ? tb.pm[n] : tb.pp[n], a);
          b = fma(xn, low ? tb.pp[n] : tb.pm[n], b);
        }
        const double flen = DIM == 1 ? 1.0 : (f < 2 ? I.hy : I.hx);
        num = fma(flen, a - b, num);
        len += flen;
      }
      if (len == 0.0) continue;
      if (DIM == 2) num *= kInvSqrt2;
      double nrm = 0.0;
      if (DIM == 1) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          double a = 0.0;
#pragma unroll
          for (int k = 0; k < NP; ++k) a = fma(uc[k], tb.pq[q][k], a);
          nrm = fmax(nrm, fabs(a));
        }
      } else {
#pragma unroll
        for (int qx = 0; qx < Q; ++qx) {
          double t[N + 1];
#pragma unroll
          for (int b = 0; b <= N; ++b) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a <= N - b; ++a) s = fma(uc[mode_idx(a, b)], tb.pq[qx][a], s);
            t[b] = s;
          }
#pragma unroll
          for (int qy = 0; qy < Q; ++qy) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b <= N; ++b) s = fma(t[b], tb.pq[qy][b], s);
            nrm = fmax(nrm, fabs(s));
          }
        }
      }
      const double den = hp * len * nrm, an = fabs(num);
      if (kx_near(an, den)) near = true;
      if (an > den) fl = 1;
    }
    flags[g] = (unsigned char)(fl | (near ? 2 : 0));
  }
  block_compact(fl, near ? 1 : 0, g, tile.inst, cnt, list_cell, list_inst);
}

// tiles: the indicator tiles of the mesh (1D: 256 cells, 2D: 32 x 8 cells), 256 threads
void launch_kxrcf(int dim, int pde, int N, const LaunchArgs& a, const double* hpow, const double* psi_m1,
                  const double* psi_p1, const double* psi_q /* [N+1][N+1] */, const double* gw,
                  unsigned char* flags, Counters* cnt, int* lc, int* li) {
  KxTab tb{};
  for (int k = 0; k <= N; ++k) {
    tb.pm[k] = psi_m1[k];
    tb.pp[k] = psi_p1[k];
    tb.w[k] = gw[k];
    for (int q = 0; q <= N; ++q) tb.pq[q][k] = psi_q[q * (N + 1) + k];
  }
#define DG_KX(D, P, NN)                                                                                     \
  k_kxrcf<D, P, NN><<<a.ntiles, 256, 0, a.st>>>(a.us, a.inst, a.tiles, a.ctot, a.bc, hpow, tb, flags, cnt, lc, li)
#define DG_KX_N(D, P) \
  do {                \
    if (N == 1) DG_KX(D, P, 1); \
    else if (N == 2) DG_KX(D, P, 2); \
    else DG_KX(D, P, 3); \
  } while (0)
  if (dim == 1) {
    if (pde == 0) DG_KX_N(1, 0);
    else DG_KX_N(1, 1);
  } else {
    if (pde == 0) DG_KX_N(2, 0);
    else DG_KX_N(2, 1);
  }
#undef DG_KX_N
#undef DG_KX
}

}  // namespace dg
