// Host-side tables of the method for one polynomial degree N (1..3).
//
// Everything here is derived at library start-up from the definitions in Sec. 2 and
// Sec. 3 of the paper (basis, quadrature rules, CSWENO reconstruction rows, linear
// weights, smoothness-indicator quadratic forms, subcell averages).
#pragma once

namespace dgt {

constexpr int kMaxN = 3;
constexpr int kMaxQ = 8;   // Gauss points (N+4 <= 7 for the initial projection)
constexpr int kMaxS = 7;   // stencil cells 2N+1
constexpr int kMaxG = 4;   // reconstruction points per direction

struct Tabs {
  int N, Q, NG, NS;
  // (N+1)-point Gauss-Legendre rule of the weak form (Eq. (5)), weights sum to 2
  double gx[kMaxQ], gw[kMaxQ];
  double psi_q[kMaxQ][kMaxN + 1], dpsi_q[kMaxQ][kMaxN + 1];
  double psi_p1[kMaxN + 1], psi_m1[kMaxN + 1], psi_0[kMaxN + 1];
  // the same basis values over psi_0 = 1/sqrt(2): sqrt(2) psi_n at the Gauss points and at 1
  double kq[kMaxQ][kMaxN + 1], kp1[kMaxN + 1];
  // CSWENO (Sec. 3, Steps 1-6)
  double rp[kMaxG], rw[kMaxG];               // Step 1 points (reference r) and weights
  double psiG[kMaxG][kMaxN + 1];             // psi_n at the Step 1 points
  double C[kMaxN + 1][kMaxG][kMaxN + 1];     // p_i(x_g) = sum_k C[i][g][k] avg[i+k]
  double gam[kMaxG][kMaxN + 1];              // Eq. (8)
  double B[kMaxN + 1][kMaxN + 1][kMaxN + 1]; // beta_i = sum_kl avg[i+k] B[i][k][l] avg[i+l]
  double SA[kMaxS][kMaxN + 1];               // average of psi_n over stencil cell k
  int OFF[kMaxS];                            // -1 / 0 / +1: neighbour holding stencil cell k
  int neg[kMaxG];                            // point g has a negative linear weight
  double gpn[kMaxG][kMaxN + 1], gmn[kMaxG][kMaxN + 1]; // normalised split weights
  double sgp[kMaxG], sgm[kMaxG];                        // sigma+, sigma-
  // initial projection: (N+4)-point Gauss rule
  int QP;
  double px[kMaxQ], pw[kMaxQ], ppsi[kMaxQ][kMaxN + 1];
  double gam_resid;                          // residual of the full Eq. (8) system
};

// Fills t for degree N; returns 0 on success.  parent: the limiter tables of the parent
// WENO limiter (whole cells j-N .. j+N) instead of CSWENO's subcells.
int build_tables(int N, Tabs* t, bool parent = false);

}  // namespace dgt
