// Derivation of the method's tables on the host (long double, then rounded once).
//
//  - Legendre polynomials by Bonnet's recurrence, psi_n = sqrt((2n+1)/2) P_n (Sec. 2).
//  - Gauss-Legendre rules: closed-form nodes and weights up to 4 points, Newton on the
//    recurrence beyond (initial projection only).
//  - CSWENO rows (Sec. 3, Step 2): the value at x of the polynomial whose averages match
//    on a run of cells is the derivative of the Lagrange interpolant of the primitive
//    function through the cell edges.
//  - Linear weights (Eq. (8)) by back substitution from the right end of the big stencil;
//    the other columns are checked (residual kept).
//  - Smoothness indicators (Eq. (13)) as quadratic forms, integrated with a 6-point Gauss
//    rule over the troubled cell in units of its width.
//  - Subcell averages of psi_n (Fig. 1) by a 6-point Gauss rule on each subcell.
#include "tables.h"

#include <cmath>
#include <cstring>

namespace dgt {
namespace {

typedef long double ld;

void legendre(int nmax, ld x, ld* P, ld* dP) {
  P[0] = 1.0L;
  dP[0] = 0.0L;
  if (nmax >= 1) {
    P[1] = x;
    dP[1] = 1.0L;
  }
  for (int n = 1; n < nmax; ++n) {
    P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1);
    dP[n + 1] = dP[n - 1] + (2 * n + 1) * P[n];
  }
}

ld psi(int n, ld x) {
  ld P[16], dP[16];
  legendre(n, x, P, dP);
  return std::sqrt((2.0L * n + 1.0L) / 2.0L) * P[n];
}

ld dpsi(int n, ld x) {
  ld P[16], dP[16];
  legendre(n, x, P, dP);
  return std::sqrt((2.0L * n + 1.0L) / 2.0L) * dP[n];
}

void gauss(int q, ld* x, ld* w) {
  if (q == 1) {
    x[0] = 0; w[0] = 2;
  } else if (q == 2) {
    x[0] = -1.0L / std::sqrt(3.0L); x[1] = -x[0]; w[0] = w[1] = 1;
  } else if (q == 3) {
    x[0] = -std::sqrt(0.6L); x[1] = 0; x[2] = -x[0];
    w[0] = w[2] = 5.0L / 9.0L; w[1] = 8.0L / 9.0L;
  } else if (q == 4) {
    ld s = std::sqrt(6.0L / 5.0L);
    ld a = std::sqrt(3.0L / 7.0L - 2.0L / 7.0L * s), b = std::sqrt(3.0L / 7.0L + 2.0L / 7.0L * s);
    ld r30 = std::sqrt(30.0L);
    x[0] = -b; x[1] = -a; x[2] = a; x[3] = b;
    w[0] = w[3] = (18.0L - r30) / 36.0L;
    w[1] = w[2] = (18.0L + r30) / 36.0L;
  } else {
    const ld pi = 3.14159265358979323846264338327950288L;
    for (int i = 0; i < q; ++i) {
      ld z = -std::cos(pi * (i + 0.75L) / (q + 0.5L));
      ld P[16], dP[16];
      for (int it = 0; it < 60; ++it) {
        legendre(q, z, P, dP);
        ld dz = P[q] / dP[q];
        z -= dz;
        if (std::fabs(dz) < 1e-30L) break;
      }
      legendre(q, z, P, dP);
      x[i] = z;
      w[i] = 2.0L / ((1.0L - z * z) * dP[q] * dP[q]);
    }
  }
}

// weights w_k such that p(x) = sum_k w_k avg_k, for the polynomial of degree n-1 with the
// given averages on the n cells between edges e[0..n] (primitive-function interpolation).
void primitive_rows(int n, const ld* e, ld x, ld* w) {
  for (int k = 0; k < n; ++k) w[k] = 0;
  for (int m = 1; m <= n; ++m) {
    ld denom = 1;
    for (int j = 0; j <= n; ++j)
      if (j != m) denom *= (e[m] - e[j]);
    ld d = 0;  // derivative of prod_{j != m} (x - e_j)
    for (int skip = 0; skip <= n; ++skip) {
      if (skip == m) continue;
      ld p = 1;
      for (int j = 0; j <= n; ++j)
        if (j != m && j != skip) p *= (x - e[j]);
      d += p;
    }
    d /= denom;
    for (int k = 0; k < m; ++k) w[k] += (e[k + 1] - e[k]) * d;
  }
}

// l-th derivative, at x, of the polynomial with unit average on cell k and zero on the
// others (n cells, edges e), via finite combinations of the primitive interpolant.
// Computed from the monomial expansion of each Lagrange basis polynomial.
void primitive_deriv_rows(int n, const ld* e, int l, ld x, ld* w) {
  for (int k = 0; k < n; ++k) w[k] = 0;
  for (int m = 1; m <= n; ++m) {
    // coefficients of L_m(x) = prod_{j != m} (x - e_j) / (e_m - e_j)
    ld c[16];
    std::memset(c, 0, sizeof(c));
    c[0] = 1;
    int deg = 0;
    for (int j = 0; j <= n; ++j) {
      if (j == m) continue;
      ld s = e[m] - e[j];
      for (int q = deg + 1; q >= 1; --q) c[q] = (c[q - 1] - e[j] * c[q]) / s;
      c[0] = (-e[j] * c[0]) / s;
      ++deg;
    }
    // (l+1)-th derivative at x
    ld d = 0;
    for (int q = l + 1; q <= deg; ++q) {
      ld f = 1;
      for (int r = 0; r <= l; ++r) f *= (q - r);
      ld xp = 1;
      for (int r = 0; r < q - l - 1; ++r) xp *= x;
      d += c[q] * f * xp;
    }
    for (int k = 0; k < m; ++k) w[k] += (e[k + 1] - e[k]) * d;
  }
}

}  // namespace

int build_tables(int N, Tabs* t, bool parent) {
  if (N < 1 || N > kMaxN) return 1;
  std::memset(t, 0, sizeof(*t));
  t->N = N;
  t->Q = N + 1;
  t->NS = 2 * N + 1;
  ld x[kMaxQ], w[kMaxQ];
  gauss(N + 1, x, w);
  for (int q = 0; q <= N; ++q) {
    t->gx[q] = (double)x[q];
    t->gw[q] = (double)w[q];
    for (int n = 0; n <= N; ++n) {
      t->psi_q[q][n] = (double)psi(n, x[q]);
      t->dpsi_q[q][n] = (double)dpsi(n, x[q]);
      t->kq[q][n] = (double)(sqrtl(2.0L) * psi(n, x[q]));
    }
  }
  for (int n = 0; n <= N; ++n) {
    t->psi_p1[n] = (double)psi(n, 1.0L);
    t->kp1[n] = (double)(sqrtl(2.0L) * psi(n, 1.0L));
    t->psi_m1[n] = (double)psi(n, -1.0L);
    t->psi_0[n] = (double)psi(n, 0.0L);
  }
  // initial projection rule
  t->QP = N + 4;
  gauss(N + 4, x, w);
  for (int q = 0; q < N + 4; ++q) {
    t->px[q] = (double)x[q];
    t->pw[q] = (double)w[q];
    for (int n = 0; n <= N; ++n) t->ppsi[q][n] = (double)psi(n, x[q]);
  }
  // Step 1 points: Gauss 2 (P1), Gauss-Lobatto 4 (P2), Gauss 4 (P3)
  ld rp[kMaxG], rw[kMaxG];
  if (N == 1) {
    t->NG = 2;
    gauss(2, rp, rw);
  } else if (N == 2) {
    t->NG = 4;
    rp[0] = -1; rp[1] = -1.0L / std::sqrt(5.0L); rp[2] = -rp[1]; rp[3] = 1;
    rw[0] = rw[3] = 1.0L / 6.0L;
    rw[1] = rw[2] = 5.0L / 6.0L;
  } else {
    t->NG = 4;
    gauss(4, rp, rw);
  }
  for (int g = 0; g < t->NG; ++g) {
    t->rp[g] = (double)rp[g];
    t->rw[g] = (double)rw[g];
    for (int n = 0; n <= N; ++n) t->psiG[g][n] = (double)psi(n, rp[g]);
  }
  // stencil edges, in units of the troubled cell's width (troubled cell = [-1/2, 1/2]):
  // CSWENO splits the immediate neighbours into N parts; the parent WENO limiter (Qiu and
  // Shu) uses the whole cells j-N .. j+N
  int ns = t->NS;
  ld e[kMaxS + 1];
  if (parent) {
    for (int k = 0; k <= ns; ++k) e[k] = -(ld)N - 0.5L + k;
  } else {
    for (int k = 0; k <= N; ++k) e[k] = -1.5L + (ld)k / N;
    for (int k = 1; k <= N; ++k) e[N + k] = 0.5L + (ld)(k - 1) / N;
    e[2 * N + 1] = 1.5L;
    // (the loop above sets e[N+1] = 0.5, the troubled cell's right edge)
  }
  for (int g = 0; g < t->NG; ++g) {
    ld xi = rp[g] / 2;
    ld Cl[kMaxN + 1][kMaxN + 1];
    for (int i = 0; i <= N; ++i) {
      primitive_rows(N + 1, e + i, xi, Cl[i]);
      for (int k = 0; k <= N; ++k) t->C[i][g][k] = (double)Cl[i][k];
    }
    ld D[kMaxS];
    primitive_rows(ns, e, xi, D);
    // back substitution: column 2N only in S_N, column 2N-1 in S_{N-1}, S_N, ...
    ld gm[kMaxN + 1];
    for (int i = N; i >= 0; --i) {
      int col = i + N;
      ld s = D[col];
      for (int j = i + 1; j <= N; ++j) s -= gm[j] * Cl[j][col - j];
      gm[i] = s / Cl[i][N];
    }
    ld res = 0;
    for (int col = 0; col < ns; ++col) {
      ld s = -D[col];
      for (int i = 0; i <= N; ++i)
        if (col >= i && col <= i + N) s += gm[i] * Cl[i][col - i];
      if (std::fabs(s) > res) res = std::fabs(s);
    }
    if ((double)res > t->gam_resid) t->gam_resid = (double)res;
    int neg = 0;
    for (int i = 0; i <= N; ++i) {
      t->gam[g][i] = (double)gm[i];
      if (gm[i] < 0) neg = 1;
    }
    t->neg[g] = neg;
    // split of Shi, Hu & Shu with theta = 3 where a weight is negative
    ld sp = 0, sm = 0, gp[kMaxN + 1], gn[kMaxN + 1];
    for (int i = 0; i <= N; ++i) {
      gp[i] = 0.5L * (gm[i] + 3.0L * std::fabs(gm[i]));
      gn[i] = gp[i] - gm[i];
      sp += gp[i];
      sm += gn[i];
    }
    t->sgp[g] = (double)sp;
    t->sgm[g] = (double)sm;
    for (int i = 0; i <= N; ++i) {
      t->gpn[g][i] = (double)(gp[i] / sp);
      t->gmn[g][i] = (double)(sm > 0 ? gn[i] / sm : 0);
    }
  }
  // Eq. (13): beta_i = sum_{l=1}^N int_{-1/2}^{1/2} (d^l p_i / dxi^l)^2 dxi
  {
    ld qx[kMaxQ], qw[kMaxQ];
    gauss(6, qx, qw);
    for (int i = 0; i <= N; ++i) {
      ld Bl[kMaxN + 1][kMaxN + 1];
      std::memset(Bl, 0, sizeof(Bl));
      for (int l = 1; l <= N; ++l)
        for (int q = 0; q < 6; ++q) {
          ld xi = qx[q] / 2, wq = qw[q] / 2;
          ld d[kMaxN + 1];
          primitive_deriv_rows(N + 1, e + i, l, xi, d);
          for (int a = 0; a <= N; ++a)
            for (int b = 0; b <= N; ++b) Bl[a][b] += wq * d[a] * d[b];
        }
      for (int a = 0; a <= N; ++a)
        for (int b = 0; b <= N; ++b) t->B[i][a][b] = (double)Bl[a][b];
    }
  }
  // subcell averages (Fig. 1): N equal parts of each neighbour, troubled cell whole
  {
    ld qx[kMaxQ], qw[kMaxQ];
    gauss(6, qx, qw);
    for (int k = 0; k < ns; ++k) {
      ld a, b;
      if (parent) {  // whole cell j + k - N: only its mean enters
        t->OFF[k] = k - N;
        t->SA[k][0] = (double)psi(0, 0.0L);
        for (int n = 1; n <= N; ++n) t->SA[k][n] = 0.0;
        continue;
      }
      if (k < N) { a = -1 + 2.0L * k / N; b = -1 + 2.0L * (k + 1) / N; t->OFF[k] = -1; }
      else if (k == N) { a = -1; b = 1; t->OFF[k] = 0; }
      else { int q = k - N - 1; a = -1 + 2.0L * q / N; b = -1 + 2.0L * (q + 1) / N; t->OFF[k] = 1; }
      for (int n = 0; n <= N; ++n) {
        ld s = 0;
        for (int q = 0; q < 6; ++q) s += qw[q] * psi(n, 0.5L * (a + b) + 0.5L * (b - a) * qx[q]);
        t->SA[k][n] = (double)(s / 2);
      }
      if (k == N)
        for (int n = 1; n <= N; ++n) t->SA[k][n] = 0.0;
    }
  }
  return 0;
}

}  // namespace dgt
