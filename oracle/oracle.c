/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU statement of the RKDG method with the
 * compact subcell WENO (CSWENO) limiter of Kochi & Ramakrishna (arXiv 1904.11147).
 * It exists to check the CUDA library against the paper: only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Every routine states the passage it follows.  Tables are derived here from their
 * definitions (long double Gaussian elimination on monomial moment matrices); the
 * paper's printed P2 values are asserted by the test-suite, not copied in.
 *
 * Storage: modes are u[cell][var][mode], cell = iy*nx + ix.  2D modes are ordered by
 * total degree d = a+b, then by b ascending: (0,0),(1,0),(0,1),(2,0),(1,1),(0,2),...
 *
 * Readings of passages the paper leaves open are listed with each routine and in the
 * design notes of the repository: orthonormal reference basis, (N+1)-point Gauss
 * quadrature in the weak form, local Lax-Friedrichs flux, TVB minmod indicator,
 * neighbours split into N equal parts, Jacobi limiter updates, mirror ghosts at
 * outflow boundaries, dimension-by-dimension (x then y) 2D reconstruction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 3
#define OR_MAXNP 10 /* 2D P3 */
#define OR_MAXV 4
#define OR_MAXS 7  /* stencil cells, 2N+1 */
#define OR_MAXG 4  /* reconstruction points per direction */
#define OR_MAXQ 8  /* Gauss points (N+4 <= 7 for the initial projection) */

typedef long double ld;

/* ------------------------------------------------------------------------------------
 * Mesh description (one instance).
 * ----------------------------------------------------------------------------------*/
typedef struct {
  int dim;   /* 1 or 2 */
  int pde;   /* 0 Burgers, 1 Euler */
  int N;     /* polynomial degree 1..3 */
  int nx, ny;/* ny = 1 in 1D */
  int bc;    /* 0 periodic, 1 outflow, 2 double Mach reflection (2D Euler) */
  double xL, xR, yL, yR;
  double gamma;
  /* bc 2: the time of the state the operators are applied to, and the problem's data:
   * post-shock (rho, u, v, p), pre-shock (rho, u, v, p), and the shock line
   * x_s(y, t) = a + b y + c t (a is also where the wall starts on the bottom side) */
  double t;
  double bcp[11];
} or_mesh;

int or_nmodes(int dim, int N) { return dim == 1 ? N + 1 : (N + 1) * (N + 2) / 2; }
int or_nvars(int dim, int pde) { return pde == 0 ? 1 : (dim == 1 ? 3 : 4); }

/* 2D mode index -> (a, b): total degree first, then b ascending. */
static void mode_ab(int m, int* a, int* b) {
  int d = 0, start = 0;
  while (m >= start + d + 1) { start += d + 1; ++d; }
  *b = m - start;
  *a = d - *b;
}

/* ------------------------------------------------------------------------------------
 * Basis (Sec. 2): orthonormalised Legendre polynomials on the reference cell [-1,1],
 * psi_n(r) = sqrt((2n+1)/2) P_n(r), with the affine map of Eq. (4).  P_n is written
 * from its explicit sum  P_n(x) = 2^-n sum_j (-1)^j C(n,j) C(2n-2j,n) x^(n-2j).
 * ----------------------------------------------------------------------------------*/
static ld binom(int n, int k) {
  ld r = 1;
  if (k < 0 || k > n) return 0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
/* coefficient of x^k in P_n */
static ld leg_coef(int n, int k) {
  if (k > n || ((n - k) & 1)) return 0;
  int j = (n - k) / 2;
  ld c = binom(n, j) * binom(2 * n - 2 * j, n);
  for (int i = 0; i < n; ++i) c /= 2;
  return (j & 1) ? -c : c;
}
static ld ipow(ld x, int k) {
  ld r = 1;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}
static ld legP(int n, ld x) {
  ld s = 0;
  for (int k = 0; k <= n; ++k) s += leg_coef(n, k) * ipow(x, k);
  return s;
}
static ld legdP(int n, ld x) {
  ld s = 0;
  for (int k = 1; k <= n; ++k) s += leg_coef(n, k) * k * ipow(x, k - 1);
  return s;
}
static ld psi(int n, ld r) { return sqrtl((2.0L * n + 1.0L) / 2.0L) * legP(n, r); }
static ld dpsi(int n, ld r) { return sqrtl((2.0L * n + 1.0L) / 2.0L) * legdP(n, r); }
/* average of psi_n over [a,b] (exact, from the antiderivative of the monomial sum) */
static ld psi_avg(int n, ld a, ld b) {
  ld s = 0;
  for (int k = 0; k <= n; ++k)
    s += leg_coef(n, k) * (ipow(b, k + 1) - ipow(a, k + 1)) / (k + 1);
  return sqrtl((2.0L * n + 1.0L) / 2.0L) * s / (b - a);
}

/* Gauss-Legendre rule with q points on [-1,1] (weights sum to 2): Newton on P_q. */
static void gauss_rule(int q, ld* x, ld* w) {
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < q; ++i) {
    ld z = cosl(pi * (i + 0.75L) / (q + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld dz = legP(q, z) / legdP(q, z);
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    ld d = legdP(q, z);
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0L / ((1.0L - z * z) * d * d);
  }
}

/* ------------------------------------------------------------------------------------
 * Small dense solver (long double, partial pivoting).  A is n x n row major, B is n x m.
 * ----------------------------------------------------------------------------------*/
static void solve_ld(int n, ld* A, int m, ld* B) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
    if (p != c) {
      for (int k = 0; k < n; ++k) { ld t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t; }
      for (int k = 0; k < m; ++k) { ld t = B[c * m + k]; B[c * m + k] = B[p * m + k]; B[p * m + k] = t; }
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      ld f = A[r * n + c] / A[c * n + c];
      for (int k = 0; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < m; ++k) B[r * m + k] -= f * B[c * m + k];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int k = 0; k < m; ++k) B[r * m + k] /= A[r * n + r];
}

/* ------------------------------------------------------------------------------------
 * CSWENO tables for degree N (Sec. 3, Fig. 1 and Steps 1-4).
 *
 * The stencil has 2N+1 cells.  The troubled cell I_j is whole; each immediate
 * neighbour is split into N equal subcells (halves for P2 as in Fig. 1; one piece,
 * i.e. plain WENO3, for P1; thirds for P3, our reading of "the same procedure ... for
 * any N").  Positions are in units of the troubled cell's width, xi = r/2, so I_j is
 * [-1/2, 1/2] and a neighbour subcell has width 1/N.
 *
 *   pt[g], wt[g]    Step 1 reconstruction points (reference r) and weights (sum 2)
 *   C[i][g][k]      Step 2/3: p_i(x_g) = sum_k C[i][g][k] * avg_k   (S_i = cells i..i+N)
 *   D[g][k]         Step 2/3: Q(x_g)   = sum_k D[g][k]   * avg_k
 *   gam[g][i]       Eq. (8) linear weights
 *   B[i][k][l]      Eq. (13): beta_i = sum_{k,l} avg_k B[i][k][l] avg_l
 *   SA[k][n]        average of psi_n over stencil cell k in the coordinate of the cell
 *                   that contains it (left neighbour, troubled cell, right neighbour)
 *   OFF[k]          -1, 0, +1: which of the three cells holds stencil cell k
 * ----------------------------------------------------------------------------------*/
typedef struct {
  int N, ns, ng;
  double pt[OR_MAXG], wt[OR_MAXG];
  double C[OR_MAXN + 1][OR_MAXG][OR_MAXS];
  double D[OR_MAXG][OR_MAXS];
  double gam[OR_MAXG][OR_MAXN + 1];
  double B[OR_MAXN + 1][OR_MAXS][OR_MAXS];
  double SA[OR_MAXS][OR_MAXN + 1];
  int OFF[OR_MAXS];
  double psiG[OR_MAXG][OR_MAXN + 1]; /* psi_n at the reconstruction points */
  double gam_resid;                   /* max residual of the full Eq. (8) system */
} or_weno_tables;

/* edges of the 2N+1 stencil cells in xi units (troubled cell [-1/2, 1/2]).  CSWENO: the
 * immediate neighbours split into N equal parts (Fig. 1).  Parent WENO (the limiter of
 * Qiu and Shu the paper compares with, ref. [qs1]): the whole cells j-N..j+N. */
static void stencil_edges(int N, int parent, ld* e) {
  if (parent) {
    for (int k = 0; k <= 2 * N + 1; ++k) e[k] = -(ld)N - 0.5L + k;
    return;
  }
  for (int k = 0; k <= N; ++k) e[k] = -1.5L + (ld)k / N;           /* left neighbour */
  e[N + 1] = 0.5L;                                                  /* troubled cell */
  for (int k = 1; k <= N; ++k) e[N + 1 + k] = 0.5L + (ld)k / N;     /* right neighbour */
}

/* Rows r (over the cells first..first+n-1) with  value_at(xi_g) = r . averages  for the
 * interpolating polynomial of degree n-1 whose averages match (monomial moments). */
static void recon_rows(int n, const ld* e, int first, int ng, const ld* xig, ld* rows /*ng x n*/,
                       ld* Ainv /* n x n, nullable */) {
  ld A[OR_MAXS * OR_MAXS], At[OR_MAXS * OR_MAXS], R[OR_MAXS * OR_MAXG];
  for (int k = 0; k < n; ++k) {
    ld a = e[first + k], b = e[first + k + 1];
    for (int j = 0; j < n; ++j) A[k * n + j] = (ipow(b, j + 1) - ipow(a, j + 1)) / ((j + 1) * (b - a));
  }
  /* rows: solve A^T c = phi(xi_g) for every g */
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j) At[j * n + k] = A[k * n + j];
  for (int j = 0; j < n; ++j)
    for (int g = 0; g < ng; ++g) R[j * ng + g] = ipow(xig[g], j);
  solve_ld(n, At, ng, R);
  for (int g = 0; g < ng; ++g)
    for (int k = 0; k < n; ++k) rows[g * n + k] = R[k * ng + g];
  if (Ainv) {
    ld I[OR_MAXS * OR_MAXS];
    for (int k = 0; k < n * n; ++k) At[k] = A[k];
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) I[r * n + c] = (r == c);
    solve_ld(n, At, n, I);
    for (int k = 0; k < n * n; ++k) Ainv[k] = I[k];
  }
}

/* parent: full-width stencil (see stencil_edges).  ng_in > 0: reconstruct at the ng_in
 * points r_in instead of the Step 1 points (tables for tests; weights then unused). */
static void weno_tables_build_g(int N, int parent, int ng_in, const double* r_in, or_weno_tables* t) {
  memset(t, 0, sizeof(*t));
  int ns = 2 * N + 1, ng;
  ld e[OR_MAXS + 1], r[OR_MAXG], w[OR_MAXG], xi[OR_MAXG];
  t->N = N;
  t->ns = ns;
  stencil_edges(N, parent, e);
  /* Step 1: the points the paper prescribes, weights of the matching rule. */
  if (ng_in > 0) {
    ng = ng_in;
    for (int g = 0; g < ng; ++g) r[g] = r_in[g];
  } else if (N == 1) {
    ng = 2;
    r[0] = -1.0L / sqrtl(3.0L); r[1] = -r[0];
  } else if (N == 2) {
    ng = 4; /* Gauss-Lobatto */
    r[0] = -1.0L; r[1] = -1.0L / sqrtl(5.0L); r[2] = -r[1]; r[3] = 1.0L;
  } else {
    ng = 4;
    r[0] = -sqrtl(525.0L + 70.0L * sqrtl(30.0L)) / 35.0L;
    r[1] = -sqrtl(525.0L - 70.0L * sqrtl(30.0L)) / 35.0L;
    r[2] = -r[1]; r[3] = -r[0];
  }
  for (int g = 0; g < ng; ++g) {
    if (ng_in > 0) {
      w[g] = 0.0L;
    } else if (N == 2) { /* Lobatto weights 2/(n(n-1) P_{n-1}(x)^2), n = 4 */
      ld p = legP(3, r[g]);
      w[g] = 2.0L / (12.0L * p * p);
    } else { /* Gauss weights 2/((1-x^2) P_n'(x)^2) */
      ld d = legdP(ng, r[g]);
      w[g] = 2.0L / ((1.0L - r[g] * r[g]) * d * d);
    }
    xi[g] = r[g] / 2.0L;
    t->pt[g] = (double)r[g];
    t->wt[g] = (double)w[g];
    for (int n = 0; n <= N; ++n) t->psiG[g][n] = (double)psi(n, r[g]);
  }
  t->ng = ng;
  /* Step 2: p_i on S_i = cells i..i+N, Q on all 2N+1 cells. */
  ld Cl[OR_MAXN + 1][OR_MAXG][OR_MAXS];
  ld Dl[OR_MAXG][OR_MAXS];
  ld Ainv[OR_MAXN + 1][OR_MAXS * OR_MAXS];
  ld rows[OR_MAXG * OR_MAXS];
  memset(Cl, 0, sizeof(Cl));
  for (int i = 0; i <= N; ++i) {
    recon_rows(N + 1, e, i, ng, xi, rows, Ainv[i]);
    for (int g = 0; g < ng; ++g)
      for (int k = 0; k <= N; ++k) Cl[i][g][i + k] = rows[g * (N + 1) + k];
  }
  recon_rows(ns, e, 0, ng, xi, rows, NULL);
  for (int g = 0; g < ng; ++g)
    for (int k = 0; k < ns; ++k) Dl[g][k] = rows[g * ns + k];
  /* Step 3, Eq. (8): sum_i gamma_i C[i][g][.] = D[g][.].  Stencil cell k < N+1 lies
   * in S_0..S_k only, so the first N+1 columns give the weights by forward
   * substitution; the remaining columns must then hold (residual recorded). */
  t->gam_resid = 0;
  for (int g = 0; g < ng; ++g) {
    ld gm[OR_MAXN + 1];
    for (int i = 0; i <= N; ++i) {
      ld s = Dl[g][i];
      for (int j = 0; j < i; ++j) s -= gm[j] * Cl[j][g][i];
      gm[i] = s / Cl[i][g][i];
    }
    for (int k = 0; k < ns; ++k) {
      ld s = -Dl[g][k];
      for (int i = 0; i <= N; ++i) s += gm[i] * Cl[i][g][k];
      if ((double)fabsl(s) > t->gam_resid) t->gam_resid = (double)fabsl(s);
    }
    for (int i = 0; i <= N; ++i) t->gam[g][i] = (double)gm[i];
    for (int k = 0; k < ns; ++k) {
      t->D[g][k] = (double)Dl[g][k];
      for (int i = 0; i <= N; ++i) t->C[i][g][k] = (double)Cl[i][g][k];
    }
  }
  /* Step 4, Eq. (13): beta_i = sum_{l=1}^{N} int_{-1/2}^{1/2} (d^l p_i / dxi^l)^2 dxi
   * (Delta x_j^{2l-1} absorbs the units when x is measured in cell widths).  With
   * p_i = sum_n a_n xi^n and a = Ainv * avg, beta_i = avg^T (Ainv^T G Ainv) avg. */
  int n1 = N + 1;
  for (int i = 0; i <= N; ++i) {
    ld G[OR_MAXS * OR_MAXS];
    for (int a = 0; a < n1; ++a)
      for (int b = 0; b < n1; ++b) {
        ld s = 0;
        for (int l = 1; l <= N; ++l) {
          if (a < l || b < l) continue;
          ld fa = 1, fb = 1;
          for (int q = 0; q < l; ++q) { fa *= (a - q); fb *= (b - q); }
          int pw = a - l + b - l;
          s += fa * fb * (ipow(0.5L, pw + 1) - ipow(-0.5L, pw + 1)) / (pw + 1);
        }
        G[a * n1 + b] = s;
      }
    for (int k = 0; k < n1; ++k)
      for (int l = 0; l < n1; ++l) {
        ld s = 0;
        for (int a = 0; a < n1; ++a)
          for (int b = 0; b < n1; ++b) s += Ainv[i][a * n1 + k] * G[a * n1 + b] * Ainv[i][b * n1 + l];
        t->B[i][i + k][i + l] = (double)s;
      }
  }
  /* Subcell averages of the neighbours' DG polynomials (Sec. 3, Fig. 1): stencil cell
   * k < N is part k of the left neighbour, k = N the troubled cell, k > N part k-N-1
   * of the right neighbour, each in its own reference coordinate. */
  for (int k = 0; k < ns; ++k) {
    ld a, b;
    if (parent) { /* whole cell j + k - N: its average is U_0 psi_0 */
      t->OFF[k] = k - N;
      for (int n = 0; n <= N; ++n) t->SA[k][n] = n == 0 ? (double)psi_avg(0, -1.0L, 1.0L) : 0.0;
      continue;
    }
    if (k < N) { a = -1.0L + 2.0L * k / N; b = -1.0L + 2.0L * (k + 1) / N; t->OFF[k] = -1; }
    else if (k == N) { a = -1.0L; b = 1.0L; t->OFF[k] = 0; }
    else { int q = k - N - 1; a = -1.0L + 2.0L * q / N; b = -1.0L + 2.0L * (q + 1) / N; t->OFF[k] = 1; }
    for (int n = 0; n <= N; ++n) t->SA[k][n] = (double)psi_avg(n, a, b);
    if (k == N)
      for (int n = 1; n <= N; ++n) t->SA[k][n] = 0.0; /* orthogonality to psi_0 */
  }
}

void or_weno_tables_build(int N, or_weno_tables* t) { weno_tables_build_g(N, 0, 0, NULL, t); }

/* ------------------------------------------------------------------------------------
 * DG tables for the weak form (Eqs. (5)-(7)): (N+1)-point Gauss rule (our reading; the
 * paper does not state the quadrature), psi and psi' at the points and at r = +-1.
 * ----------------------------------------------------------------------------------*/
typedef struct {
  int N, nq;
  double x[OR_MAXQ], w[OR_MAXQ];
  double P[OR_MAXQ][OR_MAXN + 1], dP[OR_MAXQ][OR_MAXN + 1];
  double Pm[OR_MAXN + 1], Pp[OR_MAXN + 1]; /* psi_n(-1), psi_n(+1) */
  double P0[OR_MAXN + 1];                  /* psi_n(0) */
} or_dg_tables;

static void dg_tables(int N, int nq, or_dg_tables* t) {
  ld x[OR_MAXQ], w[OR_MAXQ];
  memset(t, 0, sizeof(*t));
  t->N = N;
  t->nq = nq;
  gauss_rule(nq, x, w);
  for (int q = 0; q < nq; ++q) {
    t->x[q] = (double)x[q];
    t->w[q] = (double)w[q];
    for (int n = 0; n <= N; ++n) {
      t->P[q][n] = (double)psi(n, x[q]);
      t->dP[q][n] = (double)dpsi(n, x[q]);
    }
  }
  for (int n = 0; n <= N; ++n) {
    t->Pm[n] = (double)psi(n, -1.0L);
    t->Pp[n] = (double)psi(n, 1.0L);
    t->P0[n] = (double)psi(n, 0.0L);
  }
}

/* ------------------------------------------------------------------------------------
 * Physical fluxes.  Burgers f = g = u^2/2 (Eqs. (19), (20)); Euler with the ideal-gas
 * pressure of Eqs. (21), (23).  dir = 0: x-flux, 1: y-flux.
 * ----------------------------------------------------------------------------------*/
static void phys_flux(int dim, int pde, double gam, int dir, const double* u, double* f) {
  if (pde == 0) { f[0] = 0.5 * u[0] * u[0]; return; }
  if (dim == 1) {
    double rho = u[0], m = u[1], E = u[2];
    double vel = m / rho;
    double p = (gam - 1.0) * (E - 0.5 * m * vel);
    f[0] = m;
    f[1] = m * vel + p;
    f[2] = (E + p) * vel;
    return;
  }
  double rho = u[0], mx = u[1], my = u[2], E = u[3];
  double vx = mx / rho, vy = my / rho;
  double p = (gam - 1.0) * (E - 0.5 * (mx * vx + my * vy));
  if (dir == 0) {
    f[0] = mx; f[1] = mx * vx + p; f[2] = my * vx; f[3] = (E + p) * vx;
  } else {
    f[0] = my; f[1] = mx * vy; f[2] = my * vy + p; f[3] = (E + p) * vy;
  }
}

/* largest |eigenvalue| of the flux Jacobian in direction dir */
static double max_speed(int dim, int pde, double gam, int dir, const double* u) {
  if (pde == 0) return fabs(u[0]);
  int nv = dim == 1 ? 3 : 4;
  double rho = u[0], E = u[nv - 1];
  double vx = u[1] / rho, vy = dim == 2 ? u[2] / rho : 0.0;
  double p = (gam - 1.0) * (E - 0.5 * rho * (vx * vx + vy * vy));
  double c = sqrt(gam * p / rho);
  return fabs(dir == 0 ? vx : vy) + c;
}

/* Local Lax-Friedrichs flux (Sec. 2 names Lax-Friedrichs; local alpha is our reading):
 * f* = 1/2 (f(uL) + f(uR)) - 1/2 alpha (uR - uL), alpha = max(rho(f'(uL)), rho(f'(uR))).
 * Where either spectral radius is undefined (no real sound speed: negative density or
 * pressure at the face) alpha is NaN, whichever side it comes from. */
static void llf(int dim, int pde, double gam, int dir, const double* uL, const double* uR, double* fs) {
  int nv = or_nvars(dim, pde);
  double fL[OR_MAXV], fR[OR_MAXV];
  phys_flux(dim, pde, gam, dir, uL, fL);
  phys_flux(dim, pde, gam, dir, uR, fR);
  double aL = max_speed(dim, pde, gam, dir, uL), aR = max_speed(dim, pde, gam, dir, uR);
  double a = (isnan(aL) || isnan(aR)) ? NAN : (aL > aR ? aL : aR);
  for (int v = 0; v < nv; ++v) fs[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * a * (uR[v] - uL[v]);
}

/* ------------------------------------------------------------------------------------
 * Neighbour access with boundary conditions.  Periodic wraps.  Outflow (our reading of
 * the transmissive boundaries of Examples 7-8): the ghost cell holds the mirror image
 * of the boundary cell's polynomial, i.e. modes odd in the normal direction negated;
 * further ghosts (the parent WENO stencil reaches N cells out) mirror the interior cell
 * at the reflected position (ghost -1-k <-> cell k).
 * ----------------------------------------------------------------------------------*/
/* Conserved variables of a primitive state (rho, u, v, p), 2D Euler. */
static void prim_to_cons(double gam, const double* w, double* c) {
  c[0] = w[0];
  c[1] = w[0] * w[1];
  c[2] = w[0] * w[2];
  c[3] = w[3] / (gam - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2]);
}

/* Modes of a cell holding the constant conserved state c (2D: only U_00 = 2 c). */
static void const_modes(int nv, int np, const double* c, double* out) {
  for (int v = 0; v < nv; ++v)
    for (int k = 0; k < np; ++k) out[v * np + k] = k == 0 ? 2.0 * c[v] : 0.0;
}

/* Ghost cells of the double Mach reflection problem (Example 11, after Woodward and
 * Colella, ref. [wc]), decided by the ghost cell's centre (x_c, y_c) at the time m->t of
 * the state:
 *   left (x < xL): the post-shock state (inflow);
 *   right (x > xR): the mirror image of the boundary cell (outflow);
 *   bottom (y < yL): the post-shock state where x_c < a, else a reflecting wall: the
 *     mirror image in y with the normal momentum rho v negated;
 *   top (y > yR): the post-shock state where x_c < x_s(yR, t) = a + b yR + c t (the
 *     exact position of the moving shock on that side), else the pre-shock state.
 * The x side decides first (a corner ghost takes the left or right rule, then the bottom
 * or top rule applies to what the right rule returned).  Ghosts further out (k > 0)
 * mirror interior cell k. */
static void dmr_modes(const or_mesh* m, const double* u, int ix, int iy, double* out) {
  const int nv = 4, np = or_nmodes(2, m->N);
  const double hx = (m->xR - m->xL) / m->nx, hy = (m->yR - m->yL) / m->ny;
  const double xc = m->xL + (ix + 0.5) * hx;
  const double* b = m->bcp;
  double post[4], pre[4];
  prim_to_cons(m->gamma, b, post);
  prim_to_cons(m->gamma, b + 4, pre);
  if (ix < 0) { const_modes(nv, np, post, out); return; }
  if (iy >= m->ny) {
    const double xs = b[8] + b[9] * m->yR + b[10] * m->t;
    const_modes(nv, np, xc < xs ? post : pre, out);
    return;
  }
  if (iy < 0 && xc < b[8]) { const_modes(nv, np, post, out); return; }
  int fx = 0, fy = 0;
  if (ix >= m->nx) { ix = 2 * m->nx - 1 - ix; fx = 1; }
  if (iy < 0) { iy = -1 - iy; fy = 1; }
  if (ix < 0) ix = 0;
  if (iy >= m->ny) iy = m->ny - 1;
  const double* src = u + ((size_t)iy * m->nx + ix) * nv * np;
  for (int v = 0; v < nv; ++v)
    for (int k = 0; k < np; ++k) {
      int a, bb;
      mode_ab(k, &a, &bb);
      double s = 1.0;
      if (fx && (a & 1)) s = -s;
      if (fy && (bb & 1)) s = -s;
      if (fy && v == 2) s = -s; /* reflecting wall: rho v changes sign */
      out[v * np + k] = s * src[v * np + k];
    }
}

static void cell_modes(const or_mesh* m, const double* u, int ix, int iy, double* out) {
  int nv = or_nvars(m->dim, m->pde), np = or_nmodes(m->dim, m->N);
  int fx = 0, fy = 0;
  if (m->bc == 2 && (ix < 0 || ix >= m->nx || iy < 0 || iy >= m->ny)) {
    dmr_modes(m, u, ix, iy, out);
    return;
  }
  if (m->bc == 0) {
    ix = (ix % m->nx + m->nx) % m->nx;
    iy = (iy % m->ny + m->ny) % m->ny;
  } else {
    /* ghost -1-k is the mirror image of cell k (reflection across the boundary) */
    if (ix < 0) { ix = -1 - ix; fx = 1; }
    if (ix >= m->nx) { ix = 2 * m->nx - 1 - ix; fx = 1; }
    if (iy < 0) { iy = -1 - iy; fy = 1; }
    if (iy >= m->ny) { iy = 2 * m->ny - 1 - iy; fy = 1; }
    if (ix < 0) ix = 0;
    if (ix >= m->nx) ix = m->nx - 1;
    if (iy < 0) iy = 0;
    if (iy >= m->ny) iy = m->ny - 1;
  }
  const double* src = u + ((size_t)iy * m->nx + ix) * nv * np;
  for (int v = 0; v < nv; ++v)
    for (int k = 0; k < np; ++k) {
      int a, b;
      if (m->dim == 1) { a = k; b = 0; } else mode_ab(k, &a, &b);
      double s = 1.0;
      if (fx && (a & 1)) s = -s;
      if (fy && (b & 1)) s = -s;
      out[v * np + k] = s * src[v * np + k];
    }
}

/* ------------------------------------------------------------------------------------
 * Spatial operator L(u_h), Eq. (5) in modal form.  With the reference-orthonormal
 * basis, M = (h/2) I (Eq. (6)) in 1D and (hx hy / 4) I in 2D, and
 *   dU_i/dt = (2/h) [ sum_q w_q f(u_h(r_q)) psi_i'(r_q)  -  (f*_R psi_i(1) - f*_L psi_i(-1)) ].
 * The flux projection of Eq. (3) followed by S^T equals the quadrature of f psi_i'
 * because psi_i' has degree < N.
 * ----------------------------------------------------------------------------------*/
void or_rhs(const or_mesh* m, const double* u, double* L) {
  int N = m->N, nv = or_nvars(m->dim, m->pde), np = or_nmodes(m->dim, N);
  or_dg_tables t;
  dg_tables(N, N + 1, &t);
  int nq = t.nq;
  if (m->dim == 1) {
    double h = (m->xR - m->xL) / m->nx;
    for (int c = 0; c < m->nx; ++c) {
      double uc[OR_MAXV * (OR_MAXN + 1)], ul[OR_MAXV * (OR_MAXN + 1)], ur[OR_MAXV * (OR_MAXN + 1)];
      cell_modes(m, u, c, 0, uc);
      cell_modes(m, u, c - 1, 0, ul);
      cell_modes(m, u, c + 1, 0, ur);
      double acc[OR_MAXV][OR_MAXN + 1];
      memset(acc, 0, sizeof(acc));
      /* volume term */
      for (int q = 0; q < nq; ++q) {
        double uq[OR_MAXV], f[OR_MAXV];
        for (int v = 0; v < nv; ++v) {
          uq[v] = 0;
          for (int n = 0; n < np; ++n) uq[v] += uc[v * np + n] * t.P[q][n];
        }
        phys_flux(1, m->pde, m->gamma, 0, uq, f);
        for (int v = 0; v < nv; ++v)
          for (int n = 0; n < np; ++n) acc[v][n] += t.w[q] * f[v] * t.dP[q][n];
      }
      /* traces and LLF fluxes at x_l (face with the left cell) and x_r */
      double aL[OR_MAXV], aR[OR_MAXV], bL[OR_MAXV], bR[OR_MAXV], fl[OR_MAXV], fr[OR_MAXV];
      for (int v = 0; v < nv; ++v) {
        aL[v] = aR[v] = bL[v] = bR[v] = 0;
        for (int n = 0; n < np; ++n) {
          aL[v] += ul[v * np + n] * t.Pp[n]; /* left cell at its r = +1 */
          aR[v] += uc[v * np + n] * t.Pm[n]; /* this cell at r = -1 */
          bL[v] += uc[v * np + n] * t.Pp[n]; /* this cell at r = +1 */
          bR[v] += ur[v * np + n] * t.Pm[n]; /* right cell at r = -1 */
        }
      }
      llf(1, m->pde, m->gamma, 0, aL, aR, fl);
      llf(1, m->pde, m->gamma, 0, bL, bR, fr);
      for (int v = 0; v < nv; ++v)
        for (int n = 0; n < np; ++n)
          L[((size_t)c * nv + v) * np + n] =
              (2.0 / h) * (acc[v][n] - (fr[v] * t.Pp[n] - fl[v] * t.Pm[n]));
    }
    return;
  }
  /* 2D, tensor-product rule on the reference square; modes psi_a(r) psi_b(s). */
  double hx = (m->xR - m->xL) / m->nx, hy = (m->yR - m->yL) / m->ny;
  int A[OR_MAXNP], Bm[OR_MAXNP];
  for (int k = 0; k < np; ++k) mode_ab(k, &A[k], &Bm[k]);
  for (int iy = 0; iy < m->ny; ++iy)
    for (int ix = 0; ix < m->nx; ++ix) {
      double uc[OR_MAXV * OR_MAXNP], nb[4][OR_MAXV * OR_MAXNP];
      cell_modes(m, u, ix, iy, uc);
      cell_modes(m, u, ix - 1, iy, nb[0]);
      cell_modes(m, u, ix + 1, iy, nb[1]);
      cell_modes(m, u, ix, iy - 1, nb[2]);
      cell_modes(m, u, ix, iy + 1, nb[3]);
      double ax[OR_MAXV][OR_MAXNP], ay[OR_MAXV][OR_MAXNP];
      memset(ax, 0, sizeof(ax));
      memset(ay, 0, sizeof(ay));
      for (int qy = 0; qy < nq; ++qy)
        for (int qx = 0; qx < nq; ++qx) {
          double uq[OR_MAXV], f[OR_MAXV], g[OR_MAXV];
          for (int v = 0; v < nv; ++v) {
            uq[v] = 0;
            for (int k = 0; k < np; ++k) uq[v] += uc[v * np + k] * t.P[qx][A[k]] * t.P[qy][Bm[k]];
          }
          phys_flux(2, m->pde, m->gamma, 0, uq, f);
          phys_flux(2, m->pde, m->gamma, 1, uq, g);
          double ww = t.w[qx] * t.w[qy];
          for (int v = 0; v < nv; ++v)
            for (int k = 0; k < np; ++k) {
              ax[v][k] += ww * f[v] * t.dP[qx][A[k]] * t.P[qy][Bm[k]];
              ay[v][k] += ww * g[v] * t.P[qx][A[k]] * t.dP[qy][Bm[k]];
            }
        }
      /* faces: west (r=-1), east (r=+1), south (s=-1), north (s=+1) */
      for (int q = 0; q < nq; ++q) {
        double in[OR_MAXV], out[OR_MAXV], fs[OR_MAXV];
        /* west face: neighbour's east trace | this cell's west trace */
        for (int v = 0; v < nv; ++v) {
          out[v] = in[v] = 0;
          for (int k = 0; k < np; ++k) {
            out[v] += nb[0][v * np + k] * t.Pp[A[k]] * t.P[q][Bm[k]];
            in[v] += uc[v * np + k] * t.Pm[A[k]] * t.P[q][Bm[k]];
          }
        }
        llf(2, m->pde, m->gamma, 0, out, in, fs);
        for (int v = 0; v < nv; ++v)
          for (int k = 0; k < np; ++k) ax[v][k] += t.w[q] * fs[v] * t.Pm[A[k]] * t.P[q][Bm[k]];
        /* east face */
        for (int v = 0; v < nv; ++v) {
          out[v] = in[v] = 0;
          for (int k = 0; k < np; ++k) {
            in[v] += uc[v * np + k] * t.Pp[A[k]] * t.P[q][Bm[k]];
            out[v] += nb[1][v * np + k] * t.Pm[A[k]] * t.P[q][Bm[k]];
          }
        }
        llf(2, m->pde, m->gamma, 0, in, out, fs);
        for (int v = 0; v < nv; ++v)
          for (int k = 0; k < np; ++k) ax[v][k] -= t.w[q] * fs[v] * t.Pp[A[k]] * t.P[q][Bm[k]];
        /* south face */
        for (int v = 0; v < nv; ++v) {
          out[v] = in[v] = 0;
          for (int k = 0; k < np; ++k) {
            out[v] += nb[2][v * np + k] * t.P[q][A[k]] * t.Pp[Bm[k]];
            in[v] += uc[v * np + k] * t.P[q][A[k]] * t.Pm[Bm[k]];
          }
        }
        llf(2, m->pde, m->gamma, 1, out, in, fs);
        for (int v = 0; v < nv; ++v)
          for (int k = 0; k < np; ++k) ay[v][k] += t.w[q] * fs[v] * t.P[q][A[k]] * t.Pm[Bm[k]];
        /* north face */
        for (int v = 0; v < nv; ++v) {
          out[v] = in[v] = 0;
          for (int k = 0; k < np; ++k) {
            in[v] += uc[v * np + k] * t.P[q][A[k]] * t.Pp[Bm[k]];
            out[v] += nb[3][v * np + k] * t.P[q][A[k]] * t.Pm[Bm[k]];
          }
        }
        llf(2, m->pde, m->gamma, 1, in, out, fs);
        for (int v = 0; v < nv; ++v)
          for (int k = 0; k < np; ++k) ay[v][k] -= t.w[q] * fs[v] * t.P[q][A[k]] * t.Pp[Bm[k]];
      }
      size_t base = ((size_t)iy * m->nx + ix) * nv * np;
      for (int v = 0; v < nv; ++v)
        for (int k = 0; k < np; ++k) L[base + v * np + k] = (2.0 / hx) * ax[v][k] + (2.0 / hy) * ay[v][k];
    }
}

/* ------------------------------------------------------------------------------------
 * Third-order TVD (SSP) Runge-Kutta stage (Sec. 3, last paragraph; Shu's scheme):
 *   s=1: u1 = u^n + dt L(u^n)
 *   s=2: u2 = 3/4 u^n + 1/4 (u1 + dt L(u1))
 *   s=3: u^{n+1} = 1/3 u^n + 2/3 (u2 + dt L(u2))
 * us is u^(s-1) (= u^n for s = 1).
 * ----------------------------------------------------------------------------------*/
void or_rk_stage(const or_mesh* m, int stage, double dt, const double* un, const double* us, double* out) {
  size_t n = (size_t)m->nx * m->ny * or_nvars(m->dim, m->pde) * or_nmodes(m->dim, m->N);
  double* L = (double*)malloc(n * sizeof(double));
  or_rhs(m, us, L);
  for (size_t i = 0; i < n; ++i) {
    double e = us[i] + dt * L[i];
    if (stage == 1) out[i] = e;
    else if (stage == 2) out[i] = 0.75 * un[i] + 0.25 * e;
    else out[i] = (1.0 / 3.0) * un[i] + (2.0 / 3.0) * e;
  }
  free(L);
}

/* ------------------------------------------------------------------------------------
 * Troubled-cell indicator.  The paper uses KXRCF (Sec. 3); the method built here uses
 * the TVB modified minmod of Cockburn & Shu with constant M:
 *   u+~ = u(x_{j+1/2}^-) - ubar_j,  u-~ = ubar_j - u(x_{j-1/2}^+),
 *   flag if  mt(u+~, D+ubar, D-ubar) != u+~  or  mt(u-~, D+ubar, D-ubar) != u-~,
 *   mt(a1,a2,a3) = a1 if |a1| <= M h^2, else minmod(a1,a2,a3).
 * Conserved variables; in 2D the x test uses the east/west edge midpoints and the y test
 * the north/south ones, with h the cell width in that direction.  A cell is also counted
 * "near threshold" when one of the comparisons deciding it is within 1e-12 relative
 * (rel_near; reporting only, the flag is the exact FP64 decision).
 * ----------------------------------------------------------------------------------*/
/* Near-threshold window: two non-negative doubles x, y are near when
 * |x - y| <= 1e-12 max(x, y). */
static int rel_near(double x, double y) {
  const double mx = x > y ? x : y;
  return fabs(x - y) <= 1e-12 * mx;
}

static int tvb_changes(double a1, double a2, double a3, double Mh2, int* near) {
  double b1 = fabs(a1);
  if (rel_near(b1, Mh2)) *near = 1;
  double mt;
  if (b1 <= Mh2) return 0;
  /* a sign test decides minmod: a mean difference within 1e-12 of the largest magnitude
   * in the comparison counts as near zero */
  double s = fabs(a1) > fabs(a2) ? fabs(a1) : fabs(a2);
  s = s > fabs(a3) ? s : fabs(a3);
  if (fabs(a2) <= 1e-12 * s || fabs(a3) <= 1e-12 * s) *near = 1;
  if (a1 > 0 && a2 > 0 && a3 > 0) {
    mt = a1 < a2 ? a1 : a2;
    mt = mt < a3 ? mt : a3;
  } else if (a1 < 0 && a2 < 0 && a3 < 0) {
    mt = a1 > a2 ? a1 : a2;
    mt = mt > a3 ? mt : a3;
  } else {
    mt = 0.0;
  }
  if (mt != 0.0) {
    double m23 = fabs(a2) < fabs(a3) ? fabs(a2) : fabs(a3);
    if (rel_near(b1, m23)) *near = 1;
  }
  return mt != a1;
}

/* flags[c] = 1 if troubled; returns the count; *n_near gets the near-threshold count and
 * near_cells[c] (optional) is 1 for each near-threshold cell */
long or_flag_tvb_cells(const or_mesh* m, const double* u, double M, unsigned char* flags, unsigned char* near_cells,
                       long* n_near) {
  int N = m->N, nv = or_nvars(m->dim, m->pde), np = or_nmodes(m->dim, N);
  or_dg_tables t;
  dg_tables(N, N + 1, &t);
  long nf = 0, nn = 0;
  if (m->dim == 1) {
    double h = (m->xR - m->xL) / m->nx, Mh2 = M * h * h;
    for (int c = 0; c < m->nx; ++c) {
      double uc[OR_MAXV * 4], ul[OR_MAXV * 4], ur[OR_MAXV * 4];
      cell_modes(m, u, c, 0, uc);
      cell_modes(m, u, c - 1, 0, ul);
      cell_modes(m, u, c + 1, 0, ur);
      int fl = 0, near = 0;
      for (int v = 0; v < nv; ++v) {
        double mean = uc[v * np] * t.P0[0], mL = ul[v * np] * t.P0[0], mR = ur[v * np] * t.P0[0];
        double up = 0, um = 0;
        for (int n = 0; n < np; ++n) {
          up += uc[v * np + n] * t.Pp[n];
          um += uc[v * np + n] * t.Pm[n];
        }
        double dp = mR - mean, dm = mean - mL;
        fl |= tvb_changes(up - mean, dp, dm, Mh2, &near);
        fl |= tvb_changes(mean - um, dp, dm, Mh2, &near);
      }
      flags[c] = (unsigned char)fl;
      if (near_cells) near_cells[c] = (unsigned char)near;
      nf += fl;
      nn += near;
    }
  } else {
    double hx = (m->xR - m->xL) / m->nx, hy = (m->yR - m->yL) / m->ny;
    double Mx = M * hx * hx, My = M * hy * hy;
    int A[OR_MAXNP], Bm[OR_MAXNP];
    for (int k = 0; k < np; ++k) mode_ab(k, &A[k], &Bm[k]);
    for (int iy = 0; iy < m->ny; ++iy)
      for (int ix = 0; ix < m->nx; ++ix) {
        double uc[OR_MAXV * OR_MAXNP], nb[4][OR_MAXV * OR_MAXNP];
        cell_modes(m, u, ix, iy, uc);
        cell_modes(m, u, ix - 1, iy, nb[0]);
        cell_modes(m, u, ix + 1, iy, nb[1]);
        cell_modes(m, u, ix, iy - 1, nb[2]);
        cell_modes(m, u, ix, iy + 1, nb[3]);
        int fl = 0, near = 0;
        double c00 = t.P0[0] * t.P0[0]; /* mean = U_00 psi_0 psi_0 */
        for (int v = 0; v < nv; ++v) {
          double mean = uc[v * np] * c00;
          double mW = nb[0][v * np] * c00, mE = nb[1][v * np] * c00;
          double mS = nb[2][v * np] * c00, mN = nb[3][v * np] * c00;
          double uE = 0, uW = 0, uN = 0, uS = 0;
          for (int k = 0; k < np; ++k) {
            double ck = uc[v * np + k];
            uE += ck * (t.Pp[A[k]] * t.P0[Bm[k]]);
            uW += ck * (t.Pm[A[k]] * t.P0[Bm[k]]);
            uN += ck * (t.P0[A[k]] * t.Pp[Bm[k]]);
            uS += ck * (t.P0[A[k]] * t.Pm[Bm[k]]);
          }
          double dpx = mE - mean, dmx = mean - mW, dpy = mN - mean, dmy = mean - mS;
          fl |= tvb_changes(uE - mean, dpx, dmx, Mx, &near);
          fl |= tvb_changes(mean - uW, dpx, dmx, Mx, &near);
          fl |= tvb_changes(uN - mean, dpy, dmy, My, &near);
          fl |= tvb_changes(mean - uS, dpy, dmy, My, &near);
        }
        flags[(size_t)iy * m->nx + ix] = (unsigned char)fl;
        if (near_cells) near_cells[(size_t)iy * m->nx + ix] = (unsigned char)near;
        nf += fl;
        nn += near;
      }
  }
  if (n_near) *n_near = nn;
  return nf;
}

long or_flag_tvb(const or_mesh* m, const double* u, double M, unsigned char* flags, long* n_near) {
  return or_flag_tvb_cells(m, u, M, flags, NULL, n_near);
}

/* ------------------------------------------------------------------------------------
 * KXRCF troubled-cell indicator (Sec. 3, step 1: the paper's own choice, after
 * Krivodonova et al., ref. [kxrcf]).  For an indicator variable w of cell j,
 *   I_j = | int_{dI_j^-} (w_j - w_nb) ds | / ( r^{(N+1)/2} |dI_j^-| ||w_j|| ),
 * dI_j^- the inflow part of the boundary, r the radius of the circle circumscribing the
 * cell, ||w_j|| the largest |w_j| over the cell's (N+1)^dim Gauss points; the cell is
 * troubled when I_j > 1.  Readings (the paper prints no formula): inflow faces are those
 * whose outward normal has a negative product with the mean velocity (Euler m/rho, its
 * sign taken from the mean momentum; Burgers f'(ubar) = ubar in every direction); a
 * face integral is the (N+1)-point Gauss rule along the face (a point value in 1D, where
 * |dI^-| counts inflow faces); the indicator variables are u for Burgers and the density
 * and the total energy for Euler (either one flags the cell); neighbours follow the
 * boundary condition as in the scheme.  The decision is num > den without a division,
 * and near (reporting) when the two are within 1e-12 relative (rel_near).
 * ----------------------------------------------------------------------------------*/
static void kx_ratio(double an, double den, double* r) {
  const double q = den > 0.0 ? an / den : (an > 0.0 ? INFINITY : 0.0);
  if (q > *r) *r = q;
}

/* ratio (optional): the largest I_j over the indicator variables (0 without inflow);
 * near_cells (optional): 1 for each near-threshold cell. */
long or_flag_kxrcf_cells(const or_mesh* m, const double* u, unsigned char* flags, unsigned char* near_cells,
                         long* n_near, double* ratio) {
  const int N = m->N, nv = or_nvars(m->dim, m->pde), np = or_nmodes(m->dim, N);
  or_dg_tables t;
  dg_tables(N, N + 1, &t);
  const int nq = N + 1;
  const int wv[2] = {0, nv - 1};
  const int nw = m->pde == 0 ? 1 : 2;
  long nf = 0, nn = 0;
  if (m->dim == 1) {
    const double h = (m->xR - m->xL) / m->nx;
    const double hp = pow(0.5 * h, 0.5 * (N + 1));
    for (int c = 0; c < m->nx; ++c) {
      double uc[OR_MAXV * 4], ul[OR_MAXV * 4], ur[OR_MAXV * 4];
      cell_modes(m, u, c, 0, uc);
      cell_modes(m, u, c - 1, 0, ul);
      cell_modes(m, u, c + 1, 0, ur);
      /* mean velocity sign: Burgers ubar, Euler mbar (rho > 0) */
      const double vel = m->pde == 0 ? uc[0] : uc[np];
      int fl = 0, near = 0;
      double rmax = 0.0;
      for (int iw = 0; iw < nw; ++iw) {
        const int v = wv[iw];
        double num = 0.0, len = 0.0;
        if (vel > 0.0) { /* left face x = -1 is inflow */
          double a = 0.0, b = 0.0;
          for (int k = 0; k < np; ++k) a += uc[v * np + k] * t.Pm[k];
          for (int k = 0; k < np; ++k) b += ul[v * np + k] * t.Pp[k];
          num += a - b;
          len += 1.0;
        }
        if (vel < 0.0) { /* right face x = +1 */
          double a = 0.0, b = 0.0;
          for (int k = 0; k < np; ++k) a += uc[v * np + k] * t.Pp[k];
          for (int k = 0; k < np; ++k) b += ur[v * np + k] * t.Pm[k];
          num += a - b;
          len += 1.0;
        }
        if (len == 0.0) continue;
        double nrm = 0.0;
        for (int q = 0; q < nq; ++q) {
          double a = 0.0;
          for (int k = 0; k < np; ++k) a += uc[v * np + k] * t.P[q][k];
          if (fabs(a) > nrm) nrm = fabs(a);
        }
        const double den = hp * len * nrm, an = fabs(num);
        if (rel_near(an, den)) near = 1;
        if (an > den) fl = 1;
        kx_ratio(an, den, &rmax);
      }
      if (ratio) ratio[c] = rmax;
      flags[c] = (unsigned char)fl;
      if (near_cells) near_cells[c] = (unsigned char)near;
      nf += fl;
      nn += near;
    }
  } else {
    const double hx = (m->xR - m->xL) / m->nx, hy = (m->yR - m->yL) / m->ny;
    const double hp = pow(0.5 * sqrt(hx * hx + hy * hy), 0.5 * (N + 1));
    int A[OR_MAXNP], Bm[OR_MAXNP];
    for (int k = 0; k < np; ++k) mode_ab(k, &A[k], &Bm[k]);
    for (int iy = 0; iy < m->ny; ++iy)
      for (int ix = 0; ix < m->nx; ++ix) {
        double uc[OR_MAXV * OR_MAXNP], nb[4][OR_MAXV * OR_MAXNP];
        cell_modes(m, u, ix, iy, uc);
        cell_modes(m, u, ix - 1, iy, nb[0]);
        cell_modes(m, u, ix + 1, iy, nb[1]);
        cell_modes(m, u, ix, iy - 1, nb[2]);
        cell_modes(m, u, ix, iy + 1, nb[3]);
        const double vx = m->pde == 0 ? uc[0] : uc[np], vy = m->pde == 0 ? uc[0] : uc[2 * np];
        /* faces W, E, S, N: inflow test, face length, own side, neighbour side */
        const int in[4] = {vx > 0.0, vx < 0.0, vy > 0.0, vy < 0.0};
        const double flen[4] = {hy, hy, hx, hx};
        int fl = 0, near = 0;
        double rmax = 0.0;
        for (int iw = 0; iw < nw; ++iw) {
          const int v = wv[iw];
          double num = 0.0, len = 0.0;
          for (int f = 0; f < 4; ++f) {
            if (!in[f]) continue;
            double s = 0.0;
            for (int q = 0; q < nq; ++q) {
              double a = 0.0, b = 0.0;
              for (int k = 0; k < np; ++k) {
                /* own face point and the neighbour's matching point */
                double po, pn;
                if (f == 0) { po = t.Pm[A[k]] * t.P[q][Bm[k]]; pn = t.Pp[A[k]] * t.P[q][Bm[k]]; }
                else if (f == 1) { po = t.Pp[A[k]] * t.P[q][Bm[k]]; pn = t.Pm[A[k]] * t.P[q][Bm[k]]; }
                else if (f == 2) { po = t.P[q][A[k]] * t.Pm[Bm[k]]; pn = t.P[q][A[k]] * t.Pp[Bm[k]]; }
                else { po = t.P[q][A[k]] * t.Pp[Bm[k]]; pn = t.P[q][A[k]] * t.Pm[Bm[k]]; }
                a += uc[v * np + k] * po;
                b += nb[f][v * np + k] * pn;
              }
              s += t.w[q] * (a - b);
            }
            num += s * (0.5 * flen[f]);
            len += flen[f];
          }
          if (len == 0.0) continue;
          double nrm = 0.0;
          for (int qx = 0; qx < nq; ++qx)
            for (int qy = 0; qy < nq; ++qy) {
              double a = 0.0;
              for (int k = 0; k < np; ++k) a += uc[v * np + k] * (t.P[qx][A[k]] * t.P[qy][Bm[k]]);
              if (fabs(a) > nrm) nrm = fabs(a);
            }
          const double den = hp * len * nrm, an = fabs(num);
          if (rel_near(an, den)) near = 1;
          if (an > den) fl = 1;
          kx_ratio(an, den, &rmax);
        }
        if (ratio) ratio[(size_t)iy * m->nx + ix] = rmax;
        flags[(size_t)iy * m->nx + ix] = (unsigned char)fl;
        if (near_cells) near_cells[(size_t)iy * m->nx + ix] = (unsigned char)near;
        nf += fl;
        nn += near;
      }
  }
  if (n_near) *n_near = nn;
  return nf;
}

long or_flag_kxrcf(const or_mesh* m, const double* u, unsigned char* flags, long* n_near, double* ratio) {
  return or_flag_kxrcf_cells(m, u, flags, NULL, n_near, ratio);
}

/* ------------------------------------------------------------------------------------
 * Local characteristic decomposition for the Euler systems (Sec. 3, "local
 * characteristic field decomposition"): right/left eigenvectors of the flux Jacobian
 * in direction dir at the state u (conserved).  R columns, L rows, L R = I.
 * ----------------------------------------------------------------------------------*/
void or_euler_eigen(int dim, double gam, int dir, const double* u, double* R, double* L) {
  if (dim == 1) {
    double rho = u[0], vel = u[1] / rho, E = u[2];
    double p = (gam - 1.0) * (E - 0.5 * rho * vel * vel);
    double c = sqrt(gam * p / rho), H = (E + p) / rho;
    double b1 = (gam - 1.0) / (c * c), b2 = 0.5 * b1 * vel * vel;
    double Rm[3][3] = {{1.0, 1.0, 1.0}, {vel - c, vel, vel + c}, {H - vel * c, 0.5 * vel * vel, H + vel * c}};
    double Lm[3][3] = {{0.5 * (b2 + vel / c), 0.5 * (-b1 * vel - 1.0 / c), 0.5 * b1},
                       {1.0 - b2, b1 * vel, -b1},
                       {0.5 * (b2 - vel / c), 0.5 * (-b1 * vel + 1.0 / c), 0.5 * b1}};
    memcpy(R, Rm, sizeof(Rm));
    memcpy(L, Lm, sizeof(Lm));
    return;
  }
  double rho = u[0], E = u[3];
  double vx = u[1] / rho, vy = u[2] / rho;
  double q2 = vx * vx + vy * vy;
  double p = (gam - 1.0) * (E - 0.5 * rho * q2);
  double c = sqrt(gam * p / rho), H = (E + p) / rho;
  double b1 = (gam - 1.0) / (c * c), b2 = 0.5 * b1 * q2;
  /* normal velocity vn, tangential vt; index of the normal / tangential momentum */
  double vn = dir == 0 ? vx : vy, vt = dir == 0 ? vy : vx;
  int in = dir == 0 ? 1 : 2, it = dir == 0 ? 2 : 1;
  double Rm[4][4], Lm[4][4];
  memset(Rm, 0, sizeof(Rm));
  memset(Lm, 0, sizeof(Lm));
  /* columns: vn - c, vn (entropy), vn (shear), vn + c */
  Rm[0][0] = 1.0;     Rm[in][0] = vn - c;  Rm[it][0] = vt;  Rm[3][0] = H - vn * c;
  Rm[0][1] = 1.0;     Rm[in][1] = vn;      Rm[it][1] = vt;  Rm[3][1] = 0.5 * q2;
  Rm[0][2] = 0.0;     Rm[in][2] = 0.0;     Rm[it][2] = 1.0; Rm[3][2] = vt;
  Rm[0][3] = 1.0;     Rm[in][3] = vn + c;  Rm[it][3] = vt;  Rm[3][3] = H + vn * c;
  Lm[0][0] = 0.5 * (b2 + vn / c); Lm[0][in] = 0.5 * (-b1 * vn - 1.0 / c); Lm[0][it] = -0.5 * b1 * vt; Lm[0][3] = 0.5 * b1;
  Lm[1][0] = 1.0 - b2;           Lm[1][in] = b1 * vn;                    Lm[1][it] = b1 * vt;        Lm[1][3] = -b1;
  Lm[2][0] = -vt;                Lm[2][in] = 0.0;                        Lm[2][it] = 1.0;            Lm[2][3] = 0.0;
  Lm[3][0] = 0.5 * (b2 - vn / c); Lm[3][in] = 0.5 * (-b1 * vn + 1.0 / c); Lm[3][it] = -0.5 * b1 * vt; Lm[3][3] = 0.5 * b1;
  memcpy(R, Rm, sizeof(Rm));
  memcpy(L, Lm, sizeof(Lm));
}

/* ------------------------------------------------------------------------------------
 * One 1D WENO reconstruction (Steps 2-5) on the 2N+1 stencil averages 'avg' at every
 * reconstruction point.  Eq. (14) is read as  wbar_i = gamma_i / (eps + beta_i)^2
 * (the printed sum in the denominator is a typesetting slip), Eq. (15) as
 * u_G = sum_i omega_i p_i(x_G).  Where a linear weight is negative (P3 with thirds)
 * the split of Shi, Hu & Shu is used: gamma = sigma+ gamma~+ - sigma- gamma~-,
 * gamma+_i = (gamma_i + theta |gamma_i|)/2, theta = 3, each part normalised and
 * combined as sigma+ u+ - sigma- u-.
 * ----------------------------------------------------------------------------------*/
static void weno_1d(const or_weno_tables* t, const double* avg, double eps, double* out) {
  int N = t->N, ns = t->ns;
  /* Every p_i reproduces constants and Eq. (13) only involves derivatives, so beta_i and
   * p_i - c are unchanged when the constant c is removed from all averages.  Evaluating
   * them on the averages centred at the troubled cell's own average avoids the
   * cancellation of O(1) terms in a quadratic form whose value is O(eps). */
  double c = avg[N], d[OR_MAXS];
  for (int k = 0; k < ns; ++k) d[k] = avg[k] - c;
  double beta[OR_MAXN + 1];
  for (int i = 0; i <= N; ++i) {
    double s = 0;
    for (int k = 0; k < ns; ++k)
      for (int l = 0; l < ns; ++l) s += d[k] * t->B[i][k][l] * d[l];
    beta[i] = s;
  }
  for (int g = 0; g < t->ng; ++g) {
    double p[OR_MAXN + 1];
    int negative = 0;
    for (int i = 0; i <= N; ++i) {
      double s = 0;
      for (int k = 0; k < ns; ++k) s += t->C[i][g][k] * d[k];
      p[i] = c + s;
      if (t->gam[g][i] < 0) negative = 1;
    }
    if (!negative) {
      double wb[OR_MAXN + 1], sw = 0, r = 0;
      for (int i = 0; i <= N; ++i) {
        wb[i] = t->gam[g][i] / ((eps + beta[i]) * (eps + beta[i]));
        sw += wb[i];
      }
      for (int i = 0; i <= N; ++i) r += (wb[i] / sw) * p[i];
      out[g] = r;
    } else {
      const double theta = 3.0;
      double gp[OR_MAXN + 1], gm[OR_MAXN + 1], sp = 0, sm = 0;
      for (int i = 0; i <= N; ++i) {
        gp[i] = 0.5 * (t->gam[g][i] + theta * fabs(t->gam[g][i]));
        gm[i] = gp[i] - t->gam[g][i];
        sp += gp[i];
        sm += gm[i];
      }
      double wp[OR_MAXN + 1], wm[OR_MAXN + 1], swp = 0, swm = 0, up = 0, um = 0;
      for (int i = 0; i <= N; ++i) {
        double d = (eps + beta[i]) * (eps + beta[i]);
        wp[i] = (gp[i] / sp) / d;
        wm[i] = (gm[i] / sm) / d;
        swp += wp[i];
        swm += wm[i];
      }
      for (int i = 0; i <= N; ++i) {
        up += (wp[i] / swp) * p[i];
        um += (wm[i] / swm) * p[i];
      }
      out[g] = sp * up - sm * um;
    }
  }
}

/* ------------------------------------------------------------------------------------
 * CSWENO limiter (Sec. 3).  For every flagged cell: keep U_0 (the cell average), build
 * the stencil of subcell averages from the immediate neighbours (Fig. 1), reconstruct
 * point values at the Step 1 points by WENO (Steps 2-5; in characteristic variables
 * for Euler), and project back to modes 1..N (Eq. (16), orthonormal basis):
 *   U_i = sum_G w_G u(r_G) psi_i(r_G).
 * In 2D (our reading of the short 2D paragraph): the (2N+1)^2 array of sub-rectangle
 * averages of the 3x3 neighbourhood is swept in x (each row -> row-averaged values at
 * the x points), then in y (each x point -> point values), then projected with the
 * tensor rule onto the modes with 1 <= a+b <= N.  Characteristic fields use the x-
 * (resp. y-) Jacobian eigenvectors at the troubled cell's mean state.
 * Updates are Jacobi: every flagged cell reads the unlimited input u; results go to
 * out (which starts as a copy of u).  eps is the WENO epsilon (1e-6 in the paper).
 * ----------------------------------------------------------------------------------*/
static void weno_limit_g(const or_mesh* m, const double* u, const unsigned char* flags, double* out, double eps,
                         int parent) {
  int N = m->N, nv = or_nvars(m->dim, m->pde), np = or_nmodes(m->dim, N);
  size_t ncell = (size_t)m->nx * m->ny;
  or_weno_tables t;
  weno_tables_build_g(N, parent, 0, NULL, &t);
  int ns = t.ns, ng = t.ng;
  const int reach = parent ? N : 1; /* neighbourhood reach */
  memcpy(out, u, ncell * nv * np * sizeof(double));
  if (m->dim == 1) {
    for (int c = 0; c < m->nx; ++c) {
      if (!flags[c]) continue;
      double nbm[OR_MAXS][OR_MAXV * 4];
      for (int d = -reach; d <= reach; ++d) cell_modes(m, u, c + d, 0, nbm[d + reach]);
      /* subcell averages per conserved variable */
      double avg[OR_MAXV][OR_MAXS];
      for (int v = 0; v < nv; ++v)
        for (int k = 0; k < ns; ++k) {
          const double* src = nbm[t.OFF[k] + reach] + v * np;
          double s = 0;
          for (int n = 0; n < np; ++n) s += src[n] * t.SA[k][n];
          avg[v][k] = s;
        }
      double val[OR_MAXV][OR_MAXG];
      if (m->pde == 1) {
        double mean[3], R[9], L[9], w[3][OR_MAXS], wv[3][OR_MAXG];
        for (int v = 0; v < 3; ++v) mean[v] = nbm[reach][v * np] * t.SA[N][0];
        or_euler_eigen(1, m->gamma, 0, mean, R, L);
        for (int f = 0; f < 3; ++f)
          for (int k = 0; k < ns; ++k) {
            double s = 0;
            for (int v = 0; v < 3; ++v) s += L[f * 3 + v] * avg[v][k];
            w[f][k] = s;
          }
        for (int f = 0; f < 3; ++f) weno_1d(&t, w[f], eps, wv[f]);
        for (int v = 0; v < 3; ++v)
          for (int g = 0; g < ng; ++g) {
            double s = 0;
            for (int f = 0; f < 3; ++f) s += R[v * 3 + f] * wv[f][g];
            val[v][g] = s;
          }
      } else {
        weno_1d(&t, avg[0], eps, val[0]);
      }
      for (int v = 0; v < nv; ++v)
        for (int n = 1; n < np; ++n) {
          double s = 0;
          for (int g = 0; g < ng; ++g) s += t.wt[g] * val[v][g] * t.psiG[g][n];
          out[((size_t)c * nv + v) * np + n] = s;
        }
    }
    return;
  }
  int A[OR_MAXNP], Bm[OR_MAXNP];
  for (int k = 0; k < np; ++k) mode_ab(k, &A[k], &Bm[k]);
  for (int iy = 0; iy < m->ny; ++iy)
    for (int ix = 0; ix < m->nx; ++ix) {
      size_t c = (size_t)iy * m->nx + ix;
      if (!flags[c]) continue;
      double nbm[OR_MAXS][OR_MAXS][OR_MAXV * OR_MAXNP];
      for (int dy = -reach; dy <= reach; ++dy)
        for (int dx = -reach; dx <= reach; ++dx) cell_modes(m, u, ix + dx, iy + dy, nbm[dy + reach][dx + reach]);
      /* sub-rectangle averages avg[v][ky][kx] */
      double avg[OR_MAXV][OR_MAXS][OR_MAXS];
      for (int v = 0; v < nv; ++v)
        for (int ky = 0; ky < ns; ++ky)
          for (int kx = 0; kx < ns; ++kx) {
            const double* src = nbm[t.OFF[ky] + reach][t.OFF[kx] + reach] + v * np;
            double s = 0;
            for (int k = 0; k < np; ++k) s += src[k] * t.SA[kx][A[k]] * t.SA[ky][Bm[k]];
            avg[v][ky][kx] = s;
          }
      double mean[OR_MAXV];
      for (int v = 0; v < nv; ++v) mean[v] = nbm[reach][reach][v * np] * t.SA[N][0] * t.SA[N][0];
      double Rx[16], Lx[16], Ry[16], Ly[16];
      if (m->pde == 1) {
        or_euler_eigen(2, m->gamma, 0, mean, Rx, Lx);
        or_euler_eigen(2, m->gamma, 1, mean, Ry, Ly);
      }
      /* x-sweep: rowval[v][ky][g] = average over row ky of u(x_g, y) */
      double rowval[OR_MAXV][OR_MAXS][OR_MAXG];
      for (int ky = 0; ky < ns; ++ky) {
        if (m->pde == 1) {
          double w[4][OR_MAXS], wv[4][OR_MAXG];
          for (int f = 0; f < 4; ++f)
            for (int kx = 0; kx < ns; ++kx) {
              double s = 0;
              for (int v = 0; v < 4; ++v) s += Lx[f * 4 + v] * avg[v][ky][kx];
              w[f][kx] = s;
            }
          for (int f = 0; f < 4; ++f) weno_1d(&t, w[f], eps, wv[f]);
          for (int v = 0; v < 4; ++v)
            for (int g = 0; g < ng; ++g) {
              double s = 0;
              for (int f = 0; f < 4; ++f) s += Rx[v * 4 + f] * wv[f][g];
              rowval[v][ky][g] = s;
            }
        } else {
          weno_1d(&t, avg[0][ky], eps, rowval[0][ky]);
        }
      }
      /* y-sweep: pv[v][gy][gx] = u(x_gx, y_gy) */
      double pv[OR_MAXV][OR_MAXG][OR_MAXG];
      for (int gx = 0; gx < ng; ++gx) {
        double col[OR_MAXV][OR_MAXS];
        for (int v = 0; v < nv; ++v)
          for (int ky = 0; ky < ns; ++ky) col[v][ky] = rowval[v][ky][gx];
        if (m->pde == 1) {
          double w[4][OR_MAXS], wv[4][OR_MAXG];
          for (int f = 0; f < 4; ++f)
            for (int ky = 0; ky < ns; ++ky) {
              double s = 0;
              for (int v = 0; v < 4; ++v) s += Ly[f * 4 + v] * col[v][ky];
              w[f][ky] = s;
            }
          for (int f = 0; f < 4; ++f) weno_1d(&t, w[f], eps, wv[f]);
          for (int v = 0; v < 4; ++v)
            for (int gy = 0; gy < ng; ++gy) {
              double s = 0;
              for (int f = 0; f < 4; ++f) s += Ry[v * 4 + f] * wv[f][gy];
              pv[v][gy][gx] = s;
            }
        } else {
          double wv[OR_MAXG];
          weno_1d(&t, col[0], eps, wv);
          for (int gy = 0; gy < ng; ++gy) pv[0][gy][gx] = wv[gy];
        }
      }
      for (int v = 0; v < nv; ++v)
        for (int k = 1; k < np; ++k) {
          double s = 0;
          for (int gy = 0; gy < ng; ++gy)
            for (int gx = 0; gx < ng; ++gx)
              s += t.wt[gx] * t.wt[gy] * pv[v][gy][gx] * t.psiG[gx][A[k]] * t.psiG[gy][Bm[k]];
          out[(c * nv + v) * np + k] = s;
        }
    }
}

/* The 1D reconstruction (Steps 2-5) alone: from the 2N+1 stencil averages avg (the
 * subcells of Fig. 1, or the whole cells j-N..j+N when parent is set) to the point
 * values out[NG] at the Step 1 points (in the order or_weno_export gives them). */
void or_weno_points(int N, int parent, const double* avg, double eps, double* out) {
  or_weno_tables t;
  weno_tables_build_g(N, parent, 0, NULL, &t);
  weno_1d(&t, avg, eps, out);
}

void or_csweno_limit(const or_mesh* m, const double* u, const unsigned char* flags, double* out, double eps) {
  weno_limit_g(m, u, flags, out, eps, 0);
}

/* The parent WENO limiter of Qiu and Shu (ref. [qs1]), the paper's main comparison (Sec.
 * 4): the same reconstruction as or_csweno_limit on the whole cells j-N..j+N (their cell
 * averages) instead of subcells of the immediate neighbours; in 2D on the (2N+1)^2 cell
 * averages around the troubled cell.  Needs N cells on each side (ghosts reflect). */
void or_parent_weno_limit(const or_mesh* m, const double* u, const unsigned char* flags, double* out, double eps) {
  weno_limit_g(m, u, flags, out, eps, 1);
}

/* ------------------------------------------------------------------------------------
 * One full SSP-RK3 step with the limiter after every stage (Sec. 3, last paragraph:
 * the semi-discrete scheme "along with the limiter" is integrated in time).  limit = 0
 * gives the unlimited scheme.  Returns the number of flagged cells over the 3 stages.
 * ----------------------------------------------------------------------------------*/
long or_step(const or_mesh* m, double dt, double* u, double M, int limit, double eps, long* n_near) {
  size_t ncell = (size_t)m->nx * m->ny;
  size_t n = ncell * or_nvars(m->dim, m->pde) * or_nmodes(m->dim, m->N);
  double* un = (double*)malloc(n * sizeof(double));   /* u^n */
  double* keep = (double*)malloc(n * sizeof(double)); /* u^(s-1) for s >= 2 */
  double* a = (double*)malloc(n * sizeof(double));
  double* b = (double*)malloc(n * sizeof(double));
  unsigned char* fl = (unsigned char*)malloc(ncell);
  long nf = 0, nn = 0, near = 0;
  memcpy(un, u, n * sizeof(double));
  const double* prev = un;
  /* m->t is the time of u^n; stage s evaluates L at the time of u^(s-1) (t, t + dt,
   * t + dt/2) and its output holds at t + dt, t + dt/2, t + dt (time-dependent boundary
   * data only) */
  const double c_in[3] = {0.0, 1.0, 0.5}, c_out[3] = {1.0, 0.5, 1.0};
  or_mesh ms = *m;
  for (int s = 1; s <= 3; ++s) {
    ms.t = m->t + c_in[s - 1] * dt;
    or_rk_stage(&ms, s, dt, un, prev, a);
    ms.t = m->t + c_out[s - 1] * dt;
    if (limit) {
      nf += or_flag_tvb(&ms, a, M, fl, &near);
      nn += near;
      or_csweno_limit(&ms, a, fl, b, eps);
      double* t = a; a = b; b = t;
    }
    memcpy(keep, a, n * sizeof(double));
    prev = keep;
  }
  memcpy(u, a, n * sizeof(double));
  if (n_near) *n_near = nn;
  free(un); free(keep); free(a); free(b); free(fl);
  return nf;
}

/* ------------------------------------------------------------------------------------
 * Positivity-preserving scaling (Example 11 adds it to the limiter, following Zhang and
 * Shu, ref. [zs3]), Euler only.  For each cell with mean state Ubar (rho > 0, p > 0):
 *   eps = min(eps0, rhobar, pbar);
 *   S   = the check points: in 1D the L-point Gauss-Lobatto rule with 2L-3 >= N
 *         (L = 2 for N = 1, else 3); in 2D the union of (Gauss x Gauss-Lobatto) and
 *         (Gauss-Lobatto x Gauss) with the (N+1)-point Gauss rule of the face integrals;
 *   1) rho_min = min_S rho_h; if rho_min < eps the density's modes n >= 1 are scaled
 *      by theta1 = (rhobar - eps) / (rhobar - rho_min);
 *   2) for every q in S with p(U_q) < eps (U_q the point value after step 1), t_q in
 *      [0,1] solves p((1-t) Ubar + t U_q) = eps; theta2 = min_q t_q (1 when no point
 *      is below eps) scales the modes n >= 1 of every variable.
 * Multiplying p by the positive density turns the equation of step 2 into the quadratic
 *   A t^2 + B t + C = 0,  D = U_q - Ubar,
 *   A = (g-1) (D_E D_rho - |D_m|^2 / 2),
 *   B = (g-1) (Ebar D_rho + rhobar D_E - mbar . D_m) - eps D_rho,
 *   C = (g-1) (Ebar rhobar - |mbar|^2 / 2) - eps rhobar  (= rhobar (pbar - eps) >= 0),
 * which changes sign on [0,1] (C >= 0 > value at t = 1); its root there is taken from the
 * cancellation-free pair q = -(B + sign(B) sqrt(B^2 - 4AC)) / 2, roots q/A and C/q, and
 * moved 1e-12 (relative) towards 0: near vacuum p changes by ~1e5 per unit of t, so a
 * root rounded by one ulp could leave p below zero, while the shift raises p by far
 * more than that rounding (p is concave along the segment, so every t below the root
 * is admissible).
 * Cells whose mean is not admissible are left alone and counted in *n_bad.  Returns the
 * number of cells changed.
 * ----------------------------------------------------------------------------------*/
static double pp_pressure(int dim, double gam, const double* q) {
  const int nv = dim == 1 ? 3 : 4;
  double k = q[1] * q[1];
  if (dim == 2) k += q[2] * q[2];
  return (gam - 1.0) * (q[nv - 1] - 0.5 * k / q[0]);
}

static double pp_root(int dim, double gam, double eps, const double* ub, const double* uq) {
  const int nv = dim == 1 ? 3 : 4;
  const double g1 = gam - 1.0;
  double D[OR_MAXV];
  for (int v = 0; v < nv; ++v) D[v] = uq[v] - ub[v];
  double dm2 = D[1] * D[1], mdm = ub[1] * D[1], m2 = ub[1] * ub[1];
  if (dim == 2) { dm2 += D[2] * D[2]; mdm += ub[2] * D[2]; m2 += ub[2] * ub[2]; }
  const double A = g1 * (D[nv - 1] * D[0] - 0.5 * dm2);
  const double B = g1 * (ub[nv - 1] * D[0] + ub[0] * D[nv - 1] - mdm) - eps * D[0];
  const double C = g1 * (ub[nv - 1] * ub[0] - 0.5 * m2) - eps * ub[0];
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

long or_positivity_limit(const or_mesh* m, double* u, double eps0, long* n_bad) {
  if (m->pde != 1) return -1;
  const int dim = m->dim, N = m->N, nv = or_nvars(dim, 1), np = or_nmodes(dim, N);
  const int L = N == 1 ? 2 : 3;
  const ld glx[3] = {-1.0L, 0.0L, 1.0L}, glx2[2] = {-1.0L, 1.0L};
  const ld* gl = L == 2 ? glx2 : glx;
  ld gx[OR_MAXQ], gw[OR_MAXQ];
  gauss_rule(N + 1, gx, gw);
  /* check points (r, s) and the basis values there */
  int npt = 0;
  double phi[2 * OR_MAXQ * 3][OR_MAXNP];
  if (dim == 1) {
    for (int i = 0; i < L; ++i, ++npt)
      for (int k = 0; k < np; ++k) phi[npt][k] = (double)psi(k, gl[i]);
  } else {
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i <= N; ++i)
        for (int j = 0; j < L; ++j, ++npt) {
          const ld r = pass == 0 ? gx[i] : gl[j], t = pass == 0 ? gl[j] : gx[i];
          for (int k = 0; k < np; ++k) {
            int a, b;
            mode_ab(k, &a, &b);
            phi[npt][k] = (double)(psi(a, r) * psi(b, t));
          }
        }
  }
  const double c0 = dim == 1 ? (double)psi(0, 0) : (double)(psi(0, 0) * psi(0, 0));
  long changed = 0, bad = 0;
  for (size_t c = 0; c < (size_t)m->nx * m->ny; ++c) {
    double* uc = u + c * nv * np;
    double ub[OR_MAXV];
    for (int v = 0; v < nv; ++v) ub[v] = uc[v * np] * c0;
    const double pb = pp_pressure(dim, m->gamma, ub);
    if (!(ub[0] > 0.0) || !(pb > 0.0)) { ++bad; continue; }
    double eps = eps0;
    if (ub[0] < eps) eps = ub[0];
    if (pb < eps) eps = pb;
    int touched = 0;
    /* 1) density */
    double rmin = ub[0];
    for (int q = 0; q < npt; ++q) {
      double r = 0.0;
      for (int k = 0; k < np; ++k) r += uc[k] * phi[q][k];
      if (r < rmin) rmin = r;
    }
    if (rmin < eps) {
      const double th1 = (ub[0] - eps) / (ub[0] - rmin);
      for (int k = 1; k < np; ++k) uc[k] *= th1;
      touched = 1;
    }
    /* 2) pressure */
    double th2 = 1.0;
    for (int q = 0; q < npt; ++q) {
      double uq[OR_MAXV];
      for (int v = 0; v < nv; ++v) {
        double s = 0.0;
        for (int k = 0; k < np; ++k) s += uc[v * np + k] * phi[q][k];
        uq[v] = s;
      }
      if (pp_pressure(dim, m->gamma, uq) < eps) {
        const double t = pp_root(dim, m->gamma, eps, ub, uq);
        if (t < th2) th2 = t;
      }
    }
    if (th2 < 1.0) {
      for (int v = 0; v < nv; ++v)
        for (int k = 1; k < np; ++k) uc[v * np + k] *= th2;
      touched = 1;
    }
    changed += touched;
  }
  if (n_bad) *n_bad = bad;
  return changed;
}

/* One SSP-RK3 step as or_step with the indicator ind (0 TVB with constant M, 2 KXRCF)
 * and, when pp is set (Euler), the positivity-preserving scaling after the limiter of
 * every stage.  *n_pp (if given) receives the number of cell changes over the three
 * stages and *n_bad the cells whose mean was not admissible. */
/* Largest characteristic speed |v_d| + c over the check points of the positivity-
 * preserving scaling (the Gauss-Lobatto points in 1D; Gauss x Gauss-Lobatto and
 * Gauss-Lobatto x Gauss in 2D), per direction.  Zhang and Shu's condition for admissible
 * means bounds the time step by the wave speeds of these point values, not of the cell
 * means.  Points without a real sound speed are skipped.  Euler only (returns -1). */
int or_max_wavespeed_points(const or_mesh* m, const double* u, double* out) {
  if (m->pde != 1) return -1;
  const int dim = m->dim, N = m->N, nv = or_nvars(dim, 1), np = or_nmodes(dim, N);
  const int L = N == 1 ? 2 : 3;
  const ld glx[3] = {-1.0L, 0.0L, 1.0L}, glx2[2] = {-1.0L, 1.0L};
  const ld* gl = L == 2 ? glx2 : glx;
  ld gx[OR_MAXQ], gw[OR_MAXQ];
  gauss_rule(N + 1, gx, gw);
  int npt = 0;
  double phi[2 * OR_MAXQ * 3][OR_MAXNP];
  if (dim == 1) {
    for (int i = 0; i < L; ++i, ++npt)
      for (int k = 0; k < np; ++k) phi[npt][k] = (double)psi(k, gl[i]);
  } else {
    for (int pass = 0; pass < 2; ++pass)
      for (int i = 0; i <= N; ++i)
        for (int j = 0; j < L; ++j, ++npt) {
          const ld r = pass == 0 ? gx[i] : gl[j], t = pass == 0 ? gl[j] : gx[i];
          for (int k = 0; k < np; ++k) {
            int a, b;
            mode_ab(k, &a, &b);
            phi[npt][k] = (double)(psi(a, r) * psi(b, t));
          }
        }
  }
  out[0] = out[1] = 0.0;
  for (size_t c = 0; c < (size_t)m->nx * m->ny; ++c) {
    const double* uc = u + c * nv * np;
    for (int q = 0; q < npt; ++q) {
      double w[OR_MAXV];
      for (int v = 0; v < nv; ++v) {
        double s = 0.0;
        for (int k = 0; k < np; ++k) s += uc[v * np + k] * phi[q][k];
        w[v] = s;
      }
      for (int d = 0; d < dim; ++d) {
        const double sp = max_speed(dim, 1, m->gamma, d, w);
        if (sp > out[d]) out[d] = sp; /* a NaN speed never compares greater */
      }
    }
  }
  return 0;
}

long or_step_gen(const or_mesh* m, double dt, double* u, int ind, double M, int limit, double eps, int pp,
                 double pp_eps, long* n_near, long* n_pp, long* n_bad);
long or_step_ind(const or_mesh* m, double dt, double* u, int ind, double M, int limit, double eps, int pp,
                 double pp_eps, long* n_near, long* n_pp, long* n_bad) {
  return or_step_gen(m, dt, u, ind, M, limit, eps, pp, pp_eps, n_near, n_pp, n_bad);
}

/* limit: 0 none, 1 CSWENO, 2 parent WENO */
long or_step_gen(const or_mesh* m, double dt, double* u, int ind, double M, int limit, double eps, int pp,
                 double pp_eps, long* n_near, long* n_pp, long* n_bad) {
  size_t ncell = (size_t)m->nx * m->ny;
  size_t n = ncell * or_nvars(m->dim, m->pde) * or_nmodes(m->dim, m->N);
  double* un = (double*)malloc(n * sizeof(double));
  double* keep = (double*)malloc(n * sizeof(double));
  double* a = (double*)malloc(n * sizeof(double));
  double* b = (double*)malloc(n * sizeof(double));
  unsigned char* fl = (unsigned char*)malloc(ncell);
  long nf = 0, nn = 0, near = 0, np_ = 0, nb = 0, bad = 0;
  memcpy(un, u, n * sizeof(double));
  const double* prev = un;
  const double c_in[3] = {0.0, 1.0, 0.5}, c_out[3] = {1.0, 0.5, 1.0};  /* as in or_step */
  or_mesh ms = *m;
  for (int s = 1; s <= 3; ++s) {
    ms.t = m->t + c_in[s - 1] * dt;
    or_rk_stage(&ms, s, dt, un, prev, a);
    ms.t = m->t + c_out[s - 1] * dt;
    if (limit) {
      nf += ind == 2 ? or_flag_kxrcf(&ms, a, fl, &near, NULL) : or_flag_tvb(&ms, a, M, fl, &near);
      nn += near;
      if (limit == 2) or_parent_weno_limit(&ms, a, fl, b, eps);
      else or_csweno_limit(&ms, a, fl, b, eps);
      double* t = a; a = b; b = t;
    }
    if (pp) {
      np_ += or_positivity_limit(&ms, a, pp_eps, &bad);
      nb += bad;
    }
    memcpy(keep, a, n * sizeof(double));
    prev = keep;
  }
  memcpy(u, a, n * sizeof(double));
  if (n_near) *n_near = nn;
  if (n_pp) *n_pp = np_;
  if (n_bad) *n_bad = nb;
  free(un); free(keep); free(a); free(b); free(fl);
  return nf;
}

long or_step_pp(const or_mesh* m, double dt, double* u, double M, int limit, double eps, int pp, double pp_eps,
                long* n_near, long* n_pp, long* n_bad) {
  return or_step_ind(m, dt, u, 0, M, limit, eps, pp, pp_eps, n_near, n_pp, n_bad);
}

/* ------------------------------------------------------------------------------------
 * Largest characteristic speed over the cell means (for the CFL time step), per
 * direction: out[0] = x, out[1] = y (2D only).
 * ----------------------------------------------------------------------------------*/
void or_max_wavespeed(const or_mesh* m, const double* u, double* out) {
  int nv = or_nvars(m->dim, m->pde), np = or_nmodes(m->dim, m->N);
  double c0 = m->dim == 1 ? (double)psi(0, 0) : (double)(psi(0, 0) * psi(0, 0));
  out[0] = out[1] = 0;
  for (size_t c = 0; c < (size_t)m->nx * m->ny; ++c) {
    double mean[OR_MAXV];
    for (int v = 0; v < nv; ++v) mean[v] = u[(c * nv + v) * np] * c0;
    for (int d = 0; d < m->dim; ++d) {
      double s = max_speed(m->dim, m->pde, m->gamma, d, mean);
      if (s > out[d]) out[d] = s;
    }
  }
}

/* ------------------------------------------------------------------------------------
 * Initial L2 projection (Eq. (2)): U_n = sum_q w_q u0(x(r_q)) psi_n(r_q) with N+4 Gauss
 * points per direction (tensor rule in 2D).  Initial-condition families, params per
 * instance:
 *   0 sine (Burgers):     u = p0 + p1 sin(p2 x + p3 y)
 *   1 Riemann 1D (Euler): (rho,u,p)_L = p0..p2 for x < p6, (rho,u,p)_R = p3..p5 else
 *   2 four quadrants (2D Euler): (rho,u,v,p) for x>=p16,y>=p17 (p0..3), x<p16,y>=p17
 *     (p4..7), x<p16,y<p17 (p8..11), x>=p16,y<p17 (p12..15)
 *   3 density wave (Euler): rho = p0 + p1 sin(p2 x + p3 y), u = p4, v = p5, p = p6
 *   4 shock/entropy wave (1D Euler, Example 9): (rho,u,p) = p0..p2 for x < p3, else
 *     rho = p4 + p5 sin(p6 x), u = p7, p = p8
 *   5 isentropic vortex (2D Euler, Example 4): the printed exact solution with centre
 *     (p0, p1), strength beta = p2, evaluated at time p3 (advected with speed 1 in x)
 * ----------------------------------------------------------------------------------*/
static void ic_eval(int dim, int pde, double gam, int kind, const double* p, double x, double y, double* u) {
  if (kind == 0) { u[0] = p[0] + p[1] * sin(p[2] * x + p[3] * y); return; }
  double rho, vx, vy = 0, pr;
  if (kind == 1) {
    int left = x < p[6];
    rho = left ? p[0] : p[3]; vx = left ? p[1] : p[4]; pr = left ? p[2] : p[5];
  } else if (kind == 2) {
    int q = (x >= p[16]) ? (y >= p[17] ? 0 : 3) : (y >= p[17] ? 1 : 2);
    rho = p[4 * q]; vx = p[4 * q + 1]; vy = p[4 * q + 2]; pr = p[4 * q + 3];
  } else if (kind == 4) { /* Example 9: a shock running into an entropy (density) wave */
    int left = x < p[3];
    rho = left ? p[0] : p[4] + p[5] * sin(p[6] * x);
    vx = left ? p[1] : p[7];
    pr = left ? p[2] : p[8];
  } else if (kind == 6) { /* Example 11: post-shock state left of the line x = p8 + p9 y */
    const int post = x < p[8] + p[9] * y;
    rho = post ? p[0] : p[4]; vx = post ? p[1] : p[5]; vy = post ? p[2] : p[6]; pr = post ? p[3] : p[7];
  } else if (kind == 5) { /* Example 4: isentropic vortex (exact solution at time p3) */
    const double pi = 3.14159265358979323846;
    double dx = x - p[0] - p[3], dy = y - p[1];
    double e = exp(1.0 - (dx * dx + dy * dy));
    rho = pow(1.0 - (gam - 1.0) * p[2] * p[2] * e * e / (16.0 * gam * pi * pi), 1.0 / (gam - 1.0));
    vx = 1.0 - p[2] * e * dy / (2.0 * pi);
    vy = p[2] * e * dx / (2.0 * pi);
    pr = pow(rho, gam);
  } else {
    rho = p[0] + p[1] * sin(p[2] * x + p[3] * y); vx = p[4]; vy = p[5]; pr = p[6];
  }
  if (dim == 1) {
    u[0] = rho; u[1] = rho * vx; u[2] = pr / (gam - 1.0) + 0.5 * rho * vx * vx;
  } else {
    u[0] = rho; u[1] = rho * vx; u[2] = rho * vy; u[3] = pr / (gam - 1.0) + 0.5 * rho * (vx * vx + vy * vy);
  }
  (void)pde;
}

void or_project_ic(const or_mesh* m, int kind, const double* params, double* u) {
  int N = m->N, nv = or_nvars(m->dim, m->pde), np = or_nmodes(m->dim, N);
  or_dg_tables t;
  dg_tables(N, N + 4, &t);
  int nq = t.nq;
  double hx = (m->xR - m->xL) / m->nx, hy = m->dim == 2 ? (m->yR - m->yL) / m->ny : 0;
  int A[OR_MAXNP], Bm[OR_MAXNP];
  for (int k = 0; k < np; ++k) {
    if (m->dim == 1) { A[k] = k; Bm[k] = 0; } else mode_ab(k, &A[k], &Bm[k]);
  }
  for (int iy = 0; iy < m->ny; ++iy)
    for (int ix = 0; ix < m->nx; ++ix) {
      double acc[OR_MAXV][OR_MAXNP];
      memset(acc, 0, sizeof(acc));
      double xl = m->xL + ix * hx, yl = m->dim == 2 ? m->yL + iy * hy : 0;
      int nqy = m->dim == 2 ? nq : 1;
      for (int qy = 0; qy < nqy; ++qy)
        for (int qx = 0; qx < nq; ++qx) {
          double x = xl + 0.5 * (1.0 + t.x[qx]) * hx;
          double y = m->dim == 2 ? yl + 0.5 * (1.0 + t.x[qy]) * hy : 0.0;
          double uq[OR_MAXV];
          ic_eval(m->dim, m->pde, m->gamma, kind, params, x, y, uq);
          for (int v = 0; v < nv; ++v)
            for (int k = 0; k < np; ++k) {
              if (m->dim == 1) acc[v][k] += t.w[qx] * uq[v] * t.P[qx][k];
              else acc[v][k] += t.w[qx] * t.w[qy] * uq[v] * t.P[qx][A[k]] * t.P[qy][Bm[k]];
            }
        }
      size_t base = ((size_t)iy * m->nx + ix) * nv * np;
      for (int v = 0; v < nv; ++v)
        for (int k = 0; k < np; ++k) u[base + v * np + k] = acc[v][k];
    }
}

/* ------------------------------------------------------------------------------------
 * Table export for the tests (so that the printed P2 constants, the closed forms and
 * the invariants can be checked against what the oracle derived).
 * ----------------------------------------------------------------------------------*/
int or_weno_tables_size(void) { return (int)sizeof(or_weno_tables); }
/* parent: full-width stencil; ng_in > 0: reconstruction points r_in instead of Step 1's. */
void or_weno_export_g(int N, int parent, int ng_in, const double* r_in, double* pt, double* wt, double* C, double* D,
                      double* gam, double* B, double* SA, int* OFF, double* resid);
void or_weno_export(int N, double* pt, double* wt, double* C, double* D, double* gam, double* B,
                    double* SA, int* OFF, double* resid) {
  or_weno_export_g(N, 0, 0, NULL, pt, wt, C, D, gam, B, SA, OFF, resid);
}
void or_weno_export_g(int N, int parent, int ng_in, const double* r_in, double* pt, double* wt, double* C, double* D,
                      double* gam, double* B, double* SA, int* OFF, double* resid) {
  or_weno_tables t;
  weno_tables_build_g(N, parent, ng_in, r_in, &t);
  int ns = t.ns, ng = t.ng;
  for (int g = 0; g < ng; ++g) { pt[g] = t.pt[g]; wt[g] = t.wt[g]; }
  for (int i = 0; i <= N; ++i)
    for (int g = 0; g < ng; ++g)
      for (int k = 0; k < ns; ++k) C[(i * ng + g) * ns + k] = t.C[i][g][k];
  for (int g = 0; g < ng; ++g)
    for (int k = 0; k < ns; ++k) D[g * ns + k] = t.D[g][k];
  for (int g = 0; g < ng; ++g)
    for (int i = 0; i <= N; ++i) gam[g * (N + 1) + i] = t.gam[g][i];
  for (int i = 0; i <= N; ++i)
    for (int k = 0; k < ns; ++k)
      for (int l = 0; l < ns; ++l) B[(i * ns + k) * ns + l] = t.B[i][k][l];
  for (int k = 0; k < ns; ++k) {
    OFF[k] = t.OFF[k];
    for (int n = 0; n <= N; ++n) SA[k * (N + 1) + n] = t.SA[k][n];
  }
  *resid = t.gam_resid;
}

void or_dg_export(int N, int nq, double* x, double* w, double* P, double* dP) {
  or_dg_tables t;
  dg_tables(N, nq, &t);
  for (int q = 0; q < nq; ++q) {
    x[q] = t.x[q];
    w[q] = t.w[q];
    for (int n = 0; n <= N; ++n) {
      P[q * (N + 1) + n] = t.P[q][n];
      dP[q * (N + 1) + n] = t.dP[q][n];
    }
  }
}
