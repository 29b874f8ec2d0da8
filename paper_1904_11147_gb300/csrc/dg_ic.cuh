// Initial-condition families of dg_project_ic, evaluated at a point (conserved variables).
// Parameters per instance (dg.h lists them):
//   0 sine (Burgers):          u = p0 + p1 sin(p2 x + p3 y)
//   1 Riemann 1D (Euler):      (rho,u,p) = p0..p2 for x < p6, p3..p5 otherwise
//   2 four quadrants (2D):     (rho,u,v,p) for x>=p16,y>=p17: p0..3; x<p16,y>=p17: p4..7;
//                              x<p16,y<p17: p8..11; x>=p16,y<p17: p12..15
//   3 density wave (Euler):    rho = p0 + p1 sin(p2 x + p3 y), u = p4, v = p5, p = p6
//   4 shock/entropy wave (1D): (rho,u,p) = p0..p2 for x < p3, otherwise
//                              rho = p4 + p5 sin(p6 x), u = p7, p = p8   (Example 9)
//   5 isentropic vortex (2D):  centre (p0 + p3, p1), strength p2, at time p3 (Example 4):
//                              rho = (1 - (g-1) p2^2 e^(2(1-r^2)) / (16 g pi^2))^(1/(g-1)),
//                              u = 1 - p2 e^(1-r^2) (y - p1) / (2 pi),
//                              v = p2 e^(1-r^2) (x - p0 - p3) / (2 pi), p = rho^g
//   6 double Mach (2D):        post-shock (rho,u,v,p) = p0..p3 where x < p8 + p9 y, the
//                              pre-shock state p4..p7 elsewhere (Example 11)
#pragma once

namespace dg {

__device__ __forceinline__ void ic_prim_to_cons1(double rho, double vel, double pr, double gam, double* u) {
  u[0] = rho; u[1] = rho * vel; u[2] = pr / (gam - 1.0) + 0.5 * rho * vel * vel;
}

__device__ __forceinline__ void ic_eval1(int kind, const double* p, double x, double gam, double* u) {
  if (kind == 0) { u[0] = p[0] + p[1] * sin(p[2] * x); return; }
  double rho, vel, pr;
  if (kind == 1) {
    const bool left = x < p[6];
    rho = left ? p[0] : p[3]; vel = left ? p[1] : p[4]; pr = left ? p[2] : p[5];
  } else if (kind == 4) {
    const bool left = x < p[3];
    rho = left ? p[0] : p[4] + p[5] * sin(p[6] * x); vel = left ? p[1] : p[7]; pr = left ? p[2] : p[8];
  } else {
    rho = p[0] + p[1] * sin(p[2] * x); vel = p[4]; pr = p[6];
  }
  ic_prim_to_cons1(rho, vel, pr, gam, u);
}

__device__ __forceinline__ void ic_eval2(int kind, const double* p, double x, double y, double gam, double* u) {
  if (kind == 0) { u[0] = p[0] + p[1] * sin(p[2] * x + p[3] * y); return; }
  double rho, vx, vy, pr;
  if (kind == 2) {
    const int q = (x >= p[16]) ? (y >= p[17] ? 0 : 3) : (y >= p[17] ? 1 : 2);
    rho = p[4 * q]; vx = p[4 * q + 1]; vy = p[4 * q + 2]; pr = p[4 * q + 3];
  } else if (kind == 6) {
    const bool post = x < __dadd_rn(p[8], __dmul_rn(p[9], y));  // as the oracle rounds it
    rho = post ? p[0] : p[4]; vx = post ? p[1] : p[5]; vy = post ? p[2] : p[6]; pr = post ? p[3] : p[7];
  } else if (kind == 5) {
    const double pi = 3.14159265358979323846;
    const double dx = x - p[0] - p[3], dy = y - p[1];
    const double e = exp(1.0 - (dx * dx + dy * dy));
    rho = pow(1.0 - (gam - 1.0) * p[2] * p[2] * e * e / (16.0 * gam * pi * pi), 1.0 / (gam - 1.0));
    vx = 1.0 - p[2] * e * dy / (2.0 * pi);
    vy = p[2] * e * dx / (2.0 * pi);
    pr = pow(rho, gam);
  } else {  // density wave
    rho = p[0] + p[1] * sin(p[2] * x + p[3] * y); vx = p[4]; vy = p[5]; pr = p[6];
  }
  u[0] = rho; u[1] = rho * vx; u[2] = rho * vy; u[3] = pr / (gam - 1.0) + 0.5 * rho * (vx * vx + vy * vy);
}

}  // namespace dg
