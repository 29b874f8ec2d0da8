/*
 * dg.h -- C ABI of the GB300 (sm_103a) RKDG + CSWENO library.
 *
 * The library advances u_t + f(u)_x (+ g(u)_y) = 0 (Sec. 2, Eq. (1); Eqs. (19)-(21), (23)
 * for Burgers and the ideal-gas Euler equations) with a modal discontinuous Galerkin
 * method, u_h = sum_n U_n psi_n (Eq. (2)), psi_n the orthonormalised Legendre polynomials
 * on the reference cell (Sec. 2), third-order SSP Runge-Kutta in time (Sec. 3, last
 * paragraph) and the compact subcell WENO limiter of Sec. 3 on troubled cells.
 *
 * Conventions
 *  - All functions return a dg_status; none aborts or throws.  dg_last_error() gives a
 *    thread-local description of the last failure.
 *  - Every call is asynchronous on the mesh's CUDA stream unless it returns host data;
 *    those synchronise the stream before returning.
 *  - Modal arrays crossing the ABI use the layout [instance][cell][var][mode] with
 *    cell = iy * nx + ix, instances concatenated in creation order.  1D: mode n = degree n.
 *    2D (total degree P^N, (N+1)(N+2)/2 modes): modes are ordered by total degree
 *    d = a + b, then by b ascending: (0,0),(1,0),(0,1),(2,0),(1,1),(0,2),(3,0),... where
 *    mode (a,b) is psi_a(r) psi_b(s).  Variables: Burgers u; 1D Euler (rho, rho u, E);
 *    2D Euler (rho, rho u, rho v, E).
 *  - Pointers passed in are borrowed for the duration of the call only; the library
 *    copies what it keeps.  Device memory belongs to the mesh and is freed by
 *    dg_mesh_destroy.
 *  - The device layout (SoA planes, tiles) is private.
 */
#ifndef DG_H_
#define DG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mesh dg_mesh; /* opaque, owned by the library */

typedef enum {
  DG_OK = 0,
  DG_EINVAL = 1,      /* bad argument (sizes, enums, null pointers, order) */
  DG_ENOMEM = 2,      /* device or host allocation failed */
  DG_ECUDA = 3,       /* a CUDA runtime call failed (text in dg_last_error) */
  DG_EPOSITIVITY = 4, /* density or pressure not positive after the fallback */
  DG_ETIMEOUT = 5,    /* a bounded device wait gave up */
  DG_ESTATE = 6       /* calls out of order (e.g. stage 2 before stage 1) */
} dg_status;

typedef enum { DG_BURGERS = 0, DG_EULER = 1 } dg_pde;
/* DG_BC_DMR: the boundaries of the double Mach reflection problem (Example 11; 2D Euler
 * only, data from dg_set_boundary_data): the ghost cell outside a side is decided by its
 * centre (x_c, y_c) at the time of the state -- left: the post-shock state (inflow); right:
 * the mirror image of the boundary cell (outflow); bottom: the post-shock state where
 * x_c < a, else a reflecting wall (mirror image with rho v negated); top: the post-shock
 * state where x_c < x_s = a + b y_top + c t (the exact position of the moving shock),
 * else the pre-shock state.  The x side decides first.  Such meshes run the split stage,
 * the TVB indicator, the CSWENO limiter and the positivity scaling (DG_EINVAL for KXRCF,
 * the learned indicator and the parent limiter). */
typedef enum { DG_BC_PERIODIC = 0, DG_BC_OUTFLOW = 1, DG_BC_DMR = 2 } dg_bc;
typedef enum { DG_IND_TVB = 0, DG_IND_MLP = 1, DG_IND_KXRCF = 2 } dg_indicator;
typedef enum { DG_LIM_CSWENO = 0, DG_LIM_PARENT = 1 } dg_limiter;

/* Initial-condition families for dg_project_ic (parameters per instance):
 *   DG_IC_SINE          u = p0 + p1 sin(p2 x + p3 y)                              (4)
 *   DG_IC_RIEMANN1D     (rho,u,p) = p0..p2 for x < p6, p3..p5 otherwise           (7)
 *   DG_IC_QUADRANT      (rho,u,v,p) for x>=p16,y>=p17: p0..3; x<p16,y>=p17: p4..7;
 *                       x<p16,y<p17: p8..11; x>=p16,y<p17: p12..15                 (18)
 *   DG_IC_DENSITY_WAVE  rho = p0 + p1 sin(p2 x + p3 y), u = p4, v = p5, p = p6     (7)
 *   DG_IC_SHOCK_ENTROPY (1D, Example 9) (rho,u,p) = p0..p2 for x < p3, otherwise
 *                       rho = p4 + p5 sin(p6 x), u = p7, p = p8                     (9)
 *   DG_IC_VORTEX        (2D, Example 4) isentropic vortex centred at (p0 + p3, p1),
 *                       strength p2, at time p3: rho = (1 - (g-1) p2^2 e^{2(1-r^2)} /
 *                       (16 g pi^2))^{1/(g-1)}, u = 1 - p2 e^{1-r^2} (y-p1)/(2 pi),
 *                       v = p2 e^{1-r^2} (x-p0-p3)/(2 pi), p = rho^g               (4)
 *   DG_IC_DMR           (2D, Example 11) post-shock (rho,u,v,p) = p0..p3 where
 *                       x < p8 + p9 y, pre-shock p4..p7 elsewhere                   (10) */
typedef enum {
  DG_IC_SINE = 0,
  DG_IC_RIEMANN1D = 1,
  DG_IC_QUADRANT = 2,
  DG_IC_DENSITY_WAVE = 3,
  DG_IC_SHOCK_ENTROPY = 4,
  DG_IC_VORTEX = 5,
  DG_IC_DMR = 6
} dg_ic;

/* Create a batch of n_inst meshes sharing dim, PDE, order N and boundary condition.
 *  dim      1 or 2.  pde: dg_pde.  N: polynomial degree 1..3 (Sec. 2, P^N).
 *  nx, ny   host arrays of n_inst cell counts (ny ignored in 1D); each >= 1 (periodic
 *           meshes need >= 1 cell; the stencil wraps).
 *  box      host array n_inst * 4: xL, xR, yL, yR of each instance (yL, yR ignored in 1D).
 *  bc       dg_bc; outflow uses mirror ghost cells (our reading of the paper's
 *           transmissive shock-tube boundaries, Examples 7-8).
 *  gamma    ratio of specific heats for Euler (1.4 in the paper), ignored for Burgers.
 *  stream   a cudaStream_t (may be NULL = legacy default stream).
 * Allocates three state copies (u^n and two stage buffers) plus flag/list/limiter
 * scratch on the current device.  Errors: DG_EINVAL, DG_ENOMEM, DG_ECUDA. */
dg_status dg_mesh_create(int dim, int pde, int N, int n_inst, const int* nx, const int* ny,
                         const double* box, int bc, double gamma, void* stream, dg_mesh** out);

/* Free everything the mesh owns.  NULL is accepted. */
dg_status dg_mesh_destroy(dg_mesh* m);

/* Number of doubles of a full modal array (sum over instances of cells * vars * modes). */
size_t dg_mesh_size(const dg_mesh* m);

/* Copy modes in (u^n := modes).  modes is a host (is_device = 0) or device pointer of n
 * doubles in the ABI layout; n must equal dg_mesh_size.  The copy is ordered on the mesh
 * stream; a host buffer may be reused once the call returns. */
dg_status dg_set_modes(dg_mesh* m, const double* modes, size_t n, int is_device);

/* Copy the current state out (the output of the last stage / limiter, or u^n).
 * Synchronises the stream. */
dg_status dg_get_modes(dg_mesh* m, double* out, size_t n, int is_device);

/* Initial L2 projection (Eq. (2) applied to u0): U_n = sum_q w_q u0(x_q) psi_n(x_q) with
 * N+4 Gauss points per direction, computed on the device.  params: host array of
 * n_inst * nparams doubles (see dg_ic).  Sets u^n. */
dg_status dg_project_ic(dg_mesh* m, int ic, const double* params, int nparams);

/* Per-instance time steps (host array of n_inst doubles) used by dg_rk_stage / dg_step
 * when they are called with dt <= 0. */
dg_status dg_set_dt(dg_mesh* m, const double* dt);

/* One SSP-RK3 stage (Sec. 3, last paragraph; Shu's third-order TVD scheme) of the
 * semi-discrete scheme of Eq. (5) with the local Lax-Friedrichs flux (Sec. 2):
 *   stage 1: u1 = u^n + dt L(u^n)
 *   stage 2: u2 = 3/4 u^n + 1/4 (u1 + dt L(u1))
 *   stage 3: u^{n+1} = 1/3 u^n + 2/3 (u2 + dt L(u2))
 * L is evaluated on the current state (the previous stage, limited or not).  dt > 0 applies
 * to every instance; dt <= 0 uses the per-instance values of dg_set_dt.  No limiting.
 * FP64 arithmetic; in 2D Euler the reciprocal of the density and the sound speed's square
 * root are the hardware's approximations refined to within 1-2 ulp of the IEEE results.
 * Errors: DG_EINVAL (stage not 1..3), DG_ESTATE (stage s without stage s-1 before it). */
dg_status dg_rk_stage(dg_mesh* m, int stage, double dt);

/* Troubled-cell indicator on the current state (Sec. 3, step 1).  DG_IND_TVB: the TVB
 * modified minmod with constant tvb_M on the face values of every variable, per
 * direction.  DG_IND_KXRCF: the paper's own choice (Krivodonova et al.), troubled when
 * |int over the inflow faces of (w_j - w_nb)| > r^((N+1)/2) |inflow faces| max|w_j| over
 * the cell's Gauss points, r the circumscribed radius, inflow by the sign of the mean
 * velocity, w = u (Burgers) or density and total energy (Euler); tvb_M is ignored.
 * DG_IND_MLP: the TVB flags the learned network keeps (dg_set_indicator_mlp).  Writes the
 * device flag array and the compacted list of troubled cells used by dg_cswenolimit.
 * n_flagged, n_near and flags_out (host, one byte per cell: bit 0 troubled, bit 1 near
 * threshold) are optional; asking for any of them synchronises the stream.  A cell is near
 * threshold when a comparison deciding it (TVB: |a1| against M h^2 or against the smaller
 * neighbour difference, or a sign test; KXRCF: the two sides of I_j > 1) lies within 32768
 * units in the last place, or a mean difference within 2^-39 of the largest magnitude in
 * its comparison: a window that contains every comparison within 1e-12 relative.  Near
 * cells are reported, not treated differently.  Errors: DG_EINVAL (unknown indicator or no MLP weights). */
dg_status dg_flag_cells(dg_mesh* m, int indicator, double tvb_M, int64_t* n_flagged,
                        int64_t* n_near, uint8_t* flags_out);

/* CSWENO limiter (Sec. 3, Steps 1-6, Fig. 1) on the cells flagged by the last
 * dg_flag_cells: keeps each troubled cell's average U_0 and rebuilds modes 1..N from WENO
 * point values reconstructed on the subcells of its immediate neighbours (characteristic
 * fields for Euler; dimension by dimension in 2D).  Jacobi update: every troubled cell
 * reads the unlimited neighbours.  In 2D the reciprocals in the nonlinear weights
 * (Eq. (14)) are the hardware's approximations refined to within 1-2 ulp.  After the
 * learned indicator's flags (Euler) the positivity fallback of dg_set_indicator_mlp applies
 * as in dg_step.  Errors: DG_ESTATE if no flags exist for this state. */
dg_status dg_cswenolimit(dg_mesh* m);

/* The parent WENO limiter (Qiu and Shu, ref. [qs1]; the limiter Sec. 4 compares CSWENO
 * with) on the cells flagged by the last dg_flag_cells: the reconstruction of Sec. 3,
 * Steps 2-6, on the averages of the whole cells j-N..j+N (in 2D the (2N+1)^2 cell averages
 * around the troubled cell, x sweep then y sweep; characteristic fields for Euler).
 * Outflow ghosts mirror the interior cell at the reflected position.  Jacobi update, U_0
 * kept.  Errors: DG_ESTATE (no flags for this state), DG_EINVAL (an instance with fewer
 * than N+1 cells per side). */
dg_status dg_parent_wenolimit(dg_mesh* m);

/* Limiter used by dg_step with the TVB and KXRCF indicators: DG_LIM_CSWENO (default) or
 * DG_LIM_PARENT (the learned indicator always uses CSWENO).  The CUDA graph is rebuilt on
 * the next dg_step.  Errors: DG_EINVAL (unknown limiter, instance too small). */
dg_status dg_set_limiter(dg_mesh* m, int limiter);

/* Positivity-preserving scaling (Example 11 adds it to the limiter, following Zhang and
 * Shu, ref. [zs3]) of the current state, every cell, Euler only.  For a cell whose mean
 * Ubar has rho > 0 and p > 0, with eps = min(eps0, rhobar, pbar): the density's modes
 * n >= 1 are scaled so that rho >= eps at the check points, then every variable's modes
 * n >= 1 by the largest theta in [0,1] that keeps p >= eps there (the root of a quadratic
 * in theta per point, taken 1e-12 relative below it).  Check points: the Gauss-Lobatto
 * points -1, 0, 1 (-1, 1 for N = 1) in 1D; in 2D (Gauss x Gauss-Lobatto) and
 * (Gauss-Lobatto x Gauss) with the N+1 face Gauss points.  Means are left bitwise; cells
 * with an inadmissible mean are left alone and counted (dg_positivity_counts).
 * Asynchronous.  Errors: DG_EINVAL (Burgers, eps0 not positive and finite). */
dg_status dg_positivity_limit(dg_mesh* m, double eps0);

/* enable != 0: dg_step applies dg_positivity_limit(eps0) after the limiter of every
 * stage (the CUDA graph is rebuilt on the next dg_step); 0 switches it off (default).
 * Errors: DG_EINVAL (Burgers, eps0 not positive and finite when enabling). */
dg_status dg_set_positivity(dg_mesh* m, int enable, double eps0);

/* Running totals of the scaling since mesh creation or the last reset: cells changed and
 * cells whose mean was not admissible (left alone).  Returns DG_EPOSITIVITY when
 * bad_means > 0.  Synchronises the stream. */
dg_status dg_positivity_counts(dg_mesh* m, int64_t* changed, int64_t* bad_means, int reset);

/* Boundary data of a DG_BC_DMR mesh (Example 11, after Woodward and Colella): p[0..3] the
 * post-shock (rho, u, v, p), p[4..7] the pre-shock state, p[8..10] a, b, c of the shock
 * line x_s(y, t) = a + b y + c t (a is also where the wall starts on the bottom side).
 * n must be 11.  Required before the first stage.  Synchronises the stream.  Errors:
 * DG_EINVAL (another bc, n != 11, non-positive density or pressure). */
dg_status dg_set_boundary_data(dg_mesh* m, const double* p, int n);

/* Time of u^n per instance (host array of n_inst doubles; 0 at creation) for the
 * time-dependent boundaries of DG_BC_DMR meshes.  The stages evaluate the boundaries at
 * the SSP-RK3 stage times t, t + dt, t + dt/2; the indicator and the limiter after stage s
 * at the time of its output (t + dt, t + dt/2, t + dt); stage 3 advances t by dt.
 * dg_get_time reads it back (synchronises).  Errors: DG_EINVAL (another bc). */
dg_status dg_set_time(dg_mesh* m, const double* t);
dg_status dg_get_time(dg_mesh* m, double* t);

/* One full SSP-RK3 step: three times (stage, indicator, limiter), replayed from a CUDA
 * graph captured on the first call.  dt as in dg_rk_stage. */
dg_status dg_step(dg_mesh* m, double dt, int indicator, double tvb_M);

/* Largest characteristic speed over the cell means of each instance: out[2*i] (x) and
 * out[2*i+1] (y, 0 in 1D), host array.  Used by callers for the CFL condition.
 * Synchronises the stream. */
dg_status dg_max_wavespeed(dg_mesh* m, double* out);

/* A wave-speed bound over the check points of the positivity-preserving scaling instead of
 * the cell means (Euler): per instance and direction, max |v_d| + max c over the points of
 * all cells, which bounds the wave speeds of the face states and so the time step under
 * which the scaling keeps the next stage's means admissible (Zhang and Shu).  Points
 * without a real sound speed are skipped.  out: host [n_inst][2].  Synchronises the
 * stream.  Errors: DG_EINVAL (Burgers). */
dg_status dg_max_wavespeed_points(dg_mesh* m, double* out);

/* Autotuner: times the candidate launch configurations on this mesh's current state with
 * the time step dt (u^n is left unchanged; stage buffers and limiter scratch are
 * overwritten): the 2D stage form -- split into a face pass (one thread per face: traces,
 * local Lax-Friedrichs flux, projection onto the transverse modes) and a cell pass (volume
 * term, lifting, stage combination), reported as stage_ty = 0, or fused in one kernel per
 * tile with a tile height of 4 or 8 rows of 32 cells plus their halo warps and launched
 * one block per tile or as one persistent block per SM taking tiles from an atomic queue --
 * and the limiter's grid (2, 4, 8 or 16 blocks per SM).  The split form is the default of
 * a 2D mesh (it needs (N+1) x V doubles per face; without that memory the mesh uses the
 * fused form).  Applies the fastest
 * to the mesh and remembers them for later meshes of the same dim, PDE, N and size class
 * (floor(log2 cells)); with the environment variable DG_AUTOTUNE_FILE set, choices are also
 * appended to that file and read back by later processes.  Synchronises the stream.
 * stage_ty (0 in 1D), limit_blocks_per_sm and persistent are optional outputs.  Errors: DG_EINVAL,
 * DG_ESTATE (a step left unfinished). */
dg_status dg_autotune(dg_mesh* m, double dt, int* stage_ty, int* limit_blocks_per_sm, int* persistent);

/* Number of kernels the library launched since the mesh was created (graph replays count
 * every kernel node they contain). */
int64_t dg_kernel_launches(const dg_mesh* m);

/* Copies the CSWENO tables the library derived for degree N (host only; works without a
 * GPU).  NG = 2 for N = 1, else 4.  rp[NG], rw[NG]: Step 1 points and weights (Sec. 3);
 * C[(i*NG+g)*(N+1)+k]: p_i(x_g) from the averages of stencil cells i..i+N (Step 2);
 * gam[g*(N+1)+i]: Eq. (8); B[(i*(N+1)+k)*(N+1)+l]: Eq. (13) as a quadratic form;
 * SA[k*(N+1)+n]: average of psi_n over stencil cell k (Fig. 1).  Errors: DG_EINVAL. */
dg_status dg_limiter_tables(int N, double* rp, double* rw, double* C, double* gam, double* B, double* SA);

/* ------------------------------------------------------------------------------------
 * Learned troubled-cell indicator (the paper has none; its Sec. 3 indicator is KXRCF and
 * this library's plain indicator is the TVB minmod).  A 32-32 ReLU network maps features
 * of a cell and its cross neighbours to one logit; a cell is troubled when logit > tau.
 * Features per variable v (s_v = max_c |ubar_c - ubar_j| + sum_{n>=1} |U^j_{n,v}| + 1e-14):
 * (ubar_c - ubar_j)/s_v for the neighbours c (W, E, S, N; 1D: L, R), then U^c_{n,v}/s_v for
 * n >= 1 and c = the cell, then the neighbours in that order.  Inference runs inside the
 * flagging pass on the tensor cores (BF16 weights and features, FP32 accumulation); the
 * network is trained on the device by this library's kernels from harvested tuples.
 * ----------------------------------------------------------------------------------*/
typedef struct dg_mlp dg_mlp; /* network + Adam state, owned by the library */

/* Number of features for (dim, pde, N): V (4 + 5 (NP-1)) in 2D, V (2 + 3 N) in 1D; -1 if invalid. */
int dg_mlp_features(int dim, int pde, int N);

/* New network for n_features inputs, He-uniform weights from seed, zero biases and Adam
 * moments; its kernels run on stream.  Errors: DG_EINVAL, DG_ENOMEM. */
dg_status dg_mlp_create(int n_features, uint64_t seed, void* stream, dg_mlp** out);
dg_status dg_mlp_destroy(dg_mlp* n);

/* Parameters as one FP32 host vector: W1 [32][F] (row = hidden unit), b1 [32], W2 [32][32],
 * b2 [32], w3 [32], b3 [1]; count = 32 F + 1121.  set also resets the Adam moments. */
size_t dg_mlp_param_count(const dg_mlp* n);
dg_status dg_mlp_get_params(dg_mlp* n, float* out, size_t count);
dg_status dg_mlp_set_params(dg_mlp* n, const float* in, size_t count);

/* Gradient (host, packed as the parameters) and mean loss of the weighted binary cross
 * entropy -[pw y log s(z) + (1-y) log(1-s(z))] over B samples; X: device [B][F] FP32,
 * y: device [B] bytes (0/1).  FP32 arithmetic.  Synchronises the network's stream. */
dg_status dg_mlp_grad(dg_mlp* n, const float* X, const uint8_t* y, int64_t B, float pos_weight, float* grad_out,
                      float* loss_out);

/* One Adam step (beta 0.9/0.999, eps 1e-8, bias-corrected) on the batch; loss_out (host,
 * optional) receives the batch loss before the step and synchronises. */
dg_status dg_mlp_train_step(dg_mlp* n, const float* X, const uint8_t* y, int64_t B, float pos_weight, float lr,
                            float* loss_out);

/* FP32 logits of B samples (X device [B][F], logits device [B]), asynchronous on the
 * network's stream; for validation and for choosing the threshold. */
dg_status dg_mlp_predict(dg_mlp* n, const float* X, int64_t B, float* logits);

/* Attach the network's current weights to the mesh as DG_IND_MLP with threshold tau.
 * DG_IND_MLP flags a cell when the TVB indicator flags it and the network's logit exceeds
 * tau (the network filters the TVB list).  In dg_step (Euler), the plain TVB indicator is
 * the positivity fallback, per instance: when a TVB-flagged cell the network skipped has a
 * non-positive density or pressure at a volume or face Gauss point of its unlimited stage
 * (FP32 screen, p > 1e-6 |E| required), the instance's stage is redone with all its TVB
 * flags from the unlimited stage -- the plain method's stage. */
dg_status dg_set_indicator_mlp(dg_mesh* m, const dg_mlp* n, float tau);

/* Evaluates the network on every cell of the current state and writes the logits to the
 * device array logits [cells] (FP32); also sets the flags (logit > tau, without the TVB gate)
 * that the next dg_cswenolimit uses.  Diagnostics of the learned indicator. */
dg_status dg_indicator_logits(dg_mesh* m, float* logits);

/* Training data from the plain method on the current (post-stage, unlimited) state:
 * features X (device [cells][F] FP32), TVB flags (device [cells] bytes) and the limiter's
 * relative change (device [cells] FP32: for a flagged cell max over v and n >= 1 of
 * |limited - unlimited U_{n,v}| / s_v, 0 for the others); then applies the TVB + CSWENO
 * limiter to the state as dg_flag_cells(TVB) + dg_cswenolimit would. */
dg_status dg_harvest(dg_mesh* m, double tvb_M, float* X, uint8_t* flags, float* change);

/* Running totals over the limiter passes of dg_step (three per step): cells the TVB
 * indicator flagged, cells passed to the limiter (equal for DG_IND_TVB; for DG_IND_MLP the
 * learned subset plus the TVB-flagged cells of the instance stages the positivity fallback
 * redid) and the number of passes.  reset != 0 zeroes them.  Synchronises the stream. */
dg_status dg_flag_statistics(dg_mesh* m, int64_t* tvb_flagged, int64_t* limited, int64_t* passes, int reset);

/* Positivity fallbacks of the learned indicator since the network was attached: instance
 * stages redone with the TVB flags, and instance stages whose final state still fails the
 * screen at some cell (every cell is screened; counted only while the positivity-preserving
 * scaling is off: with it on, the scaling that follows the limiter restores the check points
 * instead).  A failure outside the cells the network skipped is one the plain method's
 * stage from the same input has as well.  Returns
 * DG_EPOSITIVITY when failures > 0.  Synchronises the stream. */
dg_status dg_positivity_report(dg_mesh* m, int64_t* fallbacks, int64_t* failures);

/* Largest mesh (cells) that dg_cswenolimit_noalloc accepts. */
#define DG_NOALLOC_MAX_CELLS 16384

/* The troubled-cell indicator (TVB, as dg_flag_cells) and the CSWENO limiter (as
 * dg_cswenolimit) for one mesh in one call that allocates no device memory.  The paper has
 * no counterpart: this entry point exists for callers that must not allocate once they run
 * -- an application whose memory manager already reserved or capped the GPU memory, a
 * latency-critical loop in which cudaMalloc/cudaFree could block on or synchronise with
 * the device, or a plugin whose host forbids allocation after initialisation.
 *  dim, pde, N, bc, gamma, tvb_M  as for dg_mesh_create / dg_flag_cells; one instance of
 *           nx x ny cells (ny ignored in 1D) on box = {xL, xR, yL, yR} (host array).
 *  u_in     device array, V*NP planes of nx*ny doubles: plane (v*NP + m) holds mode m of
 *           variable v for cell iy*nx + ix (modes and variables ordered as in the ABI layout).
 *  u_out    device array of the same shape; may equal u_in (limited in place).  Unflagged
 *           cells are copied; flagged cells keep U_0 and get limited modes 1..N.
 *  n_flagged, n_near  optional host pointers; if either is given, the call synchronises the
 *           stream and stores the number of troubled cells and the number of near-threshold
 *           cells (the window of dg_flag_cells).
 *  stream   cudaStream_t (NULL = legacy default stream); the work is ordered on it.
 * Scratch: a file-scope device array of about 5.7 MB (sized for DG_NOALLOC_MAX_CELLS cells of
 * up to 4 variables x 10 modes), created when the library's device code is loaded and kept
 * until the process exits on every GPU that loads the library.  The first call on a device
 * uploads the method's tables and looks the array up with that device current; make that
 * first call before any stream capture.  Every call uses the same array and the array keeps
 * the last call's contents (the call clears the counters it needs at zero), so calls that
 * overlap on the GPU (other streams, other host threads) race: order them.
 * Errors: DG_EINVAL (bad arguments, or more than DG_NOALLOC_MAX_CELLS cells), DG_ECUDA. */
dg_status dg_cswenolimit_noalloc(int dim, int pde, int N, int nx, int ny, const double* box, int bc, double gamma,
                                 double tvb_M, const double* u_in, double* u_out, int64_t* n_flagged, int64_t* n_near,
                                 void* stream);

/* The refined arithmetic of the FP64 kernels (not part of the method): op 0 the reciprocal,
 * op 1 the square root, as the 2D Euler fluxes and the WENO weights evaluate them -- the
 * hardware's approximation refined by one Householder step of order three, within one or
 * two ulps of the IEEE results; arguments outside the refined range (zero, subnormal,
 * |x| >= 2^1022, inf, NaN, and non-positive square-root arguments) give the IEEE result.
 * x and out are device arrays of n doubles; asynchronous on stream.  For checking that
 * arithmetic against IEEE operations.  Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_refined_arith(int op, const double* x, double* out, int64_t n, void* stream);

/* Thread-local text of the last error (never NULL). */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_H_ */
