// C ABI of the library (include/dg.h): mesh management, host<->device layout changes,
// the per-call entry points and the CUDA-graph time step.
#include <algorithm>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_shared.cuh"
#include "tables.h"

namespace dg {
// kernels_1d / kernels_2d entry points
cudaError_t upload_tables1(const dgt::Tabs* tabs);
cudaError_t upload_tables2(const dgt::Tabs* tabs);
cudaError_t prepare2(int pde, int N);
int tile_w1();
int tile_w2();
int tile_h2();
void launch_stage1(int pde, int N, const LaunchArgs& a, int stage, double dt_all);
void launch_flag1(int pde, int N, const LaunchArgs& a, double M, unsigned char* flags, Counters* cnt, int* lc, int* li);
void launch_limit1(int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt, double* lim,
                   int nblocks);
void launch_scatter1(int pde, int N, const LaunchArgs& a, const double* lim, const int* lc, const Counters* cnt,
                     int nblocks);
void launch_project1(int pde, int N, const LaunchArgs& a, const int* cell_inst, int kind, const double* params, int np);
void launch_speed1(int pde, int N, const LaunchArgs& a, const int* cell_inst, double* out);
void launch_stage2(int pde, int N, const LaunchArgs& a, int stage, double dt_all, int tys, int* queue, int grid);
void launch_stage2_split(int pde, int N, const LaunchArgs& a, int stage, double dt_all, const Tile* face_tiles,
                         int nface_tiles, double* fx, long long fxt, double* fy, long long fyt);
void launch_flag2(int pde, int N, const LaunchArgs& a, double M, unsigned char* flags, Counters* cnt, int* lc, int* li);
void launch_limit2(int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt, double* lim,
                   int nblocks);
void launch_scatter2(int pde, int N, const LaunchArgs& a, const double* lim, const int* lc, const Counters* cnt,
                     int nblocks);
void launch_project2(int pde, int N, const LaunchArgs& a, const int* cell_inst, int kind, const double* params, int np);
void launch_speed2(int pde, int N, const LaunchArgs& a, const int* cell_inst, double* out);
int mlp_features(int dim, int pde, int N);
int mlp_padded(int F);
cudaError_t prepare_mlp(int dim, int pde, int N, int FP);
void launch_features(int dim, int pde, int N, const LaunchArgs& a, double c0, float* X);
void launch_label(int dim, int pde, int N, const LaunchArgs& a, double c0, const int* lc, const int* li,
                  const Counters* cnt, const double* lim, float* label, int nblocks);
void launch_mlp_fb(cudaStream_t st, const float* X, const unsigned char* y, long long B, int F, const float* params,
                   float pw, float* h1, float* d1, float* h2, float* d2, float* dz, float* loss);
long long mlp_wgrad_chunks(long long B);
void launch_mlp_wgrad(cudaStream_t st, const float* X, long long B, int F, const float* h1, const float* d1,
                      const float* h2, const float* d2, const float* dz, float* part, float* grad);
void launch_mlp_forward(cudaStream_t st, const float* X, long long B, int F, const float* params, float* z);
void launch_mlp_adam(cudaStream_t st, float* params, const float* grad, float* m1, float* m2, int P, float lr, int t);
void launch_mlp_export(cudaStream_t st, const float* params, int F, int FP, void* W1b, float* b1, void* W2b, float* b2,
                       float* w3, float* b3);
}  // namespace dg

namespace dg {
void launch_flag_mlp(int dim, int pde, int N, const LaunchArgs& a, double c0, const MlpInfer& W, unsigned char* flags,
                     Counters* cnt, int* lc, int* li, float* logits);
cudaError_t prepare_filter(int dim, int pde, int N, int FP);
void launch_mlp_filter(int dim, int pde, int N, const LaunchArgs& a, double c0, const MlpInfer& W, const int* la_c,
                       const int* la_i, const Counters* cnt_a, unsigned char* flags, Counters* cnt_b, int* lb_c,
                       int* lb_i, int nblocks);
void launch_positivity_all(int dim, int N, const LaunchArgs& a, const double* psi_q, const double* psi_p1, double gam,
                           const int* cell_inst, unsigned int* fail, int nblocks);
void launch_positivity_skipped(int dim, int N, const LaunchArgs& a, const double* psi_q, const double* psi_p1,
                               double gam, const int* la_c, const int* la_i, const Counters* cnt_a,
                               const unsigned char* flags, unsigned int* fail, int nblocks);
void launch_scatter_unless(int dim, int pde, int N, const LaunchArgs& a, const double* lim, const int* lc,
                           const int* li, const Counters* cnt, const unsigned int* skip, int nblocks);
void launch_filter_inst(cudaStream_t st, const int* la_c, const int* la_i, const Counters* cnt_a,
                        const unsigned int* mark, Counters* cnt_c, int* lc_c, int* lc_i, int nblocks);
void launch_count_fail(cudaStream_t st, const unsigned int* fail, int n_inst, unsigned long long* total);
cudaError_t upload_tables_parent(const dgt::Tabs* tabs);
void launch_parent(int dim, int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt,
                   double* lim, int nblocks);
void launch_kxrcf(int dim, int pde, int N, const LaunchArgs& a, const double* hpow, const double* psi_m1,
                  const double* psi_p1, const double* psi_q, const double* gw, unsigned char* flags, Counters* cnt,
                  int* lc, int* li);
void launch_speed_points(int dim, int N, cudaStream_t st, const double* U, long long ctot, long long ncell,
                         const int* cell_inst, const double* pg, const double* pl, double gam, double* out,
                         unsigned int* lb, int n_inst, int* list, unsigned int* n_list, int nblocks);
void launch_positivity(int dim, int N, cudaStream_t st, double* U, long long ctot, long long ncell,
                       const double* pg, const double* pl, double c0, double gam, double eps0,
                       int* list, unsigned int* n_list, unsigned long long* counts, int nblocks);
}  // namespace dg

using namespace dg;

// ----------------------------------------------------------------------------- errors
static thread_local char g_err[512] = "";

static dg_status fail(dg_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(DG_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

extern "C" const char* dg_last_error(void) { return g_err; }

void dg_set_error_internal(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

// ----------------------------------------------------------------------------- tables
static int g_tables_dev = -2;  // device the constant tables were uploaded to (per process)
static dgt::Tabs g_tabs[3];
static dgt::Tabs g_ptabs[3];  // parent WENO limiter tables (full-width stencil)

// Derives the tables once per process and uploads them once per device.  Any host thread
// may call it (mesh creation, the no-allocation entry point); one mutex orders them.
dg_status dg_ensure_tables_internal() {
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (g_tables_dev == -2) {
    for (int n = 1; n <= 3; ++n)
      if (dgt::build_tables(n, &g_tabs[n - 1]) || dgt::build_tables(n, &g_ptabs[n - 1], true))
        return fail(DG_EINVAL, "table derivation failed for N=%d", n);
  }
  // constant memory is per device: upload once for every device that creates a mesh
  static std::vector<int> done;
  for (int d : done)
    if (d == dev) return DG_OK;
  CK(upload_tables1(g_tabs));
  CK(upload_tables2(g_tabs));
  CK(upload_tables_parent(g_ptabs));
  done.push_back(dev);
  g_tables_dev = dev;
  return DG_OK;
}

// ----------------------------------------------------------------------------- mesh
struct dg_mesh {
  int dim, pde, N, n_inst, bc, V, NP;
  double gamma;
  cudaStream_t st;
  int device;
  long long ncell, ctot;   // cells (all instances) and plane stride
  std::vector<Inst> h_inst;
  Inst* d_inst = nullptr;
  Tile* d_tiles = nullptr;
  int ntiles = 0;
  int* d_cell_inst = nullptr;
  double* U[3] = {nullptr, nullptr, nullptr};  // u^n, stage buffers
  double* lim = nullptr;                       // limiter output (compact) / transpose scratch
  unsigned char* flags = nullptr;
  int* list_cell = nullptr;
  int* list_inst = nullptr;
  Counters* cnt = nullptr;
  double* d_speed = nullptr;
  int cur = 0;          // buffer holding the current state
  int last_stage = 0;   // 0: state is u^n; s: output of stage s
  bool flags_valid = false;
  int limit_blocks = 0;
  int sms = 152;
  // 2D stage tiles (TX x stage_ty cells), chosen by the autotuner
  int stage_ty = 8;
  Tile* d_stage_tiles = nullptr;
  int n_stage_tiles = 0;
  int stage_persistent = 0;  // persistent tile queue (1) or one block per tile (0)
  int* d_queue = nullptr;
  unsigned int* d_lq = nullptr;  // work counter of the 2D Euler limiter
  // split 2D stage (face pass + cell pass; stage_ty == 0): face flux planes, x faces then
  // y faces, with their plane strides, and the face tiles
  bool stage_split = false;
  double* fbuf = nullptr;
  long long fxt = 0, fyt = 0;
  Tile* d_face_tiles = nullptr;
  int n_face_tiles = 0;
  long long launches = 0;
  // CUDA graph of one full step
  cudaGraphExec_t gexec = nullptr;
  int g_ind = -1;
  double g_M = 0.0;
  int g_kernels = 0;
  std::vector<double> last_dt;
  // learned indicator attached by dg_set_indicator_mlp: list B (TVB flags kept by the
  // network, plus the cells the positivity gate adds), per-instance screen bits
  void* mlp_buf = nullptr;
  MlpInfer mlp{};
  bool has_mlp = false;
  int *lb_cell = nullptr, *lb_inst = nullptr, *lc_cell = nullptr, *lc_inst = nullptr;
  Counters *cnt_b = nullptr, *cnt_c = nullptr;
  unsigned int* fail = nullptr;              // [2][n_inst]: the screen of skipped cells, the final one
  unsigned long long* pos_counts = nullptr;  // [0] stages redone with the TVB flags, [1] failures after it
  bool use_b = false;                        // dg_cswenolimit limits list B (learned) or A (TVB)
  unsigned long long* flag_totals = nullptr;  // TVB-flagged, limited, passes (dg_step)
  double psi_q[16], psi_p1[4];
  // positivity-preserving scaling (Euler): basis values at the check points, the
  // dg_step option and the running counts (cells changed, inadmissible means)
  double pp_g[16], pp_l[12];  // psi_n at the Gauss [N+1][N+1] and Gauss-Lobatto [L][N+1] points
  bool pp_on = false;
  double pp_eps0 = 1e-13;
  unsigned long long* pp_counts = nullptr;
  int* pp_list = nullptr;          // Euler: cells an FP32 screen leaves to an FP64 pass
  unsigned int* pp_n = nullptr;
  unsigned int* sp_lb = nullptr;   // Euler: [2 n_inst] lower bounds of the check-point wave speed
  bool g_pp = false;
  double g_pp_eps = 0.0;
  // KXRCF indicator: r^((N+1)/2) per instance (r the circumscribed radius) and the basis
  // values at r = -1, +1 and at the Gauss points, with the Gauss weights
  double* d_kx_hpow = nullptr;
  double kx_pm[4], kx_pp[4], kx_pq[16], kx_w[4];
  // limiter of dg_step with the TVB / KXRCF indicators: CSWENO (default) or parent WENO
  int limiter = DG_LIM_CSWENO;
  int g_lim = -1;
  int min_side = 1;  // smallest instance side (the parent stencil needs N+1 cells)
  // double Mach reflection boundaries (DG_BC_DMR): data and per-instance times on the
  // device (layout in dg_shared.cuh), and whether dg_set_boundary_data was called
  double* d_bcd = nullptr;
  bool bcd_set = false;
};

static size_t mesh_doubles(const dg_mesh* m) { return (size_t)m->ncell * m->V * m->NP; }

extern "C" size_t dg_mesh_size(const dg_mesh* m) { return m ? mesh_doubles(m) : 0; }

extern "C" int64_t dg_kernel_launches(const dg_mesh* m) { return m ? m->launches : 0; }

extern "C" dg_status dg_mesh_destroy(dg_mesh* m) {
  if (!m) return DG_OK;
  if (m->gexec) cudaGraphExecDestroy(m->gexec);
  cudaFree(m->d_inst);
  cudaFree(m->d_tiles);
  cudaFree(m->d_stage_tiles);
  cudaFree(m->d_queue);
  cudaFree(m->d_lq);
  cudaFree(m->fbuf);
  cudaFree(m->d_face_tiles);
  cudaFree(m->d_cell_inst);
  for (auto& p : m->U) cudaFree(p);
  cudaFree(m->lim);
  cudaFree(m->flags);
  cudaFree(m->list_cell);
  cudaFree(m->list_inst);
  cudaFree(m->cnt);
  cudaFree(m->d_speed);
  cudaFree(m->flag_totals);
  cudaFree(m->mlp_buf);
  cudaFree(m->d_bcd);
  cudaFree(m->lb_cell); cudaFree(m->lb_inst); cudaFree(m->lc_cell); cudaFree(m->lc_inst);
  cudaFree(m->cnt_b); cudaFree(m->cnt_c); cudaFree(m->fail); cudaFree(m->pos_counts);
  cudaFree(m->pp_counts); cudaFree(m->pp_list); cudaFree(m->pp_n); cudaFree(m->sp_lb);
  cudaFree(m->d_kx_hpow);
  delete m;
  return DG_OK;
}

// ----------------------------------------------------------------------------- autotuning
// Process-wide choices per (dim, pde, N, mesh-size class = floor(log2 cells)); optionally
// loaded from and appended to the text file named by DG_AUTOTUNE_FILE
// ("dim pde N class stage_ty limit_blocks_per_sm persistent" per line; stage_ty 0 = the
// split face/cell stage, 4 or 8 = the fused stage's tile height).
struct TuneKey {
  int dim, pde, N, cls;
  bool operator==(const TuneKey& o) const { return dim == o.dim && pde == o.pde && N == o.N && cls == o.cls; }
};
struct TuneVal {
  int stage_ty, limit_per_sm, persistent;
};
static std::vector<std::pair<TuneKey, TuneVal>> g_tune;
static bool g_tune_loaded = false;

static int size_class(long long cells) {
  int c = 0;
  while ((1LL << (c + 1)) <= cells) ++c;
  return c;
}

static void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* f = getenv("DG_AUTOTUNE_FILE");
  if (!f) return;
  FILE* fp = fopen(f, "r");
  if (!fp) return;
  TuneKey k;
  TuneVal v;
  while (fscanf(fp, "%d %d %d %d %d %d %d", &k.dim, &k.pde, &k.N, &k.cls, &v.stage_ty, &v.limit_per_sm,
                &v.persistent) == 7)
    if ((v.stage_ty == 0 || v.stage_ty == 4 || v.stage_ty == 8) && v.limit_per_sm >= 1 && v.limit_per_sm <= 64 &&
        (v.persistent == 0 || v.persistent == 1))
      g_tune.push_back({k, v});
  fclose(fp);
}

static const TuneVal* tune_find(const TuneKey& k) {
  for (auto it = g_tune.rbegin(); it != g_tune.rend(); ++it)
    if (it->first == k) return &it->second;
  return nullptr;
}

// (re)builds the 2D stage tile list for tile height ty
static cudaError_t build_stage_tiles(dg_mesh* m, int ty) {
  std::vector<Tile> tiles;
  for (int i = 0; i < m->n_inst; ++i) {
    const Inst& I = m->h_inst[i];
    for (int y0 = 0; y0 < I.ny; y0 += ty)
      for (int x0 = 0; x0 < I.nx; x0 += tile_w2()) tiles.push_back(Tile{i, x0, y0, 0});
  }
  if (m->d_stage_tiles) cudaFree(m->d_stage_tiles);
  m->d_stage_tiles = nullptr;
  cudaError_t e = cudaMalloc(&m->d_stage_tiles, sizeof(Tile) * tiles.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(m->d_stage_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice);
  m->n_stage_tiles = (int)tiles.size();
  m->stage_ty = ty;
  return e;
}

extern "C" dg_status dg_mesh_create(int dim, int pde, int N, int n_inst, const int* nx, const int* ny,
                                    const double* box, int bc, double gamma, void* stream, dg_mesh** out) {
  if (!out) return fail(DG_EINVAL, "out is NULL");
  *out = nullptr;
  if (dim != 1 && dim != 2) return fail(DG_EINVAL, "dim must be 1 or 2 (got %d)", dim);
  if (pde != DG_BURGERS && pde != DG_EULER) return fail(DG_EINVAL, "unknown pde %d", pde);
  if (N < 1 || N > 3) return fail(DG_EINVAL, "order N must be 1..3 (got %d)", N);
  if (n_inst < 1 || !nx || !box || (dim == 2 && !ny)) return fail(DG_EINVAL, "bad instance arrays");
  if (bc != DG_BC_PERIODIC && bc != DG_BC_OUTFLOW && bc != DG_BC_DMR) return fail(DG_EINVAL, "unknown bc %d", bc);
  if (bc == DG_BC_DMR && (dim != 2 || pde != DG_EULER))
    return fail(DG_EINVAL, "the double Mach reflection boundaries are for 2D Euler meshes");
  if (pde == DG_EULER && !(gamma > 1.0)) return fail(DG_EINVAL, "gamma must exceed 1");
  dg_status s = dg_ensure_tables_internal();
  if (s != DG_OK) return s;
  dg_mesh* m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ENOMEM, "host allocation");
  m->dim = dim; m->pde = pde; m->N = N; m->n_inst = n_inst; m->bc = bc; m->gamma = gamma;
  m->V = nv_of(dim, pde);
  m->NP = np_of(dim, N);
  m->st = (cudaStream_t)stream;
  cudaGetDevice(&m->device);
  long long off = 0, fxoff = 0, fyoff = 0;
  std::vector<Tile> tiles;
  const int TW = dim == 1 ? tile_w1() : tile_w2(), TH = dim == 1 ? 1 : tile_h2();
  for (int i = 0; i < n_inst; ++i) {
    Inst I{};
    I.nx = nx[i];
    I.ny = dim == 1 ? 1 : ny[i];
    if (I.nx < 1 || I.ny < 1 || (long long)I.nx * I.ny > (1LL << 30)) {
      delete m;
      return fail(DG_EINVAL, "instance %d: bad size %d x %d", i, nx[i], dim == 1 ? 1 : ny[i]);
    }
    const double xL = box[4 * i], xR = box[4 * i + 1], yL = box[4 * i + 2], yR = box[4 * i + 3];
    if (!(xR > xL) || (dim == 2 && !(yR > yL))) {
      delete m;
      return fail(DG_EINVAL, "instance %d: empty box", i);
    }
    I.off = off;
    I.hx = (xR - xL) / I.nx;
    I.hy = dim == 2 ? (yR - yL) / I.ny : 1.0;
    I.xL = xL;
    I.yL = dim == 2 ? yL : 0.0;
    I.dt = 0.0;
    I.fx = fxoff;
    I.fy = fyoff;
    fxoff += (long long)(I.nx + 1) * I.ny;
    fyoff += (long long)I.nx * (I.ny + 1);
    m->h_inst.push_back(I);
    for (int y0 = 0; y0 < I.ny; y0 += TH)
      for (int x0 = 0; x0 < I.nx; x0 += TW) tiles.push_back(Tile{i, x0, y0, 0});
    off += (long long)I.nx * I.ny;
  }
  if (off >= (1LL << 31)) {
    delete m;
    return fail(DG_EINVAL, "too many cells (%lld); the troubled-cell list uses 32-bit indices", off);
  }
  m->ncell = off;
  m->ctot = (off + 31) / 32 * 32;
  m->min_side = 1 << 30;
  for (const Inst& I : m->h_inst) m->min_side = std::min(m->min_side, dim == 1 ? I.nx : std::min(I.nx, I.ny));
  m->ntiles = (int)tiles.size();
  m->last_dt.assign(n_inst, 0.0);
  std::vector<int> cell_inst(off);
  for (int i = 0; i < n_inst; ++i)
    for (long long c = 0; c < (long long)m->h_inst[i].nx * m->h_inst[i].ny; ++c) cell_inst[m->h_inst[i].off + c] = i;
  const size_t plane = (size_t)m->ctot * m->V * m->NP * sizeof(double);
  auto alloc = [&](void** p, size_t bytes) -> bool { return cudaMalloc(p, bytes) == cudaSuccess; };
  bool ok = alloc((void**)&m->d_inst, sizeof(Inst) * n_inst) && alloc((void**)&m->d_tiles, sizeof(Tile) * tiles.size()) &&
            alloc((void**)&m->d_cell_inst, sizeof(int) * off) && alloc((void**)&m->U[0], plane) &&
            alloc((void**)&m->U[1], plane) && alloc((void**)&m->U[2], plane) && alloc((void**)&m->lim, plane) &&
            alloc((void**)&m->flags, m->ctot) && alloc((void**)&m->list_cell, sizeof(int) * m->ctot) &&
            alloc((void**)&m->list_inst, sizeof(int) * m->ctot) && alloc((void**)&m->cnt, sizeof(Counters)) &&
            alloc((void**)&m->d_speed, sizeof(double) * 2 * n_inst) &&
            alloc((void**)&m->flag_totals, 3 * sizeof(unsigned long long)) &&
            alloc((void**)&m->pp_counts, 2 * sizeof(unsigned long long)) &&
            (pde != DG_EULER || (alloc((void**)&m->pp_list, sizeof(int) * off) &&
                                 alloc((void**)&m->pp_n, sizeof(unsigned int)) &&
                                 alloc((void**)&m->sp_lb, sizeof(unsigned int) * 2 * n_inst))) &&
            alloc((void**)&m->d_kx_hpow, sizeof(double) * n_inst) &&
            (bc != DG_BC_DMR || alloc((void**)&m->d_bcd, sizeof(double) * (kDmrInst + kDmrStride * n_inst)));
  if (!ok) {
    cudaGetLastError();
    dg_mesh_destroy(m);
    return fail(DG_ENOMEM, "device allocation of %.3f GB failed", 4.0 * plane / 1e9);
  }
  cudaError_t e = cudaMemcpy(m->d_inst, m->h_inst.data(), sizeof(Inst) * n_inst, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->d_cell_inst, cell_inst.data(), sizeof(int) * off, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->U[0], 0, plane);
  if (e == cudaSuccess) e = cudaMemset(m->cnt, 0, sizeof(Counters));
  if (e == cudaSuccess) e = cudaMemset(m->flag_totals, 0, 3 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(m->pp_counts, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess && bc == DG_BC_DMR) {  // times 0, the top side's y per instance; data set later
    std::vector<double> bcd(kDmrInst + kDmrStride * n_inst, 0.0);
    for (int i = 0; i < n_inst; ++i) bcd[kDmrInst + kDmrStride * i + 1] = box[4 * i + 3];
    e = cudaMemcpy(m->d_bcd, bcd.data(), sizeof(double) * bcd.size(), cudaMemcpyHostToDevice);
  }
  {
    std::vector<double> hp(n_inst);
    for (int i = 0; i < n_inst; ++i) {
      const Inst& I = m->h_inst[i];
      const double r = dim == 1 ? 0.5 * I.hx : 0.5 * std::sqrt(I.hx * I.hx + I.hy * I.hy);
      hp[i] = std::pow(r, 0.5 * (N + 1));
    }
    if (e == cudaSuccess) e = cudaMemcpy(m->d_kx_hpow, hp.data(), sizeof(double) * n_inst, cudaMemcpyHostToDevice);
    const dgt::Tabs& tb = g_tabs[N - 1];
    for (int k = 0; k <= N; ++k) {
      m->kx_pm[k] = tb.psi_m1[k];
      m->kx_pp[k] = tb.psi_p1[k];
      m->kx_w[k] = tb.gw[k];
      for (int q = 0; q <= N; ++q) m->kx_pq[q * (N + 1) + k] = tb.psi_q[q][k];
    }
  }
  if (e != cudaSuccess) {
    dg_mesh_destroy(m);
    return fail(DG_ECUDA, "mesh upload: %s", cudaGetErrorString(e));
  }
  {
    // 1D bases at the check points of the positivity-preserving scaling: the N+1 Gauss
    // points and the Gauss-Lobatto points -1, 0, 1 (-1, 1 for N = 1)
    const dgt::Tabs& tb = g_tabs[N - 1];
    const double* gl[3] = {tb.psi_m1, N == 1 ? tb.psi_p1 : tb.psi_0, tb.psi_p1};
    const int L = N == 1 ? 2 : 3;
    for (int i = 0; i <= N; ++i)
      for (int k = 0; k <= N; ++k) m->pp_g[i * (N + 1) + k] = tb.psi_q[i][k];
    for (int j = 0; j < L; ++j)
      for (int k = 0; k <= N; ++k) m->pp_l[j * (N + 1) + k] = gl[j][k];
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  m->sms = sms > 0 ? sms : 152;
  m->limit_blocks = m->sms * 8;
  tune_load();
  const TuneVal* tv = tune_find(TuneKey{dim, pde, N, size_class(off)});
  if (tv) m->limit_blocks = m->sms * tv->limit_per_sm;
  if (tv) m->stage_persistent = tv->persistent;
  if (dim == 2) {
    e = prepare2(pde, N);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_lq, sizeof(unsigned int));
    if (e == cudaSuccess) e = build_stage_tiles(m, tv && tv->stage_ty ? tv->stage_ty : 8);
    if (e != cudaSuccess) {
      dg_mesh_destroy(m);
      return fail(DG_ECUDA, "stage kernel set-up: %s", cudaGetErrorString(e));
    }
    // split stage: face planes and face tiles (32 faces x 4 rows); without the memory the
    // mesh keeps the fused stage
    std::vector<Tile> ft;
    for (int i = 0; i < n_inst; ++i) {
      const Inst& I = m->h_inst[i];
      for (int y0 = 0; y0 < I.ny; y0 += 4)
        for (int x0 = 0; x0 <= I.nx; x0 += 32) ft.push_back(Tile{i, x0, y0, 0});
      for (int y0 = 0; y0 <= I.ny; y0 += 4)
        for (int x0 = 0; x0 < I.nx; x0 += 32) ft.push_back(Tile{i, x0, y0, 1});
    }
    m->fxt = (fxoff + 31) / 32 * 32;
    m->fyt = (fyoff + 31) / 32 * 32;
    const size_t fbytes = sizeof(double) * (size_t)(m->N + 1) * m->V * (size_t)(m->fxt + m->fyt);
    if (cudaMalloc(&m->fbuf, fbytes) == cudaSuccess &&
        cudaMalloc(&m->d_face_tiles, sizeof(Tile) * ft.size()) == cudaSuccess &&
        cudaMemcpy(m->d_face_tiles, ft.data(), sizeof(Tile) * ft.size(), cudaMemcpyHostToDevice) == cudaSuccess) {
      m->n_face_tiles = (int)ft.size();
      m->stage_split = !tv || tv->stage_ty == 0;
    } else {
      cudaGetLastError();
      cudaFree(m->fbuf);
      cudaFree(m->d_face_tiles);
      m->fbuf = nullptr;
      m->d_face_tiles = nullptr;
      m->stage_split = false;
    }
    if (bc == DG_BC_DMR && !m->fbuf) {
      dg_mesh_destroy(m);
      return fail(DG_ENOMEM, "the double Mach reflection boundaries need the split stage's face planes");
    }
  }
  *out = m;
  return DG_OK;
}

// ----------------------------------------------------------------------------- launches
template <typename L>
static L args(dg_mesh* m, int un, int us, int out) {
  L a;
  a.st = m->st;
  a.un = m->U[un];
  a.us = m->U[us];
  a.out = m->U[out];
  a.inst = m->d_inst;
  a.tiles = m->d_tiles;
  a.ntiles = m->ntiles;
  a.ctot = m->ctot;
  a.ncell = m->ncell;
  a.cap = m->ctot;
  a.bc = m->bc;
  a.gam = m->gamma;
  a.lq = m->d_lq;
  a.bcd = m->d_bcd;
  return a;
}

// Times of the kBcDmr boundary data after stage s of SSP-RK3: the output of stage 1 holds at
// t^n + dt, of stage 2 at t^n + dt/2, of stage 3 at t^n + dt, which becomes the new t^n.
// kBcDmr meshes run the stage, the TVB indicator, the CSWENO limiter and the positivity
// scaling; the other indicators and limiters have no double Mach reflection ghosts.
static dg_status dmr_check(const dg_mesh* m, int indicator) {
  if (m->bc != DG_BC_DMR) return DG_OK;
  if (!m->bcd_set) return fail(DG_ESTATE, "set the boundary data (dg_set_boundary_data) first");
  if (indicator != DG_IND_TVB)
    return fail(DG_EINVAL, "the double Mach reflection boundaries support the TVB indicator only");
  return DG_OK;
}

static __global__ void k_stage_time(double* __restrict__ bcd, const Inst* __restrict__ insts, int n_inst, int stage,
                                    double dt_all) {
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
    double* ti = bcd + kDmrInst + kDmrStride * i;
    const double dt = dt_all > 0.0 ? dt_all : insts[i].dt;
    if (stage == 0) {  // the current state is u^n again (dg_set_modes)
      ti[0] = ti[2];
      continue;
    }
    const double c = stage == 2 ? 0.5 : 1.0;
    ti[0] = ti[2] + c * dt;
    if (stage == 3) ti[2] = ti[0];
  }
}

static void k_stage(dg_mesh* m, int stage, int in, int out, double dt_all) {
  if (m->bc == DG_BC_DMR) {
    // the stage evaluates L at the time of its input state (bcd), then the times advance
    LaunchArgs a = args<LaunchArgs>(m, 0, in, out);
    double* fy = m->fbuf + (size_t)(m->N + 1) * m->V * m->fxt;
    launch_stage2_split(m->pde, m->N, a, stage, dt_all, m->d_face_tiles, m->n_face_tiles, m->fbuf, m->fxt, fy,
                        m->fyt);
    k_stage_time<<<1, 32, 0, m->st>>>(m->d_bcd, m->d_inst, m->n_inst, stage, dt_all);
    m->launches += 3;
    return;
  }
  if (m->dim == 1) {
    launch_stage1(m->pde, m->N, args<LaunchArgs>(m, 0, in, out), stage, dt_all);
  } else {
    LaunchArgs a = args<LaunchArgs>(m, 0, in, out);
    if (m->stage_split) {
      double* fy = m->fbuf + (size_t)(m->N + 1) * m->V * m->fxt;
      launch_stage2_split(m->pde, m->N, a, stage, dt_all, m->d_face_tiles, m->n_face_tiles, m->fbuf, m->fxt, fy,
                          m->fyt);
      m->launches += 2;
      return;
    }
    a.tiles = m->d_stage_tiles;
    a.ntiles = m->n_stage_tiles;
    if (m->stage_persistent) cudaMemsetAsync(m->d_queue, 0, sizeof(int), m->st);
    launch_stage2(m->pde, m->N, a, stage, dt_all, m->stage_ty, m->stage_persistent ? m->d_queue : nullptr, m->sms);
  }
  m->launches++;
}


// U_0 -> cell mean factor: psi_0 in 1D, psi_0^2 in 2D
static double mean_factor(const dg_mesh* m) { return m->dim == 1 ? g_tabs[0].psi_0[0] : g_tabs[0].psi_0[0] * g_tabs[0].psi_0[0]; }

// every cell's logit (diagnostics): the network on the whole mesh
static void k_flag_learned(dg_mesh* m, float* logits) {
  LaunchArgs a = args<LaunchArgs>(m, 0, m->cur, m->cur);
  launch_flag_mlp(m->dim, m->pde, m->N, a, mean_factor(m), m->mlp, m->flags, m->cnt, m->list_cell, m->list_inst, logits);
  m->launches++;
}

static void k_flag(dg_mesh* m, double M);
static void k_limit_list(dg_mesh* m, const int* lc, const int* li, const Counters* cnt);

// the learned indicator: TVB flags (list A), then the network keeps a subset (list B)
static cudaError_t learned_flags(dg_mesh* m, double M) {
  cudaError_t e = cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->cnt_b, 0, sizeof(Counters), m->st);
  if (e != cudaSuccess) return e;
  k_flag(m, M);
  LaunchArgs a = args<LaunchArgs>(m, 0, m->cur, m->cur);
  launch_mlp_filter(m->dim, m->pde, m->N, a, mean_factor(m), m->mlp, m->list_cell, m->list_inst, m->cnt, m->flags,
                    m->cnt_b, m->lb_cell, m->lb_inst, m->limit_blocks);
  m->launches++;
  return cudaSuccess;
}

// limiter on list B with the positivity fallback of the learned indicator (Euler).  The
// learned stage differs from the plain method's only in the TVB-flagged cells the network
// skipped, which stay unlimited; they are screened on their unlimited state (density and
// pressure at the volume and face Gauss points).  An instance where one fails is redone with
// the plain TVB flags (list C: all its TVB-flagged cells, limited from the unlimited stage,
// which list B's limited values have not yet overwritten) -- the stage the plain method
// produces; the other instances get list B's values.  Cells outside the skipped ones
// (unflagged, or limited on the network's list) take the same values in the plain stage,
// so a failure there is one the redo cannot change: without the positivity-preserving
// scaling a final screen of every cell of the stage counts the instances whose stage still
// fails (with the scaling on, the scaling that follows restores the check points instead).
static cudaError_t learned_limit(dg_mesh* m) {
  LaunchArgs a = args<LaunchArgs>(m, 0, m->cur, m->cur);
  if (m->pde != DG_EULER) {
    k_limit_list(m, m->lb_cell, m->lb_inst, m->cnt_b);
    return cudaSuccess;
  }
  unsigned int* redo = m->fail;
  unsigned int* fail3 = m->fail + m->n_inst;
  cudaError_t e = cudaMemsetAsync(m->fail, 0, 2 * sizeof(unsigned int) * m->n_inst, m->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->cnt_c, 0, sizeof(Counters), m->st);
  if (e != cudaSuccess) return e;
  if (m->dim == 1) launch_limit1(m->pde, m->N, a, m->lb_cell, m->lb_inst, m->cnt_b, m->lim, m->limit_blocks);
  else launch_limit2(m->pde, m->N, a, m->lb_cell, m->lb_inst, m->cnt_b, m->lim, m->limit_blocks);
  launch_positivity_skipped(m->dim, m->N, a, m->psi_q, m->psi_p1, m->gamma, m->list_cell, m->list_inst, m->cnt,
                            m->flags, redo, m->limit_blocks);
  launch_count_fail(m->st, redo, m->n_inst, m->pos_counts);
  launch_scatter_unless(m->dim, m->pde, m->N, a, m->lim, m->lb_cell, m->lb_inst, m->cnt_b, redo, m->limit_blocks);
  launch_filter_inst(m->st, m->list_cell, m->list_inst, m->cnt, redo, m->cnt_c, m->lc_cell, m->lc_inst,
                     m->limit_blocks);
  k_limit_list(m, m->lc_cell, m->lc_inst, m->cnt_c);
  m->launches += 6;
  if (!m->pp_on) {
    launch_positivity_all(m->dim, m->N, a, m->psi_q, m->psi_p1, m->gamma, m->d_cell_inst, fail3, m->sms * 8);
    launch_count_fail(m->st, fail3, m->n_inst, m->pos_counts + 1);
    m->launches += 2;
  }
  return cudaSuccess;
}

static void k_flag_kx(dg_mesh* m) {
  launch_kxrcf(m->dim, m->pde, m->N, args<LaunchArgs>(m, 0, m->cur, m->cur), m->d_kx_hpow, m->kx_pm, m->kx_pp,
               m->kx_pq, m->kx_w, m->flags, m->cnt, m->list_cell, m->list_inst);
  m->launches++;
}

static void k_flag(dg_mesh* m, double M) {
  if (m->dim == 1) launch_flag1(m->pde, m->N, args<LaunchArgs>(m, 0, m->cur, m->cur), M, m->flags, m->cnt, m->list_cell, m->list_inst);
  else launch_flag2(m->pde, m->N, args<LaunchArgs>(m, 0, m->cur, m->cur), M, m->flags, m->cnt, m->list_cell, m->list_inst);
  m->launches++;
}

static void k_parent_list(dg_mesh* m, const int* lc, const int* li, const Counters* cnt) {
  auto a = args<LaunchArgs>(m, 0, m->cur, m->cur);
  launch_parent(m->dim, m->pde, m->N, a, lc, li, cnt, m->lim, m->limit_blocks);
  if (m->dim == 1) launch_scatter1(m->pde, m->N, a, m->lim, lc, cnt, m->limit_blocks);
  else launch_scatter2(m->pde, m->N, a, m->lim, lc, cnt, m->limit_blocks);
  m->launches += 2;
}

static void k_limit_list(dg_mesh* m, const int* lc, const int* li, const Counters* cnt) {
  auto a = args<LaunchArgs>(m, 0, m->cur, m->cur);
  if (m->dim == 1) {
    launch_limit1(m->pde, m->N, a, lc, li, cnt, m->lim, m->limit_blocks);
    launch_scatter1(m->pde, m->N, a, m->lim, lc, cnt, m->limit_blocks);
  } else {
    launch_limit2(m->pde, m->N, a, lc, li, cnt, m->lim, m->limit_blocks);
    launch_scatter2(m->pde, m->N, a, m->lim, lc, cnt, m->limit_blocks);
  }
  m->launches += 2;
}

static void k_limit(dg_mesh* m) {
  if (m->use_b) k_limit_list(m, m->lb_cell, m->lb_inst, m->cnt_b);
  else k_limit_list(m, m->list_cell, m->list_inst, m->cnt);
}

// positivity-preserving scaling of the current state, every cell (Euler)
static void k_pp(dg_mesh* m, double eps0) {
  const long long want = (m->ncell + 127) / 128;
  const int nb = (int)std::max<long long>(1, std::min<long long>(want, (long long)m->sms * 16));
  launch_positivity(m->dim, m->N, m->st, m->U[m->cur], m->ctot, m->ncell, m->pp_g, m->pp_l, mean_factor(m),
                    m->gamma, eps0, m->pp_list, m->pp_n, m->pp_counts, nb);
  m->launches += 2;
}

// Adds the TVB list length and the limited list length of one pass to running totals
// (extra: the fallback list of the learned indicator, whose cells are limited as well).
static __global__ void k_accum_flags(const Counters* __restrict__ tvb, const Counters* __restrict__ limited,
                                     const Counters* __restrict__ extra, unsigned long long* __restrict__ totals) {
  if (threadIdx.x == 0) {
    totals[0] += tvb->n_flag;
    totals[1] += limited->n_flag + (extra ? extra->n_flag : 0u);
    totals[2] += 1;
  }
}

// The troubled bit (bit 0) of the flag bytes; bit 1 marks near-threshold cells.
static __global__ void k_flag_bit0(const unsigned char* __restrict__ in, unsigned char* __restrict__ out,
                                   long long n) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x)
    out[g] = in[g] & 1;
}

// The refined reciprocal (op 0) and square root (op 1) the Euler fluxes and the WENO
// weights use, on a device array (dg_refined_arith).
static __global__ void k_refined_arith(int op, const double* __restrict__ x, double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = op == 0 ? rcp_d(x[i]) : sqrt_d(x[i]);
}

// ----------------------------------------------------------------------------- layout
// ABI [cell][var][mode]  <->  device planes [var*NP + mode][ctot]
__global__ void k_aos_to_soa(const double* __restrict__ in, double* __restrict__ out, long long ncell, long long ctot,
                             int vn) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ncell; g += (long long)gridDim.x * blockDim.x)
    for (int k = 0; k < vn; ++k) out[(long long)k * ctot + g] = in[g * vn + k];
}
__global__ void k_soa_to_aos(const double* __restrict__ in, double* __restrict__ out, long long ncell, long long ctot,
                             int vn) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ncell; g += (long long)gridDim.x * blockDim.x)
    for (int k = 0; k < vn; ++k) out[g * vn + k] = in[(long long)k * ctot + g];
}

static void invalidate(dg_mesh* m) {
  m->cur = 0;
  m->last_stage = 0;
  m->flags_valid = false;
}

extern "C" dg_status dg_set_modes(dg_mesh* m, const double* modes, size_t n, int is_device) {
  if (!m || !modes) return fail(DG_EINVAL, "null argument");
  if (n != mesh_doubles(m)) return fail(DG_EINVAL, "size %zu != mesh size %zu", n, mesh_doubles(m));
  const double* src = modes;
  if (!is_device) {
    CK(cudaMemcpyAsync(m->lim, modes, n * sizeof(double), cudaMemcpyHostToDevice, m->st));
    src = m->lim;
  }
  const int vn = m->V * m->NP;
  const int nb = (int)std::min<long long>((m->ncell + 255) / 256, 65535);
  k_aos_to_soa<<<nb, 256, 0, m->st>>>(src, m->U[0], m->ncell, m->ctot, vn);
  m->launches++;
  if (m->bc == DG_BC_DMR) {
    k_stage_time<<<1, 32, 0, m->st>>>(m->d_bcd, m->d_inst, m->n_inst, 0, 0.0);
    m->launches++;
  }
  CK(cudaGetLastError());
  invalidate(m);
  return DG_OK;
}

extern "C" dg_status dg_get_modes(dg_mesh* m, double* out, size_t n, int is_device) {
  if (!m || !out) return fail(DG_EINVAL, "null argument");
  if (n != mesh_doubles(m)) return fail(DG_EINVAL, "size %zu != mesh size %zu", n, mesh_doubles(m));
  const int vn = m->V * m->NP;
  const int nb = (int)std::min<long long>((m->ncell + 255) / 256, 65535);
  double* dst = is_device ? out : m->lim;
  k_soa_to_aos<<<nb, 256, 0, m->st>>>(m->U[m->cur], dst, m->ncell, m->ctot, vn);
  m->launches++;
  CK(cudaGetLastError());
  if (!is_device) CK(cudaMemcpyAsync(out, m->lim, n * sizeof(double), cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  return DG_OK;
}

extern "C" dg_status dg_project_ic(dg_mesh* m, int ic, const double* params, int nparams) {
  if (!m || !params) return fail(DG_EINVAL, "null argument");
  static const int need[7] = {4, 7, 18, 7, 9, 4, 10};
  if (ic < 0 || ic > 6) return fail(DG_EINVAL, "unknown initial condition %d", ic);
  if (nparams < need[ic]) return fail(DG_EINVAL, "initial condition %d needs %d parameters", ic, need[ic]);
  if ((m->pde == DG_BURGERS) != (ic == DG_IC_SINE)) return fail(DG_EINVAL, "initial condition does not fit the PDE");
  if ((ic == DG_IC_RIEMANN1D || ic == DG_IC_SHOCK_ENTROPY) && m->dim != 1)
    return fail(DG_EINVAL, "1D initial data on a 2D mesh");
  if ((ic == DG_IC_QUADRANT || ic == DG_IC_VORTEX) && m->dim != 2) return fail(DG_EINVAL, "2D initial data on a 1D mesh");
  // parameters go through the limiter scratch buffer (large enough for any batch)
  const size_t bytes = sizeof(double) * (size_t)m->n_inst * nparams;
  if (bytes > (size_t)m->ctot * m->V * m->NP * sizeof(double)) return fail(DG_EINVAL, "too many parameters");
  CK(cudaMemcpyAsync(m->lim, params, bytes, cudaMemcpyHostToDevice, m->st));
  CK(cudaStreamSynchronize(m->st));
  if (m->dim == 1) launch_project1(m->pde, m->N, args<LaunchArgs>(m, 0, 0, 0), m->d_cell_inst, ic, m->lim, nparams);
  else launch_project2(m->pde, m->N, args<LaunchArgs>(m, 0, 0, 0), m->d_cell_inst, ic, m->lim, nparams);
  m->launches++;
  CK(cudaGetLastError());
  invalidate(m);
  return DG_OK;
}

extern "C" dg_status dg_set_dt(dg_mesh* m, const double* dt) {
  if (!m || !dt) return fail(DG_EINVAL, "null argument");
  for (int i = 0; i < m->n_inst; ++i) {
    if (!(dt[i] > 0.0)) return fail(DG_EINVAL, "dt[%d] must be positive", i);
    m->h_inst[i].dt = dt[i];
  }
  CK(cudaMemcpyAsync(m->d_inst, m->h_inst.data(), sizeof(Inst) * m->n_inst, cudaMemcpyHostToDevice, m->st));
  CK(cudaStreamSynchronize(m->st));
  for (int i = 0; i < m->n_inst; ++i) m->last_dt[i] = dt[i];
  return DG_OK;
}

static dg_status check_dt(dg_mesh* m, double dt) {
  if (dt > 0.0) return DG_OK;
  for (int i = 0; i < m->n_inst; ++i)
    if (!(m->h_inst[i].dt > 0.0)) return fail(DG_EINVAL, "dt <= 0 but no per-instance dt was set");
  return DG_OK;
}

// stage s reads u^(s-1) from `in` and u^n from U[0]; buffers: stage 1 -> U1, 2 -> U2, 3 -> U0
static int stage_out(int s) { return s == 1 ? 1 : (s == 2 ? 2 : 0); }

extern "C" dg_status dg_rk_stage(dg_mesh* m, int stage, double dt) {
  if (m && m->bc == DG_BC_DMR && !m->bcd_set) return fail(DG_ESTATE, "set the boundary data (dg_set_boundary_data) first");
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (stage < 1 || stage > 3) return fail(DG_EINVAL, "stage must be 1..3 (got %d)", stage);
  if (m->last_stage != stage - 1 && !(stage == 1 && m->last_stage == 3))
    return fail(DG_ESTATE, "stage %d requested after stage %d", stage, m->last_stage);
  dg_status s = check_dt(m, dt);
  if (s != DG_OK) return s;
  const int in = m->cur, out = stage_out(stage);
  k_stage(m, stage, in, out, dt > 0.0 ? dt : 0.0);
  CK(cudaGetLastError());
  m->cur = out;
  m->last_stage = stage;
  m->flags_valid = false;
  return DG_OK;
}

extern "C" dg_status dg_flag_cells(dg_mesh* m, int indicator, double tvb_M, int64_t* n_flagged, int64_t* n_near,
                                   uint8_t* flags_out) {
  if (m) {
    dg_status ds = dmr_check(m, indicator);
    if (ds != DG_OK) return ds;
  }
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (indicator != DG_IND_TVB && indicator != DG_IND_MLP && indicator != DG_IND_KXRCF)
    return fail(DG_EINVAL, "unknown indicator %d", indicator);
  if (indicator == DG_IND_MLP && !m->has_mlp) return fail(DG_EINVAL, "no learned indicator attached to the mesh");
  if (!(tvb_M >= 0.0)) return fail(DG_EINVAL, "tvb_M must be >= 0");
  if (indicator == DG_IND_MLP) {
    CK(learned_flags(m, tvb_M));
  } else if (indicator == DG_IND_KXRCF) {
    CK(cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st));
    k_flag_kx(m);
  } else {
    CK(cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st));
    k_flag(m, tvb_M);
  }
  CK(cudaGetLastError());
  m->flags_valid = true;
  m->use_b = indicator == DG_IND_MLP;
  if (n_flagged || n_near || flags_out) {
    Counters c, cb;
    CK(cudaMemcpyAsync(&c, m->cnt, sizeof(c), cudaMemcpyDeviceToHost, m->st));
    if (m->use_b) {
      CK(cudaMemcpyAsync(&cb, m->cnt_b, sizeof(cb), cudaMemcpyDeviceToHost, m->st));
    }
    if (flags_out) CK(cudaMemcpyAsync(flags_out, m->flags, m->ncell, cudaMemcpyDeviceToHost, m->st));
    CK(cudaStreamSynchronize(m->st));
    if (n_flagged) *n_flagged = m->use_b ? cb.n_flag : c.n_flag;
    if (n_near) *n_near = c.n_near;
  }
  return DG_OK;
}

extern "C" dg_status dg_cswenolimit(dg_mesh* m) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (!m->flags_valid) return fail(DG_ESTATE, "no troubled-cell flags for the current state");
  if (m->use_b) CK(learned_limit(m));  // the learned flags, with their positivity fallback
  else k_limit(m);
  CK(cudaGetLastError());
  m->flags_valid = false;
  return DG_OK;
}

extern "C" dg_status dg_parent_wenolimit(dg_mesh* m) {
  if (m && m->bc == DG_BC_DMR) return fail(DG_EINVAL, "not available with the double Mach reflection boundaries");
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (!m->flags_valid) return fail(DG_ESTATE, "no troubled-cell flags for the current state");
  if (m->min_side < m->N + 1) return fail(DG_EINVAL, "the parent WENO stencil needs %d cells per side", m->N + 1);
  if (m->use_b) k_parent_list(m, m->lb_cell, m->lb_inst, m->cnt_b);
  else k_parent_list(m, m->list_cell, m->list_inst, m->cnt);
  CK(cudaGetLastError());
  m->flags_valid = false;
  return DG_OK;
}

extern "C" dg_status dg_set_limiter(dg_mesh* m, int limiter) {
  if (m && m->bc == DG_BC_DMR && limiter != DG_LIM_CSWENO)
    return fail(DG_EINVAL, "the double Mach reflection boundaries support the CSWENO limiter only");
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (limiter != DG_LIM_CSWENO && limiter != DG_LIM_PARENT) return fail(DG_EINVAL, "unknown limiter %d", limiter);
  if (limiter == DG_LIM_PARENT && m->min_side < m->N + 1)
    return fail(DG_EINVAL, "the parent WENO stencil needs %d cells per side", m->N + 1);
  m->limiter = limiter;
  return DG_OK;
}

extern "C" dg_status dg_positivity_limit(dg_mesh* m, double eps0) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (m->pde != DG_EULER) return fail(DG_EINVAL, "the positivity-preserving scaling is defined for the Euler equations");
  if (!(eps0 > 0.0) || !std::isfinite(eps0)) return fail(DG_EINVAL, "eps0 must be positive and finite");
  k_pp(m, eps0);
  CK(cudaGetLastError());
  m->flags_valid = false;
  return DG_OK;
}

extern "C" dg_status dg_set_positivity(dg_mesh* m, int enable, double eps0) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (enable && m->pde != DG_EULER) return fail(DG_EINVAL, "the positivity-preserving scaling is defined for the Euler equations");
  if (enable && (!(eps0 > 0.0) || !std::isfinite(eps0))) return fail(DG_EINVAL, "eps0 must be positive and finite");
  m->pp_on = enable != 0;
  if (m->pp_on) m->pp_eps0 = eps0;
  return DG_OK;
}

extern "C" dg_status dg_positivity_counts(dg_mesh* m, int64_t* changed, int64_t* bad_means, int reset) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  unsigned long long c[2];
  CK(cudaMemcpyAsync(c, m->pp_counts, sizeof(c), cudaMemcpyDeviceToHost, m->st));
  if (reset) CK(cudaMemsetAsync(m->pp_counts, 0, sizeof(c), m->st));
  CK(cudaStreamSynchronize(m->st));
  if (changed) *changed = (int64_t)c[0];
  if (bad_means) *bad_means = (int64_t)c[1];
  return c[1] ? DG_EPOSITIVITY : DG_OK;
}

extern "C" dg_status dg_max_wavespeed_points(dg_mesh* m, double* out) {
  if (!m || !out) return fail(DG_EINVAL, "null argument");
  if (m->pde != DG_EULER) return fail(DG_EINVAL, "the check-point wave speed is defined for the Euler equations");
  CK(cudaMemsetAsync(m->d_speed, 0, sizeof(double) * 2 * m->n_inst, m->st));
  const long long want = (m->ncell + 127) / 128;
  const int nb = (int)std::max<long long>(1, std::min<long long>(want, (long long)m->sms * 16));
  launch_speed_points(m->dim, m->N, m->st, m->U[m->cur], m->ctot, m->ncell, m->d_cell_inst, m->pp_g, m->pp_l,
                      m->gamma, m->d_speed, m->sp_lb, m->n_inst, m->pp_list, m->pp_n, nb);
  m->launches += 3;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, m->d_speed, sizeof(double) * 2 * m->n_inst, cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  return DG_OK;
}

extern "C" dg_status dg_max_wavespeed(dg_mesh* m, double* out) {
  if (!m || !out) return fail(DG_EINVAL, "null argument");
  CK(cudaMemsetAsync(m->d_speed, 0, sizeof(double) * 2 * m->n_inst, m->st));
  if (m->dim == 1) launch_speed1(m->pde, m->N, args<LaunchArgs>(m, 0, m->cur, m->cur), m->d_cell_inst, m->d_speed);
  else launch_speed2(m->pde, m->N, args<LaunchArgs>(m, 0, m->cur, m->cur), m->d_cell_inst, m->d_speed);
  m->launches++;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, m->d_speed, sizeof(double) * 2 * m->n_inst, cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  return DG_OK;
}

// The three (stage, indicator, limiter) passes of one SSP-RK3 step, enqueued on m->st.
static dg_status enqueue_step(dg_mesh* m, int indicator, double M) {
  for (int s = 1; s <= 3; ++s) {
    const int in = s == 1 ? 0 : m->cur, out = stage_out(s);
    k_stage(m, s, in, out, 0.0);
    m->cur = out;
    if (indicator == DG_IND_MLP) {
      CK(learned_flags(m, M));
      CK(learned_limit(m));
      k_accum_flags<<<1, 32, 0, m->st>>>(m->cnt, m->cnt_b, m->pde == DG_EULER ? m->cnt_c : nullptr, m->flag_totals);
    } else {
      CK(cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st));
      if (indicator == DG_IND_KXRCF) k_flag_kx(m);
      else k_flag(m, M);
      if (m->limiter == DG_LIM_PARENT) k_parent_list(m, m->list_cell, m->list_inst, m->cnt);
      else k_limit_list(m, m->list_cell, m->list_inst, m->cnt);
      k_accum_flags<<<1, 32, 0, m->st>>>(m->cnt, m->cnt, nullptr, m->flag_totals);
    }
    m->launches++;
    if (m->pp_on) k_pp(m, m->pp_eps0);
  }
  CK(cudaGetLastError());
  return DG_OK;
}

extern "C" dg_status dg_set_boundary_data(dg_mesh* m, const double* p, int n) {
  if (!m || !p) return fail(DG_EINVAL, "null argument");
  if (m->bc != DG_BC_DMR) return fail(DG_EINVAL, "the mesh has no boundary data (bc %d)", m->bc);
  if (n != 11) return fail(DG_EINVAL, "the double Mach reflection boundaries take 11 values (got %d)", n);
  double h[kDmrInst];
  for (int k = 0; k < 2; ++k) {
    const double rho = p[4 * k], u = p[4 * k + 1], v = p[4 * k + 2], pr = p[4 * k + 3];
    if (!(rho > 0.0) || !(pr > 0.0)) return fail(DG_EINVAL, "boundary states need positive density and pressure");
    double* c = h + (k == 0 ? kDmrPost : kDmrPre);
    c[0] = rho;
    c[1] = rho * u;
    c[2] = rho * v;
    c[3] = pr / (m->gamma - 1.0) + 0.5 * rho * (u * u + v * v);
  }
  h[kDmrA] = p[8];
  h[kDmrB] = p[9];
  h[kDmrC] = p[10];
  CK(cudaMemcpyAsync(m->d_bcd, h, sizeof(h), cudaMemcpyHostToDevice, m->st));
  CK(cudaStreamSynchronize(m->st));
  m->bcd_set = true;
  return DG_OK;
}

extern "C" dg_status dg_set_time(dg_mesh* m, const double* t) {
  if (!m || !t) return fail(DG_EINVAL, "null argument");
  if (m->bc != DG_BC_DMR) return fail(DG_EINVAL, "only meshes with time-dependent boundaries keep a time");
  const size_t pitch = sizeof(double) * kDmrStride;
  CK(cudaMemcpy2DAsync(m->d_bcd + kDmrInst + 2, pitch, t, sizeof(double), sizeof(double), m->n_inst,
                       cudaMemcpyHostToDevice, m->st));
  CK(cudaMemcpy2DAsync(m->d_bcd + kDmrInst, pitch, t, sizeof(double), sizeof(double), m->n_inst,
                       cudaMemcpyHostToDevice, m->st));
  CK(cudaStreamSynchronize(m->st));
  return DG_OK;
}

extern "C" dg_status dg_get_time(dg_mesh* m, double* t) {
  if (!m || !t) return fail(DG_EINVAL, "null argument");
  if (m->bc != DG_BC_DMR) return fail(DG_EINVAL, "only meshes with time-dependent boundaries keep a time");
  CK(cudaMemcpy2DAsync(t, sizeof(double), m->d_bcd + kDmrInst + 2, sizeof(double) * kDmrStride, sizeof(double),
                       m->n_inst, cudaMemcpyDeviceToHost, m->st));
  CK(cudaStreamSynchronize(m->st));
  return DG_OK;
}

extern "C" dg_status dg_step(dg_mesh* m, double dt, int indicator, double tvb_M) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  {
    dg_status ds = dmr_check(m, indicator);
    if (ds != DG_OK) return ds;
  }
  if (indicator != DG_IND_TVB && indicator != DG_IND_MLP && indicator != DG_IND_KXRCF)
    return fail(DG_EINVAL, "unknown indicator %d", indicator);
  if (indicator == DG_IND_MLP && !m->has_mlp) return fail(DG_EINVAL, "no learned indicator attached to the mesh");
  if (m->last_stage != 0 && m->last_stage != 3) return fail(DG_ESTATE, "a step was left unfinished (stage %d)", m->last_stage);
  // the graph reads the per-instance time steps from device memory
  if (dt > 0.0) {
    bool same = true;
    for (int i = 0; i < m->n_inst; ++i) same = same && m->last_dt[i] == dt;
    if (!same) {
      std::vector<double> v(m->n_inst, dt);
      dg_status s = dg_set_dt(m, v.data());
      if (s != DG_OK) return s;
    }
  } else {
    dg_status s = check_dt(m, dt);
    if (s != DG_OK) return s;
  }
  m->cur = 0;
  if (m->st == nullptr) {  // the legacy default stream cannot be captured
    dg_status s = enqueue_step(m, indicator, tvb_M);
    m->last_stage = 3;
    m->flags_valid = false;
    return s;
  }
  if (!m->gexec || m->g_ind != indicator || m->g_M != tvb_M || m->g_pp != m->pp_on || m->g_pp_eps != m->pp_eps0 ||
      m->g_lim != m->limiter) {
    if (m->gexec) {
      cudaGraphExecDestroy(m->gexec);
      m->gexec = nullptr;
    }
    cudaGraph_t graph;
    const long long before = m->launches;
    CK(cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal));
    dg_status s = enqueue_step(m, indicator, tvb_M);
    cudaError_t e = cudaStreamEndCapture(m->st, &graph);
    if (s != DG_OK) return s;
    if (e != cudaSuccess) return fail(DG_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&m->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(DG_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    m->g_kernels = (int)(m->launches - before);
    m->launches = before;
    m->g_ind = indicator;
    m->g_M = tvb_M;
    m->g_pp = m->pp_on;
    m->g_pp_eps = m->pp_eps0;
    m->g_lim = m->limiter;
  }
  CK(cudaGraphLaunch(m->gexec, m->st));
  m->launches += m->g_kernels;
  m->cur = 0;
  m->last_stage = 3;
  m->flags_valid = false;
  return DG_OK;
}

// Times the candidate configurations on this mesh's current state (u^n is left unchanged):
// the 2D stage form on stage 1 -- split (face pass + cell pass) or fused with a tile height
// of 4 or 8 rows and one block per tile or a persistent grid taking tiles from a queue --
// then the limiter's grid (2, 4, 8 or 16 blocks per SM) on the TVB-flagged cells of that stage.  The fastest are applied to the
// mesh and remembered for meshes of the same kind and size class.
extern "C" dg_status dg_autotune(dg_mesh* m, double dt, int* stage_ty, int* limit_blocks_per_sm, int* persistent) {
  if (!m || !(dt > 0.0)) return fail(DG_EINVAL, "bad arguments");
  if (m->last_stage != 0 && m->last_stage != 3) return fail(DG_ESTATE, "a step was left unfinished");
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_it = [&](auto fn, int reps) -> float {
    fn();  // warm-up
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(e0, m->st);
      fn();
      cudaEventRecord(e1, m->st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = ms < best ? ms : best;
    }
    return best;
  };
  m->cur = 0;
  int best_ty = m->stage_split ? 0 : m->stage_ty, best_pers = m->stage_persistent;
  if (m->dim == 2) {
    float best = 1e30f;
    if (m->fbuf) {  // split stage (face pass + cell pass)
      m->stage_split = true;
      best = time_it([&] { k_stage(m, 1, 0, 1, dt); }, 3);
      best_ty = 0;
    }
    m->stage_split = false;
    for (int ty : {8, 4}) {
      if (m->bc == DG_BC_DMR) break;  // the boundary data are read by the split stage only
      cudaError_t e = build_stage_tiles(m, ty);
      if (e != cudaSuccess) return fail(DG_ECUDA, "stage tiles: %s", cudaGetErrorString(e));
      for (int pers : {0, 1}) {
        m->stage_persistent = pers;
        const float ms = time_it([&] { k_stage(m, 1, 0, 1, dt); }, 3);
        if (ms < best) { best = ms; best_ty = ty; best_pers = pers; }
      }
    }
    CK(build_stage_tiles(m, best_ty ? best_ty : 8));
    m->stage_persistent = best_pers;
    m->stage_split = best_ty == 0;
  }
  // limiter grid on the flagged cells of stage 1 (writes only the limiter scratch)
  k_stage(m, 1, 0, 1, dt);
  m->cur = 1;
  CK(cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st));
  k_flag(m, 0.01);
  int best_mult = m->limit_blocks / m->sms;
  {
    float best = 1e30f;
    for (int mult : {8, 2, 4, 16}) {
      LaunchArgs a = args<LaunchArgs>(m, 0, 1, 1);
      const float ms = time_it([&] {
        if (m->dim == 1) launch_limit1(m->pde, m->N, a, m->list_cell, m->list_inst, m->cnt, m->lim, m->sms * mult);
        else launch_limit2(m->pde, m->N, a, m->list_cell, m->list_inst, m->cnt, m->lim, m->sms * mult);
      }, 3);
      if (ms < best) { best = ms; best_mult = mult; }
    }
  }
  m->limit_blocks = m->sms * best_mult;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  m->cur = 0;
  m->last_stage = 0;
  m->flags_valid = false;
  if (m->gexec) {  // launch configurations are baked into the graph
    cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
  }
  const TuneKey k{m->dim, m->pde, m->N, size_class(m->ncell)};
  g_tune.push_back({k, TuneVal{best_ty, best_mult, best_pers}});
  if (const char* f = getenv("DG_AUTOTUNE_FILE")) {
    if (FILE* fp = fopen(f, "a")) {
      fprintf(fp, "%d %d %d %d %d %d %d\n", k.dim, k.pde, k.N, k.cls, best_ty, best_mult, best_pers);
      fclose(fp);
    }
  }
  if (stage_ty) *stage_ty = m->dim == 2 ? best_ty : 0;
  if (limit_blocks_per_sm) *limit_blocks_per_sm = best_mult;
  if (persistent) *persistent = m->dim == 2 ? best_pers : 0;
  return DG_OK;
}

// ----------------------------------------------------------------------------- diagnostics
// Copies the CSWENO tables the library derived for degree N (host only, no GPU needed):
// rp[NG], rw[NG], C[(i*NG+g)*(N+1)+k], gam[g*(N+1)+i], B[(i*(N+1)+k)*(N+1)+l], SA[k*(N+1)+n].
extern "C" dg_status dg_limiter_tables(int N, double* rp, double* rw, double* C, double* gam, double* B, double* SA) {
  if (N < 1 || N > 3 || !rp || !rw || !C || !gam || !B || !SA) return fail(DG_EINVAL, "bad arguments");
  dgt::Tabs t;
  if (dgt::build_tables(N, &t)) return fail(DG_EINVAL, "table derivation failed");
  const int N1 = N + 1, NG = t.NG;
  for (int g = 0; g < NG; ++g) {
    rp[g] = t.rp[g];
    rw[g] = t.rw[g];
    for (int i = 0; i < N1; ++i) gam[g * N1 + i] = t.gam[g][i];
  }
  for (int i = 0; i < N1; ++i)
    for (int g = 0; g < NG; ++g)
      for (int k = 0; k < N1; ++k) C[(i * NG + g) * N1 + k] = t.C[i][g][k];
  for (int i = 0; i < N1; ++i)
    for (int k = 0; k < N1; ++k)
      for (int l = 0; l < N1; ++l) B[(i * N1 + k) * N1 + l] = t.B[i][k][l];
  for (int k = 0; k < 2 * N + 1; ++k)
    for (int n = 0; n < N1; ++n) SA[k * N1 + n] = t.SA[k][n];
  return DG_OK;
}

// ----------------------------------------------------------------------------- learned indicator
struct dg_mlp {
  int F = 0, FP = 0, P = 0, t = 0;
  cudaStream_t st = nullptr;
  float *params = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *loss = nullptr;
  void* infer = nullptr;  // BF16 W1 [32][FP], BF16 W2 [32][32], FP32 b1, b2, w3, b3
  long long cap = 0;
  float *h1 = nullptr, *d1 = nullptr, *h2 = nullptr, *d2 = nullptr, *dz = nullptr;
  float* part = nullptr;  // per-chunk weight gradients [chunks][P]
};

static const int kHidden = 32;

static size_t infer_bytes(int FP) { return 2 * (size_t)kHidden * FP + 2 * kHidden * kHidden + 4 * (3 * kHidden + 4); }

static MlpInfer infer_view(void* buf, int FP, float tau) {
  unsigned char* p = static_cast<unsigned char*>(buf);
  MlpInfer w{};
  w.W1 = p;
  w.W2 = p + 2 * (size_t)kHidden * FP;
  float* f = reinterpret_cast<float*>(p + 2 * (size_t)kHidden * FP + 2 * kHidden * kHidden);
  w.b1 = f;
  w.b2 = f + kHidden;
  w.w3 = f + 2 * kHidden;
  w.b3 = f + 3 * kHidden;
  w.FP = FP;
  w.tau = tau;
  return w;
}

static void mlp_export(dg_mlp* n) {
  MlpInfer w = infer_view(n->infer, n->FP, 0.f);
  launch_mlp_export(n->st, n->params, n->F, n->FP, const_cast<void*>(w.W1), const_cast<float*>(w.b1),
                    const_cast<void*>(w.W2), const_cast<float*>(w.b2), const_cast<float*>(w.w3),
                    const_cast<float*>(w.b3));
}

extern "C" int dg_mlp_features(int dim, int pde, int N) {
  if ((dim != 1 && dim != 2) || (pde != 0 && pde != 1) || N < 1 || N > 3) return -1;
  return mlp_features(dim, pde, N);
}

extern "C" size_t dg_mlp_param_count(const dg_mlp* n) { return n ? (size_t)n->P : 0; }

extern "C" dg_status dg_mlp_destroy(dg_mlp* n) {
  if (!n) return DG_OK;
  cudaFree(n->params); cudaFree(n->grad); cudaFree(n->m1); cudaFree(n->m2); cudaFree(n->loss); cudaFree(n->infer);
  cudaFree(n->h1); cudaFree(n->d1); cudaFree(n->h2); cudaFree(n->d2); cudaFree(n->dz); cudaFree(n->part);
  delete n;
  return DG_OK;
}

extern "C" dg_status dg_mlp_create(int n_features, uint64_t seed, void* stream, dg_mlp** out) {
  if (!out) return fail(DG_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_features < 1 || n_features > 4096) return fail(DG_EINVAL, "bad feature count %d", n_features);
  dg_mlp* n = new (std::nothrow) dg_mlp();
  if (!n) return fail(DG_ENOMEM, "host allocation");
  n->F = n_features;
  n->FP = mlp_padded(n_features);
  n->P = kHidden * n_features + kHidden + kHidden * kHidden + kHidden + kHidden + 1;
  n->st = (cudaStream_t)stream;
  const size_t pb = sizeof(float) * n->P;
  if (cudaMalloc(&n->params, pb) != cudaSuccess || cudaMalloc(&n->grad, pb) != cudaSuccess ||
      cudaMalloc(&n->m1, pb) != cudaSuccess || cudaMalloc(&n->m2, pb) != cudaSuccess ||
      cudaMalloc(&n->loss, sizeof(float)) != cudaSuccess || cudaMalloc(&n->infer, infer_bytes(n->FP)) != cudaSuccess) {
    cudaGetLastError();
    dg_mlp_destroy(n);
    return fail(DG_ENOMEM, "device allocation for the network");
  }
  // He-uniform initial weights from a splitmix64 stream, zero biases
  std::vector<float> h(n->P, 0.0f);
  uint64_t x = seed;
  auto uni = [&]() {
    x += 0x9e3779b97f4a7c15ULL;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  };
  const double a1 = std::sqrt(6.0 / n_features), a2 = std::sqrt(6.0 / kHidden);
  size_t o = 0;
  for (int i = 0; i < kHidden * n_features; ++i) h[o++] = (float)((2 * uni() - 1) * a1);
  o += kHidden;
  for (int i = 0; i < kHidden * kHidden; ++i) h[o++] = (float)((2 * uni() - 1) * a2);
  o += kHidden;
  for (int i = 0; i < kHidden; ++i) h[o++] = (float)((2 * uni() - 1) * a2);
  cudaError_t e = cudaMemcpy(n->params, h.data(), pb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m1, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(n->m2, 0, pb);
  if (e != cudaSuccess) {
    dg_mlp_destroy(n);
    return fail(DG_ECUDA, "network upload: %s", cudaGetErrorString(e));
  }
  mlp_export(n);
  *out = n;
  return DG_OK;
}

extern "C" dg_status dg_mlp_get_params(dg_mlp* n, float* out, size_t count) {
  if (!n || !out) return fail(DG_EINVAL, "null argument");
  if (count != (size_t)n->P) return fail(DG_EINVAL, "parameter count %zu != %d", count, n->P);
  CK(cudaMemcpyAsync(out, n->params, sizeof(float) * n->P, cudaMemcpyDeviceToHost, n->st));
  CK(cudaStreamSynchronize(n->st));
  return DG_OK;
}

extern "C" dg_status dg_mlp_set_params(dg_mlp* n, const float* in, size_t count) {
  if (!n || !in) return fail(DG_EINVAL, "null argument");
  if (count != (size_t)n->P) return fail(DG_EINVAL, "parameter count %zu != %d", count, n->P);
  CK(cudaMemcpyAsync(n->params, in, sizeof(float) * n->P, cudaMemcpyHostToDevice, n->st));
  CK(cudaMemsetAsync(n->m1, 0, sizeof(float) * n->P, n->st));
  CK(cudaMemsetAsync(n->m2, 0, sizeof(float) * n->P, n->st));
  n->t = 0;
  mlp_export(n);
  CK(cudaStreamSynchronize(n->st));
  return DG_OK;
}

static dg_status mlp_backward(dg_mlp* n, const float* X, const uint8_t* y, int64_t B, float pw) {
  if (B > n->cap) {
    cudaFree(n->h1); cudaFree(n->d1); cudaFree(n->h2); cudaFree(n->d2); cudaFree(n->dz); cudaFree(n->part);
    n->h1 = n->d1 = n->h2 = n->d2 = n->dz = n->part = nullptr;
    const size_t hb = sizeof(float) * kHidden * (size_t)B;
    if (cudaMalloc(&n->h1, hb) != cudaSuccess || cudaMalloc(&n->d1, hb) != cudaSuccess ||
        cudaMalloc(&n->h2, hb) != cudaSuccess || cudaMalloc(&n->d2, hb) != cudaSuccess ||
        cudaMalloc(&n->dz, sizeof(float) * (size_t)B) != cudaSuccess ||
        cudaMalloc(&n->part, sizeof(float) * (size_t)n->P * (size_t)mlp_wgrad_chunks(B)) != cudaSuccess) {
      cudaGetLastError();
      n->cap = 0;
      return fail(DG_ENOMEM, "training scratch for %lld samples", (long long)B);
    }
    n->cap = B;
  }
  CK(cudaMemsetAsync(n->loss, 0, sizeof(float), n->st));
  launch_mlp_fb(n->st, X, y, B, n->F, n->params, pw, n->h1, n->d1, n->h2, n->d2, n->dz, n->loss);
  launch_mlp_wgrad(n->st, X, B, n->F, n->h1, n->d1, n->h2, n->d2, n->dz, n->part, n->grad);
  CK(cudaGetLastError());
  return DG_OK;
}

extern "C" dg_status dg_mlp_grad(dg_mlp* n, const float* X, const uint8_t* y, int64_t B, float pos_weight,
                                 float* grad_out, float* loss_out) {
  if (!n || !X || !y || B < 1) return fail(DG_EINVAL, "bad arguments");
  dg_status s = mlp_backward(n, X, y, B, pos_weight);
  if (s != DG_OK) return s;
  if (grad_out) CK(cudaMemcpyAsync(grad_out, n->grad, sizeof(float) * n->P, cudaMemcpyDeviceToHost, n->st));
  if (loss_out) CK(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->st));
  CK(cudaStreamSynchronize(n->st));
  return DG_OK;
}

extern "C" dg_status dg_mlp_train_step(dg_mlp* n, const float* X, const uint8_t* y, int64_t B, float pos_weight,
                                       float lr, float* loss_out) {
  if (!n || !X || !y || B < 1 || !(lr > 0.f)) return fail(DG_EINVAL, "bad arguments");
  dg_status s = mlp_backward(n, X, y, B, pos_weight);
  if (s != DG_OK) return s;
  n->t += 1;
  launch_mlp_adam(n->st, n->params, n->grad, n->m1, n->m2, n->P, lr, n->t);
  mlp_export(n);
  CK(cudaGetLastError());
  if (loss_out) {
    CK(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->st));
    CK(cudaStreamSynchronize(n->st));
  }
  return DG_OK;
}

extern "C" dg_status dg_mlp_predict(dg_mlp* n, const float* X, int64_t B, float* logits) {
  if (!n || !X || !logits || B < 1) return fail(DG_EINVAL, "bad arguments");
  launch_mlp_forward(n->st, X, B, n->F, n->params, logits);
  CK(cudaGetLastError());
  return DG_OK;
}

extern "C" dg_status dg_set_indicator_mlp(dg_mesh* m, const dg_mlp* n, float tau) {
  if (m && m->bc == DG_BC_DMR) return fail(DG_EINVAL, "not available with the double Mach reflection boundaries");
  if (!m || !n) return fail(DG_EINVAL, "null argument");
  const int F = mlp_features(m->dim, m->pde, m->N);
  if (F != n->F) return fail(DG_EINVAL, "network has %d features, this mesh needs %d", n->F, F);
  if (!m->mlp_buf) {
    bool ok = cudaMalloc(&m->mlp_buf, infer_bytes(n->FP)) == cudaSuccess &&
              cudaMalloc(&m->lb_cell, sizeof(int) * m->ctot) == cudaSuccess &&
              cudaMalloc(&m->lb_inst, sizeof(int) * m->ctot) == cudaSuccess &&
              cudaMalloc(&m->lc_cell, sizeof(int) * m->ctot) == cudaSuccess &&
              cudaMalloc(&m->lc_inst, sizeof(int) * m->ctot) == cudaSuccess &&
              cudaMalloc(&m->cnt_b, sizeof(Counters)) == cudaSuccess &&
              cudaMalloc(&m->cnt_c, sizeof(Counters)) == cudaSuccess &&
              cudaMalloc(&m->fail, 2 * sizeof(unsigned int) * m->n_inst) == cudaSuccess &&
              cudaMalloc(&m->pos_counts, 2 * sizeof(unsigned long long)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return fail(DG_ENOMEM, "device allocation for the learned indicator");
    }
    CK(cudaMemset(m->pos_counts, 0, 2 * sizeof(unsigned long long)));
    CK(cudaMemset(m->cnt_b, 0, sizeof(Counters)));
    CK(prepare_mlp(m->dim, m->pde, m->N, n->FP));
    CK(prepare_filter(m->dim, m->pde, m->N, n->FP));
    const dgt::Tabs& tb = g_tabs[m->N - 1];
    for (int q = 0; q <= m->N; ++q)
      for (int k = 0; k <= m->N; ++k) m->psi_q[q * (m->N + 1) + k] = tb.psi_q[q][k];
    for (int k = 0; k <= m->N; ++k) m->psi_p1[k] = tb.psi_p1[k];
  }
  // the network's stream must have finished its last update before the copy
  CK(cudaStreamSynchronize(n->st));
  CK(cudaMemcpyAsync(m->mlp_buf, n->infer, infer_bytes(n->FP), cudaMemcpyDeviceToDevice, m->st));
  m->mlp = infer_view(m->mlp_buf, n->FP, tau);
  m->has_mlp = true;
  if (m->gexec && m->g_ind == DG_IND_MLP) {  // the threshold is a kernel argument of the graph
    cudaGraphExecDestroy(m->gexec);
    m->gexec = nullptr;
  }
  return DG_OK;
}

extern "C" dg_status dg_flag_statistics(dg_mesh* m, int64_t* tvb_flagged, int64_t* limited, int64_t* passes,
                                        int reset) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  unsigned long long c[3];
  CK(cudaMemcpyAsync(c, m->flag_totals, sizeof(c), cudaMemcpyDeviceToHost, m->st));
  if (reset) CK(cudaMemsetAsync(m->flag_totals, 0, sizeof(c), m->st));
  CK(cudaStreamSynchronize(m->st));
  if (tvb_flagged) *tvb_flagged = (int64_t)c[0];
  if (limited) *limited = (int64_t)c[1];
  if (passes) *passes = (int64_t)c[2];
  return DG_OK;
}

extern "C" dg_status dg_positivity_report(dg_mesh* m, int64_t* fallbacks, int64_t* failures) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  unsigned long long c[2] = {0, 0};
  if (m->pos_counts) {
    CK(cudaMemcpyAsync(c, m->pos_counts, sizeof(c), cudaMemcpyDeviceToHost, m->st));
    CK(cudaStreamSynchronize(m->st));
  }
  if (fallbacks) *fallbacks = (int64_t)c[0];
  if (failures) *failures = (int64_t)c[1];
  return c[1] ? DG_EPOSITIVITY : DG_OK;
}

extern "C" dg_status dg_indicator_logits(dg_mesh* m, float* logits) {
  if (m && m->bc == DG_BC_DMR) return fail(DG_EINVAL, "not available with the double Mach reflection boundaries");
  if (!m || !logits) return fail(DG_EINVAL, "null argument");
  if (!m->has_mlp) return fail(DG_EINVAL, "no learned indicator attached to the mesh");
  CK(cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st));
  k_flag_learned(m, logits);
  CK(cudaGetLastError());
  m->flags_valid = true;
  m->use_b = false;
  return DG_OK;
}

extern "C" dg_status dg_refined_arith(int op, const double* x, double* out, int64_t n, void* stream) {
  if ((op != 0 && op != 1) || !x || !out || n < 0) return fail(DG_EINVAL, "bad arguments");
  if (n == 0) return DG_OK;
  const cudaStream_t st = (cudaStream_t)stream;
  k_refined_arith<<<(int)std::min<long long>((n + 255) / 256, 65535), 256, 0, st>>>(op, x, out, n);
  CK(cudaGetLastError());
  return DG_OK;
}

extern "C" dg_status dg_harvest(dg_mesh* m, double tvb_M, float* X, uint8_t* flags, float* change) {
  if (m && m->bc == DG_BC_DMR) return fail(DG_EINVAL, "not available with the double Mach reflection boundaries");
  if (!m || !X || !flags || !change) return fail(DG_EINVAL, "null argument");
  LaunchArgs a = args<LaunchArgs>(m, 0, m->cur, m->cur);
  const double c0 = mean_factor(m);
  m->use_b = false;
  launch_features(m->dim, m->pde, m->N, a, c0, X);
  CK(cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st));
  k_flag(m, tvb_M);
  CK(cudaMemsetAsync(change, 0, sizeof(float) * m->ncell, m->st));
  if (m->dim == 1) launch_limit1(m->pde, m->N, a, m->list_cell, m->list_inst, m->cnt, m->lim, m->limit_blocks);
  else launch_limit2(m->pde, m->N, a, m->list_cell, m->list_inst, m->cnt, m->lim, m->limit_blocks);
  launch_label(m->dim, m->pde, m->N, a, c0, m->list_cell, m->list_inst, m->cnt, m->lim, change, m->limit_blocks);
  k_flag_bit0<<<(int)std::min<long long>((m->ncell + 255) / 256, 65535), 256, 0, m->st>>>(m->flags, flags, m->ncell);
  if (m->dim == 1) launch_scatter1(m->pde, m->N, a, m->lim, m->list_cell, m->cnt, m->limit_blocks);
  else launch_scatter2(m->pde, m->N, a, m->lim, m->list_cell, m->cnt, m->limit_blocks);
  m->launches += 5;
  CK(cudaGetLastError());
  m->flags_valid = false;
  return DG_OK;
}
