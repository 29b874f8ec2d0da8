// C ABI of the library (include/dg.h): mesh management, host<->device layout changes,
// the per-call entry points and the CUDA-graph time step.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
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
void launch_stage2(int pde, int N, const LaunchArgs& a, int stage, double dt_all);
void launch_flag2(int pde, int N, const LaunchArgs& a, double M, unsigned char* flags, Counters* cnt, int* lc, int* li);
void launch_limit2(int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt, double* lim,
                   int nblocks);
void launch_scatter2(int pde, int N, const LaunchArgs& a, const double* lim, const int* lc, const Counters* cnt,
                     int nblocks);
void launch_project2(int pde, int N, const LaunchArgs& a, const int* cell_inst, int kind, const double* params, int np);
void launch_speed2(int pde, int N, const LaunchArgs& a, const int* cell_inst, double* out);
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

dg_status dg_ensure_tables_internal() {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (g_tables_dev == -2) {
    for (int n = 1; n <= 3; ++n)
      if (dgt::build_tables(n, &g_tabs[n - 1])) return fail(DG_EINVAL, "table derivation failed for N=%d", n);
  }
  // constant memory is per device: upload once for every device that creates a mesh
  static std::vector<int> done;
  for (int d : done)
    if (d == dev) return DG_OK;
  CK(upload_tables1(g_tabs));
  CK(upload_tables2(g_tabs));
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
  long long launches = 0;
  // CUDA graph of one full step
  cudaGraphExec_t gexec = nullptr;
  int g_ind = -1;
  double g_M = 0.0;
  int g_kernels = 0;
  std::vector<double> last_dt;
};

static size_t mesh_doubles(const dg_mesh* m) { return (size_t)m->ncell * m->V * m->NP; }

extern "C" size_t dg_mesh_size(const dg_mesh* m) { return m ? mesh_doubles(m) : 0; }

extern "C" int64_t dg_kernel_launches(const dg_mesh* m) { return m ? m->launches : 0; }

extern "C" dg_status dg_mesh_destroy(dg_mesh* m) {
  if (!m) return DG_OK;
  if (m->gexec) cudaGraphExecDestroy(m->gexec);
  cudaFree(m->d_inst);
  cudaFree(m->d_tiles);
  cudaFree(m->d_cell_inst);
  for (auto& p : m->U) cudaFree(p);
  cudaFree(m->lim);
  cudaFree(m->flags);
  cudaFree(m->list_cell);
  cudaFree(m->list_inst);
  cudaFree(m->cnt);
  cudaFree(m->d_speed);
  delete m;
  return DG_OK;
}

extern "C" dg_status dg_mesh_create(int dim, int pde, int N, int n_inst, const int* nx, const int* ny,
                                    const double* box, int bc, double gamma, void* stream, dg_mesh** out) {
  if (!out) return fail(DG_EINVAL, "out is NULL");
  *out = nullptr;
  if (dim != 1 && dim != 2) return fail(DG_EINVAL, "dim must be 1 or 2 (got %d)", dim);
  if (pde != DG_BURGERS && pde != DG_EULER) return fail(DG_EINVAL, "unknown pde %d", pde);
  if (N < 1 || N > 3) return fail(DG_EINVAL, "order N must be 1..3 (got %d)", N);
  if (n_inst < 1 || !nx || !box || (dim == 2 && !ny)) return fail(DG_EINVAL, "bad instance arrays");
  if (bc != DG_BC_PERIODIC && bc != DG_BC_OUTFLOW) return fail(DG_EINVAL, "unknown bc %d", bc);
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
  long long off = 0;
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
            alloc((void**)&m->d_speed, sizeof(double) * 2 * n_inst);
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
  if (e != cudaSuccess) {
    dg_mesh_destroy(m);
    return fail(DG_ECUDA, "mesh upload: %s", cudaGetErrorString(e));
  }
  if (dim == 2) {
    e = prepare2(pde, N);
    if (e != cudaSuccess) {
      dg_mesh_destroy(m);
      return fail(DG_ECUDA, "stage kernel attributes: %s", cudaGetErrorString(e));
    }
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  m->limit_blocks = (sms > 0 ? sms : 152) * 8;
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
  return a;
}

static void k_stage(dg_mesh* m, int stage, int in, int out, double dt_all) {
  if (m->dim == 1) launch_stage1(m->pde, m->N, args<LaunchArgs>(m, 0, in, out), stage, dt_all);
  else launch_stage2(m->pde, m->N, args<LaunchArgs>(m, 0, in, out), stage, dt_all);
  m->launches++;
}

static void k_flag(dg_mesh* m, double M) {
  if (m->dim == 1) launch_flag1(m->pde, m->N, args<LaunchArgs>(m, 0, m->cur, m->cur), M, m->flags, m->cnt, m->list_cell, m->list_inst);
  else launch_flag2(m->pde, m->N, args<LaunchArgs>(m, 0, m->cur, m->cur), M, m->flags, m->cnt, m->list_cell, m->list_inst);
  m->launches++;
}

static void k_limit(dg_mesh* m) {
  if (m->dim == 1) {
    auto a = args<LaunchArgs>(m, 0, m->cur, m->cur);
    launch_limit1(m->pde, m->N, a, m->list_cell, m->list_inst, m->cnt, m->lim, m->limit_blocks);
    launch_scatter1(m->pde, m->N, a, m->lim, m->list_cell, m->cnt, m->limit_blocks);
  } else {
    auto a = args<LaunchArgs>(m, 0, m->cur, m->cur);
    launch_limit2(m->pde, m->N, a, m->list_cell, m->list_inst, m->cnt, m->lim, m->limit_blocks);
    launch_scatter2(m->pde, m->N, a, m->lim, m->list_cell, m->cnt, m->limit_blocks);
  }
  m->launches += 2;
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
  static const int need[4] = {4, 7, 18, 7};
  if (ic < 0 || ic > 3) return fail(DG_EINVAL, "unknown initial condition %d", ic);
  if (nparams < need[ic]) return fail(DG_EINVAL, "initial condition %d needs %d parameters", ic, need[ic]);
  if ((m->pde == DG_BURGERS) != (ic == DG_IC_SINE)) return fail(DG_EINVAL, "initial condition does not fit the PDE");
  if (ic == DG_IC_RIEMANN1D && m->dim != 1) return fail(DG_EINVAL, "1D Riemann data on a 2D mesh");
  if (ic == DG_IC_QUADRANT && m->dim != 2) return fail(DG_EINVAL, "quadrant data on a 1D mesh");
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
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (indicator != DG_IND_TVB) return fail(DG_EINVAL, "indicator %d is not available", indicator);
  if (!(tvb_M >= 0.0)) return fail(DG_EINVAL, "tvb_M must be >= 0");
  CK(cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st));
  k_flag(m, tvb_M);
  CK(cudaGetLastError());
  m->flags_valid = true;
  if (n_flagged || n_near || flags_out) {
    Counters c;
    CK(cudaMemcpyAsync(&c, m->cnt, sizeof(c), cudaMemcpyDeviceToHost, m->st));
    if (flags_out) CK(cudaMemcpyAsync(flags_out, m->flags, m->ncell, cudaMemcpyDeviceToHost, m->st));
    CK(cudaStreamSynchronize(m->st));
    if (n_flagged) *n_flagged = c.n_flag;
    if (n_near) *n_near = c.n_near;
  }
  return DG_OK;
}

extern "C" dg_status dg_cswenolimit(dg_mesh* m) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (!m->flags_valid) return fail(DG_ESTATE, "no troubled-cell flags for the current state");
  k_limit(m);
  CK(cudaGetLastError());
  m->flags_valid = false;
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
static dg_status enqueue_step(dg_mesh* m, double M) {
  for (int s = 1; s <= 3; ++s) {
    const int in = s == 1 ? 0 : m->cur, out = stage_out(s);
    k_stage(m, s, in, out, 0.0);
    m->cur = out;
    CK(cudaMemsetAsync(m->cnt, 0, sizeof(Counters), m->st));
    k_flag(m, M);
    k_limit(m);
  }
  CK(cudaGetLastError());
  return DG_OK;
}

extern "C" dg_status dg_step(dg_mesh* m, double dt, int indicator, double tvb_M) {
  if (!m) return fail(DG_EINVAL, "null mesh");
  if (indicator != DG_IND_TVB) return fail(DG_EINVAL, "indicator %d is not available", indicator);
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
    dg_status s = enqueue_step(m, tvb_M);
    m->last_stage = 3;
    m->flags_valid = false;
    return s;
  }
  if (!m->gexec || m->g_ind != indicator || m->g_M != tvb_M) {
    if (m->gexec) {
      cudaGraphExecDestroy(m->gexec);
      m->gexec = nullptr;
    }
    cudaGraph_t graph;
    const long long before = m->launches;
    CK(cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal));
    dg_status s = enqueue_step(m, tvb_M);
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
  }
  CK(cudaGraphLaunch(m->gexec, m->st));
  m->launches += m->g_kernels;
  m->cur = 0;
  m->last_stage = 3;
  m->flags_valid = false;
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
