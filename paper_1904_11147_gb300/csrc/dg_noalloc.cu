// dg_cswenolimit_noalloc: the troubled-cell indicator and the CSWENO limiter for one mesh
// in a single call that allocates no device memory.
//
// Who needs it: callers that must not allocate device memory once they are running -- a
// host application whose memory manager has already reserved or capped the GPU memory, a
// latency-critical loop in which cudaMalloc/cudaFree could block on or synchronise with
// the device, or a plugin whose host forbids allocation after initialisation.  They pass
// their own input and output arrays; every other buffer the limiter needs (the flag bytes,
// the compacted list of troubled cells, the counters, the limited modes, the mesh and
// tile descriptors) lives in the file-scope array below, which the CUDA runtime creates
// when this library's device code is loaded and keeps until the process exits, on every
// GPU that loads the library.
//
// The kernels are the ones the mesh-based entry points launch; only the place of their
// scratch differs.
#include <cstdio>
#include <mutex>

#include "../../include/dg.h"
#include "dg_shared.cuh"

namespace dg {
void launch_flag1(int pde, int N, const LaunchArgs& a, double M, unsigned char* flags, Counters* cnt, int* lc, int* li);
void launch_limit1(int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt, double* lim,
                   int nblocks);
void launch_scatter1(int pde, int N, const LaunchArgs& a, const double* lim, const int* lc, const Counters* cnt,
                     int nblocks);
void launch_flag2(int pde, int N, const LaunchArgs& a, double M, unsigned char* flags, Counters* cnt, int* lc, int* li);
void launch_limit2(int pde, int N, const LaunchArgs& a, const int* lc, const int* li, const Counters* cnt, double* lim,
                   int nblocks);
void launch_scatter2(int pde, int N, const LaunchArgs& a, const double* lim, const int* lc, const Counters* cnt,
                     int nblocks);
int tile_w1();
int tile_w2();
int tile_h2();
}  // namespace dg

dg_status dg_ensure_tables_internal();
void dg_set_error_internal(const char* msg);

using namespace dg;

namespace {

constexpr long long kMaxCells = DG_NOALLOC_MAX_CELLS;
constexpr int kMaxVN = 40;  // variables x modes of the largest case (2D Euler P3)

// byte offsets inside the scratch array (all 256-byte aligned)
constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffCnt = 0;
constexpr size_t kOffInst = al(kOffCnt + sizeof(Counters));
constexpr size_t kOffTiles = al(kOffInst + sizeof(Inst));
constexpr size_t kOffFlags = al(kOffTiles + sizeof(Tile) * kMaxCells);  // at most one tile per cell
constexpr size_t kOffListC = al(kOffFlags + kMaxCells);
constexpr size_t kOffListI = al(kOffListC + sizeof(int) * kMaxCells);
constexpr size_t kOffLim = al(kOffListI + sizeof(int) * kMaxCells);
constexpr size_t kScratchBytes = al(kOffLim + sizeof(double) * kMaxVN * kMaxCells);

// The scratch of every call, on every device that loads the library (about 5.7 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Writes the single mesh descriptor and its tile list into the scratch.
__global__ void k_noalloc_setup(Inst I, Inst* inst_out, Tile* tiles, int tw, int th, int ntx, int ntiles) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) *inst_out = I;
  if (t < ntiles) tiles[t] = Tile{0, (t % ntx) * tw, (t / ntx) * th, 0};
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {nullptr};

dg_status fail(dg_status s, const char* m, cudaError_t e = cudaSuccess) {
  char msg[256];
  if (e != cudaSuccess) snprintf(msg, sizeof(msg), "%s: %s", m, cudaGetErrorString(e));
  else snprintf(msg, sizeof(msg), "%s", m);
  dg_set_error_internal(msg);
  return s;
}

}  // namespace

extern "C" dg_status dg_cswenolimit_noalloc(int dim, int pde, int N, int nx, int ny, const double* box, int bc,
                                            double gamma, double tvb_M, const double* u_in, double* u_out,
                                            int64_t* n_flagged, int64_t* n_near, void* stream) {
  if (dim != 1 && dim != 2) return fail(DG_EINVAL, "dim must be 1 or 2");
  if (pde != DG_BURGERS && pde != DG_EULER) return fail(DG_EINVAL, "unknown pde");
  if (N < 1 || N > 3) return fail(DG_EINVAL, "order N must be 1..3");
  if (bc != DG_BC_PERIODIC && bc != DG_BC_OUTFLOW) return fail(DG_EINVAL, "unknown bc");
  if (!box || !u_in || !u_out) return fail(DG_EINVAL, "null pointer");
  if (pde == DG_EULER && !(gamma > 1.0)) return fail(DG_EINVAL, "gamma must exceed 1");
  if (!(tvb_M >= 0.0)) return fail(DG_EINVAL, "tvb_M must be >= 0");
  if (dim == 1) ny = 1;
  if (nx < 1 || ny < 1) return fail(DG_EINVAL, "mesh sizes must be >= 1");
  const long long ncell = (long long)nx * ny;
  if (ncell > kMaxCells) {
    char msg[160];
    snprintf(msg, sizeof(msg), "mesh of %lld cells exceeds the no-allocation limit of %lld cells", ncell, kMaxCells);
    return fail(DG_EINVAL, msg);
  }
  if (!(box[1] > box[0]) || (dim == 2 && !(box[3] > box[2]))) return fail(DG_EINVAL, "empty box");
  // device tables and the scratch address (first call on each device)
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(DG_ECUDA, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) return fail(DG_EINVAL, "device index out of range");
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
      dg_status s = dg_ensure_tables_internal();
      if (s != DG_OK) return s;
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return fail(DG_ECUDA, "cudaGetSymbolAddress", e);
      g_dev_ptr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_dev_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  Counters* cnt = reinterpret_cast<Counters*>(base + kOffCnt);
  Inst* inst = reinterpret_cast<Inst*>(base + kOffInst);
  Tile* tiles = reinterpret_cast<Tile*>(base + kOffTiles);
  unsigned char* flags = base + kOffFlags;
  int* list_c = reinterpret_cast<int*>(base + kOffListC);
  int* list_i = reinterpret_cast<int*>(base + kOffListI);
  double* lim = reinterpret_cast<double*>(base + kOffLim);

  Inst I{};
  I.nx = nx;
  I.ny = ny;
  I.off = 0;
  I.hx = (box[1] - box[0]) / nx;
  I.hy = dim == 2 ? (box[3] - box[2]) / ny : 1.0;
  I.xL = box[0];
  I.yL = dim == 2 ? box[2] : 0.0;
  I.dt = 0.0;
  const int tw = dim == 1 ? tile_w1() : tile_w2(), th = dim == 1 ? 1 : tile_h2();
  const int ntx = (nx + tw - 1) / tw, nty = (ny + th - 1) / th, ntiles = ntx * nty;
  const int V = nv_of(dim, pde), NP = np_of(dim, N);
  k_noalloc_setup<<<(ntiles + 255) / 256, 256, 0, st>>>(I, inst, tiles, tw, th, ntx, ntiles);
  // the counters must start at zero; the previous call's list, flags and modes are dead
  e = cudaMemsetAsync(cnt, 0, sizeof(Counters), st);
  if (e != cudaSuccess) return fail(DG_ECUDA, "clearing the counters", e);
  if (u_out != u_in) {
    e = cudaMemcpyAsync(u_out, u_in, sizeof(double) * (size_t)V * NP * ncell, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(DG_ECUDA, "copying the input", e);
  }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  LaunchArgs a{};
  a.st = st;
  a.un = u_in;
  a.us = u_in;
  a.out = u_out;
  a.inst = inst;
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.ctot = ncell;
  a.ncell = ncell;
  a.cap = kMaxCells;
  a.bc = bc;
  a.gam = gamma;
  if (dim == 1) {
    launch_flag1(pde, N, a, tvb_M, flags, cnt, list_c, list_i);
    launch_limit1(pde, N, a, list_c, list_i, cnt, lim, sms * 8);
    launch_scatter1(pde, N, a, lim, list_c, cnt, sms * 8);
  } else {
    launch_flag2(pde, N, a, tvb_M, flags, cnt, list_c, list_i);
    launch_limit2(pde, N, a, list_c, list_i, cnt, lim, sms * 8);
    launch_scatter2(pde, N, a, lim, list_c, cnt, sms * 8);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DG_ECUDA, "kernel launch", e);
  if (n_flagged || n_near) {
    Counters c;
    e = cudaMemcpyAsync(&c, cnt, sizeof(c), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(DG_ECUDA, "reading the troubled-cell count", e);
    if (n_flagged) *n_flagged = c.n_flag;
    if (n_near) *n_near = c.n_near;
  }
  return DG_OK;
}
