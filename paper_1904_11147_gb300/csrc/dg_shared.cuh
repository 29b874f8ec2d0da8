// Device helpers shared by the 1D and 2D kernel files: block compaction of flagged
// cells, the scatter of limited modes, and an atomic max on non-negative doubles.
#pragma once

#include "dg_common.cuh"

namespace dg {

// Arguments shared by the launchers of one kernel family (1D or 2D).
struct LaunchArgs {
  cudaStream_t st;
  const double *un, *us;
  double* out;
  const Inst* inst;
  const Tile* tiles;
  int ntiles;
  long long ctot, ncell, cap;
  int bc;
  double gam;
  unsigned int* lq;  // work counter of the 2D Euler limiter (zeroed by its launcher), or null
  const double* bcd;  // boundary data of kBcDmr meshes (see dmr_ghost), or null
};

// ----------------------------------------------------------------------------- boundaries
// Boundary condition codes: 0 periodic, 1 outflow (mirror ghosts), 2 the double Mach
// reflection problem (Example 11, after Woodward and Colella; 2D Euler).
constexpr int kBcDmr = 2;
// Layout of the kBcDmr boundary data: post-shock and pre-shock conserved states, the shock
// line x_s(y, t) = a + b y + c t, then per instance the time of the current state, the
// top side's y and the time of u^n.
constexpr int kDmrPost = 0, kDmrPre = 4, kDmrA = 8, kDmrB = 9, kDmrC = 10, kDmrInst = 11, kDmrStride = 3;
__device__ __forceinline__ double dmr_time(const double* __restrict__ bcd, int inst, int which) {
  return bcd[kDmrInst + kDmrStride * inst + which];  // 0: current state, 2: u^n
}

// The ghost cell (ix, iy) outside instance `inst` of a kBcDmr mesh, decided by its centre
// at the time t of the state it borders: on the left the post-shock state (inflow); on the
// right the mirror image of the boundary cell (outflow); below, the post-shock state where
// the centre lies left of a, else a reflecting wall (mirror image, rho v negated); above,
// the post-shock state left of the shock's position on the top side, x_s(y_top, t), else
// the pre-shock state.  The x side decides first.  Returns the constant state's conserved
// variables (c != null), or the interior cell to mirror and its flips.
struct Ghost {
  const double* c;   // constant ghost: conserved state, else null
  int jx, jy;        // interior cell of a mirrored ghost
  bool fx, fy, fv;   // odd modes in x / in y negated; rho v negated (wall)
};
__device__ __forceinline__ Ghost dmr_ghost(const Inst& I, int inst, int ix, int iy, const double* __restrict__ bcd,
                                           double t) {
  Ghost gh{nullptr, ix, iy, false, false, false};
  const double xc = __dadd_rn(I.xL, __dmul_rn((double)ix + 0.5, I.hx));
  if (ix < 0) {
    gh.c = bcd + kDmrPost;
    return gh;
  }
  if (iy >= I.ny) {
    const double ytop = bcd[kDmrInst + kDmrStride * inst + 1];
    const double xs = __dadd_rn(__dadd_rn(bcd[kDmrA], __dmul_rn(bcd[kDmrB], ytop)), __dmul_rn(bcd[kDmrC], t));
    gh.c = xc < xs ? bcd + kDmrPost : bcd + kDmrPre;
    return gh;
  }
  if (iy < 0 && xc < bcd[kDmrA]) {
    gh.c = bcd + kDmrPost;
    return gh;
  }
  if (ix >= I.nx) {
    gh.jx = 2 * I.nx - 1 - ix;
    gh.fx = true;
  }
  if (iy < 0) {
    gh.jy = -1 - iy;
    gh.fy = gh.fv = true;
  }
  gh.jx = gh.jx < 0 ? 0 : (gh.jx >= I.nx ? I.nx - 1 : gh.jx);
  gh.jy = gh.jy < 0 ? 0 : (gh.jy >= I.ny ? I.ny - 1 : gh.jy);
  return gh;
}

// Inference weights of the learned indicator (device pointers): W1 BF16 [32][FP] (rows
// padded with zeros to FP columns), b1 FP32 [32], W2 BF16 [32][32], b2, w3 FP32 [32], b3.
struct MlpInfer {
  const void* W1;
  const float* b1;
  const void* W2;
  const float* b2;
  const float* w3;
  const float* b3;
  int FP;
  float tau;
};

// Per-call device counters (one struct per mesh, zeroed before each indicator pass).
struct Counters {
  unsigned int n_flag;   // number of troubled cells in the list
  unsigned int n_near;   // cells decided within 1e-12 relative of a threshold
  unsigned int status;   // device error bits
  unsigned int pad;
};

// Compacts the calling block's flagged cells into list[] with one atomic per block.
// Every thread of the block must call it (flag = 0 for inactive threads).
// Warp ballot + shared-memory scan of the warp totals (up to 32 warps per block).
__device__ __forceinline__ void block_compact(int flag, int near, long long cell, int inst,
                                              Counters* cnt, int* list_cell, int* list_inst) {
  __shared__ unsigned int s_warp[32];
  __shared__ unsigned int s_base;
  __shared__ unsigned int s_near;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  if (threadIdx.x == 0) s_near = 0;
  unsigned int bal = __ballot_sync(0xffffffffu, flag);
  unsigned int nbal = __ballot_sync(0xffffffffu, near);
  if (lane == 0) s_warp[w] = __popc(bal);
  __syncthreads();
  if (lane == 0 && nbal) atomicAdd(&s_near, (unsigned)__popc(nbal));
  if (threadIdx.x == 0) {
    unsigned int run = 0;
    for (int i = 0; i < nw; ++i) {
      unsigned int c = s_warp[i];
      s_warp[i] = run;
      run += c;
    }
    s_base = run ? atomicAdd(&cnt->n_flag, run) : 0u;
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_near) atomicAdd(&cnt->n_near, s_near);
  if (flag) {
    unsigned int pos = s_base + s_warp[w] + __popc(bal & ((1u << lane) - 1u));
    list_cell[pos] = (int)cell;
    list_inst[pos] = inst;
  }
}

// Writes the limited modes 1..NP-1 of every listed cell back into the state planes.
// lim is [(v*NP + m) * cap + i] (compact, list order).
template <int V, int NP>
__global__ void k_scatter(double* __restrict__ U, long long ctot, const double* __restrict__ lim, long long cap,
                          const int* __restrict__ list_cell, const Counters* __restrict__ cnt) {
  const unsigned int n = cnt->n_flag;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    long long g = list_cell[i];
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int m = 1; m < NP; ++m) U[(long long)(v * NP + m) * ctot + g] = lim[(long long)(v * NP + m) * cap + i];
  }
}

// TVB modified-minmod decision of Cockburn and Shu, taken on the IEEE-754 bit patterns:
// returns true when mt(a1, a2, a3) != a1 with mt(a1, ...) = a1 if |a1| <= M h^2, else
// minmod(a1, a2, a3).  For finite doubles, |x| is the pattern with the sign bit cleared,
// comparisons of non-negative values are comparisons of their patterns as integers, and
// x > 0 / x < 0 are sign-and-nonzero tests, so this is exactly the FP64 decision while
// keeping the slow FP64 pipe free.  near (reporting only): a deciding comparison within
// kNearUlp units in the last place, or a mean difference within 2^-39 of the largest
// magnitude.  Both windows contain the 1e-12 relative ones: two non-negative doubles with
// |x - y| <= 1e-12 max(x, y) are at most 1e-12 * 2^54 < 18015 representable steps apart
// (a step is at least 2^-54 of the larger value), and 2^-39 = 1.8e-12 > 1e-12.  So every
// cell near the threshold by the 1e-12 relative definition is reported, with a few more.
constexpr long long kNearUlp = 32768;

__device__ __forceinline__ bool tvb_changes_bits(double a1d, double a2d, double a3d, long long mh2, bool& near) {
  const long long kAbs = 0x7fffffffffffffffLL, kWin = kNearUlp;
  const long long a1 = __double_as_longlong(a1d), a2 = __double_as_longlong(a2d), a3 = __double_as_longlong(a3d);
  const long long b1 = a1 & kAbs, b2 = a2 & kAbs, b3 = a3 & kAbs;
  const long long d = b1 - mh2;
  if (d <= kWin && d >= -kWin) near = true;
  if (b1 <= mh2) return false;
  const long long s = max(max(b1, b2), b3);
  const long long thr = s >= (40LL << 52) ? s - (39LL << 52) : 0LL;  // s * 2^-39
  if (b2 <= thr || b3 <= thr) near = true;
  const bool pos = a1 > 0 && a2 > 0 && a3 > 0;
  const bool neg = a1 < 0 && b1 != 0 && a2 < 0 && b2 != 0 && a3 < 0 && b3 != 0;
  if (!(pos || neg)) return true;  // minmod = 0, and a1 != 0 here
  const long long m23 = min(b2, b3), d2 = b1 - m23;
  if (d2 <= kWin && d2 >= -kWin) near = true;
  return !(b1 <= b2 && b1 <= b3);
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns as signed 64-bit integers
  atomicMax(reinterpret_cast<long long*>(addr), __double_as_longlong(v));
}

}  // namespace dg
