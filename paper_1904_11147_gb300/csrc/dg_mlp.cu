// Learned troubled-cell indicator: features, fused tensor-core inference in the flagging
// pass, and the training kernels (forward/backward per sample, weight gradients, Adam).
//
// Features of a cell (per variable v; cross neighbours W, E, S, N in 2D, L, R in 1D):
//   s_v = max_c |ubar_c - ubar_j| + sum_{n>=1} |U^j_{n,v}| + 1e-14,
//   (ubar_c - ubar_j) / s_v, then U^c_{n,v} / s_v (n >= 1) for c = j and the neighbours.
// Network: 32-32 ReLU MLP with one logit; a cell is troubled when the logit exceeds tau.
// Inference multiplies BF16 features by BF16 weights with FP32 accumulation on the tensor
// cores (mma.sync m16n8k16), 32 cells per warp.
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_bf16.h>

#include "dg_convert.cuh"
#include "dg_shared.cuh"

namespace dg {

constexpr int kHid = 32;
// Row strides (BF16 elements) of the per-warp feature block [32][FP] and of the hidden layer
// [32][32] in shared memory: 8 elements of padding put the eight rows an mma fragment load
// reads (and the 32 rows the feature writes touch) on different banks.
constexpr int kPadX = 8;
constexpr int kLdH = kHid + 8;

template <int DIM, int PDE, int N>
struct FeatDims {
  static constexpr int V = nv_of(DIM, PDE), NP = np_of(DIM, N), NB = DIM == 1 ? 2 : 4;
  static constexpr int F = V * (NB + (NB + 1) * (NP - 1));
  static constexpr int FP = (F + 15) / 16 * 16;  // padded to the mma K step
};

int mlp_features(int dim, int pde, int N) {
  const int V = nv_of(dim, pde), NP = np_of(dim, N), NB = dim == 1 ? 2 : 4;
  return V * (NB + (NB + 1) * (NP - 1));
}
int mlp_padded(int F) { return (F + 15) / 16 * 16; }

// Loads the modes of a cell with the boundary condition (periodic wrap; outflow mirror).
template <int DIM, int V, int NP>
__device__ __forceinline__ void load_modes(const double* __restrict__ U, long long ctot, const Inst& I, int ix,
                                           int iy, int bc, double (&u)[V][NP]) {
  bool fx = false, fy = false;
  if (bc == 0) {
    ix = ix < 0 ? ix + I.nx : (ix >= I.nx ? ix - I.nx : ix);
    iy = iy < 0 ? iy + I.ny : (iy >= I.ny ? iy - I.ny : iy);
  } else {
    if (ix < 0) { ix = 0; fx = true; }
    if (ix >= I.nx) { ix = I.nx - 1; fx = true; }
    if (iy < 0) { iy = 0; fy = true; }
    if (iy >= I.ny) { iy = I.ny - 1; fy = true; }
  }
  const long long g = I.off + (long long)iy * I.nx + ix;
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      const double x = __ldg(U + (long long)(v * NP + m) * ctot + g);
      const int a = DIM == 1 ? m : mode_a(m), b = DIM == 1 ? 0 : mode_b(m);
      const bool flip = (fx && (a & 1)) != (fy && (b & 1));
      u[v][m] = neg_if(x, flip);
    }
}

// Plane offset and mirror flags of cell (ix, iy) with the boundary condition (periodic wrap;
// outflow: the boundary cell, odd modes in the normal direction negated).
struct CellRef {
  long long g;
  bool fx, fy;
};
__device__ __forceinline__ CellRef cell_ref(const Inst& I, int ix, int iy, int bc) {
  bool fx = false, fy = false;
  if (bc == 0) {
    ix = ix < 0 ? ix + I.nx : (ix >= I.nx ? ix - I.nx : ix);
    iy = iy < 0 ? iy + I.ny : (iy >= I.ny ? iy - I.ny : iy);
  } else {
    if (ix < 0) { ix = 0; fx = true; }
    if (ix >= I.nx) { ix = I.nx - 1; fx = true; }
    if (iy < 0) { iy = 0; fy = true; }
    if (iy >= I.ny) { iy = I.ny - 1; fy = true; }
  }
  return CellRef{I.off + (long long)iy * I.nx + ix, fx, fy};
}

// The NP modes of variable v of a cell.
template <int DIM, int NP>
__device__ __forceinline__ void load_var(const double* __restrict__ U, long long ctot, const CellRef& c, int v,
                                         double (&u)[NP]) {
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    const double x = __ldg(U + (long long)(v * NP + m) * ctot + c.g);
    const int a = DIM == 1 ? m : mode_a(m), b = DIM == 1 ? 0 : mode_b(m);
    u[m] = neg_if(x, (c.fx && (a & 1)) != (c.fy && (b & 1)));
  }
}

// Writes the F features of cell (ix, iy) through `put`, one variable at a time (the modes
// of one variable of the cell and its neighbours are live at once).
template <int DIM, int PDE, int N, typename Put>
__device__ __forceinline__ void cell_features(const double* __restrict__ U, long long ctot, const Inst& I, int ix,
                                              int iy, int bc, double c0, Put put) {
  using D = FeatDims<DIM, PDE, N>;
  constexpr int V = D::V, NP = D::NP, NB = D::NB;
  CellRef cr[NB + 1];
  cr[0] = cell_ref(I, ix, iy, bc);
  cr[1] = cell_ref(I, ix - 1, iy, bc);
  cr[2] = cell_ref(I, ix + 1, iy, bc);
  if constexpr (DIM == 2) {
    cr[3] = cell_ref(I, ix, iy - 1, bc);
    cr[4] = cell_ref(I, ix, iy + 1, bc);
  }
  int k = 0;
#pragma unroll 1
  for (int v = 0; v < V; ++v) {
    double own[NP];
    load_var<DIM, NP>(U, ctot, cr[0], v, own);
    const double mj = own[0] * c0;
    float d[NB];
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < NB; ++c) {  // neighbour means first (U_0 has no mirror sign)
      d[c] = d2f_trunc(__ldg(U + (long long)(v * NP) * ctot + cr[c + 1].g) * c0 - mj);
      s = fmaxf(s, fabsf(d[c]));
    }
#pragma unroll
    for (int m = 1; m < NP; ++m) s += fabsf(d2f_trunc(own[m]));
    const float inv = 1.0f / (s + 1e-14f);
#pragma unroll
    for (int c = 0; c < NB; ++c) put(k++, d[c] * inv);
#pragma unroll
    for (int m = 1; m < NP; ++m) put(k++, d2f_trunc(own[m]) * inv);
    // then one neighbour's higher modes at a time (few registers live)
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double nb[NP];
      load_var<DIM, NP>(U, ctot, cr[c + 1], v, nb);
#pragma unroll
      for (int m = 1; m < NP; ++m) put(k++, d2f_trunc(nb[m]) * inv);
    }
  }
}

// cell of thread (lane, warp) in a tile: 2D rows of 32, 1D runs of 256
template <int DIM>
__device__ __forceinline__ void tile_cell(const Tile& t, int& ix, int& iy) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (DIM == 2) { ix = t.x0 + lane; iy = t.y0 + w; }
  else { ix = t.x0 + (int)threadIdx.x; iy = 0; }
}

// ----------------------------------------------------------------------------- features
template <int DIM, int PDE, int N>
__global__ void __launch_bounds__(256) k_features(const double* __restrict__ U, const Inst* __restrict__ insts,
                                                  const Tile* __restrict__ tiles, long long ctot, int bc, double c0,
                                                  float* __restrict__ X) {
  using D = FeatDims<DIM, PDE, N>;
  const Tile t = tiles[blockIdx.x];
  const Inst I = insts[t.inst];
  int ix, iy;
  tile_cell<DIM>(t, ix, iy);
  if (ix >= I.nx || iy >= I.ny) return;
  const long long g = I.off + (long long)iy * I.nx + ix;
  float* row = X + g * D::F;
  cell_features<DIM, PDE, N>(U, ctot, I, ix, iy, bc, c0, [&](int k, float v) { row[k] = v; });
}

// ----------------------------------------------------------------------------- inference
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3, unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const unsigned*>(p); }

// The 32-32-1 network on the 32 cells of a warp.  Xs: this warp's [32][FP] BF16 features
// with row stride FP + kPadX (reused for the hidden layer); returns the logit of the lane's cell.
__device__ __forceinline__ float warp_mlp(__nv_bfloat16* Xs, int FP, const MlpInfer& W) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int LX = FP + kPadX;
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0.f;
  __syncwarp();
  for (int k0 = 0; k0 < FP; k0 += 16) {
    unsigned a[2][4], b[4][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const __nv_bfloat16* r0 = Xs + (mt * 16 + g) * LX + k0 + 2 * t;
      const __nv_bfloat16* r1 = r0 + 8 * LX;
      a[mt][0] = ld_pair(r0);
      a[mt][1] = ld_pair(r1);
      a[mt][2] = ld_pair(r0 + 8);
      a[mt][3] = ld_pair(r1 + 8);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const __nv_bfloat16* wr = static_cast<const __nv_bfloat16*>(W.W1) + (nt * 8 + g) * FP + k0 + 2 * t;
      b[nt][0] = __ldg(reinterpret_cast<const unsigned*>(wr));
      b[nt][1] = __ldg(reinterpret_cast<const unsigned*>(wr + 8));
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
  }
  __syncwarp();
  // hidden layer 1: bias + ReLU, back to shared memory as BF16 [32][32]
  __nv_bfloat16* Hs = Xs;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + 2 * t;
      const float bb0 = __ldg(W.b1 + col), bb1 = __ldg(W.b1 + col + 1);
      Hs[(mt * 16 + g) * kLdH + col] = __float2bfloat16_rn(fmaxf(acc[mt][nt][0] + bb0, 0.f));
      Hs[(mt * 16 + g) * kLdH + col + 1] = __float2bfloat16_rn(fmaxf(acc[mt][nt][1] + bb1, 0.f));
      Hs[(mt * 16 + g + 8) * kLdH + col] = __float2bfloat16_rn(fmaxf(acc[mt][nt][2] + bb0, 0.f));
      Hs[(mt * 16 + g + 8) * kLdH + col + 1] = __float2bfloat16_rn(fmaxf(acc[mt][nt][3] + bb1, 0.f));
      acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
    }
  __syncwarp();
#pragma unroll
  for (int k0 = 0; k0 < kHid; k0 += 16) {
    unsigned a[2][4], b[4][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const __nv_bfloat16* r0 = Hs + (mt * 16 + g) * kLdH + k0 + 2 * t;
      const __nv_bfloat16* r1 = r0 + 8 * kLdH;
      a[mt][0] = ld_pair(r0);
      a[mt][1] = ld_pair(r1);
      a[mt][2] = ld_pair(r0 + 8);
      a[mt][3] = ld_pair(r1 + 8);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const __nv_bfloat16* wr = static_cast<const __nv_bfloat16*>(W.W2) + (nt * 8 + g) * kHid + k0 + 2 * t;
      b[nt][0] = __ldg(reinterpret_cast<const unsigned*>(wr));
      b[nt][1] = __ldg(reinterpret_cast<const unsigned*>(wr + 8));
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
  }
  // output layer: z = w3 . relu(acc + b2) + b3, reduced over the 4 lanes of a row group
  float z[2][2];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    float lo = 0.f, hi = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + 2 * t;
      const float bb0 = __ldg(W.b2 + col), bb1 = __ldg(W.b2 + col + 1);
      const float w0 = __ldg(W.w3 + col), w1 = __ldg(W.w3 + col + 1);
      lo += fmaxf(acc[mt][nt][0] + bb0, 0.f) * w0 + fmaxf(acc[mt][nt][1] + bb1, 0.f) * w1;
      hi += fmaxf(acc[mt][nt][2] + bb0, 0.f) * w0 + fmaxf(acc[mt][nt][3] + bb1, 0.f) * w1;
    }
    lo += __shfl_xor_sync(0xffffffffu, lo, 1);
    lo += __shfl_xor_sync(0xffffffffu, lo, 2);
    hi += __shfl_xor_sync(0xffffffffu, hi, 1);
    hi += __shfl_xor_sync(0xffffffffu, hi, 2);
    z[mt][0] = lo;
    z[mt][1] = hi;
  }
  // the logit of cell c sits in lane 4 * (c % 8) of row group: c = mt*16 + g (+8)
  float* zs = reinterpret_cast<float*>(Xs);
  __syncwarp();
  if (t == 0) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      zs[mt * 16 + g] = z[mt][0];
      zs[mt * 16 + g + 8] = z[mt][1];
    }
  }
  __syncwarp();
  const float r = zs[lane] + __ldg(W.b3);
  __syncwarp();
  return r;
}

// Flagging pass with the learned indicator: features -> BF16 shared memory -> tensor-core
// MLP -> logit > tau -> ballot/scan compaction (same list as the TVB pass).  Tiles that
// belong to no instance needing work (skip != null and skip[inst] == 0) flag nothing.
template <int DIM, int PDE, int N>
__global__ void __launch_bounds__(256)
    k_flag_mlp(const double* __restrict__ U, const Inst* __restrict__ insts, const Tile* __restrict__ tiles,
               long long ctot, int bc, double c0, MlpInfer W, unsigned char* __restrict__ flags, Counters* cnt,
               int* __restrict__ list_cell, int* __restrict__ list_inst, float* __restrict__ logits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int FP = W.FP;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(smem_raw) + w * 32 * (FP + kPadX);
  const Tile t = tiles[blockIdx.x];
  const Inst I = insts[t.inst];
  int ix, iy;
  tile_cell<DIM>(t, ix, iy);
  const bool active = ix < I.nx && iy < I.ny;
  __nv_bfloat16* row = Xs + lane * (FP + kPadX);
  using D = FeatDims<DIM, PDE, N>;
  if (active) {
    cell_features<DIM, PDE, N>(U, ctot, I, ix, iy, bc, c0, [&](int k, float v) { row[k] = __float2bfloat16_rn(v); });
  } else {
    for (int k = 0; k < D::F; ++k) row[k] = __float2bfloat16_rn(0.f);
  }
  for (int k = D::F; k < FP; ++k) row[k] = __float2bfloat16_rn(0.f);
  const float z = warp_mlp(Xs, FP, W);
  int fl = 0;
  long long g = 0;
  if (active) {
    g = I.off + (long long)iy * I.nx + ix;
    fl = z > W.tau ? 1 : 0;
    flags[g] = (unsigned char)fl;
    if (logits) logits[g] = z;
  }
  block_compact(fl, 0, g, t.inst, cnt, list_cell, list_inst);
}


// ----------------------------------------------------------------------------- learned filter
// The learned indicator keeps a TVB-flagged cell only when the network's logit exceeds
// tau: every warp takes 32 consecutive entries of the TVB list (A), computes their
// features, runs the network on the tensor cores and appends the kept cells to list B
// (warp ballot + one atomic per warp).  flags[] receives the final decision in bit 0 and
// keeps the TVB pass's near-threshold bit 1.  Three blocks per SM (80 registers): the kernel is
// latency-bound (gathered loads, shared memory), so more resident warps hide more of it.
template <int DIM, int PDE, int N>
__global__ void __launch_bounds__(256, 3)
    k_mlp_filter(const double* __restrict__ U, const Inst* __restrict__ insts, long long ctot, int bc, double c0,
                 MlpInfer W, const int* __restrict__ la_cell, const int* __restrict__ la_inst,
                 const Counters* __restrict__ cnt_a, unsigned char* __restrict__ flags, Counters* cnt_b,
                 int* __restrict__ lb_cell, int* __restrict__ lb_inst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using D = FeatDims<DIM, PDE, N>;
  const int FP = W.FP;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(smem_raw) + w * 32 * (FP + kPadX);
  __nv_bfloat16* row = Xs + lane * (FP + kPadX);
  const unsigned int n = cnt_a->n_flag;
  const unsigned int warps_total = gridDim.x * (blockDim.x >> 5);
  for (unsigned int base = (blockIdx.x * (blockDim.x >> 5) + w) * 32u; base < n; base += warps_total * 32u) {
    const unsigned int i = base + lane;
    const bool active = i < n;
    long long g = 0;
    int ii = 0;
    if (active) {
      g = la_cell[i];
      ii = la_inst[i];
      const Inst I = insts[ii];
      const int loc = (int)(g - I.off);
      cell_features<DIM, PDE, N>(U, ctot, I, loc % I.nx, loc / I.nx, bc, c0,
                                 [&](int k, float v) { row[k] = __float2bfloat16_rn(v); });
    } else {
      for (int k = 0; k < D::F; ++k) row[k] = __float2bfloat16_rn(0.f);
    }
    for (int k = D::F; k < FP; ++k) row[k] = __float2bfloat16_rn(0.f);
    const float z = warp_mlp(Xs, FP, W);
    const bool keep = active && z > W.tau;
    if (active) flags[g] = (unsigned char)((flags[g] & 2) | (keep ? 1 : 0));
    const unsigned int bal = __ballot_sync(0xffffffffu, keep);
    unsigned int pos0 = 0;
    if (lane == 0 && bal) pos0 = atomicAdd(&cnt_b->n_flag, (unsigned)__popc(bal));
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    if (keep) {
      const unsigned int p = pos0 + __popc(bal & ((1u << lane) - 1u));
      lb_cell[p] = (int)g;
      lb_inst[p] = ii;
    }
  }
}

// Positivity screen (Euler): density and pressure at the (N+1)-point Gauss points of the
// cell and of its faces, evaluated in FP32 from the modes; a point fails when rho <= 0,
// p <= 1e-6 |E| (a margin that covers the FP32 rounding of E - |m|^2 / (2 rho)) or a value
// is not finite.
struct PosTab {
  float P[4][4];  // psi_n(x_q), q < N+1
  float P1[4];    // psi_n(1)
  float gm1;
};

// True when the cell's density or pressure fails the screen at one of its points.
template <int DIM, int N>
__device__ __forceinline__ bool screen_fails(const double* __restrict__ U, long long ctot, long long g,
                                             const PosTab& tb) {
  constexpr int V = DIM == 1 ? 3 : 4, NP = np_of(DIM, N), Q = N + 1;
  float u[V][NP];
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int m = 0; m < NP; ++m) u[v][m] = d2f_trunc(__ldg(U + (long long)(v * NP + m) * ctot + g));
  bool bad = false;
  auto check = [&](const float* q) {
    const float rho = q[0], E = q[V - 1];
    float k = q[1] * q[1];
    if (DIM == 2) k += q[2] * q[2];
    const float p = tb.gm1 * (E - 0.5f * k / rho);
    if (!(rho > 0.f) || !(p > 1e-6f * fabsf(E)) || !isfinite(p)) bad = true;
  };
  if constexpr (DIM == 1) {
#pragma unroll
    for (int q = 0; q < Q + 2; ++q) {
      float val[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const float b = q < Q ? tb.P[q][m] : ((q == Q || !(m & 1)) ? tb.P1[m] : -tb.P1[m]);
          s = fmaf(u[v][m], b, s);
        }
        val[v] = s;
      }
      check(val);
    }
  } else {
    // points: Q x Q volume points, then (r = +-1, s_q) and (r_q, s = +-1)
#pragma unroll
    for (int q = 0; q < Q * Q + 4 * Q; ++q) {
      float val[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const int a = mode_a(m), b = mode_b(m);
          float fa, fb;
          if (q < Q * Q) { fa = tb.P[q % Q][a]; fb = tb.P[q / Q][b]; }
          else {
            const int f = (q - Q * Q) / Q, j = (q - Q * Q) % Q;
            const bool minus = (f & 1) != 0;  // faces: +1 then -1
            if (f < 2) { fa = ((a & 1) && minus) ? -tb.P1[a] : tb.P1[a]; fb = tb.P[j][b]; }
            else { fa = tb.P[j][a]; fb = ((b & 1) && minus) ? -tb.P1[b] : tb.P1[b]; }
          }
          s = fmaf(u[v][m], fa * fb, s);
        }
        val[v] = s;
      }
      check(val);
    }
  }
  return bad;
}

// Screens every cell of the mesh and marks the instances of failing ones in fail[].
template <int DIM, int N>
__global__ void __launch_bounds__(128) k_positivity_all(const double* __restrict__ U, long long ctot, long long ncell,
                                                        const int* __restrict__ cell_inst, PosTab tb,
                                                        unsigned int* __restrict__ fail) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ncell; g += (long long)gridDim.x * blockDim.x)
    if (screen_fails<DIM, N>(U, ctot, g, tb)) atomicOr(fail + cell_inst[g], 1u);
}

// Positivity screen of the cells the learned indicator skipped: every cell of list A (the
// TVB list) with bit 0 of flags[g] clear whose unlimited state fails the screen marks its
// instance in fail[].
template <int DIM, int N>
__global__ void __launch_bounds__(128) k_positivity_skipped(const double* __restrict__ U, long long ctot,
                                                            const int* __restrict__ la_cell,
                                                            const int* __restrict__ la_inst,
                                                            const Counters* __restrict__ cnt_a,
                                                            const unsigned char* __restrict__ flags, PosTab tb,
                                                            unsigned int* __restrict__ fail) {
  const unsigned int n = cnt_a->n_flag;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long g = la_cell[i];
    if (!(flags[g] & 1) && screen_fails<DIM, N>(U, ctot, g, tb)) atomicOr(fail + la_inst[i], 1u);
  }
}

// Writes the limited modes 1..NP-1 of the listed cells whose instance is not marked in skip[].
template <int V, int NP>
__global__ void k_scatter_unless(double* __restrict__ Ust, long long ctot, const double* __restrict__ lim,
                                 long long cap, const int* __restrict__ list_cell, const int* __restrict__ list_inst,
                                 const Counters* __restrict__ cnt, const unsigned int* __restrict__ skip) {
  const unsigned int n = cnt->n_flag;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (skip[list_inst[i]]) continue;
    const long long g = list_cell[i];
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int m = 1; m < NP; ++m) Ust[(long long)(v * NP + m) * ctot + g] = lim[(long long)(v * NP + m) * cap + i];
  }
}

// List C = the entries of list A that belong to marked instances.
__global__ void k_filter_inst(const int* __restrict__ la_cell, const int* __restrict__ la_inst,
                              const Counters* __restrict__ cnt_a, const unsigned int* __restrict__ mark, Counters* cnt_c,
                              int* __restrict__ lc_cell, int* __restrict__ lc_inst) {
  const unsigned int n = cnt_a->n_flag;
  const int lane = threadIdx.x & 31;
  const unsigned int stride = gridDim.x * blockDim.x;
  for (unsigned int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
    const unsigned int i = base + lane;
    const bool keep = i < n && mark[la_inst[i]];
    const unsigned int bal = __ballot_sync(0xffffffffu, keep);
    unsigned int pos0 = 0;
    if (lane == 0 && bal) pos0 = atomicAdd(&cnt_c->n_flag, (unsigned)__popc(bal));
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    if (keep) {
      const unsigned int p = pos0 + __popc(bal & ((1u << lane) - 1u));
      lc_cell[p] = la_cell[i];
      lc_inst[p] = la_inst[i];
    }
  }
}

// Adds the failing instances to the running count and, with `final_`, to the failures.
__global__ void k_count_fail(const unsigned int* __restrict__ fail, int n_inst, unsigned long long* total) {
  int c = 0;
  for (int i = threadIdx.x; i < n_inst; i += blockDim.x) c += fail[i] != 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(total, (unsigned long long)c);
}

// ----------------------------------------------------------------------------- harvest label
// change[g] = max over v and n >= 1 of |limited - unlimited U_{n,v}| / s_v for a listed
// (TVB-flagged) cell: how much the limiter changes the cell relative to its local scale.
template <int DIM, int PDE, int N>
__global__ void k_label(const double* __restrict__ U, const Inst* __restrict__ insts, long long ctot, int bc, double c0,
                        const int* __restrict__ list_cell, const int* __restrict__ list_inst,
                        const Counters* __restrict__ cnt, const double* __restrict__ lim, long long cap,
                        float* __restrict__ change) {
  using D = FeatDims<DIM, PDE, N>;
  constexpr int V = D::V, NP = D::NP, NB = D::NB;
  const unsigned int n = cnt->n_flag;
  for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long g = list_cell[i];
    const Inst I = insts[list_inst[i]];
    const int loc = (int)(g - I.off), ix = loc % I.nx, iy = loc / I.nx;
    double own[V][NP];
    load_modes<DIM, V, NP>(U, ctot, I, ix, iy, bc, own);
    const int dx[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
    double mx[V];
#pragma unroll
    for (int v = 0; v < V; ++v) mx[v] = 0.0;
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      double nb[V][NP];
      load_modes<DIM, V, NP>(U, ctot, I, ix + dx[c], iy + dy[c], bc, nb);
#pragma unroll
      for (int v = 0; v < V; ++v) mx[v] = fmax(mx[v], fabs(nb[v][0] * c0 - own[v][0] * c0));
    }
    double r = 0.0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      double s = mx[v];
#pragma unroll
      for (int m = 1; m < NP; ++m) s += fabs(own[v][m]);
      s += 1e-14;
      double dmax = 0.0;
#pragma unroll
      for (int m = 1; m < NP; ++m) dmax = fmax(dmax, fabs(lim[(long long)(v * NP + m) * cap + i] - own[v][m]));
      r = fmax(r, dmax / s);
    }
    change[g] = (float)r;
  }
}

// ----------------------------------------------------------------------------- training
// Per sample: forward pass, loss, and the backpropagated deltas of both hidden layers.
// Weights in shared memory (FP32): W1 [32][F], b1, W2 [32][32], b2, w3, b3.
__global__ void k_mlp_fb(const float* __restrict__ X, const unsigned char* __restrict__ y, long long B, int F,
                         const float* __restrict__ params, float pw, float* __restrict__ h1s, float* __restrict__ d1s,
                         float* __restrict__ h2s, float* __restrict__ d2s, float* __restrict__ dzs,
                         float* __restrict__ loss_acc) {
  extern __shared__ float sp[];
  const int P = kHid * F + kHid + kHid * kHid + kHid + kHid + 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) sp[i] = params[i];
  __syncthreads();
  const float* W1 = sp;
  const float* b1 = W1 + kHid * F;
  const float* W2 = b1 + kHid;
  const float* b2 = W2 + kHid * kHid;
  const float* w3 = b2 + kHid;
  const float b3 = w3[kHid];
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float lossv = 0.f;
  if (b < B) {
    float a1[kHid];
#pragma unroll
    for (int o = 0; o < kHid; ++o) a1[o] = b1[o];
    const float* x = X + b * F;
    for (int i = 0; i < F; ++i) {
      const float xi = __ldg(x + i);
#pragma unroll
      for (int o = 0; o < kHid; ++o) a1[o] = fmaf(W1[o * F + i], xi, a1[o]);
    }
    float a2[kHid];
#pragma unroll
    for (int o = 0; o < kHid; ++o) a2[o] = b2[o];
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
      const float hi = fmaxf(a1[i], 0.f);
#pragma unroll
      for (int o = 0; o < kHid; ++o) a2[o] = fmaf(W2[o * kHid + i], hi, a2[o]);
    }
    float z = b3;
#pragma unroll
    for (int i = 0; i < kHid; ++i) z = fmaf(w3[i], fmaxf(a2[i], 0.f), z);
    const float yy = y[b] ? 1.f : 0.f;
    // log(1 + e^z) and log(1 + e^-z), computed without overflow
    const float spz = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
    const float spn = spz - z;
    lossv = pw * yy * spn + (1.f - yy) * spz;
    const float sig = 1.f / (1.f + expf(-z));
    const float dz = (pw * yy * (sig - 1.f) + (1.f - yy) * sig) / (float)B;
    dzs[b] = dz;
    float d2[kHid];
#pragma unroll
    for (int o = 0; o < kHid; ++o) {
      d2[o] = a2[o] > 0.f ? dz * w3[o] : 0.f;
      h2s[b * kHid + o] = fmaxf(a2[o], 0.f);
      d2s[b * kHid + o] = d2[o];
      h1s[b * kHid + o] = fmaxf(a1[o], 0.f);
    }
#pragma unroll
    for (int i = 0; i < kHid; ++i) {
      float s = 0.f;
#pragma unroll
      for (int o = 0; o < kHid; ++o) s = fmaf(W2[o * kHid + i], d2[o], s);
      d1s[b * kHid + i] = a1[i] > 0.f ? s : 0.f;
    }
  }
  // loss: warp sum then one atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lossv += __shfl_xor_sync(0xffffffffu, lossv, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss_acc, lossv / (float)B);
}

// FP32 forward pass only (validation and threshold calibration).
__global__ void k_mlp_forward(const float* __restrict__ X, long long B, int F, const float* __restrict__ params,
                              float* __restrict__ z_out) {
  extern __shared__ float sp[];
  const int P = kHid * F + kHid + kHid * kHid + kHid + kHid + 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) sp[i] = params[i];
  __syncthreads();
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* W1 = sp;
  const float* b1 = W1 + kHid * F;
  const float* W2 = b1 + kHid;
  const float* b2 = W2 + kHid * kHid;
  const float* w3 = b2 + kHid;
  float a1[kHid];
#pragma unroll
  for (int o = 0; o < kHid; ++o) a1[o] = b1[o];
  for (int i = 0; i < F; ++i) {
    const float xi = __ldg(X + b * F + i);
#pragma unroll
    for (int o = 0; o < kHid; ++o) a1[o] = fmaf(W1[o * F + i], xi, a1[o]);
  }
  float z = w3[kHid];
#pragma unroll
  for (int o = 0; o < kHid; ++o) {
    float a2 = b2[o];
#pragma unroll
    for (int i = 0; i < kHid; ++i) a2 = fmaf(W2[o * kHid + i], fmaxf(a1[i], 0.f), a2);
    z = fmaf(w3[o], fmaxf(a2, 0.f), z);
  }
  z_out[b] = z;
}

// Weight gradients over a chunk of samples: part[chunk][p] = sum_b delta[b][o] * input[b][i]
// over the chunk's samples; k_mlp_wsum adds the chunks in a fixed order, so that training is
// reproducible bit for bit.
constexpr int kChunk = 64;
__global__ void k_mlp_wgrad(const float* __restrict__ X, long long B, int F, const float* __restrict__ h1s,
                            const float* __restrict__ d1s, const float* __restrict__ h2s, const float* __restrict__ d2s,
                            const float* __restrict__ dzs, float* __restrict__ part) {
  const long long b0 = (long long)blockIdx.x * kChunk;
  const int nb = (int)min((long long)kChunk, B - b0);
  const int P = kHid * F + kHid + kHid * kHid + kHid + kHid + 1;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    float s = 0.f;
    if (p < kHid * F) {  // W1[o][i]
      const int o = p / F, i = p % F;
      for (int j = 0; j < nb; ++j) s = fmaf(d1s[(b0 + j) * kHid + o], X[(b0 + j) * F + i], s);
    } else if (p < kHid * F + kHid) {  // b1
      const int o = p - kHid * F;
      for (int j = 0; j < nb; ++j) s += d1s[(b0 + j) * kHid + o];
    } else if (p < kHid * F + kHid + kHid * kHid) {  // W2[o][i]
      const int q = p - kHid * F - kHid, o = q / kHid, i = q % kHid;
      for (int j = 0; j < nb; ++j) s = fmaf(d2s[(b0 + j) * kHid + o], h1s[(b0 + j) * kHid + i], s);
    } else if (p < kHid * F + 2 * kHid + kHid * kHid) {  // b2
      const int o = p - kHid * F - kHid - kHid * kHid;
      for (int j = 0; j < nb; ++j) s += d2s[(b0 + j) * kHid + o];
    } else if (p < P - 1) {  // w3
      const int i = p - kHid * F - 2 * kHid - kHid * kHid;
      for (int j = 0; j < nb; ++j) s = fmaf(dzs[b0 + j], h2s[(b0 + j) * kHid + i], s);
    } else {  // b3
      for (int j = 0; j < nb; ++j) s += dzs[b0 + j];
    }
    part[(long long)blockIdx.x * P + p] = s;
  }
}

__global__ void k_mlp_wsum(const float* __restrict__ part, int nchunks, int P, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float s = 0.f;
  for (int c = 0; c < nchunks; ++c) s += part[(long long)c * P + p];
  grad[p] = s;
}

// Adam with bias correction on the FP32 master parameters; refreshes the inference copy
// (BF16 W1 padded to FP columns, BF16 W2, FP32 biases and output layer).
__global__ void k_mlp_adam(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m1,
                           float* __restrict__ m2, int P, float lr, float beta1, float beta2, float eps, float c1,
                           float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float gv = grad[p];
  const float a = beta1 * m1[p] + (1.f - beta1) * gv;
  const float v = beta2 * m2[p] + (1.f - beta2) * gv * gv;
  m1[p] = a;
  m2[p] = v;
  params[p] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

__global__ void k_mlp_export(const float* __restrict__ params, int F, int FP, __nv_bfloat16* __restrict__ W1b,
                             float* __restrict__ b1, __nv_bfloat16* __restrict__ W2b, float* __restrict__ b2,
                             float* __restrict__ w3, float* __restrict__ b3) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kHid * FP) {
    const int o = p / FP, i = p % FP;
    W1b[p] = __float2bfloat16_rn(i < F ? params[o * F + i] : 0.f);
  }
  const float* q = params + kHid * F;
  if (p < kHid) {
    b1[p] = q[p];
    b2[p] = q[kHid + kHid * kHid + p];
    w3[p] = q[2 * kHid + kHid * kHid + p];
  }
  if (p < kHid * kHid) W2b[p] = __float2bfloat16_rn(q[kHid + p]);
  if (p == 0) b3[0] = q[3 * kHid + kHid * kHid];
}

// ----------------------------------------------------------------------------- dispatch
#define DG_DISPATCH_ALL(DIM, PDE, N, CALL)                                                  \
  do {                                                                                      \
    if ((DIM) == 1) {                                                                       \
      if ((PDE) == 0 && (N) == 1) { constexpr int D_ = 1, P_ = 0, N_ = 1; CALL; }           \
      else if ((PDE) == 0 && (N) == 2) { constexpr int D_ = 1, P_ = 0, N_ = 2; CALL; }      \
      else if ((PDE) == 0 && (N) == 3) { constexpr int D_ = 1, P_ = 0, N_ = 3; CALL; }      \
      else if ((PDE) == 1 && (N) == 1) { constexpr int D_ = 1, P_ = 1, N_ = 1; CALL; }      \
      else if ((PDE) == 1 && (N) == 2) { constexpr int D_ = 1, P_ = 1, N_ = 2; CALL; }      \
      else { constexpr int D_ = 1, P_ = 1, N_ = 3; CALL; }                                  \
    } else {                                                                                \
      if ((PDE) == 0 && (N) == 1) { constexpr int D_ = 2, P_ = 0, N_ = 1; CALL; }           \
      else if ((PDE) == 0 && (N) == 2) { constexpr int D_ = 2, P_ = 0, N_ = 2; CALL; }      \
      else if ((PDE) == 0 && (N) == 3) { constexpr int D_ = 2, P_ = 0, N_ = 3; CALL; }      \
      else if ((PDE) == 1 && (N) == 1) { constexpr int D_ = 2, P_ = 1, N_ = 1; CALL; }      \
      else if ((PDE) == 1 && (N) == 2) { constexpr int D_ = 2, P_ = 1, N_ = 2; CALL; }      \
      else { constexpr int D_ = 2, P_ = 1, N_ = 3; CALL; }                                  \
    }                                                                                       \
  } while (0)

void launch_features(int dim, int pde, int N, const LaunchArgs& a, double c0, float* X) {
  DG_DISPATCH_ALL(dim, pde, N, (k_features<D_, P_, N_><<<a.ntiles, 256, 0, a.st>>>(a.us, a.inst, a.tiles, a.ctot, a.bc,
                                                                                    c0, X)));
}

size_t flag_mlp_smem(int FP) { return sizeof(__nv_bfloat16) * 256 * (size_t)(FP + kPadX); }

cudaError_t prepare_mlp(int dim, int pde, int N, int FP) {
  cudaError_t e = cudaSuccess;
  DG_DISPATCH_ALL(dim, pde, N, (e = cudaFuncSetAttribute(k_flag_mlp<D_, P_, N_>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)flag_mlp_smem(FP))));
  return e;
}

void launch_flag_mlp(int dim, int pde, int N, const LaunchArgs& a, double c0, const MlpInfer& W, unsigned char* flags,
                     Counters* cnt, int* lc, int* li, float* logits) {
  DG_DISPATCH_ALL(dim, pde, N, (k_flag_mlp<D_, P_, N_><<<a.ntiles, 256, flag_mlp_smem(W.FP), a.st>>>(
                                   a.us, a.inst, a.tiles, a.ctot, a.bc, c0, W, flags, cnt, lc, li, logits)));
}


cudaError_t prepare_filter(int dim, int pde, int N, int FP) {
  cudaError_t e = cudaSuccess;
  DG_DISPATCH_ALL(dim, pde, N, (e = cudaFuncSetAttribute(k_mlp_filter<D_, P_, N_>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          (int)flag_mlp_smem(FP))));
  return e;
}

void launch_mlp_filter(int dim, int pde, int N, const LaunchArgs& a, double c0, const MlpInfer& W, const int* la_c,
                       const int* la_i, const Counters* cnt_a, unsigned char* flags, Counters* cnt_b, int* lb_c,
                       int* lb_i, int nblocks) {
  DG_DISPATCH_ALL(dim, pde, N, (k_mlp_filter<D_, P_, N_><<<nblocks, 256, flag_mlp_smem(W.FP), a.st>>>(
                                   a.us, a.inst, a.ctot, a.bc, c0, W, la_c, la_i, cnt_a, flags, cnt_b, lb_c, lb_i)));
}

static PosTab pos_tab(int N, const double* psi_q /* [N+1][N+1] */, const double* psi_p1, double gam) {
  PosTab tb{};
  for (int q = 0; q <= N; ++q)
    for (int m = 0; m <= N; ++m) tb.P[q][m] = (float)psi_q[q * (N + 1) + m];
  for (int m = 0; m <= N; ++m) tb.P1[m] = (float)psi_p1[m];
  tb.gm1 = (float)(gam - 1.0);
  return tb;
}

#define DG_POS_DISPATCH(dim, N, CALL)     \
  do {                                    \
    if ((dim) == 1) {                     \
      if ((N) == 1) { constexpr int D_ = 1, N_ = 1; CALL; }      \
      else if ((N) == 2) { constexpr int D_ = 1, N_ = 2; CALL; } \
      else { constexpr int D_ = 1, N_ = 3; CALL; }               \
    } else {                              \
      if ((N) == 1) { constexpr int D_ = 2, N_ = 1; CALL; }      \
      else if ((N) == 2) { constexpr int D_ = 2, N_ = 2; CALL; } \
      else { constexpr int D_ = 2, N_ = 3; CALL; }               \
    }                                     \
  } while (0)

void launch_positivity_all(int dim, int N, const LaunchArgs& a, const double* psi_q, const double* psi_p1, double gam,
                           const int* cell_inst, unsigned int* fail, int nblocks) {
  const PosTab tb = pos_tab(N, psi_q, psi_p1, gam);
  DG_POS_DISPATCH(dim, N, (k_positivity_all<D_, N_><<<nblocks, 128, 0, a.st>>>(a.us, a.ctot, a.ncell, cell_inst, tb,
                                                                                  fail)));
}

void launch_positivity_skipped(int dim, int N, const LaunchArgs& a, const double* psi_q, const double* psi_p1,
                               double gam, const int* la_c, const int* la_i, const Counters* cnt_a,
                               const unsigned char* flags, unsigned int* fail, int nblocks) {
  const PosTab tb = pos_tab(N, psi_q, psi_p1, gam);
  DG_POS_DISPATCH(dim, N, (k_positivity_skipped<D_, N_><<<nblocks, 128, 0, a.st>>>(a.us, a.ctot, la_c, la_i, cnt_a,
                                                                                      flags, tb, fail)));
}

void launch_scatter_unless(int dim, int pde, int N, const LaunchArgs& a, const double* lim, const int* lc,
                           const int* li, const Counters* cnt, const unsigned int* skip, int nblocks) {
  DG_DISPATCH_ALL(dim, pde, N, (k_scatter_unless<nv_of(D_, P_), np_of(D_, N_)><<<nblocks, 256, 0, a.st>>>(
                                   a.out, a.ctot, lim, a.cap, lc, li, cnt, skip)));
}

void launch_filter_inst(cudaStream_t st, const int* la_c, const int* la_i, const Counters* cnt_a,
                        const unsigned int* mark, Counters* cnt_c, int* lc_c, int* lc_i, int nblocks) {
  k_filter_inst<<<nblocks, 256, 0, st>>>(la_c, la_i, cnt_a, mark, cnt_c, lc_c, lc_i);
}

void launch_count_fail(cudaStream_t st, const unsigned int* fail, int n_inst, unsigned long long* total) {
  k_count_fail<<<1, 256, 0, st>>>(fail, n_inst, total);
}

void launch_label(int dim, int pde, int N, const LaunchArgs& a, double c0, const int* lc, const int* li,
                  const Counters* cnt, const double* lim, float* label, int nblocks) {
  DG_DISPATCH_ALL(dim, pde, N, (k_label<D_, P_, N_><<<nblocks, 128, 0, a.st>>>(a.us, a.inst, a.ctot, a.bc, c0, lc, li,
                                                                               cnt, lim, a.cap, label)));
}

void launch_mlp_fb(cudaStream_t st, const float* X, const unsigned char* y, long long B, int F, const float* params,
                   float pw, float* h1, float* d1, float* h2, float* d2, float* dz, float* loss) {
  const int P = kHid * F + kHid + kHid * kHid + kHid + kHid + 1;
  const size_t smem = sizeof(float) * (size_t)P;
  static int attr_for = -1;
  if (attr_for != F) {
    cudaFuncSetAttribute(k_mlp_fb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_for = F;
  }
  k_mlp_fb<<<(unsigned)((B + 127) / 128), 128, smem, st>>>(X, y, B, F, params, pw, h1, d1, h2, d2, dz, loss);
}

void launch_mlp_forward(cudaStream_t st, const float* X, long long B, int F, const float* params, float* z) {
  const int P = kHid * F + kHid + kHid * kHid + kHid + kHid + 1;
  const size_t smem = sizeof(float) * (size_t)P;
  static int attr_for = -1;
  if (attr_for != F) {
    cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr_for = F;
  }
  k_mlp_forward<<<(unsigned)((B + 127) / 128), 128, smem, st>>>(X, B, F, params, z);
}

long long mlp_wgrad_chunks(long long B) { return (B + kChunk - 1) / kChunk; }

void launch_mlp_wgrad(cudaStream_t st, const float* X, long long B, int F, const float* h1, const float* d1,
                      const float* h2, const float* d2, const float* dz, float* part, float* grad) {
  const long long nc = mlp_wgrad_chunks(B);
  const int P = kHid * F + kHid + kHid * kHid + kHid + kHid + 1;
  k_mlp_wgrad<<<(unsigned)nc, 256, 0, st>>>(X, B, F, h1, d1, h2, d2, dz, part);
  k_mlp_wsum<<<(P + 255) / 256, 256, 0, st>>>(part, (int)nc, P, grad);
}

void launch_mlp_adam(cudaStream_t st, float* params, const float* grad, float* m1, float* m2, int P, float lr,
                     int t) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_mlp_adam<<<(P + 255) / 256, 256, 0, st>>>(params, grad, m1, m2, P, lr, b1, b2, 1e-8f, c1, c2);
}

void launch_mlp_export(cudaStream_t st, const float* params, int F, int FP, void* W1b, float* b1, void* W2b, float* b2,
                       float* w3, float* b3) {
  const int n = kHid * FP > kHid * kHid ? kHid * FP : kHid * kHid;
  k_mlp_export<<<(n + 255) / 256, 256, 0, st>>>(params, F, FP, (__nv_bfloat16*)W1b, b1, (__nv_bfloat16*)W2b, b2, w3,
                                               b3);
}

}  // namespace dg
