// Agent sweep kernels: one explicit Euler step of the alignment dynamics (Eq. MAsystem,
// Eq. ellipsoid, Eq. kernel) and one step of its exact discrete adjoint with the
// control-derivative partials D^n (Section 3.1, Algorithm 1).
//
// Both steps are FP32-ALU bound: every pixel visits its (2R+1)^2 window.  Design:
//  * a CTA owns a TH x TW tile of output pixels; it stages the tile plus an R-pixel halo
//    of the input field(s) in shared memory, de-interleaved into one plane per channel
//    (NHWC in HBM -> planar in SMEM), with out-of-image cells zero-filled;
//  * each thread owns PXH pixel pairs (one pixel in each half of the tile, same offsets)
//    and walks the window row by row: it loads that window row's entries once into
//    registers (16-byte reads) and reuses them for all its pairs (register blocking);
//  * the arithmetic of a pair runs in packed float2 instructions (sm_100+ FFMA2/FADD2/
//    FMUL2), halving issued instructions; per lane the operations are the scalar ones;
//  * the spatial part of r_ij is uniform over pixels, so it is a per-offset constant; the
//    forward step stages the colours scaled by sqrt(eps_c / 2), so that r - 1 is the
//    colour distance's FMA chain started from that constant, and the adjoint forms 1 - r
//    with one FMA; phi is branch-free (t = max(1 - r, 0));
//  * interior tiles skip all bounds handling; tiles whose halo leaves the image multiply
//    each interaction weight by a 0/1 validity plane (exact: out-of-image cells hold 0,
//    so the weight times a finite difference is exactly 0);
//  * the pixel's own cell (dy = dx = 0) is not skipped: its difference is exactly 0, so
//    it adds exactly 0 to every sum, and keeping it keeps the inner loop branch-free.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace agents {

// Tile geometry.  A CTA owns TH x TW output pixels, TW = 2 HALF.  Thread tx of row ty owns
// PXH pixel PAIRS: the pixel at tile column tx*PXH + p of the left half and the pixel
// HALF columns to its right.  Both pixels of a pair see the same window offsets, so all of
// their arithmetic runs as packed float2 operations (one instruction, two lanes).  Shared
// memory holds each tile row (with its R-cell halo) as float2 entries
// e -> (cell e, cell e + HALF), e < HALF + 2R, so the two operands of a pair come from
// one 8-byte entry and a thread's window row is a run of consecutive entries read with
// 16-byte loads.
template <int R, int C, int PXH, int BX, int BY>
struct Tile {
  static constexpr int HALF = BX * PXH;          // pixels per half-row
  static constexpr int TW = 2 * HALF;            // tile width (pixels)
  static constexpr int TH = BY;                  // tile height (pixels)
  static constexpr int NT = BX * BY;             // threads
  static constexpr int NE = HALF + 2 * R;        // paired entries per loaded row
  static constexpr int SEG = ((PXH + 2 * R + 1) / 2) * 2;   // entries a thread reads per row
  static constexpr int SW0 = (BX - 1) * PXH + SEG;
  static constexpr int SWm = SW0 > NE ? SW0 : NE;
  static constexpr int SW = ((SWm + 1) / 2) * 2; // row stride (entries), 16-byte multiple
  static constexpr int SH = TH + 2 * R;
  static constexpr int PLANE = SH * SW;          // float2 entries per channel plane
  static_assert(PXH % 2 == 0, "a thread's first entry must be 16-byte aligned");
};

template <int SEG>
__device__ __forceinline__ void load_row(const float2* __restrict__ row, float2 (&seg)[SEG]) {
#pragma unroll
  for (int q = 0; q < SEG / 2; ++q) {
    const float4 t = reinterpret_cast<const float4*>(row)[q];
    seg[2 * q + 0] = make_float2(t.x, t.y);
    seg[2 * q + 1] = make_float2(t.z, t.w);
  }
}

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

__device__ __forceinline__ float2 max0(float2 a) {
  return make_float2(fmaxf(a.x, 0.0f), fmaxf(a.y, 0.0f));
}

// Stage NF fields (NHWC, C channels each) of the tile + halo into paired planar shared
// memory, field 0 multiplied by s0.  Returns true when the halo leaves the image (the
// validity plane is then filled with 1/0 per cell).
// Global loads of a sweep's inputs: through the non-coherent cache path when the data
// was written before the launch, through L2 (COH) when another block of the same launch
// may have written it.
template <bool COH>
__device__ __forceinline__ float ld_in(const float* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}

template <class T, int R, int C, int NF, bool COH = false>
__device__ __forceinline__ bool load_tile(float2* __restrict__ sm, float2* __restrict__ smask,
                                          const float* __restrict__ f0,
                                          const float* __restrict__ f1, const SweepGeom& g,
                                          int x0, int y0, float s0 = 1.0f) {
  const bool border = (x0 - R < 0) || (y0 - R < 0) || (x0 + T::TW + R > g.W) ||
                      (y0 + T::TH + R > g.H);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  // A fixed trip count, unrolled: every load of the tile is issued before the first
  // shared-memory store waits on one, so staging costs one global-memory latency, not
  // one per pass.
  constexpr int kPasses = (T::PLANE + T::NT - 1) / T::NT;
#pragma unroll
  for (int pass = 0; pass < kPasses; ++pass) {
    const int idx = tid + pass * T::NT;
    if (idx >= T::PLANE) break;
    const int yy = idx / T::SW;
    const int k = idx - yy * T::SW;
    const int gy = y0 - R + yy;
    const int ga = x0 - R + k, gb = ga + T::HALF;
    const bool rowok = k < T::NE && gy >= 0 && gy < g.H;
    const bool oka = rowok && ga >= 0 && ga < g.W;
    const bool okb = rowok && gb >= 0 && gb < g.W;
    const size_t ba = oka ? ((size_t)gy * g.W + ga) * C : 0;
    const size_t bb = okb ? ((size_t)gy * g.W + gb) * C : 0;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      sm[ch * T::PLANE + idx] = make_float2(oka ? s0 * ld_in<COH>(f0 + ba + ch) : 0.0f,
                                            okb ? s0 * ld_in<COH>(f0 + bb + ch) : 0.0f);
      if constexpr (NF == 2)
        sm[(C + ch) * T::PLANE + idx] = make_float2(oka ? ld_in<COH>(f1 + ba + ch) : 0.0f,
                                                    okb ? ld_in<COH>(f1 + bb + ch) : 0.0f);
    }
    if (border) smask[idx] = make_float2(oka ? 1.0f : 0.0f, okb ? 1.0f : 0.0f);
  }
  __syncthreads();
  return border;
}

// Store the pair (left, right) of a thread's p-th pixel pair.
template <class T, int C, int PXH>
__device__ __forceinline__ void store_pairs(float* __restrict__ out, const SweepGeom& g,
                                            const float2 (&base)[PXH][C],
                                            const float2 (&acc)[PXH][C], int x0, int y0) {
  const int gy = y0 + threadIdx.y;
  if (gy >= g.H) return;
#pragma unroll
  for (int p = 0; p < PXH; ++p) {
    const int ga = x0 + threadIdx.x * PXH + p, gb = ga + T::HALF;
    if (ga < g.W) {
      float* o = out + ((size_t)gy * g.W + ga) * C;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) o[ch] = fmaf(g.scale, acc[p][ch].x, base[p][ch].x);
    }
    if (gb < g.W) {
      float* o = out + ((size_t)gy * g.W + gb) * C;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) o[ch] = fmaf(g.scale, acc[p][ch].y, base[p][ch].y);
    }
  }
}

// ------------------------------------------------------------------ forward step
// The tile holds the colours scaled by sk = sqrt(eps_c / 2), so that for d = sk (c_j - c_i)
//   r - 1 = |d|^2 + (eps_x / 2 |x_j - x_i|^2 - 1),
// one FMA per channel from a per-offset constant; t = max(1 - r, 0), phi = t^4 (5 - 4t),
// and the update sum_j phi d is taken back to colour units once per pixel
// (c^{n+1} = c^n + (dt / M) / sk * sum_j phi d, with c^n read unscaled).  Every operation
// of an interaction is a packed pair except the clamp.
template <class T, int C, int PXH, bool COH = false>
__device__ __forceinline__ void store_update(float* __restrict__ out,
                                             const float* __restrict__ src, const SweepGeom& g,
                                             const float2 (&acc)[PXH][C], float mult, int x0,
                                             int y0) {
  const int gy = y0 + threadIdx.y;
  if (gy >= g.H) return;
#pragma unroll
  for (int p = 0; p < PXH; ++p) {
    const int ga = x0 + threadIdx.x * PXH + p, gb = ga + T::HALF;
    if (ga < g.W) {
      const size_t k = ((size_t)gy * g.W + ga) * C;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) out[k + ch] = fmaf(mult, acc[p][ch].x, ld_in<COH>(src + k + ch));
    }
    if (gb < g.W) {
      const size_t k = ((size_t)gy * g.W + gb) * C;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) out[k + ch] = fmaf(mult, acc[p][ch].y, ld_in<COH>(src + k + ch));
    }
  }
}

__device__ __forceinline__ float2 max0_neg(float2 a) {
  return make_float2(fmaxf(-a.x, 0.0f), fmaxf(-a.y, 0.0f));
}

// Scale of the staged colours: sqrt(eps_c / 2), with eps_c = 0 read as a tiny positive
// value (its colour term, below 1e-30 |c_j - c_i|^2, is far under float32 resolution).
__device__ __forceinline__ float colour_scale(float kc) { return sqrtf(fmaxf(kc, 1e-30f)); }

template <class T, int R, int C, int PXH, bool BORDER, bool COH = false>
__device__ __forceinline__ void forward_body(const float2* __restrict__ sm,
                                             const float2* __restrict__ smask,
                                             const float* __restrict__ src,
                                             float* __restrict__ out, const SweepGeom& g,
                                             float kx, float ky, float mult, int x0, int y0) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int sx = tx * PXH;
  float2 nci[PXH][C], acc[PXH][C];
#pragma unroll
  for (int p = 0; p < PXH; ++p)
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      const float2 ci = sm[ch * T::PLANE + (ty + R) * T::SW + sx + R + p];
      nci[p][ch] = make_float2(-ci.x, -ci.y);
      acc[p][ch] = f2(0.0f);
    }
  const float2 m4 = f2(-4.0f), five = f2(5.0f);
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
    const int row = (ty + R + dy) * T::SW + sx;
    float2 seg[C][T::SEG];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) load_row<T::SEG>(sm + ch * T::PLANE + row, seg[ch]);
    float2 mseg[BORDER ? T::SEG : 1];
    if constexpr (BORDER) load_row<T::SEG>(smask + row, mseg);
    const float syn = fmaf(ky, (float)(dy * dy), -1.0f);
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const float2 spn = f2(fmaf(kx, (float)(dx * dx), syn));  // spatial part of r, minus 1
#pragma unroll
      for (int p = 0; p < PXH; ++p) {
        const int e = p + R + dx;
        float2 d[C];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) d[ch] = __fadd2_rn(seg[ch][e], nci[p][ch]);
        float2 u = spn;                                          // r - 1
#pragma unroll
        for (int ch = 0; ch < C; ++ch) u = __ffma2_rn(d[ch], d[ch], u);
        const float2 t = max0_neg(u);                            // max(1 - r, 0)
        const float2 t2 = __fmul2_rn(t, t);
        float2 ph = __fmul2_rn(__fmul2_rn(t2, t2), __ffma2_rn(m4, t, five));
        if constexpr (BORDER) ph = __fmul2_rn(ph, mseg[e]);
#pragma unroll
        for (int ch = 0; ch < C; ++ch) acc[p][ch] = __ffma2_rn(ph, d[ch], acc[p][ch]);
      }
    }
  }
  store_update<T, C, PXH, COH>(out, src, g, acc, mult, x0, y0);
}

template <int R, int C, int PXH, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
forward_tile_kernel(const float* __restrict__ c, float* __restrict__ out,
                    const double* __restrict__ eps_n, SweepGeom g) {
  using T = Tile<R, C, PXH, BX, BY>;
  extern __shared__ __align__(16) float2 smem2[];
  float2* sm = smem2;
  float2* smask = smem2 + C * T::PLANE;
  const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
  // Programmatic dependent launch: the next Euler step may be launched once every block
  // of this one has started, and waits (in hardware) for this grid's completion before
  // it reads c^{n+1}; launched without the attribute, both instructions do nothing.
  // Every global read comes after the wait: the control of a trial sweep is written by the
  // kernel just before its first step.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2;
  const float sk = colour_scale(0.5f * ec), mult = g.scale / sk;
  const bool border = load_tile<T, R, C, 1>(sm, smask, c, nullptr, g, x0, y0, sk);
  if (border)
    forward_body<T, R, C, PXH, true>(sm, smask, c, out, g, kx, ky, mult, x0, y0);
  else
    forward_body<T, R, C, PXH, false>(sm, smask, c, out, g, kx, ky, mult, x0, y0);
}

// ------------------------------------------------------------------ adjoint step
// (J_F^T lam)_k = (1/M) sum_{j in W(k)} [phi'(r) eps_c delta (delta . dlam) + phi(r) dlam],
//   delta = c_j - c_k, dlam = lam_j - lam_k (gather form: the Jacobian blocks are
//   symmetric because r_kj = r_jk, the window is symmetric and M is constant);
// D_x = sum_k sum_j phi'(r_kj) |x_j - x_k|^2 (lam_k . delta) (times 1/(2M) later), and
// D_c likewise with |delta|^2.  phi' and both distances are symmetric in (k, j), delta is
// antisymmetric and the window is symmetric, so pairing (k, j) with (j, k) gives
//   D_x = -1/2 sum_k sum_j phi'(r_kj) |x_j - x_k|^2 (delta . dlam),
// which reuses delta . dlam (already needed for J^T lam) instead of a third dot product
// lam_k . delta, and adds each pair's contribution once instead of as two nearly
// cancelling terms.  The identity holds for the image total, which is what D is; a
// block's partial alone has no meaning.
// phi' = 20 t^3 (t - 1) with t = max(1 - r, 0); the factor -20/2 is applied once per
// thread.
template <class T, int R, int C, int PXH, bool BORDER>
__device__ __forceinline__ void adjoint_body(const float2* __restrict__ sm,
                                             const float2* __restrict__ smask,
                                             float* __restrict__ out, double* __restrict__ partial,
                                             const SweepGeom& g, float kx, float ky, float kc,
                                             float ec, int x0, int y0) {
  const float2* sc = sm;
  const float2* sl = sm + C * T::PLANE;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int sx = tx * PXH;
  float2 lk[PXH][C], nck[PXH][C], nlk[PXH][C], acc[PXH][C];
  // Validity of the thread's own pixels (border tiles): the paired D terms of a pixel
  // outside the image are not zero by themselves (its zero-filled lam_k makes
  // dlam = lam_j), so they are masked like those of a neighbour outside the image.
  float2 vk[BORDER ? PXH : 1];
#pragma unroll
  for (int p = 0; p < PXH; ++p) {
    if constexpr (BORDER) vk[p] = smask[(ty + R) * T::SW + sx + R + p];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      const int o = ch * T::PLANE + (ty + R) * T::SW + sx + R + p;
      const float2 ck = sc[o];
      lk[p][ch] = sl[o];
      nck[p][ch] = make_float2(-ck.x, -ck.y);
      nlk[p][ch] = make_float2(-lk[p][ch].x, -lk[p][ch].y);
      acc[p][ch] = f2(0.0f);
    }
  }
  const float2 nkc = f2(-kc), m4 = f2(-4.0f), five = f2(5.0f), m1 = f2(-1.0f);
  const float2 ec20 = f2(20.0f * ec);
  float2 Dx = f2(0.0f), Dc = f2(0.0f);
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
    const int row = (ty + R + dy) * T::SW + sx;
    float2 cseg[C][T::SEG], lseg[C][T::SEG];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      load_row<T::SEG>(sc + ch * T::PLANE + row, cseg[ch]);
      load_row<T::SEG>(sl + ch * T::PLANE + row, lseg[ch]);
    }
    float2 mseg[BORDER ? T::SEG : 1];
    if constexpr (BORDER) load_row<T::SEG>(smask + row, mseg);
    const float sy = fmaf(-ky, (float)(dy * dy), 1.0f);
    const float d2y = g.inv_h2 * (float)(dy * dy);
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const float2 sp = f2(fmaf(-kx, (float)(dx * dx), sy));  // 1 - spatial part of r
      const float2 d2 = f2(fmaf(g.inv_w2, (float)(dx * dx), d2y));
#pragma unroll
      for (int p = 0; p < PXH; ++p) {
        const int e = p + R + dx;
        float2 d[C], dl[C];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
          d[ch] = __fadd2_rn(cseg[ch][e], nck[p][ch]);
          dl[ch] = __fadd2_rn(lseg[ch][e], nlk[p][ch]);
        }
        float2 s2 = __fmul2_rn(d[0], d[0]);
        float2 proj = __fmul2_rn(d[0], dl[0]);
#pragma unroll
        for (int ch = 1; ch < C; ++ch) {
          s2 = __ffma2_rn(d[ch], d[ch], s2);
          proj = __ffma2_rn(d[ch], dl[ch], proj);
        }
        const float2 t = max0(__ffma2_rn(nkc, s2, sp));        // max(1 - r, 0)
        const float2 t2 = __fmul2_rn(t, t);
        const float2 t3 = __fmul2_rn(t2, t);
        float2 ph = __fmul2_rn(__fmul2_rn(t2, t2), __ffma2_rn(m4, t, five));
        float2 dph = __fmul2_rn(t3, __fadd2_rn(t, m1));         // phi' / 20
        if constexpr (BORDER) {
          const float2 m = __fmul2_rn(mseg[e], vk[p]);
          ph = __fmul2_rn(ph, m);
          dph = __fmul2_rn(dph, m);
        }
        const float2 gk = __fmul2_rn(dph, proj);
        const float2 coef = __fmul2_rn(gk, ec20);
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
          acc[p][ch] = __ffma2_rn(coef, d[ch], acc[p][ch]);
          acc[p][ch] = __ffma2_rn(ph, dl[ch], acc[p][ch]);
        }
        Dx = __ffma2_rn(gk, d2, Dx);
        Dc = __ffma2_rn(gk, s2, Dc);
      }
    }
  }
  store_pairs<T, C, PXH>(out, g, lk, acc, x0, y0);
  __shared__ double red[2 * 32];
  double v[2] = {-10.0 * ((double)Dx.x + (double)Dx.y), -10.0 * ((double)Dc.x + (double)Dc.y)};
  double tot[2];
  block_sum<2>(v, red, tot);
  if (threadIdx.x == 0 && threadIdx.y == 0) {   // partial points at this tile's pair
    partial[0] = tot[0];
    partial[1] = tot[1];
  }
}

template <int R, int C, int PXH, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
adjoint_tile_kernel(const float* __restrict__ c, const float* __restrict__ lam,
                    float* __restrict__ out, const double* __restrict__ eps_n,
                    double* __restrict__ partial, SweepGeom g) {
  using T = Tile<R, C, PXH, BX, BY>;
  extern __shared__ __align__(16) float2 smem2[];
  float2* sm = smem2;
  float2* smask = smem2 + 2 * C * T::PLANE;
  const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
  // Programmatic dependent launch, as in forward_tile_kernel: the next adjoint step may
  // be launched once every block of this one has started; all global reads follow the
  // wait for the previous grid.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
  const bool border = load_tile<T, R, C, 2>(sm, smask, c, lam, g, x0, y0);
  double* part = partial + 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
  if (border)
    adjoint_body<T, R, C, PXH, true>(sm, smask, out, part, g, kx, ky, kc, ec, x0, y0);
  else
    adjoint_body<T, R, C, PXH, false>(sm, smask, out, part, g, kx, ky, kc, ec, x0, y0);
}

// ------------------------------------------------------------------ batched (persistent)
// One launch processes step n for every (image, tile) job of a batch; the tile bodies are
// the single-image ones, so every pixel's result is bitwise the same.  The grid is sized
// to the resident capacity and walks the job list; jobs of inactive images are skipped.
__device__ __forceinline__ const float* batch_state(const BatchSweepImg& im, int n) {
  return n == 0 ? im.c0 : im.traj + (size_t)(n - 1) * im.g.H * im.g.W * im.g.C;
}

template <int R, int C, int PXH, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
forward_batch_kernel(const BatchSweepImg* __restrict__ imgs, const BatchJob* __restrict__ jobs,
                     int njobs, const int* __restrict__ active, int n, int kind) {
  using T = Tile<R, C, PXH, BX, BY>;
  extern __shared__ __align__(16) float2 smem2[];
  float2* sm = smem2;
  float2* smask = smem2 + C * T::PLANE;
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchSweepImg& im = imgs[job.img];
    const SweepGeom g = im.g;
    const size_t nc = (size_t)g.H * g.W * C;
    const float* src;
    float* dst;
    const double* eps_n;
    if (kind == kSweepStore) {
      src = batch_state(im, n);
      dst = n == im.nsteps - 1 ? im.cT : im.traj + (size_t)n * nc;
      eps_n = im.eps + 2 * n;
    } else {
      src = n == 0 ? im.c0 : ((n - 1) & 1 ? im.work1 : im.work0);
      dst = n == im.nsteps - 1 ? im.trial_c : (n & 1 ? im.work1 : im.work0);
      eps_n = im.trial_eps + 2 * n;
    }
    const int x0 = job.tx * T::TW, y0 = job.ty * T::TH;
    const float ex = (float)eps_n[0], ec = (float)eps_n[1];
    const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2;
    const float sk = colour_scale(0.5f * ec), mult = g.scale / sk;
    const bool border = load_tile<T, R, C, 1>(sm, smask, src, nullptr, g, x0, y0, sk);
    if (border)
      forward_body<T, R, C, PXH, true>(sm, smask, src, dst, g, kx, ky, mult, x0, y0);
    else
      forward_body<T, R, C, PXH, false>(sm, smask, src, dst, g, kx, ky, mult, x0, y0);
    __syncthreads();  // the next job reuses shared memory
  }
}

template <int R, int C, int PXH, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
adjoint_batch_kernel(const BatchSweepImg* __restrict__ imgs, const BatchJob* __restrict__ jobs,
                     int njobs, const int* __restrict__ active, int n) {
  using T = Tile<R, C, PXH, BX, BY>;
  extern __shared__ __align__(16) float2 smem2[];
  float2* sm = smem2;
  float2* smask = smem2 + 2 * C * T::PLANE;
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchSweepImg& im = imgs[job.img];
    const SweepGeom g = im.g;
    const int li = (im.nsteps - 1 - n) & 1;
    const float* lin = li ? im.lam1 : im.lam0;
    float* lout = li ? im.lam0 : im.lam1;
    const double* eps_n = im.eps + 2 * n;
    const int x0 = job.tx * T::TW, y0 = job.ty * T::TH;
    const float ex = (float)eps_n[0], ec = (float)eps_n[1];
    const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
    const bool border = load_tile<T, R, C, 2>(sm, smask, batch_state(im, n), lin, g, x0, y0);
    const int tiles_x = (g.W + T::TW - 1) / T::TW;
    // this tile's partial pair, in the single-image kernel's order (row-major tiles)
    double* part = im.part_adj + ((size_t)n * im.ntiles + (size_t)job.ty * tiles_x + job.tx) * 2;
    if (border)
      adjoint_body<T, R, C, PXH, true>(sm, smask, lout, part, g, kx, ky, kc, ec, x0, y0);
    else
      adjoint_body<T, R, C, PXH, false>(sm, smask, lout, part, g, kx, ky, kc, ec, x0, y0);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ any R, any C
// One thread per pixel, window clipped by loop bounds, fields read through the cache.
// Used for channel counts or radii without a tiled instantiation.
constexpr int kGenericMaxC = 64;

__global__ void forward_generic_kernel(const float* __restrict__ c, float* __restrict__ out,
                                       const double* __restrict__ eps_n, SweepGeom g);
__global__ void adjoint_generic_kernel(const float* __restrict__ c,
                                       const float* __restrict__ lam, float* __restrict__ out,
                                       const double* __restrict__ eps_n,
                                       double* __restrict__ partial, SweepGeom g);
__global__ void forward_generic_batch_kernel(const BatchSweepImg* __restrict__ imgs,
                                             const BatchJob* __restrict__ jobs, int njobs,
                                             const int* __restrict__ active, int n, int kind);
__global__ void adjoint_generic_batch_kernel(const BatchSweepImg* __restrict__ imgs,
                                             const BatchJob* __restrict__ jobs, int njobs,
                                             const int* __restrict__ active, int n);

}  // namespace agents
