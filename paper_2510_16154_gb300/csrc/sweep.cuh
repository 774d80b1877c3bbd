// Agent sweep kernels: one explicit Euler step of the alignment dynamics (Eq. MAsystem,
// Eq. ellipsoid, Eq. kernel) and one step of its exact discrete adjoint with the
// control-derivative partials D^n (Section 3.1, Algorithm 1).
//
// Both steps are FP32-ALU bound: every pixel visits its (2R+1)^2 window.  Design:
//  * a CTA owns a TH x TW tile of output pixels; it stages the tile plus an R-pixel halo
//    of the input field(s) in shared memory, de-interleaved into one plane per channel
//    (NHWC in HBM -> planar in SMEM), with out-of-image cells zero-filled;
//  * each thread owns PX consecutive pixels of one row and walks the window row by row:
//    it loads the PX + 2R cells of that window row once into registers (16- or 8-byte
//    vector reads) and reuses them for all PX pixels (register blocking);
//  * the spatial part of r_ij is uniform over pixels, so it is folded into one FMA per
//    (dy, dx) per thread; phi is branch-free (r clamped at 1);
//  * interior tiles skip all bounds handling; tiles whose halo leaves the image multiply
//    each interaction weight by a 0/1 validity plane (exact: out-of-image cells hold 0,
//    so the weight times a finite difference is exactly 0);
//  * the pixel's own cell (dy = dx = 0) is not skipped: its difference is exactly 0, so
//    it adds exactly 0 to every sum, and keeping it keeps the inner loop branch-free.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace agents {

template <int R, int C, int PX, int BX, int BY>
struct Tile {
  static constexpr int TW = BX * PX;           // tile width (pixels)
  static constexpr int TH = BY;                // tile height (pixels)
  static constexpr int NT = BX * BY;           // threads
  static constexpr int VEC = (PX % 4 == 0) ? 4 : 2;
  static constexpr int SEG = ((PX + 2 * R + VEC - 1) / VEC) * VEC;  // cells read per row
  static constexpr int LW = TW + 2 * R;        // loaded width
  static constexpr int SW0 = (BX - 1) * PX + SEG;
  static constexpr int SWm = SW0 > LW ? SW0 : LW;
  static constexpr int SW = ((SWm + 3) / 4) * 4;  // row stride (floats), 16-byte multiple
  static constexpr int SH = TH + 2 * R;
  static constexpr int PLANE = SH * SW;
  static_assert(PX % 2 == 0, "PX must be even");
};

template <int VEC, int SEG>
__device__ __forceinline__ void load_row(const float* __restrict__ row, float (&seg)[SEG]) {
  if constexpr (VEC == 4) {
#pragma unroll
    for (int q = 0; q < SEG / 4; ++q) {
      const float4 t = reinterpret_cast<const float4*>(row)[q];
      seg[4 * q + 0] = t.x; seg[4 * q + 1] = t.y; seg[4 * q + 2] = t.z; seg[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < SEG / 2; ++q) {
      const float2 t = reinterpret_cast<const float2*>(row)[q];
      seg[2 * q + 0] = t.x; seg[2 * q + 1] = t.y;
    }
  }
}

// Stage NF fields (NHWC, C channels each) of the tile + halo into planar shared memory.
// Returns true when the halo leaves the image (the validity plane is then filled).
template <class T, int R, int C, int NF>
__device__ __forceinline__ bool load_tile(float* __restrict__ sm, float* __restrict__ smask,
                                          const float* __restrict__ f0,
                                          const float* __restrict__ f1, const SweepGeom& g,
                                          int x0, int y0) {
  const bool border = (x0 - R < 0) || (y0 - R < 0) || (x0 + T::TW + R > g.W) ||
                      (y0 + T::TH + R > g.H);
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int idx = tid; idx < T::PLANE; idx += T::NT) {
    const int yy = idx / T::SW;
    const int xx = idx - yy * T::SW;
    const int gy = y0 - R + yy, gx = x0 - R + xx;
    const bool ok = xx < T::LW && gy >= 0 && gy < g.H && gx >= 0 && gx < g.W;
    const size_t base = ok ? ((size_t)gy * g.W + gx) * C : 0;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      sm[ch * T::PLANE + idx] = ok ? __ldg(f0 + base + ch) : 0.0f;
      if constexpr (NF == 2) sm[(C + ch) * T::PLANE + idx] = ok ? __ldg(f1 + base + ch) : 0.0f;
    }
    if (border) smask[idx] = ok ? 1.0f : 0.0f;
  }
  __syncthreads();
  return border;
}

// ------------------------------------------------------------------ forward step
template <class T, int R, int C, int PX, bool BORDER>
__device__ __forceinline__ void forward_body(const float* __restrict__ sm,
                                             const float* __restrict__ smask,
                                             float* __restrict__ out, const SweepGeom& g,
                                             float kx, float ky, float kc, int x0, int y0) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int sx = tx * PX;
  float ci[PX][C], acc[PX][C];
#pragma unroll
  for (int p = 0; p < PX; ++p)
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      ci[p][ch] = sm[ch * T::PLANE + (ty + R) * T::SW + sx + R + p];
      acc[p][ch] = 0.0f;
    }
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
    const int row = (ty + R + dy) * T::SW + sx;
    float seg[C][T::SEG];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) load_row<T::VEC, T::SEG>(sm + ch * T::PLANE + row, seg[ch]);
    float mseg[BORDER ? T::SEG : 1];
    if constexpr (BORDER) load_row<T::VEC, T::SEG>(smask + row, mseg);
    const float sy = ky * (float)(dy * dy);
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const float sp = fmaf(kx, (float)(dx * dx), sy);
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        const int j = p + R + dx;
        float d[C];
        float s2 = 0.0f;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
          d[ch] = seg[ch][j] - ci[p][ch];
          s2 = fmaf(d[ch], d[ch], s2);
        }
        float ph = wendland_phi(fmaf(kc, s2, sp));
        if constexpr (BORDER) ph *= mseg[j];
#pragma unroll
        for (int ch = 0; ch < C; ++ch) acc[p][ch] = fmaf(ph, d[ch], acc[p][ch]);
      }
    }
  }
  const int gy = y0 + ty;
  if (gy < g.H) {
#pragma unroll
    for (int p = 0; p < PX; ++p) {
      const int gx = x0 + sx + p;
      if (gx < g.W) {
        float* o = out + ((size_t)gy * g.W + gx) * C;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) o[ch] = fmaf(g.scale, acc[p][ch], ci[p][ch]);
      }
    }
  }
}

template <int R, int C, int PX, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
forward_tile_kernel(const float* __restrict__ c, float* __restrict__ out,
                    const double* __restrict__ eps_n, SweepGeom g) {
  using T = Tile<R, C, PX, BX, BY>;
  extern __shared__ __align__(16) float smem[];
  float* sm = smem;
  float* smask = smem + C * T::PLANE;
  const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
  const bool border = load_tile<T, R, C, 1>(sm, smask, c, nullptr, g, x0, y0);
  if (border)
    forward_body<T, R, C, PX, true>(sm, smask, out, g, kx, ky, kc, x0, y0);
  else
    forward_body<T, R, C, PX, false>(sm, smask, out, g, kx, ky, kc, x0, y0);
}

// ------------------------------------------------------------------ adjoint step
// (J_F^T lam)_k = (1/M) sum_{j in W(k)} [phi'(r) eps_c delta (delta . dlam) + phi(r) dlam],
//   delta = c_j - c_k, dlam = lam_j - lam_k (gather form: the Jacobian blocks are
//   symmetric because r_kj = r_jk, the window is symmetric and M is constant);
// D_x partial = sum_k sum_j phi'(r_kj) |x_j - x_k|^2 (lam_k . delta),
// D_c partial = sum_k sum_j phi'(r_kj) |delta|^2     (lam_k . delta)   (times 1/(2M) later).
template <class T, int R, int C, int PX, bool BORDER>
__device__ __forceinline__ void adjoint_body(const float* __restrict__ sm,
                                             const float* __restrict__ smask,
                                             float* __restrict__ out, double* __restrict__ partial,
                                             const SweepGeom& g, float kx, float ky, float kc,
                                             float ec, int x0, int y0) {
  const float* sc = sm;
  const float* sl = sm + C * T::PLANE;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int sx = tx * PX;
  float ck[PX][C], lk[PX][C], acc[PX][C];
#pragma unroll
  for (int p = 0; p < PX; ++p)
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      const int o = ch * T::PLANE + (ty + R) * T::SW + sx + R + p;
      ck[p][ch] = sc[o];
      lk[p][ch] = sl[o];
      acc[p][ch] = 0.0f;
    }
  float Dx = 0.0f, Dc = 0.0f;
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
    const int row = (ty + R + dy) * T::SW + sx;
    float cseg[C][T::SEG], lseg[C][T::SEG];
#pragma unroll
    for (int ch = 0; ch < C; ++ch) {
      load_row<T::VEC, T::SEG>(sc + ch * T::PLANE + row, cseg[ch]);
      load_row<T::VEC, T::SEG>(sl + ch * T::PLANE + row, lseg[ch]);
    }
    float mseg[BORDER ? T::SEG : 1];
    if constexpr (BORDER) load_row<T::VEC, T::SEG>(smask + row, mseg);
    const float sy = ky * (float)(dy * dy);
    const float d2y = g.inv_h2 * (float)(dy * dy);
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const float sp = fmaf(kx, (float)(dx * dx), sy);
      const float d2 = fmaf(g.inv_w2, (float)(dx * dx), d2y);
#pragma unroll
      for (int p = 0; p < PX; ++p) {
        const int j = p + R + dx;
        float d[C], dl[C];
        float s2 = 0.0f, proj = 0.0f, lkd = 0.0f;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
          d[ch] = cseg[ch][j] - ck[p][ch];
          dl[ch] = lseg[ch][j] - lk[p][ch];
          s2 = fmaf(d[ch], d[ch], s2);
          proj = fmaf(d[ch], dl[ch], proj);
          lkd = fmaf(lk[p][ch], d[ch], lkd);
        }
        float ph, dph;
        wendland_phi_dphi(fmaf(kc, s2, sp), ph, dph);
        if constexpr (BORDER) {
          ph *= mseg[j];
          dph *= mseg[j];
        }
        const float coef = (dph * ec) * proj;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) {
          acc[p][ch] = fmaf(coef, d[ch], acc[p][ch]);
          acc[p][ch] = fmaf(ph, dl[ch], acc[p][ch]);
        }
        const float gk = dph * lkd;
        Dx = fmaf(gk, d2, Dx);
        Dc = fmaf(gk, s2, Dc);
      }
    }
  }
  const int gy = y0 + ty;
  if (gy < g.H) {
#pragma unroll
    for (int p = 0; p < PX; ++p) {
      const int gx = x0 + sx + p;
      if (gx < g.W) {
        float* o = out + ((size_t)gy * g.W + gx) * C;
#pragma unroll
        for (int ch = 0; ch < C; ++ch) o[ch] = fmaf(g.scale, acc[p][ch], lk[p][ch]);
      }
    }
  }
  __shared__ double red[2 * 32];
  double v[2] = {(double)Dx, (double)Dc};
  double tot[2];
  block_sum<2>(v, red, tot);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    partial[2 * b + 0] = tot[0];
    partial[2 * b + 1] = tot[1];
  }
}

template <int R, int C, int PX, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
adjoint_tile_kernel(const float* __restrict__ c, const float* __restrict__ lam,
                    float* __restrict__ out, const double* __restrict__ eps_n,
                    double* __restrict__ partial, SweepGeom g) {
  using T = Tile<R, C, PX, BX, BY>;
  extern __shared__ __align__(16) float smem[];
  float* sm = smem;
  float* smask = smem + 2 * C * T::PLANE;
  const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
  const bool border = load_tile<T, R, C, 2>(sm, smask, c, lam, g, x0, y0);
  if (border)
    adjoint_body<T, R, C, PX, true>(sm, smask, out, partial, g, kx, ky, kc, ec, x0, y0);
  else
    adjoint_body<T, R, C, PX, false>(sm, smask, out, partial, g, kx, ky, kc, ec, x0, y0);
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

}  // namespace agents
