// Total-variation kernels of the ADMM splitting (Section 4.1): the terminal adjoint and
// objective L~ (Eq. complete_square, Eq. admm_terminal), the shrinkage v-step
// (Eq. soft_threshold), the multiplier update with its residuals (Eq. dual_ascent), the
// control projection of Algorithm 1, and deterministic float64 reductions.
//
// All are HBM-bound point/stencil kernels.  G is the central-difference gradient with
// reflective boundaries (Definition discrete_gradient, Eq. reflective_boundary): along
// x it is (c[q+1] - c[q-1]) / (2 dx) for 1 <= q <= W-2 and exactly 0 on the first and
// last column (the mirrored neighbour equals the other one); likewise along y.  Its
// exact transpose is therefore (G_x^T w)[q] = (w[q-1] [q-1 interior] - w[q+1]
// [q+1 interior]) / (2 dx).  Each thread handles kPPT pixels of one row (strided by the
// block width, so warps stay coalesced), sums its per-pixel terms in float32 and the
// block then reduces in float64 with a fixed shuffle tree, writing one partial per block;
// launch_reduce_rows adds the partials in a fixed order (bitwise reproducible).
#include "common.cuh"
#include "fp_bits.cuh"
#include "kernels.h"

#include <algorithm>

namespace agents {

constexpr int kTvBX = 32, kTvBY = 8, kPPT = 4;
constexpr int kTvMaxC = 64;

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

int tv_num_blocks(const TvGeom& g) {
  return cdiv(g.W, kTvBX * kPPT) * cdiv(g.H, kTvBY);
}

template <int CT>
__device__ __forceinline__ int nch(const TvGeom& g) { return CT ? CT : g.C; }

// (G c) at pixel (r, q), channel ch.
__device__ __forceinline__ float grad_x(const float* __restrict__ c, const TvGeom& g, int r, int q,
                                        int C, int ch) {
  if (q < 1 || q > g.W - 2) return 0.0f;
  const size_t k = (size_t)r * g.W + q;
  return (__ldg(c + (k + 1) * C + ch) - __ldg(c + (k - 1) * C + ch)) * g.inv2hx;
}
__device__ __forceinline__ float grad_y(const float* __restrict__ c, const TvGeom& g, int r, int q,
                                        int C, int ch) {
  if (r < 1 || r > g.H - 2) return 0.0f;
  const size_t k = (size_t)r * g.W + q;
  return (__ldg(c + (k + g.W) * C + ch) - __ldg(c + (k - g.W) * C + ch)) * g.inv2hy;
}

// ------------------------------------------------------------------ objective / terminal
// Per-pixel term of L~ / (dx dy):  rho/2 |v - Gc + mu/rho|^2 + |v| + alpha/2 |c - c0|^2.
// With LAMBDA, also lam = -dx dy [G^T (rho G c - rho v - mu) + alpha (c - c0)].
// A hint to L2 for a line of global memory (no register is written, nothing waits on it).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The TV kernels' threads walk kPPT pixels of a row one after another; asking L2 for the
// later pixels' lines of the fields they read at the start lets those DRAM latencies
// overlap the first pixel's work.  f[j] holds per[j] floats per pixel (NHWC).  Used by
// the terminal adjoint and the multiplier update (measured faster); the trial objective
// and the v-step measured slower or the same with it.
template <int NF>
__device__ __forceinline__ void prefetch_later_pixels(int bx, int r, const TvGeom& g,
                                                      const float* const (&f)[NF],
                                                      const int (&per)[NF]) {
#pragma unroll
  for (int i = 1; i < kPPT; ++i) {
    const int q = bx * (kTvBX * kPPT) + i * kTvBX + threadIdx.x;
    if (q < g.W) {
      const size_t k = (size_t)r * g.W + q;
#pragma unroll
      for (int j = 0; j < NF; ++j)
        if (f[j]) prefetch_l2(f[j] + k * per[j]);
    }
  }
}

// The per-thread part of one block (bx, by) of pixels; returns the thread's float32 sum.
template <int CT, bool LAMBDA>
__device__ __forceinline__ float objective_block(int bx, int by, const float* __restrict__ c,
                                                 const float* __restrict__ c0,
                                                 const float* __restrict__ v,
                                                 const float* __restrict__ mu,
                                                 float* __restrict__ lam, const TvGeom& g) {
  const int C = nch<CT>(g);
  const int r = by * kTvBY + threadIdx.y;
  float acc = 0.0f;
  if (r < g.H) {
#pragma unroll
    for (int i = 0; i < kPPT; ++i) {
      const int q = bx * (kTvBX * kPPT) + i * kTvBX + threadIdx.x;
      if (q >= g.W) break;
      const size_t k = (size_t)r * g.W + q;
      const float* vk = v + k * 2 * C;
      const float* mk = mu + k * 2 * C;
      float pen = 0.0f, fid = 0.0f, vv = 0.0f, tvs = 0.0f;
      for (int ch = 0; ch < C; ++ch) {
        const float gx = grad_x(c, g, r, q, C, ch), gy = grad_y(c, g, r, q, C, ch);
        const float vx = __ldg(vk + ch), vy = __ldg(vk + C + ch);
        const float qx = fmaf(__ldg(mk + ch), g.inv_rho, vx - gx);
        const float qy = fmaf(__ldg(mk + C + ch), g.inv_rho, vy - gy);
        pen = fmaf(qx, qx, fmaf(qy, qy, pen));
        const float e = __ldg(c + k * C + ch) - __ldg(c0 + k * C + ch);
        fid = fmaf(e, e, fid);
        if (g.tv_mode == 0) vv = fmaf(vx, vx, fmaf(vy, vy, vv));
        else tvs += sqrtf(fmaf(vx, vx, vy * vy));
        if constexpr (LAMBDA) {
          // (G^T w)_k with w = rho G c - rho v - mu, evaluated at the four neighbours
          float gtw = 0.0f;
          if (q - 1 >= 1) {  // q - 1 <= W - 2 always holds
            const size_t m = k - 1;
            const float w = g.rho * (grad_x(c, g, r, q - 1, C, ch) - __ldg(v + m * 2 * C + ch)) -
                            __ldg(mu + m * 2 * C + ch);
            gtw = fmaf(w, g.inv2hx, gtw);
          }
          if (q + 1 <= g.W - 2) {
            const size_t m = k + 1;
            const float w = g.rho * (grad_x(c, g, r, q + 1, C, ch) - __ldg(v + m * 2 * C + ch)) -
                            __ldg(mu + m * 2 * C + ch);
            gtw = fmaf(-w, g.inv2hx, gtw);
          }
          if (r - 1 >= 1) {
            const size_t m = k - g.W;
            const float w = g.rho * (grad_y(c, g, r - 1, q, C, ch) - __ldg(v + m * 2 * C + C + ch)) -
                            __ldg(mu + m * 2 * C + C + ch);
            gtw = fmaf(w, g.inv2hy, gtw);
          }
          if (r + 1 <= g.H - 2) {
            const size_t m = k + g.W;
            const float w = g.rho * (grad_y(c, g, r + 1, q, C, ch) - __ldg(v + m * 2 * C + C + ch)) -
                            __ldg(mu + m * 2 * C + C + ch);
            gtw = fmaf(-w, g.inv2hy, gtw);
          }
          lam[k * C + ch] = -(float)g.cell * fmaf(g.alpha, e, gtw);
        }
      }
      const float tv = g.tv_mode == 0 ? sqrtf(vv) : tvs;
      acc += fmaf(0.5f * g.rho, pen, fmaf(0.5f * g.alpha, fid, tv));
    }
  }
  return acc;
}

// Terminal adjoint for C in {1, 3} with w = rho G c - rho v - mu formed once per cell.
// The block's w is kept in shared memory: x-components for its rows and one extra column
// on either side, y-components for its columns and one extra row above and below.  G^T w
// then takes four shared loads per pixel and channel instead of recomputing w at the four
// neighbours from global memory (26 global loads per pixel and channel become about 14).
// Each thread owns the same pixels as in objective_block and forms the L~ terms with the
// same expressions in the same order, so the block's value is bitwise the one the trial
// objective (objective_block<CT, false>) returns for the same fields; G^T w adds the four
// neighbour terms in objective_block's order.
struct TermTile {
  static constexpr int BW = kTvBX * kPPT;   // pixel columns of a block
  static constexpr int XW = BW + 2;         // w_x cells per row: columns x0 - 1 .. x0 + BW
  static constexpr int YH = kTvBY + 2;      // w_y rows: y0 - 1 .. y0 + kTvBY
};

template <int CT>
__device__ __forceinline__ float terminal_block(int bx, int by, const float* __restrict__ c,
                                                const float* __restrict__ c0,
                                                const float* __restrict__ v,
                                                const float* __restrict__ mu,
                                                float* __restrict__ lam, const TvGeom& g) {
  using TT = TermTile;
  __shared__ float wx_s[kTvBY * TT::XW * CT];
  __shared__ float wy_s[TT::YH * TT::BW * CT];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = bx * TT::BW, y0 = by * kTvBY;
  const int r = y0 + ty;
  float acc = 0.0f;
  float e_own[kPPT][CT];
  // Phase 1: the L~ terms of the thread's own pixels, and w at their cells.
  if (r < g.H) {
    prefetch_later_pixels<4>(bx, r, g, {v, mu, c, c0}, {2 * CT, 2 * CT, CT, CT});
#pragma unroll
    for (int i = 0; i < kPPT; ++i) {
      const int q = x0 + i * kTvBX + tx;
      if (q >= g.W) break;
      const size_t k = (size_t)r * g.W + q;
      const float* vk = v + k * 2 * CT;
      const float* mk = mu + k * 2 * CT;
      const int j = q - x0;
      float pen = 0.0f, fid = 0.0f, vv = 0.0f, tvs = 0.0f;
#pragma unroll
      for (int ch = 0; ch < CT; ++ch) {
        const float gx = grad_x(c, g, r, q, CT, ch), gy = grad_y(c, g, r, q, CT, ch);
        const float vx = __ldg(vk + ch), vy = __ldg(vk + CT + ch);
        const float mx = __ldg(mk + ch), my = __ldg(mk + CT + ch);
        const float qx = fmaf(mx, g.inv_rho, vx - gx);
        const float qy = fmaf(my, g.inv_rho, vy - gy);
        pen = fmaf(qx, qx, fmaf(qy, qy, pen));
        const float e = __ldg(c + k * CT + ch) - __ldg(c0 + k * CT + ch);
        fid = fmaf(e, e, fid);
        if (g.tv_mode == 0) vv = fmaf(vx, vx, fmaf(vy, vy, vv));
        else tvs += sqrtf(fmaf(vx, vx, vy * vy));
        e_own[i][ch] = e;
        wx_s[(ty * TT::XW + j + 1) * CT + ch] = fmaf(g.rho, gx - vx, -mx);
        wy_s[((ty + 1) * TT::BW + j) * CT + ch] = fmaf(g.rho, gy - vy, -my);
      }
      const float tv = g.tv_mode == 0 ? sqrtf(vv) : tvs;
      acc += fmaf(0.5f * g.rho, pen, fmaf(0.5f * g.alpha, fid, tv));
    }
  }
  // Phase 1b: w at the halo cells that G^T can read (interior cells only: G is zero on
  // the first and last row and column, so w there never enters G^T w).
  const int tid = ty * kTvBX + tx;
  for (int h = tid; h < 2 * TT::BW + 2 * kTvBY; h += kTvBX * kTvBY) {
    if (h < 2 * TT::BW) {
      const int side = h / TT::BW, j = h - side * TT::BW;
      const int rr = side ? y0 + kTvBY : y0 - 1, q = x0 + j;
      if (rr >= 1 && rr <= g.H - 2 && q < g.W) {
        const size_t m = (size_t)rr * g.W + q;
#pragma unroll
        for (int ch = 0; ch < CT; ++ch)
          wy_s[((side ? TT::YH - 1 : 0) * TT::BW + j) * CT + ch] =
              fmaf(g.rho, grad_y(c, g, rr, q, CT, ch) - __ldg(v + m * 2 * CT + CT + ch),
                   -__ldg(mu + m * 2 * CT + CT + ch));
      }
    } else {
      const int hh = h - 2 * TT::BW, side = hh / kTvBY, t = hh - side * kTvBY;
      const int rr = y0 + t, q = side ? x0 + TT::BW : x0 - 1;
      if (rr < g.H && q >= 1 && q <= g.W - 2) {
        const size_t m = (size_t)rr * g.W + q;
#pragma unroll
        for (int ch = 0; ch < CT; ++ch)
          wx_s[(t * TT::XW + (side ? TT::XW - 1 : 0)) * CT + ch] =
              fmaf(g.rho, grad_x(c, g, rr, q, CT, ch) - __ldg(v + m * 2 * CT + ch),
                   -__ldg(mu + m * 2 * CT + ch));
      }
    }
  }
  __syncthreads();
  // Phase 2: lam = -dx dy [G^T w + alpha (c - c0)] from the shared w.
  if (r < g.H) {
#pragma unroll
    for (int i = 0; i < kPPT; ++i) {
      const int q = x0 + i * kTvBX + tx;
      if (q >= g.W) break;
      const size_t k = (size_t)r * g.W + q;
      const int j = q - x0;
#pragma unroll
      for (int ch = 0; ch < CT; ++ch) {
        float gtw = 0.0f;
        if (q - 1 >= 1) gtw = fmaf(wx_s[(ty * TT::XW + j) * CT + ch], g.inv2hx, gtw);
        if (q + 1 <= g.W - 2) gtw = fmaf(-wx_s[(ty * TT::XW + j + 2) * CT + ch], g.inv2hx, gtw);
        if (r - 1 >= 1) gtw = fmaf(wy_s[(ty * TT::BW + j) * CT + ch], g.inv2hy, gtw);
        if (r + 1 <= g.H - 2) gtw = fmaf(-wy_s[((ty + 2) * TT::BW + j) * CT + ch], g.inv2hy, gtw);
        lam[k * CT + ch] = -(float)g.cell * fmaf(g.alpha, e_own[i][ch], gtw);
      }
    }
  }
  return acc;
}

// The block's L~ share: the shared-w terminal form for C in {1, 3}, objective_block else.
template <int CT, bool LAMBDA>
__device__ __forceinline__ float objective_or_terminal(int bx, int by, const float* c,
                                                       const float* c0, const float* v,
                                                       const float* mu, float* lam,
                                                       const TvGeom& g) {
  if constexpr (LAMBDA && CT != 0) return terminal_block<CT>(bx, by, c, c0, v, mu, lam, g);
  else return objective_block<CT, LAMBDA>(bx, by, c, c0, v, mu, lam, g);
}

template <int CT, bool LAMBDA>
__global__ void __launch_bounds__(kTvBX * kTvBY)
objective_kernel(const float* __restrict__ c, const float* __restrict__ c0,
                 const float* __restrict__ v, const float* __restrict__ mu,
                 float* __restrict__ lam, double* __restrict__ partial, TvGeom g) {
  const float acc = objective_or_terminal<CT, LAMBDA>(blockIdx.x, blockIdx.y, c, c0, v, mu,
                                                      lam, g);
  __shared__ double red[32];
  double vals[1] = {(double)acc}, tot[1];
  block_sum<1>(vals, red, tot);
  if (threadIdx.x == 0 && threadIdx.y == 0)
    partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tot[0] * g.cell;
}

cudaError_t launch_objective(const float* c, const float* c0, const float* v, const float* mu,
                             float* lam, double* partial, const TvGeom& g, cudaStream_t s) {
  dim3 grid(cdiv(g.W, kTvBX * kPPT), cdiv(g.H, kTvBY)), block(kTvBX, kTvBY);
  if (g.C > kTvMaxC) return cudaErrorInvalidValue;
  if (lam) {
    if (g.C == 3) objective_kernel<3, true><<<grid, block, 0, s>>>(c, c0, v, mu, lam, partial, g);
    else if (g.C == 1) objective_kernel<1, true><<<grid, block, 0, s>>>(c, c0, v, mu, lam, partial, g);
    else objective_kernel<0, true><<<grid, block, 0, s>>>(c, c0, v, mu, lam, partial, g);
  } else {
    if (g.C == 3) objective_kernel<3, false><<<grid, block, 0, s>>>(c, c0, v, mu, lam, partial, g);
    else if (g.C == 1) objective_kernel<1, false><<<grid, block, 0, s>>>(c, c0, v, mu, lam, partial, g);
    else objective_kernel<0, false><<<grid, block, 0, s>>>(c, c0, v, mu, lam, partial, g);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ v-step (shrinkage)
// a = G c - mu/rho;  v = a * max(0, 1 - (1/rho)/|a|)  (v = 0 when |a| <= 1/rho).
template <int CT>
__device__ __forceinline__ void pd_tv_block(int bx, int by, const float* __restrict__ c,
                                            const float* __restrict__ mu,
                                            float* __restrict__ v, const TvGeom& g) {
  const int C = nch<CT>(g);
  const int r = by * kTvBY + threadIdx.y;
  if (r >= g.H) return;
  const float theta = g.inv_rho;
#pragma unroll
  for (int i = 0; i < kPPT; ++i) {
    const int q = bx * (kTvBX * kPPT) + i * kTvBX + threadIdx.x;
    if (q >= g.W) break;
    const size_t k = (size_t)r * g.W + q;
    const float* mk = mu + k * 2 * C;
    float* vk = v + k * 2 * C;
    if (g.tv_mode == 0) {
      float n2 = 0.0f;
      for (int ch = 0; ch < C; ++ch) {
        const float ax = fmaf(-__ldg(mk + ch), g.inv_rho, grad_x(c, g, r, q, C, ch));
        const float ay = fmaf(-__ldg(mk + C + ch), g.inv_rho, grad_y(c, g, r, q, C, ch));
        n2 = fmaf(ax, ax, fmaf(ay, ay, n2));
      }
      const float n = sqrtf(n2);
      const float f = n > theta ? 1.0f - theta / n : 0.0f;
      for (int ch = 0; ch < C; ++ch) {
        const float ax = fmaf(-__ldg(mk + ch), g.inv_rho, grad_x(c, g, r, q, C, ch));
        const float ay = fmaf(-__ldg(mk + C + ch), g.inv_rho, grad_y(c, g, r, q, C, ch));
        vk[ch] = ax * f;
        vk[C + ch] = ay * f;
      }
    } else {
      for (int ch = 0; ch < C; ++ch) {
        const float ax = fmaf(-__ldg(mk + ch), g.inv_rho, grad_x(c, g, r, q, C, ch));
        const float ay = fmaf(-__ldg(mk + C + ch), g.inv_rho, grad_y(c, g, r, q, C, ch));
        const float n = sqrtf(fmaf(ax, ax, ay * ay));
        const float f = n > theta ? 1.0f - theta / n : 0.0f;
        vk[ch] = ax * f;
        vk[C + ch] = ay * f;
      }
    }
  }
}

template <int CT>
__global__ void __launch_bounds__(kTvBX * kTvBY)
pd_tv_kernel(const float* __restrict__ c, const float* __restrict__ mu, float* __restrict__ v,
             TvGeom g) {
  pd_tv_block<CT>(blockIdx.x, blockIdx.y, c, mu, v, g);
}

cudaError_t launch_pd_tv_step(const float* c, const float* mu, float* v, const TvGeom& g,
                              cudaStream_t s) {
  if (g.C > kTvMaxC) return cudaErrorInvalidValue;
  dim3 grid(cdiv(g.W, kTvBX * kPPT), cdiv(g.H, kTvBY)), block(kTvBX, kTvBY);
  if (g.C == 3) pd_tv_kernel<3><<<grid, block, 0, s>>>(c, mu, v, g);
  else if (g.C == 1) pd_tv_kernel<1><<<grid, block, 0, s>>>(c, mu, v, g);
  else pd_tv_kernel<0><<<grid, block, 0, s>>>(c, mu, v, g);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ multiplier update
// mu <- mu + gamma (v - G c) with float64 arithmetic, rounded once to float32.  GB300's
// float64 pipe is narrow (about two lanes per SM and clock), so the residual
// R = v - k (c[+1] - c[-1]) (k = 1/(2 dx) or 1/(2 dy)) is formed with error-free float32
// transformations as an unevaluated pair s + lo (TwoSum of the difference, TwoProduct by
// k, TwoSum with v; |R - (s + lo)| is below 2^-46 max(|v|, |k (c[+1] - c[-1])|), where
// the float64 formula's own rounding is 2^-53 of the same), and the float64 pipe does only
// S = s + lo and mu + gamma S: two operations per component instead of five.  The
// conversions between the formats are the integer ones of fp_bits.cuh.  Every float32
// operation of the transformations is an explicitly rounded intrinsic, so the compiler
// cannot fuse or reorder them.  The result is the correctly rounded float32 value of the
// float64 update except when that value lies within about 2^-46 gamma max(|v|, |k dc|) of
// a rounding boundary, and within one float32 ulp of the exact update.
// Per-block partial sums: |v - Gc|^2, |G^T (v - v_prev)|^2, |c - c_prev|^2, |c|^2 and
// K(c)/(dx dy) = sum |G c_i| + alpha/2 |c_i - c0_i|^2 (float32 terms, float64 blocks).
struct ResidualPair {
  float s, lo;  // v - k (a - b) = s + lo (to 2^-46 of the larger operand)
  float g;      // k (a - b) rounded: the gradient component for K(c)
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

__device__ __forceinline__ ResidualPair residual_pair(float v, float a, float b, float k) {
  float d, de;
  two_sum(a, -b, d, de);               // a - b = d + de exactly
  const float p = __fmul_rn(k, d);
  const float pe = fmaf(k, d, -p);     // k d = p + pe exactly
  const float q = __fmul_rn(k, de);    // k de, |q| <= k ulp(d) / 2
  float s, t;
  two_sum(v, -p, s, t);                // v - p = s + t exactly
  return {s, __fsub_rn(__fsub_rn(t, pe), q), p};
}

// mu + gamma (s + lo) in float64.  Where every lane of the warp has lo = 0 (the residual
// is exactly a float32: the usual case on v = 0 pixels with a power-of-two 1/(2 dx)), the
// float64 addition forming s + lo is skipped.
__device__ __forceinline__ float mu_update(float mu, const ResidualPair& r, double gam) {
  double S = widen(r.s);
  if (__any_sync(__activemask(), r.lo != 0.0f)) S += widen(r.lo);
  return narrow(fma(gam, S, widen(mu)));
}

// Deterministic block sum of NV float32 partials per thread, in float64, with few
// float64 operations: the partials are staged in shared memory, NV * kSegs threads each
// add NT / kSegs consecutive ones (widened exactly with integer operations) in index
// order, and NV threads add those kSegs results in order.  Thread 0 receives the totals
// in out[] (other threads: unspecified).  Bitwise reproducible.
template <int NV, int NT>
__device__ __forceinline__ void block_sum_staged(const float (&v)[NV], double (&out)[NV]) {
  constexpr int kSegs = 8, kLen = NT / kSegs;
  static_assert(NT % kSegs == 0 && NV * kSegs <= NT, "block too small for the staged sum");
  __shared__ float part[NV * NT];
  __shared__ double seg[NV * kSegs];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
#pragma unroll
  for (int k = 0; k < NV; ++k) part[k * NT + tid] = v[k];
  __syncthreads();
  if (tid < NV * kSegs) {
    const float* p = part + (tid / kSegs) * NT + (tid % kSegs) * kLen;
    double acc = 0.0;
#pragma unroll 8
    for (int i = 0; i < kLen; ++i) acc += widen(p[i]);
    seg[tid] = acc;
  }
  __syncthreads();
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double acc = 0.0;
#pragma unroll
      for (int j = 0; j < kSegs; ++j) acc += seg[k * kSegs + j];
      out[k] = acc;
    }
  }
}

template <int CT>
__device__ __forceinline__ void alm_block(int bx, int by, const float* __restrict__ c,
                                          const float* __restrict__ c_prev,
                                          const float* __restrict__ c0,
                                          const float* __restrict__ v,
                                          const float* __restrict__ v_prev,
                                          float* __restrict__ mu, const TvGeom& g,
                                          float (&out)[5]) {
  const int C = nch<CT>(g);
  const int r = by * kTvBY + threadIdx.y;
  float a_r2 = 0.0f, a_s2 = 0.0f, a_dc2 = 0.0f, a_cn2 = 0.0f, a_K = 0.0f;
  const double gam = g.gamma;
  if (r < g.H) {
    // the gradient along an axis vanishes on its first and last index (and on sides of
    // length 1 or 2): there k = 0 and the neighbours are the pixel itself
    const bool yin = r >= 1 && r <= g.H - 2;
    const float ky = yin ? g.inv2hy : 0.0f;
    const int up = yin ? g.W : 0;
    prefetch_later_pixels<6>(bx, r, g, {v, mu, c, c0, c_prev, v_prev},
                             {2 * C, 2 * C, C, C, C, 2 * C});
#pragma unroll
    for (int i = 0; i < kPPT; ++i) {
      const int q = bx * (kTvBX * kPPT) + i * kTvBX + threadIdx.x;
      if (q >= g.W) break;
      const bool xin = q >= 1 && q <= g.W - 2;
      const float kx = xin ? g.inv2hx : 0.0f;
      const int rt = xin ? 1 : 0;
      const size_t k = (size_t)r * g.W + q;
      const float* ck = c + k * C;
      const float* vk = v + k * 2 * C;
      float* mk = mu + k * 2 * C;
      float gg2 = 0.0f, tvs = 0.0f, fid = 0.0f;
      for (int ch = 0; ch < C; ++ch) {
        const ResidualPair rx = residual_pair(__ldg(vk + ch), __ldg(ck + rt * C + ch),
                                              __ldg(ck - rt * C + ch), kx);
        const ResidualPair ry = residual_pair(__ldg(vk + C + ch),
                                              __ldg(ck + (size_t)up * C + ch),
                                              __ldg(ck - (size_t)up * C + ch), ky);
        mk[ch] = mu_update(mk[ch], rx, gam);
        mk[C + ch] = mu_update(mk[C + ch], ry, gam);
        a_r2 = fmaf(rx.s, rx.s, fmaf(ry.s, ry.s, a_r2));
        if (g.tv_mode == 0) gg2 = fmaf(rx.g, rx.g, fmaf(ry.g, ry.g, gg2));
        else tvs += sqrtf(fmaf(rx.g, rx.g, ry.g * ry.g));
        const float cc = __ldg(ck + ch);
        const float e = cc - __ldg(c0 + k * C + ch);
        fid = fmaf(e, e, fid);
        a_cn2 = fmaf(cc, cc, a_cn2);
        if (c_prev) {
          const float dc = cc - __ldg(c_prev + k * C + ch);
          a_dc2 = fmaf(dc, dc, a_dc2);
        }
        if (v_prev) {
          // (G^T (v - v_prev))_k
          float gt = 0.0f;
          if (q - 1 >= 1) {
            const size_t m = (k - 1) * 2 * C + ch;
            gt = fmaf(__ldg(v + m) - __ldg(v_prev + m), g.inv2hx, gt);
          }
          if (q + 1 <= g.W - 2) {
            const size_t m = (k + 1) * 2 * C + ch;
            gt = fmaf(-(__ldg(v + m) - __ldg(v_prev + m)), g.inv2hx, gt);
          }
          if (r - 1 >= 1) {
            const size_t m = (k - g.W) * 2 * C + C + ch;
            gt = fmaf(__ldg(v + m) - __ldg(v_prev + m), g.inv2hy, gt);
          }
          if (r + 1 <= g.H - 2) {
            const size_t m = (k + g.W) * 2 * C + C + ch;
            gt = fmaf(-(__ldg(v + m) - __ldg(v_prev + m)), g.inv2hy, gt);
          }
          a_s2 = fmaf(gt, gt, a_s2);
        }
      }
      const float tv = g.tv_mode == 0 ? sqrtf(gg2) : tvs;
      a_K += fmaf(0.5f * g.alpha, fid, tv);
    }
  }
  out[0] = a_r2; out[1] = a_s2; out[2] = a_dc2; out[3] = a_cn2; out[4] = a_K;
}

template <int CT>
__global__ void __launch_bounds__(kTvBX * kTvBY, 3)
alm_kernel(const float* __restrict__ c, const float* __restrict__ c_prev,
           const float* __restrict__ c0, const float* __restrict__ v,
           const float* __restrict__ v_prev, float* __restrict__ mu, double* __restrict__ partial,
           TvGeom g) {
  float a[5];
  alm_block<CT>(blockIdx.x, blockIdx.y, c, c_prev, c0, v, v_prev, mu, g, a);
  double tot[5];
  block_sum_staged<5, kTvBX * kTvBY>(a, tot);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int j = 0; j < 5; ++j) partial[5 * b + j] = tot[j];
  }
}

cudaError_t launch_alm_update(const float* c, const float* c_prev, const float* c0,
                              const float* v, const float* v_prev, float* mu, double* partial,
                              const TvGeom& g, cudaStream_t s) {
  if (g.C > kTvMaxC) return cudaErrorInvalidValue;
  dim3 grid(cdiv(g.W, kTvBX * kPPT), cdiv(g.H, kTvBY)), block(kTvBX, kTvBY);
  if (g.C == 3) alm_kernel<3><<<grid, block, 0, s>>>(c, c_prev, c0, v, v_prev, mu, partial, g);
  else if (g.C == 1) alm_kernel<1><<<grid, block, 0, s>>>(c, c_prev, c0, v, v_prev, mu, partial, g);
  else alm_kernel<0><<<grid, block, 0, s>>>(c, c_prev, c0, v, v_prev, mu, partial, g);
  return cudaGetLastError();
}

// stats = {sqrt(r2), rho sqrt(s2), gamma dx dy r2, sqrt(dc2 / cn2), dx dy K} from the raw
// sums {r2, s2, dc2, cn2, K} (one thread).
__global__ void alm_finalize_kernel(const double* __restrict__ raw, double* __restrict__ st,
                                    double rho, double gamma, double cell) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  st[0] = sqrt(raw[0]);
  st[1] = rho * sqrt(raw[1]);
  st[2] = gamma * cell * raw[0];
  st[3] = raw[3] > 0.0 ? sqrt(raw[2] / raw[3]) : 0.0;
  st[4] = cell * raw[4];
}

cudaError_t launch_alm_finalize(const double* raw, double* stats, double rho, double gamma,
                                double cell, cudaStream_t s) {
  alm_finalize_kernel<<<1, 32, 0, s>>>(raw, stats, rho, gamma, cell);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ reductions
constexpr int kRedThreads = 256;

__global__ void __launch_bounds__(kRedThreads)
reduce_rows_kernel(const double* __restrict__ partial, int nblocks, int nv, double scale,
                   double* __restrict__ out) {
  const int n = blockIdx.x;
  __shared__ double red[32];
  for (int k = 0; k < nv; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kRedThreads)
      s += partial[((size_t)n * nblocks + b) * nv + k];
    double vals[1] = {s}, tot[1];
    block_sum<1>(vals, red, tot);
    if (threadIdx.x == 0) out[(size_t)n * nv + k] = tot[0] * scale;
    __syncthreads();
  }
}

cudaError_t launch_reduce_rows(const double* partial, int nblocks, int nv, int rows,
                               double scale, double* out, cudaStream_t s) {
  reduce_rows_kernel<<<rows, kRedThreads, 0, s>>>(partial, nblocks, nv, scale, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ batched
int tv_block_w() { return kTvBX * kPPT; }
int tv_block_h() { return kTvBY; }

template <int CT, bool LAMBDA>
__global__ void __launch_bounds__(kTvBX * kTvBY)
objective_batch_kernel(const BatchTvArgs* __restrict__ args, const BatchJob* __restrict__ jobs,
                       int njobs, const int* __restrict__ active) {
  __shared__ double red[32];
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchTvArgs& a = args[job.img];
    const float acc = objective_or_terminal<CT, LAMBDA>(job.tx, job.ty, a.c, a.c0, a.v, a.mu,
                                                        a.lam, a.g);
    double vals[1] = {(double)acc}, tot[1];
    block_sum<1>(vals, red, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0)
      a.partial[(size_t)job.ty * a.tiles_x + job.tx] = tot[0] * a.g.cell;
    __syncthreads();
  }
}

template <int CT>
__global__ void __launch_bounds__(kTvBX * kTvBY)
pd_tv_batch_kernel(const BatchTvArgs* __restrict__ args, const BatchJob* __restrict__ jobs,
                   int njobs, const int* __restrict__ active) {
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchTvArgs& a = args[job.img];
    pd_tv_block<CT>(job.tx, job.ty, a.c, a.mu, a.v_out, a.g);
  }
}

template <int CT>
__global__ void __launch_bounds__(kTvBX * kTvBY, 3)
alm_batch_kernel(const BatchTvArgs* __restrict__ args, const BatchJob* __restrict__ jobs,
                 int njobs, const int* __restrict__ active) {
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchTvArgs& a = args[job.img];
    float o[5];
    alm_block<CT>(job.tx, job.ty, a.c, a.c_prev, a.c0, a.v, a.v_prev, a.mu_io, a.g, o);
    double tot[5];
    block_sum_staged<5, kTvBX * kTvBY>(o, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const size_t b = (size_t)job.ty * a.tiles_x + job.tx;
#pragma unroll
      for (int k = 0; k < 5; ++k) a.partial[5 * b + k] = tot[k];
    }
    __syncthreads();
  }
}

static int tv_batch_grid(int njobs) { return njobs < 8192 ? njobs : 8192; }

cudaError_t launch_objective_batch(const BatchTvArgs* args, const BatchJob* jobs, int njobs,
                                   const int* active, int C, bool lambda, cudaStream_t s) {
  const int grid = tv_batch_grid(njobs);
  if (grid <= 0) return cudaSuccess;
  const dim3 block(kTvBX, kTvBY);
  if (C > kTvMaxC) return cudaErrorInvalidValue;
  if (lambda) {
    if (C == 3) objective_batch_kernel<3, true><<<grid, block, 0, s>>>(args, jobs, njobs, active);
    else if (C == 1) objective_batch_kernel<1, true><<<grid, block, 0, s>>>(args, jobs, njobs, active);
    else objective_batch_kernel<0, true><<<grid, block, 0, s>>>(args, jobs, njobs, active);
  } else {
    if (C == 3) objective_batch_kernel<3, false><<<grid, block, 0, s>>>(args, jobs, njobs, active);
    else if (C == 1) objective_batch_kernel<1, false><<<grid, block, 0, s>>>(args, jobs, njobs, active);
    else objective_batch_kernel<0, false><<<grid, block, 0, s>>>(args, jobs, njobs, active);
  }
  return cudaGetLastError();
}

cudaError_t launch_pd_tv_batch(const BatchTvArgs* args, const BatchJob* jobs, int njobs,
                               const int* active, int C, cudaStream_t s) {
  const int grid = tv_batch_grid(njobs);
  if (grid <= 0) return cudaSuccess;
  const dim3 block(kTvBX, kTvBY);
  if (C > kTvMaxC) return cudaErrorInvalidValue;
  if (C == 3) pd_tv_batch_kernel<3><<<grid, block, 0, s>>>(args, jobs, njobs, active);
  else if (C == 1) pd_tv_batch_kernel<1><<<grid, block, 0, s>>>(args, jobs, njobs, active);
  else pd_tv_batch_kernel<0><<<grid, block, 0, s>>>(args, jobs, njobs, active);
  return cudaGetLastError();
}

cudaError_t launch_alm_batch(const BatchTvArgs* args, const BatchJob* jobs, int njobs,
                             const int* active, int C, cudaStream_t s) {
  const int grid = tv_batch_grid(njobs);
  if (grid <= 0) return cudaSuccess;
  const dim3 block(kTvBX, kTvBY);
  if (C > kTvMaxC) return cudaErrorInvalidValue;
  if (C == 3) alm_batch_kernel<3><<<grid, block, 0, s>>>(args, jobs, njobs, active);
  else if (C == 1) alm_batch_kernel<1><<<grid, block, 0, s>>>(args, jobs, njobs, active);
  else alm_batch_kernel<0><<<grid, block, 0, s>>>(args, jobs, njobs, active);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRedThreads)
reduce_segments_kernel(const ReduceSeg* __restrict__ segs, int nv) {
  const int n = blockIdx.x;
  const ReduceSeg sg = segs[blockIdx.y];
  __shared__ double red[32];
  for (int k = 0; k < nv; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < sg.nblocks; b += kRedThreads)
      s += sg.partial[((size_t)n * sg.nblocks + b) * nv + k];
    double vals[1] = {s}, tot[1];
    block_sum<1>(vals, red, tot);
    if (threadIdx.x == 0) sg.out[(size_t)n * nv + k] = tot[0] * sg.scale;
    __syncthreads();
  }
}

cudaError_t launch_reduce_segments(const ReduceSeg* segs, int nseg, int nv, int rows,
                                   cudaStream_t s) {
  if (nseg <= 0 || rows <= 0) return cudaSuccess;
  reduce_segments_kernel<<<dim3(rows, nseg), kRedThreads, 0, s>>>(segs, nv);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ control step
// trial = Pi_E(eps + tau D): componentwise clip onto the box E (Algorithm 1).
__global__ void control_step_kernel(const double* __restrict__ eps, const double* __restrict__ D,
                                    double tau, const double* __restrict__ lo_hi,
                                    double* __restrict__ trial, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = i & 1;
    const double e = fma(tau, D[i], eps[i]);
    trial[i] = fmin(fmax(e, lo_hi[k]), lo_hi[2 + k]);
  }
}

// y = a x over n floats (16-byte aligned fields: four at a time, then the tail).
__global__ void scale_f32_kernel(const float* __restrict__ x, float a, float* __restrict__ y,
                                 size_t n) {
  const size_t n4 = n / 4;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
    const float4 v = reinterpret_cast<const float4*>(x)[i];
    reinterpret_cast<float4*>(y)[i] = make_float4(a * v.x, a * v.y, a * v.z, a * v.w);
  }
  for (size_t i = 4 * n4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    y[i] = a * x[i];
}

cudaError_t launch_scale_f32(const float* x, float a, float* y, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t want = (n / 4 + 255) / 256;
  const int grid = (int)std::max<size_t>(1, std::min<size_t>(want, (size_t)sms * 8));
  scale_f32_kernel<<<grid, 256, 0, s>>>(x, a, y, n);
  return cudaGetLastError();
}

cudaError_t launch_control_step(const double* eps, const double* D, double tau,
                                const double* lo_hi, double* trial, int T, cudaStream_t s) {
  const int n = 2 * T;
  control_step_kernel<<<cdiv(n, 256), 256, 0, s>>>(eps, D, tau, lo_hi, trial, n);
  return cudaGetLastError();
}

}  // namespace agents
