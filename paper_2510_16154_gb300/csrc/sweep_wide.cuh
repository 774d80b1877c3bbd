// Agent sweep kernels for wide channel counts (hyperspectral images, C = 31): one pixel
// per thread on 32 x 4 pixel tiles, every channel of the tile and its halo staged in
// channel-planar shared memory (plane ch holds channel ch of the tile), and the channel
// loop unrolled in registers.  Each interaction reads C floats of the neighbour from
// shared memory and does about 3C FMAs, so the kernels sit near the balance of the
// shared-memory and FP32 rates.  Tile loads read each tile row as one flat, coalesced
// NHWC segment; the results are staged back through shared memory and stored the same
// way.  The 32 x 4 tile is the generic kernels' tile, so per-tile partial sums and batch
// job lists are laid out alike (32 x 8 tiles for R <= 6: see wide_by).
#pragma once

#include "sweep.cuh"

namespace agents {

constexpr int kWideBX = 32, kWideBY = 4;
constexpr int kWideC = 31;          // the channel count with a wide instantiation

// R <= 7: the adjoint's two fields and validity plane of a 32 x 4 tile with an R = 8 halo
// would need 242 KB of shared memory (227 KB per block at most).
inline bool wide_shape(int R, int C) { return R >= 1 && R <= 7 && C == kWideC; }

// Tile height: 8 rows where the adjoint's tile of both fields still fits (R <= 6: 190 KB
// at R = 5, 222 KB at R = 6), else 4.  Taller tiles load fewer halo cells per output
// pixel and run twice the warps per block.
template <int R>
constexpr int wide_by() { return R <= 6 ? 8 : kWideBY; }
inline int wide_tile_h(int R) { return R <= 6 ? 8 : kWideBY; }

template <int R, int C>
struct Wide {
  static constexpr int TW = kWideBX, TH = wide_by<R>(), NT = kWideBX * wide_by<R>();
  static constexpr int SW = TW + 2 * R, SH = TH + 2 * R, PLANE = SW * SH;
  // planes: NF fields x C channels, then the validity plane
  static constexpr size_t smem(int nf) { return (size_t)(nf * C + 1) * PLANE * sizeof(float); }
};

// 4-byte asynchronous copy global -> shared: a thread issues all its copies of a tile
// without waiting on each load, and waits once (wide_load_wait).
__device__ __forceinline__ void wide_cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// Stage NF fields (NHWC, C channels) of the tile at (x0, y0) plus its halo.  Cells outside
// the image hold 0 and, when the halo leaves the image, the validity plane marks them 0.
template <class T, int R, int C, int NF>
__device__ __forceinline__ bool wide_load(float* __restrict__ sm, const float* __restrict__ f0,
                                          const float* __restrict__ f1, const SweepGeom& g,
                                          int x0, int y0) {
  const bool border = (x0 - R < 0) || (y0 - R < 0) || (x0 + T::TW + R > g.W) ||
                      (y0 + T::TH + R > g.H);
  float* mask = sm + NF * C * T::PLANE;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int gx0 = x0 - R;
  const int xa = max(0, -gx0), xb = min(T::SW, g.W - gx0);   // valid columns [xa, xb)
  for (int yy = 0; yy < T::SH; ++yy) {
    const int gy = y0 - R + yy;
    const bool rowok = gy >= 0 && gy < g.H;
    const int nval = (rowok && xb > xa) ? (xb - xa) * C : 0;
    const size_t base = rowok ? ((size_t)gy * g.W + (gx0 + xa)) * C : 0;
    float* row = sm + yy * T::SW + xa;
    for (int f = tid; f < nval; f += T::NT) {
      const int px = f / C, ch = f - px * C;
      wide_cp_async4(row + ch * T::PLANE + px, f0 + base + f);
      if constexpr (NF == 2) wide_cp_async4(row + (C + ch) * T::PLANE + px, f1 + base + f);
    }
    for (int xx = tid; xx < T::SW; xx += T::NT) {
      const bool ok = rowok && xx >= xa && xx < xb;
      if (!ok) {
#pragma unroll 4
        for (int ch = 0; ch < NF * C; ++ch) sm[ch * T::PLANE + yy * T::SW + xx] = 0.0f;
      }
      if (border) mask[yy * T::SW + xx] = ok ? 1.0f : 0.0f;
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  return border;
}

// Write the tile's results (val[C] per thread) to out (NHWC) through shared memory, so
// that every tile row is stored as one flat segment.  `stage` needs TW*TH*C floats.
template <class T, int C>
__device__ __forceinline__ void wide_store(float* __restrict__ stage, const float (&val)[C],
                                           float* __restrict__ out, const SweepGeom& g, int x0,
                                           int y0) {
  __syncthreads();                                   // the tile data is no longer needed
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int ch = 0; ch < C; ++ch) stage[(ty * T::TW + tx) * C + ch] = val[ch];
  __syncthreads();
  const int tid = ty * blockDim.x + tx;
  const int ncol = min(T::TW, g.W - x0);
  for (int r = 0; r < T::TH; ++r) {
    const int gy = y0 + r;
    if (gy >= g.H) break;
    float* dst = out + ((size_t)gy * g.W + x0) * C;
    const float* src = stage + r * T::TW * C;
    for (int f = tid; f < ncol * C; f += T::NT) dst[f] = src[f];
  }
}

// Forward step of the pixel at (x0 + tx, y0 + ty): c + dt/M sum_j phi(r_kj) (c_j - c_k).
template <class T, int R, int C, bool BORDER>
__device__ __forceinline__ void wide_forward_body(float* __restrict__ sm, float* __restrict__ out,
                                                  const SweepGeom& g, float kx, float ky,
                                                  float kc, int x0, int y0) {
  const float* mask = sm + C * T::PLANE;
  const int cen = (threadIdx.y + R) * T::SW + threadIdx.x + R;
  float ci[C], acc[C];
#pragma unroll
  for (int ch = 0; ch < C; ++ch) {
    ci[ch] = sm[ch * T::PLANE + cen];
    acc[ch] = 0.0f;
  }
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
    const float sy = fmaf(-ky, (float)(dy * dy), 1.0f);
#pragma unroll 1
    for (int dx = -R; dx <= R; ++dx) {
      const int e = cen + dy * T::SW + dx;
      float d[C];
      float s2p[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // four independent chains
#pragma unroll
      for (int ch = 0; ch < C; ++ch) {
        d[ch] = sm[ch * T::PLANE + e] - ci[ch];
        s2p[ch & 3] = fmaf(d[ch], d[ch], s2p[ch & 3]);
      }
      const float s2 = (s2p[0] + s2p[1]) + (s2p[2] + s2p[3]);
      const float t = fmaxf(fmaf(-kc, s2, fmaf(-kx, (float)(dx * dx), sy)), 0.0f);
      const float t2 = t * t;
      float ph = (t2 * t2) * fmaf(-4.0f, t, 5.0f);
      if constexpr (BORDER) ph *= mask[e];
#pragma unroll
      for (int ch = 0; ch < C; ++ch) acc[ch] = fmaf(ph, d[ch], acc[ch]);
    }
  }
#pragma unroll
  for (int ch = 0; ch < C; ++ch) acc[ch] = fmaf(g.scale, acc[ch], ci[ch]);
  wide_store<T, C>(sm, acc, out, g, x0, y0);
}

// Adjoint step (gather form, as adjoint_body): lam_k + dt/M sum_j [phi' eps_c delta
// (delta . dlam) + phi dlam]; the block's D partial sums go to partial[0..1].
template <class T, int R, int C, bool BORDER>
__device__ __forceinline__ void wide_adjoint_body(float* __restrict__ sm, float* __restrict__ out,
                                                  double* __restrict__ partial, const SweepGeom& g,
                                                  float kx, float ky, float kc, float ec, int x0,
                                                  int y0) {
  const float* sc = sm;
  const float* sl = sm + C * T::PLANE;
  const float* mask = sm + 2 * C * T::PLANE;
  const int cen = (threadIdx.y + R) * T::SW + threadIdx.x + R;
  float ck[C], lk[C], acc[C];
#pragma unroll
  for (int ch = 0; ch < C; ++ch) {
    ck[ch] = sc[ch * T::PLANE + cen];
    lk[ch] = sl[ch * T::PLANE + cen];
    acc[ch] = 0.0f;
  }
  const float ec20 = 20.0f * ec;
  float Dx = 0.0f, Dc = 0.0f;
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
    const float sy = fmaf(-ky, (float)(dy * dy), 1.0f);
    const float d2y = g.inv_h2 * (float)(dy * dy);
#pragma unroll 1
    for (int dx = -R; dx <= R; ++dx) {
      const int e = cen + dy * T::SW + dx;
      float d[C], dl[C];
      // each channel sum in four independent chains (latency of the FMA chains)
      float s2p[4] = {0.0f, 0.0f, 0.0f, 0.0f}, pp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      float lp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ch = 0; ch < C; ++ch) {
        d[ch] = sc[ch * T::PLANE + e] - ck[ch];
        dl[ch] = sl[ch * T::PLANE + e] - lk[ch];
        s2p[ch & 3] = fmaf(d[ch], d[ch], s2p[ch & 3]);
        pp[ch & 3] = fmaf(d[ch], dl[ch], pp[ch & 3]);
        lp[ch & 3] = fmaf(lk[ch], d[ch], lp[ch & 3]);
      }
      const float s2 = (s2p[0] + s2p[1]) + (s2p[2] + s2p[3]);
      const float proj = (pp[0] + pp[1]) + (pp[2] + pp[3]);
      const float lkd = (lp[0] + lp[1]) + (lp[2] + lp[3]);
      const float t = fmaxf(fmaf(-kc, s2, fmaf(-kx, (float)(dx * dx), sy)), 0.0f);
      const float t2 = t * t, t3 = t2 * t;
      float ph = (t2 * t2) * fmaf(-4.0f, t, 5.0f);
      float dph = t3 * (t - 1.0f);                       // phi' / 20
      if constexpr (BORDER) {
        ph *= mask[e];
        dph *= mask[e];
      }
      const float coef = (dph * ec20) * proj;
#pragma unroll
      for (int ch = 0; ch < C; ++ch) acc[ch] = fmaf(ph, dl[ch], fmaf(coef, d[ch], acc[ch]));
      const float gk = dph * lkd;
      Dx = fmaf(gk, fmaf(g.inv_w2, (float)(dx * dx), d2y), Dx);
      Dc = fmaf(gk, s2, Dc);
    }
  }
#pragma unroll
  for (int ch = 0; ch < C; ++ch) acc[ch] = fmaf(g.scale, acc[ch], lk[ch]);
  __shared__ double red[2 * 32];
  double v[2] = {20.0 * (double)Dx, 20.0 * (double)Dc};
  double tot[2];
  block_sum<2>(v, red, tot);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    partial[0] = tot[0];
    partial[1] = tot[1];
  }
  wide_store<T, C>(sm, acc, out, g, x0, y0);
}

template <int R, int C>
__global__ void __launch_bounds__(kWideBX * wide_by<R>())
wide_forward_kernel(const float* __restrict__ c, float* __restrict__ out,
                    const double* __restrict__ eps_n, SweepGeom g) {
  using T = Wide<R, C>;
  extern __shared__ __align__(16) float wsm[];
  const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
  if (wide_load<T, R, C, 1>(wsm, c, nullptr, g, x0, y0))
    wide_forward_body<T, R, C, true>(wsm, out, g, kx, ky, kc, x0, y0);
  else
    wide_forward_body<T, R, C, false>(wsm, out, g, kx, ky, kc, x0, y0);
}

template <int R, int C>
__global__ void __launch_bounds__(kWideBX * wide_by<R>())
wide_adjoint_kernel(const float* __restrict__ c, const float* __restrict__ lam,
                    float* __restrict__ out, const double* __restrict__ eps_n,
                    double* __restrict__ partial, SweepGeom g) {
  using T = Wide<R, C>;
  extern __shared__ __align__(16) float wsm[];
  const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
  double* part = partial + 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
  if (wide_load<T, R, C, 2>(wsm, c, lam, g, x0, y0))
    wide_adjoint_body<T, R, C, true>(wsm, out, part, g, kx, ky, kc, ec, x0, y0);
  else
    wide_adjoint_body<T, R, C, false>(wsm, out, part, g, kx, ky, kc, ec, x0, y0);
}

// Batched (persistent) versions: step n of every (image, tile) job of the batch.
template <int R, int C>
__global__ void __launch_bounds__(kWideBX * wide_by<R>())
wide_forward_batch_kernel(const BatchSweepImg* __restrict__ imgs, const BatchJob* __restrict__ jobs,
                          int njobs, const int* __restrict__ active, int n, int kind) {
  using T = Wide<R, C>;
  extern __shared__ __align__(16) float wsm[];
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
    const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
    if (wide_load<T, R, C, 1>(wsm, src, nullptr, g, x0, y0))
      wide_forward_body<T, R, C, true>(wsm, dst, g, kx, ky, kc, x0, y0);
    else
      wide_forward_body<T, R, C, false>(wsm, dst, g, kx, ky, kc, x0, y0);
    __syncthreads();
  }
}

template <int R, int C>
__global__ void __launch_bounds__(kWideBX * wide_by<R>())
wide_adjoint_batch_kernel(const BatchSweepImg* __restrict__ imgs, const BatchJob* __restrict__ jobs,
                          int njobs, const int* __restrict__ active, int n) {
  using T = Wide<R, C>;
  extern __shared__ __align__(16) float wsm[];
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
    const int tiles_x = (g.W + T::TW - 1) / T::TW;
    double* part = im.part_adj + ((size_t)n * im.ntiles + (size_t)job.ty * tiles_x + job.tx) * 2;
    if (wide_load<T, R, C, 2>(wsm, batch_state(im, n), lin, g, x0, y0))
      wide_adjoint_body<T, R, C, true>(wsm, lout, part, g, kx, ky, kc, ec, x0, y0);
    else
      wide_adjoint_body<T, R, C, false>(wsm, lout, part, g, kx, ky, kc, ec, x0, y0);
    __syncthreads();
  }
}

// Launchers (sweep_wide.cu).
cudaError_t launch_wide_forward(const float* c_in, float* c_out, const double* eps_n,
                                const SweepGeom& g, cudaStream_t s);
cudaError_t launch_wide_adjoint(const float* c_n, const float* lam_next, float* lam_out,
                                const double* eps_n, double* partial, const SweepGeom& g,
                                cudaStream_t s);
cudaError_t launch_wide_forward_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                      const int* active, int n, int kind, int R, cudaStream_t s);
cudaError_t launch_wide_adjoint_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                      const int* active, int n, int R, cudaStream_t s);

}  // namespace agents
