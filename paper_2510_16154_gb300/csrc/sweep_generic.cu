// Agent sweep kernels for any window radius and channel count (up to 64 channels): one
// thread per pixel, the window clipped to the image by the loop bounds.
#include "sweep.cuh"

namespace agents {

__device__ __forceinline__ void forward_generic_pixel(const float* __restrict__ c,
                                                      float* __restrict__ out,
                                                      const double* __restrict__ eps_n,
                                                      const SweepGeom& g, int q, int r) {
  if (q >= g.W || r >= g.H) return;
  const int C = g.C, R = g.R;
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
  const float* ci = c + ((size_t)r * g.W + q) * C;
  float acc[kGenericMaxC];
  for (int ch = 0; ch < C; ++ch) acc[ch] = 0.0f;
  const int y0 = max(r - R, 0), y1 = min(r + R, g.H - 1);
  const int x0 = max(q - R, 0), x1 = min(q + R, g.W - 1);
  for (int y = y0; y <= y1; ++y) {
    const int dy = y - r;
    const float sy = ky * (float)(dy * dy);
    for (int x = x0; x <= x1; ++x) {
      const int dx = x - q;
      const float* cj = c + ((size_t)y * g.W + x) * C;
      float s2 = 0.0f;
      for (int ch = 0; ch < C; ++ch) {
        const float d = cj[ch] - ci[ch];
        s2 = fmaf(d, d, s2);
      }
      const float ph = wendland_phi(fmaf(kc, s2, fmaf(kx, (float)(dx * dx), sy)));
      for (int ch = 0; ch < C; ++ch) acc[ch] = fmaf(ph, cj[ch] - ci[ch], acc[ch]);
    }
  }
  float* o = out + ((size_t)r * g.W + q) * C;
  for (int ch = 0; ch < C; ++ch) o[ch] = fmaf(g.scale, acc[ch], ci[ch]);
}

__global__ void forward_generic_kernel(const float* __restrict__ c, float* __restrict__ out,
                                       const double* __restrict__ eps_n, SweepGeom g) {
  forward_generic_pixel(c, out, eps_n, g, blockIdx.x * blockDim.x + threadIdx.x,
                        blockIdx.y * blockDim.y + threadIdx.y);
}

// One pixel of the adjoint step; returns its D partial sums in Dx, Dc (the paired form
// of adjoint_body: the caller scales them by -1/2).
__device__ __forceinline__ void adjoint_generic_pixel(const float* __restrict__ c,
                                                      const float* __restrict__ lam,
                                                      float* __restrict__ out,
                                                      const double* __restrict__ eps_n,
                                                      const SweepGeom& g, int q, int r,
                                                      float& Dx, float& Dc) {
  Dx = 0.0f;
  Dc = 0.0f;
  if (q < g.W && r < g.H) {
    const int C = g.C, R = g.R;
    const float ex = (float)eps_n[0], ec = (float)eps_n[1];
    const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
    const size_t k = (size_t)r * g.W + q;
    const float* ck = c + k * C;
    const float* lk = lam + k * C;
    float acc[kGenericMaxC];
    for (int ch = 0; ch < C; ++ch) acc[ch] = 0.0f;
    const int y0 = max(r - R, 0), y1 = min(r + R, g.H - 1);
    const int x0 = max(q - R, 0), x1 = min(q + R, g.W - 1);
    for (int y = y0; y <= y1; ++y) {
      const int dy = y - r;
      for (int x = x0; x <= x1; ++x) {
        const int dx = x - q;
        const size_t j = (size_t)y * g.W + x;
        const float* cj = c + j * C;
        const float* lj = lam + j * C;
        float s2 = 0.0f, proj = 0.0f;
        for (int ch = 0; ch < C; ++ch) {
          const float d = cj[ch] - ck[ch];
          s2 = fmaf(d, d, s2);
          proj = fmaf(d, lj[ch] - lk[ch], proj);
        }
        const float sp = fmaf(kx, (float)(dx * dx), ky * (float)(dy * dy));
        float ph, dph;
        wendland_phi_dphi(fmaf(kc, s2, sp), ph, dph);
        const float gk = dph * proj;      // D in the paired form of adjoint_body
        const float coef = gk * ec;
        for (int ch = 0; ch < C; ++ch) {
          const float d = cj[ch] - ck[ch];
          acc[ch] = fmaf(coef, d, acc[ch]);
          acc[ch] = fmaf(ph, lj[ch] - lk[ch], acc[ch]);
        }
        const float d2 = fmaf(g.inv_w2, (float)(dx * dx), g.inv_h2 * (float)(dy * dy));
        Dx = fmaf(gk, d2, Dx);
        Dc = fmaf(gk, s2, Dc);
      }
    }
    float* o = out + k * C;
    for (int ch = 0; ch < C; ++ch) o[ch] = fmaf(g.scale, acc[ch], lk[ch]);
  }
}

__global__ void adjoint_generic_kernel(const float* __restrict__ c,
                                       const float* __restrict__ lam, float* __restrict__ out,
                                       const double* __restrict__ eps_n,
                                       double* __restrict__ partial, SweepGeom g) {
  float Dx, Dc;
  adjoint_generic_pixel(c, lam, out, eps_n, g, blockIdx.x * blockDim.x + threadIdx.x,
                        blockIdx.y * blockDim.y + threadIdx.y, Dx, Dc);
  __shared__ double red[2 * 32];
  double v[2] = {-0.5 * (double)Dx, -0.5 * (double)Dc};
  double tot[2];
  block_sum<2>(v, red, tot);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    partial[2 * b + 0] = tot[0];
    partial[2 * b + 1] = tot[1];
  }
}

// ------------------------------------------------------------------ batched
__global__ void forward_generic_batch_kernel(const BatchSweepImg* __restrict__ imgs,
                                             const BatchJob* __restrict__ jobs, int njobs,
                                             const int* __restrict__ active, int n, int kind) {
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchSweepImg& im = imgs[job.img];
    const SweepGeom g = im.g;
    const size_t nc = (size_t)g.H * g.W * g.C;
    const float* src;
    float* dst;
    const double* eps_n;
    if (kind == kSweepStore) {
      src = n == 0 ? im.c0 : im.traj + (size_t)(n - 1) * nc;
      dst = n == im.nsteps - 1 ? im.cT : im.traj + (size_t)n * nc;
      eps_n = im.eps + 2 * n;
    } else {
      src = n == 0 ? im.c0 : ((n - 1) & 1 ? im.work1 : im.work0);
      dst = n == im.nsteps - 1 ? im.trial_c : (n & 1 ? im.work1 : im.work0);
      eps_n = im.trial_eps + 2 * n;
    }
    forward_generic_pixel(src, dst, eps_n, g, job.tx * blockDim.x + threadIdx.x,
                          job.ty * blockDim.y + threadIdx.y);
  }
}

__global__ void adjoint_generic_batch_kernel(const BatchSweepImg* __restrict__ imgs,
                                             const BatchJob* __restrict__ jobs, int njobs,
                                             const int* __restrict__ active, int n) {
  __shared__ double red[2 * 32];
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchSweepImg& im = imgs[job.img];
    const SweepGeom g = im.g;
    const size_t nc = (size_t)g.H * g.W * g.C;
    const int li = (im.nsteps - 1 - n) & 1;
    const float* lin = li ? im.lam1 : im.lam0;
    float* lout = li ? im.lam0 : im.lam1;
    const float* cn = n == 0 ? im.c0 : im.traj + (size_t)(n - 1) * nc;
    float Dx, Dc;
    adjoint_generic_pixel(cn, lin, lout, im.eps + 2 * n, g, job.tx * blockDim.x + threadIdx.x,
                          job.ty * blockDim.y + threadIdx.y, Dx, Dc);
    double v[2] = {-0.5 * (double)Dx, -0.5 * (double)Dc};
    double tot[2];
    block_sum<2>(v, red, tot);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const int tiles_x = (g.W + blockDim.x - 1) / blockDim.x;
      double* part = im.part_adj + ((size_t)n * im.ntiles + (size_t)job.ty * tiles_x + job.tx) * 2;
      part[0] = tot[0];
      part[1] = tot[1];
    }
    __syncthreads();
  }
}

}  // namespace agents
