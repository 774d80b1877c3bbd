// Whole agent sweeps in one persistent launch (dataflow between tiles).
//
// One launch per Euler or adjoint step ends every step with a ramp-down (the last tiles
// of the step run on a partly idle GPU) and starts the next with a ramp-up (every block
// staging its tile at once); at 1024^2 that costs about a sixth of each step.  Here a
// grid of resident blocks takes (step, tile) jobs in step-major order from one counter.
// A job of step k needs the step-(k - 1) outputs of the 3 x 3 tiles around its own (used
// only where the window radius is at most the tile height and width, so that the halo
// reaches no further), and waits
// for their completion flags; tiles of step k start while the last tiles of step k - 1
// are still running.
//
// Deadlock freedom: jobs are taken in increasing order, and a job only waits for jobs
// with smaller indices, all of which have been taken by blocks that are running; the
// oldest unfinished job therefore never waits.  The waits are still bounded in time
// (FusedSync::wait_ns); one that runs out sets *status and the launch winds down
// (every block checks the status before each job and while it waits).
//
// Write-after-read: job (k, t) overwrites its tile of a buffer that the neighbours'
// jobs of earlier steps may read.  It starts only after the 3 x 3 neighbours finished
// step k - 1, and each of those waited for its own neighbours at k - 2, which include
// every tile that reads t's region; so no earlier reader is still running.
//
// Memory ordering: every thread fences its stores, the block synchronises, and one
// thread publishes the flag with a release store; waiters read flags with acquire
// loads, synchronise the block, and all inputs written during the launch are read
// through L2 (ld.global.cg), never the non-coherent path.
#pragma once

#include "sweep.cuh"

namespace agents {

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sequence numbers wrap; a flag has reached `target` when it is at most 2^31 - 1 past it.
__device__ __forceinline__ bool seq_reached(unsigned int flag, unsigned int target) {
  return (int)(flag - target) >= 0;
}

// Wait until *flag reaches target.  Returns false when the launch gives up: the status
// was set by another block, or this wait ran out of time (then it sets the status).
// Polls at most kMaxPolls times as a second bound should the timer not advance.  The
// pause between polls doubles from 64 ns to 1 us, so that many waiting blocks do not load
// L2 with polls while the job they wait for still runs.
__device__ __forceinline__ bool wait_flag(const unsigned int* flag, unsigned int target,
                                          unsigned int* status, long long wait_ns) {
  if (seq_reached(ld_acquire_u32(flag), target)) return true;
  constexpr int kMaxPolls = 1 << 24;
  const unsigned long long t0 = global_ns();
  unsigned int pause = 64;
  for (int it = 0; it < kMaxPolls; ++it) {
    __nanosleep(pause);
    if (pause < 1024) pause *= 2;
    if (seq_reached(ld_acquire_u32(flag), target)) return true;
    if (ld_relaxed_u32(status) != 0) return false;
    if ((long long)(global_ns() - t0) > wait_ns) break;
  }
  atomicCAS(status, 0u, 1u);
  return false;
}

// The job loop shared by the fused forward and adjoint kernels.  body(k, tx, ty) stages,
// computes and stores one tile of step k; it may use __syncthreads.  The job's
// coordinates live in shared memory, not in registers across the body, so that the loop
// adds nothing to the tile body's register budget.
template <class T, int R, class Body>
__device__ __forceinline__ void fused_jobs(const FusedSync& s, int nsteps, const SweepGeom& g,
                                           Body body) {
  __shared__ int s_job[4];  // step, tile, tile x, tile y (step -1: no job left)
  for (;;) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      const int tiles_x = (g.W + T::TW - 1) / T::TW, tiles_y = (g.H + T::TH - 1) / T::TH;
      const long long ntiles = (long long)tiles_x * tiles_y;
      const long long j =
          ld_relaxed_u32(s.status) != 0 ? -1 : (long long)atomicAdd(s.next, 1ULL);
      if (j < 0 || j >= ntiles * nsteps) {
        s_job[0] = -1;
      } else {
        const int k = (int)(j / ntiles);
        const int t = (int)(j - (long long)k * ntiles);
        s_job[0] = k;
        s_job[1] = t;
        s_job[2] = t % tiles_x;
        s_job[3] = t / tiles_x;
      }
    }
    __syncthreads();
    const int k = s_job[0];
    if (k < 0) break;
    if (k > 0) {
      bool ok = true;
      const int tid = threadIdx.y * blockDim.x + threadIdx.x;
      if (tid < 9) {
        const int tiles_x = (g.W + T::TW - 1) / T::TW, tiles_y = (g.H + T::TH - 1) / T::TH;
        const int nx = s_job[2] + tid % 3 - 1, ny = s_job[3] + tid / 3 - 1;
        if (nx >= 0 && nx < tiles_x && ny >= 0 && ny < tiles_y)
          ok = wait_flag(s.flags + (size_t)ny * tiles_x + nx,
                         s.seq0 + (unsigned int)k + s.wait_skew, s.status, s.wait_ns);
      }
      if (!__syncthreads_and(ok)) break;
    }
    body(k, s_job[2], s_job[3]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0)
      st_release_u32(s.flags + s_job[1], s.seq0 + (unsigned int)s_job[0] + 1u);
  }
  // The last block to leave re-arms the counters for the next launch on the stream.
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    if (atomicAdd(s.done, 1u) == gridDim.x - 1) {
      *s.next = 0ULL;
      *s.done = 0u;
      __threadfence();
    }
  }
}

// Register budgets of the one-launch-per-step kernels (64 and 128 per thread: 8 and 4
// blocks of 128 threads per SM), which the job loop must not raise.
template <int R, int C, int PXH, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, 1024 / (BX * BY))
forward_fused_kernel(const FusedForwardArgs a, SweepGeom g, FusedSync s) {
  using T = Tile<R, C, PXH, BX, BY>;
  if constexpr (R > T::TH || R > T::TW) {
    return;  // never launched: fused_num_tiles is 0 when the halo leaves the 3 x 3 tiles
  } else {
  extern __shared__ __align__(16) float2 smem2[];
  float2* sm = smem2;
  float2* smask = smem2 + C * T::PLANE;
  fused_jobs<T, R>(s, a.nsteps, g, [&](int k, int tx, int ty) {
    const float* src = k == 0 ? a.src0 : a.dst[k - 1];
    float* dst = a.dst[k];
    const double* eps_n = a.eps + 2 * k;
    const int x0 = tx * T::TW, y0 = ty * T::TH;
    const float ex = (float)eps_n[0], ec = (float)eps_n[1];
    const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2;
    const float sk = colour_scale(0.5f * ec), mult = g.scale / sk;
    const bool border = load_tile<T, R, C, 1, true>(sm, smask, src, nullptr, g, x0, y0, sk);
    if (border)
      forward_body<T, R, C, PXH, true, true>(sm, smask, src, dst, g, kx, ky, mult, x0, y0);
    else
      forward_body<T, R, C, PXH, false, true>(sm, smask, src, dst, g, kx, ky, mult, x0, y0);
  });
  }
}

template <int R, int C, int PXH, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, 512 / (BX * BY))
adjoint_fused_kernel(const FusedAdjointArgs a, SweepGeom g, FusedSync s) {
  using T = Tile<R, C, PXH, BX, BY>;
  if constexpr (R > T::TH || R > T::TW) {
    return;  // never launched: fused_num_tiles is 0 when the halo leaves the 3 x 3 tiles
  } else {
  extern __shared__ __align__(16) float2 smem2[];
  float2* sm = smem2;
  float2* smask = smem2 + 2 * C * T::PLANE;
  fused_jobs<T, R>(s, a.n_hi - a.n_lo + 1, g, [&](int k, int tx, int ty) {
    const int n = a.n_hi - k;
    const float* cn = n == 0 ? a.c0 : a.traj + (size_t)(n - 1) * a.nc;
    const float* lin = (k & 1) ? a.lam[1] : a.lam[0];
    float* lout = (k & 1) ? a.lam[0] : a.lam[1];
    const double* eps_n = a.eps + 2 * n;
    const int x0 = tx * T::TW, y0 = ty * T::TH;
    const float ex = (float)eps_n[0], ec = (float)eps_n[1];
    const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
    const bool border = load_tile<T, R, C, 2, true>(sm, smask, cn, lin, g, x0, y0);
    const int tiles_x = (g.W + T::TW - 1) / T::TW;
    double* part = a.part + (size_t)n * a.pstride + 2 * ((size_t)ty * tiles_x + tx);
    if (border)
      adjoint_body<T, R, C, PXH, true>(sm, smask, lout, part, g, kx, ky, kc, ec, x0, y0);
    else
      adjoint_body<T, R, C, PXH, false>(sm, smask, lout, part, g, kx, ky, kc, ec, x0, y0);
  });
  }
}

}  // namespace agents
