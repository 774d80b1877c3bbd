// Forward Euler step launcher: tiled kernels for (R <= 8, C in {1, 3}), generic otherwise.
#include "sweep_config.cuh"
#include "sweep_fused.cuh"
#include "sweep_wide.cuh"

namespace agents {

template <int R, int C>
static cudaError_t forward_tiled(const float* c_in, float* c_out, const double* eps_n,
                                 const SweepGeom& g, cudaStream_t s) {
  using T = Tile<R, C, kFwdPX, kFwdBX, kFwdBY>;
  const size_t smem = (size_t)(C + 1) * T::PLANE * sizeof(float2);
  auto kern = forward_tile_kernel<R, C, kFwdPX, kFwdBX, kFwdBY>;
  if (smem > 48 * 1024) {
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_set = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ceil_div(g.W, T::TW), ceil_div(g.H, T::TH));
  cfg.blockDim = dim3(kFwdBX, kFwdBY);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, c_in, c_out, eps_n, g);
}

static cudaError_t forward_generic(const float* c_in, float* c_out, const double* eps_n,
                                   const SweepGeom& g, cudaStream_t s) {
  if (g.C > kGenericMaxC) return cudaErrorInvalidValue;
  dim3 grid(ceil_div(g.W, kGenBX), ceil_div(g.H, kGenBY));
  forward_generic_kernel<<<grid, dim3(kGenBX, kGenBY), 0, s>>>(c_in, c_out, eps_n, g);
  return cudaGetLastError();
}

template <int R, int C, int PXH, int BX, int BY>
static cudaError_t forward_batch_tiled(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                       const int* active, int n, int kind, cudaStream_t s) {
  using T = Tile<R, C, PXH, BX, BY>;
  const size_t smem = (size_t)(C + 1) * T::PLANE * sizeof(float2);
  auto kern = forward_batch_kernel<R, C, PXH, BX, BY>;
  static int cached = 0;
  int grid = 0;
  cudaError_t e = persistent_grid(kern, BX * BY, smem, &cached, &grid);
  if (e != cudaSuccess) return e;
  grid = grid < njobs ? grid : njobs;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, dim3(BX, BY), smem, s>>>(imgs, jobs, njobs, active, n, kind);
  return cudaGetLastError();
}

int batch_tile_w(int shape) { return shape == 2 ? 32 : 64; }
int batch_tile_h(int shape) { return shape == 1 ? 4 : 8; }
bool batch_tiled(int R, int C) { return tiled_shape(R, C); }

cudaError_t launch_forward_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                 const int* active, int n, int kind, int R, int C, int shape,
                                 cudaStream_t s) {
  if (!tiled_shape(R, C)) {
    if (wide_shape(R, C)) return launch_wide_forward_batch(imgs, jobs, njobs, active, n, kind, R, s);
    if (C > kGenericMaxC) return cudaErrorInvalidValue;
    const int grid = njobs < 4096 ? njobs : 4096;
    if (grid <= 0) return cudaSuccess;
    forward_generic_batch_kernel<<<grid, dim3(kGenBX, kGenBY), 0, s>>>(imgs, jobs, njobs, active,
                                                                      n, kind);
    return cudaGetLastError();
  }
#define AGENTS_FB(R_, C_, P_, BX_, BY_) \
  forward_batch_tiled<R_, C_, P_, BX_, BY_>(imgs, jobs, njobs, active, n, kind, s)
#define AGENTS_FWD_B(R_, C_) AGENTS_BATCH_SHAPES(AGENTS_FB, R_, C_)
  AGENTS_DISPATCH_RC(R, C, AGENTS_FWD_B, cudaErrorInvalidValue);
#undef AGENTS_FWD_B
#undef AGENTS_FB
}

template <int R, int C>
static cudaError_t forward_fused(const FusedForwardArgs& a, const SweepGeom& g,
                                 const FusedSync& s, cudaStream_t st) {
  using T = Tile<R, C, kFwdPX, kFwdBX, kFwdBY>;
  const size_t smem = (size_t)(C + 1) * T::PLANE * sizeof(float2);
  auto kern = forward_fused_kernel<R, C, kFwdPX, kFwdBX, kFwdBY>;
  static int cached = 0;
  int grid = 0;
  cudaError_t e = persistent_grid(kern, kFwdBX * kFwdBY, smem, &cached, &grid);
  if (e != cudaSuccess) return e;
  const long long jobs = (long long)ceil_div(g.W, T::TW) * ceil_div(g.H, T::TH) * a.nsteps;
  if (jobs <= 0) return cudaSuccess;
  if (jobs < grid) grid = (int)jobs;
  kern<<<grid, dim3(kFwdBX, kFwdBY), smem, st>>>(a, g, s);
  return cudaGetLastError();
}

size_t fused_sync_words(int ntiles) { return 4 + (size_t)(ntiles > 0 ? ntiles : 0); }

FusedSync fused_sync_at(unsigned int* base, int ntiles) {
  (void)ntiles;
  FusedSync s{};
  s.next = reinterpret_cast<unsigned long long*>(base);
  s.done = base + 2;
  s.status = base + 3;
  s.flags = base + 4;
  return s;
}

int fused_num_tiles(const SweepGeom& g) {
  if (!tiled_shape(g.R, g.C)) return 0;
  if (g.R > kFwdBY || g.R > 2 * kFwdBX * kFwdPX) return 0;  // halo beyond the 3 x 3 tiles
  static_assert(kFwdPX == kAdjPX && kFwdBX == kAdjBX && kFwdBY == kAdjBY,
                "the fused sweeps share one tile grid and one set of flags");
  return ceil_div(g.W, 2 * kFwdBX * kFwdPX) * ceil_div(g.H, kFwdBY);
}

cudaError_t launch_forward_fused(const FusedForwardArgs& a, const SweepGeom& g,
                                 const FusedSync& s, cudaStream_t st) {
  if (a.nsteps < 1 || a.nsteps > kFusedMaxSteps) return cudaErrorInvalidValue;
#define AGENTS_FWD(R, C) forward_fused<R, C>(a, g, s, st)
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_FWD, cudaErrorInvalidValue);
#undef AGENTS_FWD
}

cudaError_t launch_forward_step(const float* c_in, float* c_out, const double* eps_n,
                                const SweepGeom& g, cudaStream_t s) {
#define AGENTS_FWD(R, C) forward_tiled<R, C>(c_in, c_out, eps_n, g, s)
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_FWD,
                     wide_shape(g.R, g.C) ? launch_wide_forward(c_in, c_out, eps_n, g, s)
                                          : forward_generic(c_in, c_out, eps_n, g, s));
#undef AGENTS_FWD
}

}  // namespace agents
