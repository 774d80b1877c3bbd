// Adjoint step launcher: tiled kernels for (R <= 8, C in {1, 3}), generic otherwise.
#include "sweep_config.cuh"
#include "sweep_fused.cuh"
#include "sweep_wide.cuh"

namespace agents {

template <int R, int C>
static cudaError_t adjoint_tiled(const float* c_n, const float* lam_next, float* lam_out,
                                 const double* eps_n, double* partial, const SweepGeom& g,
                                 cudaStream_t s) {
  using T = Tile<R, C, kAdjPX, kAdjBX, kAdjBY>;
  const size_t smem = (size_t)(2 * C + 1) * T::PLANE * sizeof(float2);
  auto kern = adjoint_tile_kernel<R, C, kAdjPX, kAdjBX, kAdjBY>;
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
  cfg.blockDim = dim3(kAdjBX, kAdjBY);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, c_n, lam_next, lam_out, eps_n, partial, g);
}

static cudaError_t adjoint_generic(const float* c_n, const float* lam_next, float* lam_out,
                                   const double* eps_n, double* partial, const SweepGeom& g,
                                   cudaStream_t s) {
  if (g.C > kGenericMaxC) return cudaErrorInvalidValue;
  dim3 grid(ceil_div(g.W, kGenBX), ceil_div(g.H, kGenBY));
  adjoint_generic_kernel<<<grid, dim3(kGenBX, kGenBY), 0, s>>>(c_n, lam_next, lam_out, eps_n,
                                                               partial, g);
  return cudaGetLastError();
}

template <int R, int C, int PXH, int BX, int BY>
static cudaError_t adjoint_batch_tiled(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                       const int* active, int n, cudaStream_t s) {
  using T = Tile<R, C, PXH, BX, BY>;
  const size_t smem = (size_t)(2 * C + 1) * T::PLANE * sizeof(float2);
  auto kern = adjoint_batch_kernel<R, C, PXH, BX, BY>;
  static int cached = 0;
  int grid = 0;
  cudaError_t e = persistent_grid(kern, BX * BY, smem, &cached, &grid);
  if (e != cudaSuccess) return e;
  grid = grid < njobs ? grid : njobs;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, dim3(BX, BY), smem, s>>>(imgs, jobs, njobs, active, n);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                 const int* active, int n, int R, int C, int shape,
                                 cudaStream_t s) {
  if (!tiled_shape(R, C)) {
    if (wide_shape(R, C)) return launch_wide_adjoint_batch(imgs, jobs, njobs, active, n, R, s);
    if (C > kGenericMaxC) return cudaErrorInvalidValue;
    const int grid = njobs < 4096 ? njobs : 4096;
    if (grid <= 0) return cudaSuccess;
    adjoint_generic_batch_kernel<<<grid, dim3(kGenBX, kGenBY), 0, s>>>(imgs, jobs, njobs, active, n);
    return cudaGetLastError();
  }
#define AGENTS_AB(R_, C_, P_, BX_, BY_) \
  adjoint_batch_tiled<R_, C_, P_, BX_, BY_>(imgs, jobs, njobs, active, n, s)
#define AGENTS_ADJ_B(R_, C_) AGENTS_BATCH_SHAPES(AGENTS_AB, R_, C_)
  AGENTS_DISPATCH_RC(R, C, AGENTS_ADJ_B, cudaErrorInvalidValue);
#undef AGENTS_ADJ_B
#undef AGENTS_AB
}

template <int R, int C>
static int adjoint_blocks_tiled(const SweepGeom& g) {
  using T = Tile<R, C, kAdjPX, kAdjBX, kAdjBY>;
  return ceil_div(g.W, T::TW) * ceil_div(g.H, T::TH);
}

int adjoint_num_blocks(const SweepGeom& g) {
#define AGENTS_NB(R, C) adjoint_blocks_tiled<R, C>(g)
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_NB,
                     ceil_div(g.W, kGenBX) * ceil_div(g.H, untiled_tile_h(g.R, g.C)));
#undef AGENTS_NB
}

template <int R, int C>
static cudaError_t adjoint_fused(const FusedAdjointArgs& a, const SweepGeom& g,
                                 const FusedSync& s, cudaStream_t st) {
  using T = Tile<R, C, kAdjPX, kAdjBX, kAdjBY>;
  const size_t smem = (size_t)(2 * C + 1) * T::PLANE * sizeof(float2);
  auto kern = adjoint_fused_kernel<R, C, kAdjPX, kAdjBX, kAdjBY>;
  static int cached = 0;
  int grid = 0;
  cudaError_t e = persistent_grid(kern, kAdjBX * kAdjBY, smem, &cached, &grid);
  if (e != cudaSuccess) return e;
  const long long jobs =
      (long long)ceil_div(g.W, T::TW) * ceil_div(g.H, T::TH) * (a.n_hi - a.n_lo + 1);
  if (jobs <= 0) return cudaSuccess;
  if (jobs < grid) grid = (int)jobs;
  kern<<<grid, dim3(kAdjBX, kAdjBY), smem, st>>>(a, g, s);
  return cudaGetLastError();
}

template <int R, int C>
static int adjoint_fused_capacity_rc() {
  using T = Tile<R, C, kAdjPX, kAdjBX, kAdjBY>;
  const size_t smem = (size_t)(2 * C + 1) * T::PLANE * sizeof(float2);
  static int cached = 0;
  int grid = 0;
  if (persistent_grid(adjoint_fused_kernel<R, C, kAdjPX, kAdjBX, kAdjBY>, kAdjBX * kAdjBY, smem,
                      &cached, &grid) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return grid;
}

int fused_adjoint_capacity(const SweepGeom& g) {
#define AGENTS_CAP(R, C) adjoint_fused_capacity_rc<R, C>()
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_CAP, 0);
#undef AGENTS_CAP
}

cudaError_t launch_adjoint_fused(const FusedAdjointArgs& a, const SweepGeom& g,
                                 const FusedSync& s, cudaStream_t st) {
  if (a.n_lo < 0 || a.n_hi < a.n_lo) return cudaErrorInvalidValue;
#define AGENTS_ADJ(R, C) adjoint_fused<R, C>(a, g, s, st)
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_ADJ, cudaErrorInvalidValue);
#undef AGENTS_ADJ
}

cudaError_t launch_adjoint_step(const float* c_n, const float* lam_next, float* lam_out,
                                const double* eps_n, double* partial, const SweepGeom& g,
                                cudaStream_t s) {
#define AGENTS_ADJ(R, C) adjoint_tiled<R, C>(c_n, lam_next, lam_out, eps_n, partial, g, s)
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_ADJ,
                     wide_shape(g.R, g.C)
                         ? launch_wide_adjoint(c_n, lam_next, lam_out, eps_n, partial, g, s)
                         : adjoint_generic(c_n, lam_next, lam_out, eps_n, partial, g, s));
#undef AGENTS_ADJ
}

}  // namespace agents
