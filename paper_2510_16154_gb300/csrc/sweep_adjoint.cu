// Adjoint step launcher: tiled kernels for (R <= 8, C in {1, 3}), generic otherwise.
#include "sweep_config.cuh"

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
  dim3 grid(ceil_div(g.W, T::TW), ceil_div(g.H, T::TH));
  kern<<<grid, dim3(kAdjBX, kAdjBY), smem, s>>>(c_n, lam_next, lam_out, eps_n, partial, g);
  return cudaGetLastError();
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

template <int R, int C>
static int adjoint_blocks_tiled(const SweepGeom& g) {
  using T = Tile<R, C, kAdjPX, kAdjBX, kAdjBY>;
  return ceil_div(g.W, T::TW) * ceil_div(g.H, T::TH);
}

int adjoint_num_blocks(const SweepGeom& g) {
#define AGENTS_NB(R, C) adjoint_blocks_tiled<R, C>(g)
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_NB, ceil_div(g.W, kGenBX) * ceil_div(g.H, kGenBY));
#undef AGENTS_NB
}

cudaError_t launch_adjoint_step(const float* c_n, const float* lam_next, float* lam_out,
                                const double* eps_n, double* partial, const SweepGeom& g,
                                cudaStream_t s) {
#define AGENTS_ADJ(R, C) adjoint_tiled<R, C>(c_n, lam_next, lam_out, eps_n, partial, g, s)
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_ADJ,
                     adjoint_generic(c_n, lam_next, lam_out, eps_n, partial, g, s));
#undef AGENTS_ADJ
}

}  // namespace agents
