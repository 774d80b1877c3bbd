// Forward Euler step launcher: tiled kernels for (R <= 8, C in {1, 3}), generic otherwise.
#include "sweep_config.cuh"

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
  dim3 grid(ceil_div(g.W, T::TW), ceil_div(g.H, T::TH));
  kern<<<grid, dim3(kFwdBX, kFwdBY), smem, s>>>(c_in, c_out, eps_n, g);
  return cudaGetLastError();
}

static cudaError_t forward_generic(const float* c_in, float* c_out, const double* eps_n,
                                   const SweepGeom& g, cudaStream_t s) {
  if (g.C > kGenericMaxC) return cudaErrorInvalidValue;
  dim3 grid(ceil_div(g.W, kGenBX), ceil_div(g.H, kGenBY));
  forward_generic_kernel<<<grid, dim3(kGenBX, kGenBY), 0, s>>>(c_in, c_out, eps_n, g);
  return cudaGetLastError();
}

cudaError_t launch_forward_step(const float* c_in, float* c_out, const double* eps_n,
                                const SweepGeom& g, cudaStream_t s) {
#define AGENTS_FWD(R, C) forward_tiled<R, C>(c_in, c_out, eps_n, g, s)
  AGENTS_DISPATCH_RC(g.R, g.C, AGENTS_FWD, forward_generic(c_in, c_out, eps_n, g, s));
#undef AGENTS_FWD
}

}  // namespace agents
