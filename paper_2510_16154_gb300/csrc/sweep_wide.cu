// Launchers of the wide-channel sweep kernels (sweep_wide.cuh): R = 1..7, C = 31.
#include "sweep_config.cuh"
#include "sweep_wide.cuh"

namespace agents {

namespace {

template <class K>
cudaError_t opt_in_smem(K kern, size_t smem, bool& done) {
  if (done || smem <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int R>
cudaError_t fwd(const float* c_in, float* c_out, const double* eps_n, const SweepGeom& g,
                cudaStream_t s) {
  using T = Wide<R, kWideC>;
  const size_t smem = T::smem(1);
  auto kern = wide_forward_kernel<R, kWideC>;
  static bool attr = false;
  cudaError_t e = opt_in_smem(kern, smem, attr);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(g.W, T::TW), ceil_div(g.H, T::TH));
  kern<<<grid, dim3(kWideBX, T::TH), smem, s>>>(c_in, c_out, eps_n, g);
  return cudaGetLastError();
}

template <int R>
cudaError_t adj(const float* c_n, const float* lam_next, float* lam_out, const double* eps_n,
                double* partial, const SweepGeom& g, cudaStream_t s) {
  using T = Wide<R, kWideC>;
  const size_t smem = T::smem(2);
  auto kern = wide_adjoint_kernel<R, kWideC>;
  static bool attr = false;
  cudaError_t e = opt_in_smem(kern, smem, attr);
  if (e != cudaSuccess) return e;
  dim3 grid(ceil_div(g.W, T::TW), ceil_div(g.H, T::TH));
  kern<<<grid, dim3(kWideBX, T::TH), smem, s>>>(c_n, lam_next, lam_out, eps_n, partial, g);
  return cudaGetLastError();
}

template <int R>
cudaError_t fwd_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                      const int* active, int n, int kind, cudaStream_t s) {
  using T = Wide<R, kWideC>;
  const size_t smem = T::smem(1);
  auto kern = wide_forward_batch_kernel<R, kWideC>;
  static int cached = 0;
  int grid = 0;
  cudaError_t e = persistent_grid(kern, T::NT, smem, &cached, &grid);
  if (e != cudaSuccess) return e;
  grid = grid < njobs ? grid : njobs;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, dim3(kWideBX, T::TH), smem, s>>>(imgs, jobs, njobs, active, n, kind);
  return cudaGetLastError();
}

template <int R>
cudaError_t adj_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                      const int* active, int n, cudaStream_t s) {
  using T = Wide<R, kWideC>;
  const size_t smem = T::smem(2);
  auto kern = wide_adjoint_batch_kernel<R, kWideC>;
  static int cached = 0;
  int grid = 0;
  cudaError_t e = persistent_grid(kern, T::NT, smem, &cached, &grid);
  if (e != cudaSuccess) return e;
  grid = grid < njobs ? grid : njobs;
  if (grid <= 0) return cudaSuccess;
  kern<<<grid, dim3(kWideBX, T::TH), smem, s>>>(imgs, jobs, njobs, active, n);
  return cudaGetLastError();
}

}  // namespace

int untiled_tile_h(int R, int C) { return wide_shape(R, C) ? wide_tile_h(R) : kGenBY; }

#define AGENTS_WIDE_R(R_, CALL)                                   \
  switch (R_) {                                                   \
    case 1: return CALL(1); case 2: return CALL(2);               \
    case 3: return CALL(3); case 4: return CALL(4);               \
    case 5: return CALL(5); case 6: return CALL(6);               \
    case 7: return CALL(7);                                       \
    default: return cudaErrorInvalidValue;                        \
  }

cudaError_t launch_wide_forward(const float* c_in, float* c_out, const double* eps_n,
                                const SweepGeom& g, cudaStream_t s) {
  if (g.C != kWideC) return cudaErrorInvalidValue;
#define CALL(R) fwd<R>(c_in, c_out, eps_n, g, s)
  AGENTS_WIDE_R(g.R, CALL)
#undef CALL
}

cudaError_t launch_wide_adjoint(const float* c_n, const float* lam_next, float* lam_out,
                                const double* eps_n, double* partial, const SweepGeom& g,
                                cudaStream_t s) {
  if (g.C != kWideC) return cudaErrorInvalidValue;
#define CALL(R) adj<R>(c_n, lam_next, lam_out, eps_n, partial, g, s)
  AGENTS_WIDE_R(g.R, CALL)
#undef CALL
}

cudaError_t launch_wide_forward_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                      const int* active, int n, int kind, int R, cudaStream_t s) {
#define CALL(R_) fwd_batch<R_>(imgs, jobs, njobs, active, n, kind, s)
  AGENTS_WIDE_R(R, CALL)
#undef CALL
}

cudaError_t launch_wide_adjoint_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                      const int* active, int n, int R, cudaStream_t s) {
#define CALL(R_) adj_batch<R_>(imgs, jobs, njobs, active, n, s)
  AGENTS_WIDE_R(R, CALL)
#undef CALL
}

}  // namespace agents
