// Internal launcher interface between the C ABI (agents.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace agents {

// Geometry and constants of one agent sweep step.
struct SweepGeom {
  int H, W, C, R;
  float inv_w2, inv_h2;  // dx^2 = 1/W^2, dy^2 = 1/H^2 (positions in the unit square)
  float scale;           // dt / M
};

// Geometry and constants of the TV kernels.
struct TvGeom {
  int H, W, C;
  float inv2hx, inv2hy;  // 1/(2 dx) = W/2, 1/(2 dy) = H/2
  float rho, inv_rho, alpha;
  double gamma;          // dual step; float64 because the multiplier update is float64
  double cell;           // dx dy
  int tv_mode;
};

// ---- agent sweeps (sweep_*.cu) ----
// One explicit Euler step c_out = c_in + dt F(c_in, eps_n); eps_n points at the device
// pair (eps_x^n, eps_c^n).
cudaError_t launch_forward_step(const float* c_in, float* c_out, const double* eps_n,
                                const SweepGeom& g, cudaStream_t s);
// One adjoint step lam_out = lam_next + dt J_F(c_n)^T lam_next, and per-block partial
// sums of D^n (before the 1/(2M) factor) written to partial[2 * block].
cudaError_t launch_adjoint_step(const float* c_n, const float* lam_next, float* lam_out,
                                const double* eps_n, double* partial, const SweepGeom& g,
                                cudaStream_t s);
// Number of per-block D partial pairs one adjoint step writes.
int adjoint_num_blocks(const SweepGeom& g);

// ---- reductions (tv.cu) ----
// out[n * nv + k] = scale * sum_b partial[(n * nblocks + b) * nv + k], for n < rows.
cudaError_t launch_reduce_rows(const double* partial, int nblocks, int nv, int rows,
                               double scale, double* out, cudaStream_t s);

// ---- TV kernels (tv.cu) ----
int tv_num_blocks(const TvGeom& g);
// Per-block partials of L~(c, v, mu) (already times dx dy); lam (may be null) receives
// -dL~/dc.
cudaError_t launch_objective(const float* c, const float* c0, const float* v, const float* mu,
                             float* lam, double* partial, const TvGeom& g, cudaStream_t s);
cudaError_t launch_pd_tv_step(const float* c, const float* mu, float* v, const TvGeom& g,
                              cudaStream_t s);
// mu += gamma (v - G c) in float64; partial[5 * block + k] = {|v-Gc|^2, |G^T(v-v_prev)|^2,
// |c-c_prev|^2, |c|^2, K(c)/(dx dy)}.
cudaError_t launch_alm_update(const float* c, const float* c_prev, const float* c0,
                              const float* v, const float* v_prev, float* mu, double* partial,
                              const TvGeom& g, cudaStream_t s);
// Multiplier-update statistics from the reduced raw sums (see alm_update in agents.h).
cudaError_t launch_alm_finalize(const double* raw, double* stats, double rho, double gamma,
                                double cell, cudaStream_t s);
// trial[n] = clip(eps[n] + tau * D[n], lo, hi) for the T x 2 control.
cudaError_t launch_control_step(const double* eps, const double* D, double tau,
                                const double* lo_hi, double* trial, int T, cudaStream_t s);

// ---- labels (labels.cu) ----
cudaError_t launch_labels(const float* c, int H, int W, int C, float threshold, int32_t* labels,
                          int32_t* count, int32_t* status, cudaStream_t s);

}  // namespace agents
