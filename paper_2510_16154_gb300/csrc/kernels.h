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

// ---- batched sweeps over many images (one launch per step and (R, C) class) ----
// Per-image buffers of one context in a batch (full trajectory storage).
struct BatchSweepImg {
  SweepGeom g;
  int nsteps;
  const float* c0;
  float* traj;        // c^1 .. c^{T-1}
  float* work0;       // trial sweep ping-pong
  float* work1;
  float* cT;          // c^T of the stored sweep
  float* trial_c;     // c^T of the trial sweep
  float* lam0;        // adjoint ping-pong (lam0 holds lambda^T at the start)
  float* lam1;
  const double* eps;        // control of the stored sweep, [T][2]
  const double* trial_eps;  // control of the trial sweep, [T][2]
  double* part_adj;         // D partials, [T][tiles][2]
  int ntiles;               // tiles of this image for the shape in use
};
struct BatchJob {
  int img, tx, ty;    // image index and tile (or TV block) coordinates
};
enum { kSweepStore = 0, kSweepTrial = 1 };
// Tile shapes the batched sweeps can use: 64x8, 64x4, 32x8 pixels.
constexpr int kNumShapes = 3;
int batch_tile_w(int shape);
int batch_tile_h(int shape);
// Tile height of the kernels without a tiled (R, C) instantiation (tile width 32): the
// wide-channel tiles for C = 31, the generic kernels' 4 rows otherwise.
int untiled_tile_h(int R, int C);
bool batch_tiled(int R, int C);
// Step n of the forward sweep of `kind` for every job whose image is active.
cudaError_t launch_forward_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                 const int* active, int n, int kind, int R, int C, int shape,
                                 cudaStream_t s);
// Step n of the adjoint sweep (reads lam[(T-1-n)&1], writes lam[(T-n)&1], partials of D).
cudaError_t launch_adjoint_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                 const int* active, int n, int R, int C, int shape,
                                 cudaStream_t s);

// Per-image arguments of a batched TV kernel (the roles each kernel reads are set).
struct BatchTvArgs {
  TvGeom g;
  const float* c;
  const float* c0;
  const float* v;
  const float* mu;
  float* lam;          // objective: -dL~/dc (may be null)
  float* v_out;        // pd_tv_step output
  const float* c_prev; // alm_update
  const float* v_prev;
  float* mu_io;
  double* partial;     // this image's per-block partials
  int tiles_x;         // TV blocks along x
};
int tv_block_w();      // pixels per TV block along x (and kTvBY along y)
int tv_block_h();
cudaError_t launch_objective_batch(const BatchTvArgs* args, const BatchJob* jobs, int njobs,
                                   const int* active, int C, bool lambda, cudaStream_t s);
cudaError_t launch_pd_tv_batch(const BatchTvArgs* args, const BatchJob* jobs, int njobs,
                               const int* active, int C, cudaStream_t s);
cudaError_t launch_alm_batch(const BatchTvArgs* args, const BatchJob* jobs, int njobs,
                             const int* active, int C, cudaStream_t s);
// out_s[n * nv + k] = scale_s * sum_b partial_s[(n * nblocks_s + b) * nv + k] for each
// segment s (blockIdx.y) and row n < rows, in the order of launch_reduce_rows.
struct ReduceSeg {
  const double* partial;
  int nblocks;
  double scale;
  double* out;
};
cudaError_t launch_reduce_segments(const ReduceSeg* segs, int nseg, int nv, int rows,
                                   cudaStream_t s);

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

// ---- whole sweeps in one launch (sweep_fused.cuh) ----
// A persistent grid takes (step, tile) jobs in step-major order from a counter; a job of
// step k waits until the 3 x 3 tiles around its own have finished step k - 1 (their
// outputs are its halo, and once they have finished, nothing reads the buffer it
// overwrites any more).  Every job whose dependencies have been taken is held by a
// running block, so the waits always end; each is still bounded in time, after which
// the launch gives up and records a status.  Per-tile results are bitwise those of the
// one-launch-per-step kernels.
struct FusedSync {
  unsigned long long* next;  // job counter, 0 between launches
  unsigned int* done;        // blocks that have left, 0 between launches
  unsigned int* status;      // 0, or 1 when a wait ran out of time (sticky until reset)
  unsigned int* flags;       // per tile: sequence number of the last completed step
  unsigned int seq0;         // flags of every tile when the launch starts
  unsigned int wait_skew;    // added to every wait target (0; a test sets it so that no
                             // flag ever reaches its target)
  long long wait_ns;         // time limit of one wait
};
// Words of a FusedSync block for `ntiles` tiles (one allocation, zero-initialised).
size_t fused_sync_words(int ntiles);
FusedSync fused_sync_at(unsigned int* base, int ntiles);

constexpr int kFusedMaxSteps = 128;  // forward steps per launch (destination table size)
struct FusedForwardArgs {
  const float* src0;                 // state before the first step
  const double* eps;                 // (eps_x, eps_c) of step k at eps + 2 k
  float* dst[kFusedMaxSteps];        // output of step k; the input of step k + 1
  int nsteps;
};
// Adjoint steps n = n_hi, n_hi - 1, ..., n_lo: c^n = n == 0 ? c0 : traj + (n - 1) nc; the
// k-th step of the launch reads lam[k & 1] and writes lam[(k & 1) ^ 1]; D partials of step
// n at part + n * pstride (tiles in row-major order).
struct FusedAdjointArgs {
  const float* c0;
  const float* traj;
  size_t nc;
  float* lam[2];
  const double* eps;                 // eps of step n at eps + 2 n
  double* part;
  size_t pstride;
  int n_hi, n_lo;
};
// Tiles of the sweep kernels for (R, C); 0 when (R, C) has no tiled kernel (those sweeps
// keep one launch per step).
int fused_num_tiles(const SweepGeom& g);
cudaError_t launch_forward_fused(const FusedForwardArgs& a, const SweepGeom& g,
                                 const FusedSync& s, cudaStream_t st);
cudaError_t launch_adjoint_fused(const FusedAdjointArgs& a, const SweepGeom& g,
                                 const FusedSync& s, cudaStream_t st);
// Blocks of the fused adjoint kernel resident on the whole device (0 if not tiled).
int fused_adjoint_capacity(const SweepGeom& g);

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
// y = a x over n floats (x, y 16-byte aligned; x == y allowed).
cudaError_t launch_scale_f32(const float* x, float a, float* y, size_t n, cudaStream_t s);
// trial[n] = clip(eps[n] + tau * D[n], lo, hi) for the T x 2 control.
cudaError_t launch_control_step(const double* eps, const double* D, double tau,
                                const double* lo_hi, double* trial, int T, cudaStream_t s);

// ---- labels (labels.cu) ----
// loop_cap bounds every union-find loop (0: the pixel count, which a forest whose links
// decrease never reaches); a loop that reaches it gives up and sets *status = 1.
cudaError_t launch_labels(const float* c, int H, int W, int C, float threshold, int loop_cap,
                          int32_t* labels, int32_t* count, int32_t* status, cudaStream_t s);

}  // namespace agents
