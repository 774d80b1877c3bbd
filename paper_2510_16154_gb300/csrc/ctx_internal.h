// Internal definition of the library context (shared by agents.cu and batch.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "agents.h"
#include "kernels.h"

struct agents_ctx {
  agents_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::string err;

  int N = 0, C = 0, T = 0;
  size_t nc = 0, nv = 0;  // floats per colour field, per TV field
  agents::SweepGeom sg{};
  agents::TvGeom tg{};
  double M = 1.0;

  // colour fields
  float* c0 = nullptr;       // input image c^0
  float* cT = nullptr;       // c^T of the last stored forward
  float* work[2] = {nullptr, nullptr};
  float* lam[2] = {nullptr, nullptr};
  float* traj = nullptr;     // stored states (mode 0: c^1..c^{T-1}; mode k: checkpoints)
  float* seg = nullptr;      // mode k: recomputed states of one checkpoint segment
  int ckpt_every = 0;        // 0: full store; k: checkpoint every k steps
  int nckpt = 0;

  // control and reductions
  double* d_eps = nullptr;       // [T][2]
  double* d_trial[2] = {nullptr, nullptr};
  double* d_D = nullptr;         // [T][2]
  double* d_lohi = nullptr;      // [4]
  double* d_part_adj = nullptr;  // [T][nb_adj][2]
  double* d_part_tv = nullptr;   // [nb_tv][5]
  double* d_scal = nullptr;      // [16] small device results; slot 15: sweep wait status
  double* h_scal = nullptr;      // pinned [16]
  int nb_adj = 0, nb_tv = 0;

  // labels
  int32_t* d_labels = nullptr;
  int32_t* d_lstat = nullptr;    // [2] = {count, status}

  // stored-trajectory bookkeeping
  bool stored = false;
  std::vector<double> stored_eps;

  // solve workspaces (allocated on first solve)
  float *s_c = nullptr, *s_cn = nullptr, *s_v = nullptr, *s_vn = nullptr, *s_mu = nullptr;
  float* s_trial_c = nullptr;

  // trajectory reuse in full-store mode: Armijo trials store their trajectories in
  // traj_alt/cT_alt; an accepted trial's buffers are swapped in, so the next DAL
  // iteration and the multiplier step need no forward sweep (traj_ok: ctx->traj holds
  // the trajectory of the control in d_eps).  Off when the buffers cannot be allocated.
  float* traj_alt[2] = {nullptr, nullptr};
  float* cT_alt[2] = {nullptr, nullptr};
  bool reuse = false;
  bool reuse_tried = false;
  bool traj_ok = false;

  // whole-sweep launches: per-tile flags and job counters (FusedSync), the sequence
  // number every flag holds between launches, and whether a launch has run since the
  // last read of its status
  unsigned int* d_fsync = nullptr;
  int fused_tiles = 0;            // 0: no tiled kernels for (R, C), one launch per step
  int fused_cap_adj = 0;          // resident blocks of the fused adjoint kernel
  unsigned int fused_seq = 0;
  bool fused_pending = false;

  int64_t launches = 0;           // kernels launched by this context (for accounting)
  std::vector<agents_iter_record> log;  // per-DAL-iteration records of the last solve()
  std::vector<agents_outer_record> outer_log;  // per-multiplier-step records
  std::vector<void*> allocs;
  size_t held_bytes = 0;          // bytes of allocs counted against the memory limit
};

namespace agents {
// Helpers implemented in agents.cu for other translation units.
int ctx_fail(agents_ctx* ctx, int code, const char* msg);
int ctx_forward_sweep(agents_ctx* ctx, const double* d_eps, float* dst_T, bool store);
// Context-owned device allocation counted against agents_set_memory_limit's cap
// (AGENTS_ENOMEM with the message in ctx->err when the cap or cudaMalloc refuses).
int ctx_alloc(agents_ctx* ctx, void** out, size_t bytes);
bool mem_reserve(size_t bytes);
void mem_release(size_t bytes);
// Loop bound of the label union-find set by agents_debug_set_label_loop_cap (0: default).
int32_t label_loop_cap();
}  // namespace agents
