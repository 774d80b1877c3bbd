// C ABI of the agent-based optimal-control image solver: context and workspace
// management, the per-sweep entry points, and solve() -- Algorithm 2 (ADMM) with
// Algorithm 1 (direct-adjoint loop with projected two-way Armijo) as its eps-step.
//
// Host code drives the iteration: the Armijo accept/reject test needs one float64
// objective per trial on the host, the only host/device round trip of a DAL iteration.
// Everything else (Euler steps, adjoint steps, control projection, reductions) runs in
// the kernels declared in kernels.h, stream-ordered on the context's stream.
#include "agents.h"
#include "ctx_internal.h"
#include "kernels.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <nvtx3/nvToolsExt.h>

using namespace agents;

namespace {

thread_local std::string g_init_error;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace agents {
// Message returned by agents_last_error(NULL) for calls that have no context.
void set_global_error(const std::string& msg) { g_init_error = msg; }

// Process-wide accounting of the device memory held by contexts, against an optional
// cap (agents_set_memory_limit; 0 = no cap).
namespace {
std::atomic<uint64_t> g_mem_limit{0};
std::atomic<uint64_t> g_mem_held{0};
std::atomic<int32_t> g_label_loop_cap{0};
// Whole-sweep launches (sweep_fused.cuh): 0 never, 1 where they measured faster (the
// default), 2 for every tiled sweep; the time limit of one wait; a one-shot offset of the
// next launch's wait targets that no flag reaches (tests of the time limit).
std::atomic<int32_t> g_fused_enabled{1};
std::atomic<int64_t> g_fused_wait_ns{2000000000LL};
std::atomic<uint32_t> g_fused_skew{0};
}  // namespace

bool mem_reserve(size_t bytes) {
  uint64_t held = g_mem_held.load();
  for (;;) {
    const uint64_t lim = g_mem_limit.load();
    if (lim != 0 && (held > lim || bytes > lim - held)) return false;
    if (g_mem_held.compare_exchange_weak(held, held + bytes)) return true;
  }
}

void mem_release(size_t bytes) { g_mem_held.fetch_sub(bytes); }

// cudaMalloc of a context-owned buffer, counted against the limit.  Returns AGENTS_OK,
// or AGENTS_ENOMEM (limit reached or cudaMalloc failed) with the message in ctx->err.
int ctx_alloc(agents_ctx* ctx, void** out, size_t bytes) {
  if (bytes == 0) bytes = 1;
  if (!mem_reserve(bytes))
    return ctx_fail(ctx, AGENTS_ENOMEM,
                    ("allocation of " + std::to_string(bytes) + " bytes exceeds the memory "
                     "limit of " + std::to_string(g_mem_limit.load()) + " bytes (" +
                     std::to_string(g_mem_held.load()) + " held)").c_str());
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mem_release(bytes);
    return ctx_fail(ctx, AGENTS_ENOMEM,
                    ("cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                     cudaGetErrorString(e)).c_str());
  }
  ctx->allocs.push_back(p);
  ctx->held_bytes += bytes;
  *out = p;
  return AGENTS_OK;
}

int32_t label_loop_cap() { return g_label_loop_cap.load(); }
}  // namespace agents

int agents_set_memory_limit(uint64_t bytes) {
  agents::g_mem_limit.store(bytes);
  return AGENTS_OK;
}

uint64_t agents_memory_held(void) { return agents::g_mem_held.load(); }

int agents_debug_set_fused(int32_t enable, int64_t wait_ns, uint32_t skew_once) {
  if (wait_ns < 0) {
    agents::set_global_error("agents_debug_set_fused: wait_ns must be >= 0");
    return AGENTS_EINVAL;
  }
  if (enable < 0 || enable > 2) {
    agents::set_global_error("agents_debug_set_fused: enable must be 0, 1 or 2");
    return AGENTS_EINVAL;
  }
  agents::g_fused_enabled.store(enable);
  agents::g_fused_wait_ns.store(wait_ns > 0 ? wait_ns : 2000000000LL);
  agents::g_fused_skew.store(skew_once);
  return AGENTS_OK;
}

int agents_debug_set_label_loop_cap(int32_t cap) {
  if (cap < 0) {
    agents::set_global_error("agents_debug_set_label_loop_cap: cap must be >= 0");
    return AGENTS_EINVAL;
  }
  agents::g_label_loop_cap.store(cap);
  return AGENTS_OK;
}

// struct agents_ctx is defined in ctx_internal.h

namespace {

int fail(agents_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  else g_init_error = buf;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? AGENTS_ENOMEM : AGENTS_ECUDA, \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define TRY(expr)              \
  do {                         \
    int st_ = (expr);          \
    if (st_ != AGENTS_OK) return st_; \
  } while (0)

// NVTX range over a scope (named in profiler timelines; no cost without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

template <class T>
int dalloc(agents_ctx* ctx, T** out, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  TRY(ctx_alloc(ctx, &p, count * sizeof(T)));
  *out = static_cast<T*>(p);
  return AGENTS_OK;
}

int validate(const agents_params* p) {
  if (!p) return fail(nullptr, AGENTS_EINVAL, "params is NULL");
  if (p->height < 1 || p->width < 1 || p->channels < 1)
    return fail(nullptr, AGENTS_EINVAL, "height, width and channels must be >= 1");
  if ((int64_t)p->height * p->width > (int64_t)1 << 30)
    return fail(nullptr, AGENTS_EINVAL, "image too large (more than 2^30 pixels)");
  if (p->channels > 64) return fail(nullptr, AGENTS_EINVAL, "channels must be <= 64");
  if (p->radius < 1) return fail(nullptr, AGENTS_EINVAL, "radius must be >= 1");
  if (p->nsteps < 1) return fail(nullptr, AGENTS_EINVAL, "nsteps must be >= 1");
  if (!(p->dt > 0) || !(p->alpha > 0) || !(p->rho > 0) || !(p->gamma > 0))
    return fail(nullptr, AGENTS_EINVAL, "dt, alpha, rho and gamma must be > 0");
  for (int k = 0; k < 2; ++k)
    if (!(p->eps_lo[k] >= 0) || !(p->eps_lo[k] <= p->eps_hi[k]) || !std::isfinite(p->eps_hi[k]))
      return fail(nullptr, AGENTS_EINVAL, "need 0 <= eps_lo <= eps_hi < inf");
  if (p->norm_mode != 0 && p->norm_mode != 1)
    return fail(nullptr, AGENTS_EINVAL, "norm_mode must be 0 or 1");
  if (p->tv_mode != 0 && p->tv_mode != 1) return fail(nullptr, AGENTS_EINVAL, "tv_mode must be 0 or 1");
  if (p->traj_mode < 0) return fail(nullptr, AGENTS_EINVAL, "traj_mode must be >= 0");
  return AGENTS_OK;
}

// Copy n bytes from src (host or device) into device dst on the context stream.
int to_device(agents_ctx* ctx, void* dst, const void* src, size_t n) {
  CK(cudaMemcpyAsync(dst, src, n, is_device_ptr(src) ? cudaMemcpyDeviceToDevice
                                                      : cudaMemcpyHostToDevice,
                     ctx->stream));
  return AGENTS_OK;
}

constexpr int kStatusSlot = 15;  // d_scal slot of the whole-sweep wait status
int fused_check(agents_ctx* ctx);

// Copy n bytes from device src into dst (host or device); host destinations are
// complete when this returns.
int from_device(agents_ctx* ctx, void* dst, const void* src, size_t n) {
  if (is_device_ptr(dst)) {
    CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    TRY(fused_check(ctx));
  }
  return AGENTS_OK;
}

int check_aligned(agents_ctx* ctx, const void* p, const char* name) {
  if (p && (reinterpret_cast<uintptr_t>(p) & 15u))
    return fail(ctx, AGENTS_EINVAL, "%s must be 16-byte aligned", name);
  return AGENTS_OK;
}

int need(agents_ctx* ctx, const void* p, const char* name) {
  if (!p) return fail(ctx, AGENTS_EINVAL, "%s is NULL", name);
  return check_aligned(ctx, p, name);
}

// ------------------------------------------------------------------ sweeps
// Whole-sweep launches.  The status word of their waits is the last slot of d_scal, so
// that every read of the small device results also reads it.
unsigned int* fused_status_dev(agents_ctx* ctx) {
  return reinterpret_cast<unsigned int*>(ctx->d_scal + kStatusSlot);
}

// Where whole-sweep launches pay (GB300, RGB, R = 5, T = 50): the per-SM warp scheduler
// favours the oldest blocks, so in a persistent grid the youngest block's job lags and
// the jobs that need its tile wait; the saving at the end of every step has to outweigh
// that.  Measured: the adjoint of a 1024^2 image 129 vs 135 us per step (4 resident
// blocks per SM, 3.4 tiles per block and step); 2048^2 497 vs 491 us; the forward step
// (8 resident blocks per SM) 64.5 vs 64.3 us at 1024^2 and slower at every other size.
// So by default only adjoint sweeps of at most 4 tiles per resident block are fused.
constexpr int kFusedAdjointMaxTilesPerBlock = 4;

bool use_fused_forward(const agents_ctx* ctx) {
  return ctx->fused_tiles > 0 && g_fused_enabled.load() == 2;
}

bool use_fused_adjoint(const agents_ctx* ctx) {
  const int mode = g_fused_enabled.load();
  if (ctx->fused_tiles <= 0 || mode == 0) return false;
  if (mode == 2) return true;
  return (int64_t)ctx->fused_tiles <= (int64_t)kFusedAdjointMaxTilesPerBlock * ctx->fused_cap_adj;
}

FusedSync fused_sync(agents_ctx* ctx) {
  FusedSync s = fused_sync_at(ctx->d_fsync, ctx->fused_tiles);
  s.status = fused_status_dev(ctx);
  s.seq0 = ctx->fused_seq;
  s.wait_skew = g_fused_skew.exchange(0);
  s.wait_ns = g_fused_wait_ns.load();
  return s;
}

// Called after a synchronisation that copied d_scal[kStatusSlot] into h_scal: a fused
// launch that gave up leaves invalid results and inconsistent flags; the flags are
// re-armed and the call fails with AGENTS_ETIMEOUT.
int fused_status_after_sync(agents_ctx* ctx) {
  if (!ctx->fused_pending) return AGENTS_OK;
  ctx->fused_pending = false;
  unsigned int st = 0;
  std::memcpy(&st, ctx->h_scal + kStatusSlot, sizeof(st));
  if (st == 0) return AGENTS_OK;
  CK(cudaMemsetAsync(ctx->d_fsync, 0, fused_sync_words(ctx->fused_tiles) * sizeof(unsigned int),
                     ctx->stream));
  CK(cudaMemsetAsync(ctx->d_scal + kStatusSlot, 0, sizeof(double), ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->fused_seq = 0;
  return fail(ctx, AGENTS_ETIMEOUT,
              "a whole-sweep launch gave up waiting for a neighbouring tile (time limit); "
              "its results are invalid");
}

int fused_check(agents_ctx* ctx) {
  if (!ctx->fused_pending) return AGENTS_OK;
  CK(cudaMemcpyAsync(ctx->h_scal + kStatusSlot, ctx->d_scal + kStatusSlot, sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return fused_status_after_sync(ctx);
}

// Euler steps k = 0 .. n-1 from src0 under the device control d_eps (2 values per
// step); step k writes dsts[k], which step k + 1 reads.  One launch per kFusedMaxSteps
// steps when the tiled kernels apply, one launch per step otherwise.
int run_forward(agents_ctx* ctx, const float* src0, const double* d_eps,
                float* const* dsts, int n) {
  for (int k = 0; k < n; ++k)
    if (dsts[k] == (k == 0 ? src0 : dsts[k - 1]))
      return fail(ctx, AGENTS_EINVAL, "an Euler step would overwrite its own input");
  if (use_fused_forward(ctx)) {
    for (int n0 = 0; n0 < n; n0 += kFusedMaxSteps) {
      FusedForwardArgs a{};
      a.src0 = n0 == 0 ? src0 : dsts[n0 - 1];
      a.eps = d_eps + 2 * n0;
      a.nsteps = std::min(kFusedMaxSteps, n - n0);
      for (int k = 0; k < a.nsteps; ++k) a.dst[k] = dsts[n0 + k];
      CK(launch_forward_fused(a, ctx->sg, fused_sync(ctx), ctx->stream));
      ctx->fused_seq += (unsigned int)a.nsteps;
      ctx->fused_pending = true;
      ++ctx->launches;
    }
    return AGENTS_OK;
  }
  const float* cur = src0;
  for (int k = 0; k < n; ++k) {
    CK(launch_forward_step(cur, dsts[k], d_eps + 2 * k, ctx->sg, ctx->stream));
    ++ctx->launches;
    cur = dsts[k];
  }
  return AGENTS_OK;
}

// Pointer to stored state c^n (0 <= n < T) for the full-store mode.
const float* full_state(agents_ctx* ctx, int n) {
  return n == 0 ? ctx->c0 : ctx->traj + (size_t)(n - 1) * ctx->nc;
}

// Forward sweep under the device control d_eps; c^T goes to dst_T.  With store, the
// states the adjoint needs are kept (all of them, or every k-th).
int forward_sweep(agents_ctx* ctx, const double* d_eps, float* dst_T, bool store) {
  NvtxRange nr("forward_sweep");
  const int T = ctx->T;
  const float* cur = ctx->c0;
  int wi = 0;
  std::vector<float*> dsts(T);
  for (int n = 0; n < T; ++n) {
    float* dst;
    if (n == T - 1) {
      dst = dst_T;
    } else if (store && ctx->ckpt_every == 0) {
      dst = ctx->traj + (size_t)n * ctx->nc;
    } else if (store && (n + 1) % ctx->ckpt_every == 0) {
      dst = ctx->traj + (size_t)((n + 1) / ctx->ckpt_every - 1) * ctx->nc;
    } else {
      dst = ctx->work[wi];
      if (dst == cur) dst = ctx->work[wi ^ 1];
      wi = (dst == ctx->work[0]) ? 1 : 0;
    }
    dsts[n] = dst;
    cur = dst;
  }
  return run_forward(ctx, ctx->c0, d_eps, dsts.data(), T);
}

// L~(c, v, mu) into d_scal[slot] (device); lam (optional) = -dL~/dc.
int objective(agents_ctx* ctx, const float* c, const float* v, const float* mu, float* lam,
              int slot) {
  CK(launch_objective(c, ctx->c0, v, mu, lam, ctx->d_part_tv, ctx->tg, ctx->stream));
  CK(launch_reduce_rows(ctx->d_part_tv, ctx->nb_tv, 1, 1, 1.0, ctx->d_scal + slot, ctx->stream));
  ctx->launches += 2;
  return AGENTS_OK;
}

int fetch_scalar(agents_ctx* ctx, int slot, double* out) {
  // slot .. kStatusSlot in one copy: the status of the whole-sweep launches comes along
  CK(cudaMemcpyAsync(ctx->h_scal + slot, ctx->d_scal + slot,
                     (size_t)(kStatusSlot + 1 - slot) * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  TRY(fused_status_after_sync(ctx));
  *out = ctx->h_scal[slot];
  return AGENTS_OK;
}

// Reverse sweep from lambda^T held in ctx->lam[0]; D^n (times 1/(2M)) into ctx->d_D.
// Returns the final lambda^0 buffer in *lam_out.
int adjoint_sweep_from(agents_ctx* ctx, const double* d_eps, float** lam_out) {
  NvtxRange nr("adjoint_sweep");
  const int T = ctx->T;
  int li = 0;
  const size_t pstride = (size_t)ctx->nb_adj * 2;
  auto step = [&](int n, const float* cn) -> int {
    CK(launch_adjoint_step(cn, ctx->lam[li], ctx->lam[li ^ 1], d_eps + 2 * n,
                           ctx->d_part_adj + (size_t)n * pstride, ctx->sg, ctx->stream));
    ++ctx->launches;
    li ^= 1;
    return AGENTS_OK;
  };
  if (ctx->ckpt_every == 0 && use_fused_adjoint(ctx)) {
    FusedAdjointArgs a{};
    a.c0 = ctx->c0;
    a.traj = ctx->traj;
    a.nc = ctx->nc;
    a.lam[0] = ctx->lam[0];
    a.lam[1] = ctx->lam[1];
    a.eps = d_eps;
    a.part = ctx->d_part_adj;
    a.pstride = pstride;
    a.n_hi = T - 1;
    a.n_lo = 0;
    CK(launch_adjoint_fused(a, ctx->sg, fused_sync(ctx), ctx->stream));
    ctx->fused_seq += (unsigned int)T;
    ctx->fused_pending = true;
    ++ctx->launches;
    li = T & 1;
  } else if (ctx->ckpt_every == 0) {
    for (int n = T - 1; n >= 0; --n) TRY(step(n, full_state(ctx, n)));
  } else {
    const int k = ctx->ckpt_every;
    const int nseg = (T + k - 1) / k;
    for (int m = nseg - 1; m >= 0; --m) {
      const int n0 = m * k, len = std::min(k, T - n0);
      const float* base = m == 0 ? ctx->c0 : ctx->traj + (size_t)(m - 1) * ctx->nc;
      // recompute c^{n0+1} .. c^{n0+len-1} into seg[0..len-2]
      std::vector<float*> dsts(len > 1 ? len - 1 : 0);
      for (int i = 1; i < len; ++i) dsts[i - 1] = ctx->seg + (size_t)(i - 1) * ctx->nc;
      if (len > 1) TRY(run_forward(ctx, base, d_eps + 2 * n0, dsts.data(), len - 1));
      for (int i = len - 1; i >= 0; --i) {
        const float* cn = i == 0 ? base : ctx->seg + (size_t)(i - 1) * ctx->nc;
        TRY(step(n0 + i, cn));
      }
    }
  }
  CK(launch_reduce_rows(ctx->d_part_adj, ctx->nb_adj, 2, T, 1.0 / (2.0 * ctx->M), ctx->d_D,
                        ctx->stream));
  ++ctx->launches;
  *lam_out = ctx->lam[li];
  return AGENTS_OK;
}

// Reverse sweep from lambda^T = -dL~/dc(c^T) (the terminal cost of Eq. complete_square).
int adjoint_sweep(agents_ctx* ctx, const double* d_eps, const float* v, const float* mu,
                  int obj_slot, float** lam_out) {
  TRY(objective(ctx, ctx->cT, v, mu, ctx->lam[0], obj_slot));
  return adjoint_sweep_from(ctx, d_eps, lam_out);
}

int alm(agents_ctx* ctx, const float* c, const float* c_prev, const float* v,
        const float* v_prev, float* mu, double* h_stats /*host[5]*/, double* d_stats) {
  CK(launch_alm_update(c, c_prev, ctx->c0, v, v_prev, mu, ctx->d_part_tv, ctx->tg, ctx->stream));
  CK(launch_reduce_rows(ctx->d_part_tv, ctx->nb_tv, 5, 1, 1.0, ctx->d_scal + 8, ctx->stream));
  ctx->launches += 2;
  if (d_stats) {
    CK(launch_alm_finalize(ctx->d_scal + 8, d_stats, ctx->p.rho, ctx->p.gamma, ctx->tg.cell,
                           ctx->stream));
    ++ctx->launches;
  }
  if (h_stats) {
    double raw[5];
    CK(cudaMemcpyAsync(ctx->h_scal + 8, ctx->d_scal + 8, (kStatusSlot + 1 - 8) * sizeof(double),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    TRY(fused_status_after_sync(ctx));
    std::memcpy(raw, ctx->h_scal + 8, sizeof(raw));
    const double cell = ctx->tg.cell;
    h_stats[0] = std::sqrt(raw[0]);
    h_stats[1] = ctx->p.rho * std::sqrt(raw[1]);
    h_stats[2] = ctx->p.gamma * cell * raw[0];
    h_stats[3] = raw[3] > 0 ? std::sqrt(raw[2] / raw[3]) : 0.0;
    h_stats[4] = cell * raw[4];
  }
  return AGENTS_OK;
}

// Trial-trajectory buffers for trajectory reuse (full-store mode only); if they do not
// fit, solve() recomputes trajectories as before.
void ensure_reuse_buffers(agents_ctx* ctx) {
  if (ctx->reuse_tried) return;
  ctx->reuse_tried = true;
  if (ctx->ckpt_every != 0 || ctx->T < 2) return;
  void* p[4] = {nullptr, nullptr, nullptr, nullptr};
  const size_t sizes[4] = {(size_t)(ctx->T - 1) * ctx->nc, (size_t)(ctx->T - 1) * ctx->nc,
                           ctx->nc, ctx->nc};
  // only when a quarter of the device stays free afterwards
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const size_t need = (sizes[0] + sizes[1] + sizes[2] + sizes[3]) * sizeof(float);
  if (free_b < need || free_b - need < total_b / 4) return;
  if (!mem_reserve(need)) return;  // optional buffers: skipped under the memory limit
  for (int k = 0; k < 4; ++k) {
    if (cudaMalloc(&p[k], sizes[k] * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      for (int m = 0; m < k; ++m) cudaFree(p[m]);
      mem_release(need);
      return;
    }
  }
  for (int k = 0; k < 4; ++k) ctx->allocs.push_back(p[k]);
  ctx->held_bytes += need;
  ctx->traj_alt[0] = static_cast<float*>(p[0]);
  ctx->traj_alt[1] = static_cast<float*>(p[1]);
  ctx->cT_alt[0] = static_cast<float*>(p[2]);
  ctx->cT_alt[1] = static_cast<float*>(p[3]);
  ctx->reuse = true;
}

// Full-store forward sweep into a given trajectory buffer and final state.
int forward_sweep_into(agents_ctx* ctx, const double* d_eps, float* traj, float* dst_T) {
  NvtxRange nr("trial_sweep");
  const int T = ctx->T;
  std::vector<float*> dsts(T);
  for (int n = 0; n < T; ++n) dsts[n] = n == T - 1 ? dst_T : traj + (size_t)n * ctx->nc;
  return run_forward(ctx, ctx->c0, d_eps, dsts.data(), T);
}

// c(T) of the control in d_eps into dst: a copy of the stored final state when the stored
// trajectory belongs to that control, else a forward sweep.  Returns the steps executed.
int final_state(agents_ctx* ctx, float* dst, int64_t& steps) {
  if (ctx->reuse && ctx->traj_ok) {
    CK(cudaMemcpyAsync(dst, ctx->cT, ctx->nc * sizeof(float), cudaMemcpyDeviceToDevice,
                       ctx->stream));
    return AGENTS_OK;
  }
  TRY(forward_sweep(ctx, ctx->d_eps, dst, false));
  steps += ctx->T;
  return AGENTS_OK;
}

int ensure_solve_buffers(agents_ctx* ctx) {
  ensure_reuse_buffers(ctx);
  // each buffer on its own: an allocation refused part-way leaves the others usable
  if (!ctx->s_c) TRY(dalloc(ctx, &ctx->s_c, ctx->nc));
  if (!ctx->s_cn) TRY(dalloc(ctx, &ctx->s_cn, ctx->nc));
  if (!ctx->s_trial_c) TRY(dalloc(ctx, &ctx->s_trial_c, ctx->nc));
  if (!ctx->s_v) TRY(dalloc(ctx, &ctx->s_v, ctx->nv));
  if (!ctx->s_vn) TRY(dalloc(ctx, &ctx->s_vn, ctx->nv));
  if (!ctx->s_mu) TRY(dalloc(ctx, &ctx->s_mu, ctx->nv));
  return AGENTS_OK;
}

int read_control(agents_ctx* ctx, const double* eps, std::vector<double>& host) {
  host.resize(2 * (size_t)ctx->T);
  if (is_device_ptr(eps)) {
    CK(cudaMemcpyAsync(host.data(), eps, host.size() * sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    std::memcpy(host.data(), eps, host.size() * sizeof(double));
  }
  for (double e : host) {
    if (!std::isfinite(e)) return fail(ctx, AGENTS_EINVAL, "control contains NaN/Inf");
    if (e < 0.0) return fail(ctx, AGENTS_EINVAL, "control entries must be >= 0 (Eq. ellipsoid)");
  }
  return AGENTS_OK;
}

// One iteration of Algorithm 1 on L~(c(T; eps), v, mu), the control in ctx->d_eps:
// forward sweep with store, terminal adjoint and L~, reverse sweep, then the projected
// two-way Armijo search (stationarity, sufficient decrease with |P D|^2, strict decrease).
// Sets `ended` when the eps-step ends (stationary control or no admissible step); appends
// one record to ctx->log.  Returns AGENTS_EDIVERGED on a NaN/Inf objective.
int dal_iteration(agents_ctx* ctx, const agents_solve_opts& o, const float* v, const float* mu,
                  int outer, double& sigma, agents_solve_info& inf, std::vector<double>& Dh,
                  std::vector<double>& eps_h, bool& ended) {
  NvtxRange nr("dal_iteration");
  const int T = ctx->T;
  const double dt = ctx->p.dt;
  const double lo[2] = {ctx->p.eps_lo[0], ctx->p.eps_lo[1]};
  const double hi[2] = {ctx->p.eps_hi[0], ctx->p.eps_hi[1]};
  auto count_fwd = [&]() { inf.forward_steps += T; };
  ended = false;
  if (!(ctx->reuse && ctx->traj_ok)) {
    TRY(forward_sweep(ctx, ctx->d_eps, ctx->cT, true));
    count_fwd();
    ctx->traj_ok = ctx->reuse;
  }
  float* lam0 = nullptr;
  TRY(adjoint_sweep(ctx, ctx->d_eps, v, mu, 0, &lam0));
  inf.adjoint_steps += T;
  inf.tv_sweeps += 1;
  if (ctx->ckpt_every) inf.forward_steps += T - 1 - ctx->nckpt;
  double L0;
  TRY(fetch_scalar(ctx, 0, &L0));
  CK(cudaMemcpyAsync(Dh.data(), ctx->d_D, Dh.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(eps_h.data(), ctx->d_eps, eps_h.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ++inf.inner_done;
  agents_iter_record rec{outer, 0, 0, 0, L0, L0, 0.0, 0.0};
  if (!std::isfinite(L0)) return AGENTS_EDIVERGED;
  // Components the projection onto E does not block; |P D|^2 over those only.
  double g2 = 0.0;
  bool any_free = false;
  for (size_t i = 0; i < Dh.size(); ++i) {
    const int k = (int)(i & 1);
    const double d = Dh[i], e = eps_h[i];
    if (d != 0.0 && (e < hi[k] || d < 0.0) && (e > lo[k] || d > 0.0)) {
      any_free = true;
      g2 += d * d;
    }
  }
  g2 *= dt;
  rec.gnorm2 = g2;
  if (!std::isfinite(g2)) return AGENTS_EDIVERGED;
  if (!any_free) {  // variational inequality holds: the control is stationary
    ++inf.stationary;
    rec.status = 2;
    ctx->log.push_back(rec);
    ended = true;
    return AGENTS_OK;
  }
  int cur = 0, best = -1;
  double best_tau = 0.0, best_L = L0;
  auto trial = [&](double tau, bool& ok) -> int {
    CK(launch_control_step(ctx->d_eps, ctx->d_D, tau, ctx->d_lohi, ctx->d_trial[cur], T,
                           ctx->stream));
    ++ctx->launches;
    float* trial_c = ctx->s_trial_c;
    if (ctx->reuse) {   // keep the trial's trajectory: it is the next stored one if accepted
      trial_c = ctx->cT_alt[cur];
      TRY(forward_sweep_into(ctx, ctx->d_trial[cur], ctx->traj_alt[cur], trial_c));
    } else {
      TRY(forward_sweep(ctx, ctx->d_trial[cur], trial_c, false));
    }
    count_fwd();
    TRY(objective(ctx, trial_c, v, mu, nullptr, 1));
    inf.tv_sweeps += 1;
    ++inf.trials;
    double L;
    TRY(fetch_scalar(ctx, 1, &L));
    if (!std::isfinite(L)) return AGENTS_EDIVERGED;
    ok = (L < L0) && (L <= L0 - o.ls_c * tau * g2);
    if (ok) {
      best = cur;
      best_tau = tau;
      best_L = L;
      cur ^= 1;  // keep the passing trial; write the next one into the other buffer
    }
    return AGENTS_OK;
  };
  double tau = sigma;
  bool ok = false;
  int ntr = 1;
  int ts = trial(tau, ok);
  if (ts != AGENTS_OK) return ts;
  if (ok) {
    while (ntr < o.max_ls) {
      tau = tau / o.ls_b;
      ++ntr;
      ts = trial(tau, ok);
      if (ts != AGENTS_OK || !ok) break;
    }
  } else {
    while (ntr < o.max_ls) {
      tau = tau * o.ls_b;
      ++ntr;
      ts = trial(tau, ok);
      if (ts != AGENTS_OK || ok) break;
    }
  }
  if (ts != AGENTS_OK) return ts;
  rec.trials = ntr;
  if (best < 0) {
    ++inf.stalls;
    rec.status = 1;
    ctx->log.push_back(rec);
    ended = true;
    return AGENTS_OK;
  }
  rec.L = best_L;
  rec.tau = best_tau;
  ctx->log.push_back(rec);
  CK(cudaMemcpyAsync(ctx->d_eps, ctx->d_trial[best], 2 * (size_t)T * sizeof(double),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  if (ctx->reuse) {   // the accepted trial's trajectory becomes the stored one
    std::swap(ctx->traj, ctx->traj_alt[best]);
    std::swap(ctx->cT, ctx->cT_alt[best]);
    ctx->traj_ok = true;
  }
  sigma = best_tau;
  return AGENTS_OK;
}

int validate_opts(agents_ctx* ctx, const agents_solve_opts& o) {
  if (o.k_out < 0 || o.k_in < 0 || o.max_ls < 1 || !(o.sigma0 > 0) || !(o.ls_b > 0 && o.ls_b < 1) ||
      !(o.ls_c > 0 && o.ls_c < 1) || !(o.tol >= 0))
    return fail(ctx, AGENTS_EINVAL, "invalid solve options");
  return AGENTS_OK;
}

}  // namespace

namespace agents {
int ctx_fail(agents_ctx* ctx, int code, const char* msg) { return fail(ctx, code, "%s", msg); }
int ctx_forward_sweep(agents_ctx* ctx, const double* d_eps, float* dst_T, bool store) {
  return forward_sweep(ctx, d_eps, dst_T, store);
}
}  // namespace agents

// ====================================================================== C ABI
extern "C" {

void agents_default_params(agents_params* p, int32_t height, int32_t width, int32_t channels,
                           int32_t radius, int32_t nsteps) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->height = height;
  p->width = width;
  p->channels = channels;
  p->radius = radius;
  p->nsteps = nsteps;
  p->dt = 0.25;
  p->alpha = 3000.0;
  p->rho = 1e-2;
  p->gamma = 1e-2;
  p->eps_lo[0] = p->eps_lo[1] = 2.0;
  p->eps_hi[0] = p->eps_hi[1] = 1100.0;
  p->norm_mode = 0;
  p->tv_mode = 0;
  p->traj_mode = 0;
}

void agents_default_solve_opts(agents_solve_opts* o) {
  if (!o) return;
  o->k_out = 10;
  o->k_in = 30;
  o->max_ls = 30;
  o->sigma0 = 1.0;
  o->ls_b = 0.5;
  o->ls_c = 1e-4;
  o->tol = 0.0;
}

const char* agents_last_error(const agents_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_init_error.c_str();
}

int agents_destroy(agents_ctx* ctx) {
  if (!ctx) return AGENTS_OK;
  DeviceGuard dg(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (void* p : ctx->allocs) cudaFree(p);
  mem_release(ctx->held_bytes);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  delete ctx;
  return AGENTS_OK;
}

int agents_init(const agents_params* p, const float* c0, void* cuda_stream, agents_ctx** out) {
  g_init_error.clear();
  if (!out) return fail(nullptr, AGENTS_EINVAL, "out is NULL");
  *out = nullptr;
  TRY(validate(p));
  if (!c0) return fail(nullptr, AGENTS_EINVAL, "c0 is NULL");
  agents_ctx* ctx = new (std::nothrow) agents_ctx();
  if (!ctx) return fail(nullptr, AGENTS_ENOMEM, "host allocation failed");
  ctx->p = *p;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&ctx->device);
  const int H = p->height, W = p->width, C = p->channels, T = p->nsteps;
  ctx->N = H * W;
  ctx->C = C;
  ctx->T = T;
  ctx->nc = (size_t)ctx->N * C;
  ctx->nv = ctx->nc * 2;
  ctx->M = p->norm_mode == 0 ? (double)(2 * p->radius + 1) * (2 * p->radius + 1) : (double)ctx->N;
  ctx->sg = SweepGeom{H, W, C, p->radius, (float)(1.0 / ((double)W * W)),
                      (float)(1.0 / ((double)H * H)), (float)(p->dt / ctx->M)};
  ctx->tg = TvGeom{H, W, C, (float)(0.5 * W), (float)(0.5 * H), (float)p->rho,
                   (float)(1.0 / p->rho), (float)p->alpha, p->gamma,
                   1.0 / ((double)W * (double)H), p->tv_mode};
  ctx->ckpt_every = p->traj_mode >= T ? 0 : p->traj_mode;
  ctx->nb_adj = adjoint_num_blocks(ctx->sg);
  ctx->nb_tv = tv_num_blocks(ctx->tg);

  auto bail = [&](int st) {
    std::string msg = ctx->err;
    agents_destroy(ctx);
    g_init_error = msg;
    return st;
  };
  int st = AGENTS_OK;
#define INIT_TRY(expr)                \
  do {                                \
    st = (expr);                      \
    if (st != AGENTS_OK) return bail(st); \
  } while (0)
  INIT_TRY(dalloc(ctx, &ctx->c0, ctx->nc));
  INIT_TRY(dalloc(ctx, &ctx->cT, ctx->nc));
  INIT_TRY(dalloc(ctx, &ctx->work[0], ctx->nc));
  INIT_TRY(dalloc(ctx, &ctx->work[1], ctx->nc));
  INIT_TRY(dalloc(ctx, &ctx->lam[0], ctx->nc));
  INIT_TRY(dalloc(ctx, &ctx->lam[1], ctx->nc));
  if (ctx->ckpt_every == 0) {
    ctx->nckpt = T - 1;
    INIT_TRY(dalloc(ctx, &ctx->traj, ctx->nc * (size_t)std::max(T - 1, 1)));
  } else {
    const int k = ctx->ckpt_every;
    ctx->nckpt = (T - 1) / k;  // states k, 2k, ... <= T-1
    INIT_TRY(dalloc(ctx, &ctx->traj, ctx->nc * (size_t)std::max(ctx->nckpt, 1)));
    INIT_TRY(dalloc(ctx, &ctx->seg, ctx->nc * (size_t)std::max(k - 1, 1)));
  }
  INIT_TRY(dalloc(ctx, &ctx->d_eps, 2 * (size_t)T));
  INIT_TRY(dalloc(ctx, &ctx->d_trial[0], 2 * (size_t)T));
  INIT_TRY(dalloc(ctx, &ctx->d_trial[1], 2 * (size_t)T));
  INIT_TRY(dalloc(ctx, &ctx->d_D, 2 * (size_t)T));
  INIT_TRY(dalloc(ctx, &ctx->d_lohi, 4));
  INIT_TRY(dalloc(ctx, &ctx->d_part_adj, (size_t)T * ctx->nb_adj * 2));
  INIT_TRY(dalloc(ctx, &ctx->d_part_tv, (size_t)ctx->nb_tv * 5));
  INIT_TRY(dalloc(ctx, &ctx->d_scal, 16));
  ctx->fused_tiles = fused_num_tiles(ctx->sg);
  ctx->fused_cap_adj = ctx->fused_tiles > 0 ? fused_adjoint_capacity(ctx->sg) : 0;
  if (ctx->fused_tiles > 0)
    INIT_TRY(dalloc(ctx, &ctx->d_fsync, fused_sync_words(ctx->fused_tiles)));
  INIT_TRY(dalloc(ctx, &ctx->d_labels, (size_t)ctx->N));
  INIT_TRY(dalloc(ctx, &ctx->d_lstat, 2));
  {
    cudaError_t e = cudaMallocHost(&ctx->h_scal, 16 * sizeof(double));
    if (e != cudaSuccess) {
      ctx->err = std::string("cudaMallocHost failed: ") + cudaGetErrorString(e);
      return bail(AGENTS_ENOMEM);
    }
  }
  const double lohi[4] = {p->eps_lo[0], p->eps_lo[1], p->eps_hi[0], p->eps_hi[1]};
  {
    cudaError_t e = cudaMemcpyAsync(ctx->d_lohi, lohi, sizeof(lohi), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e != cudaSuccess) {
      ctx->err = std::string("copy of the box failed: ") + cudaGetErrorString(e);
      return bail(AGENTS_ECUDA);
    }
  }
  {
    cudaError_t e = cudaMemsetAsync(ctx->d_scal, 0, 16 * sizeof(double), ctx->stream);
    if (e == cudaSuccess && ctx->d_fsync)
      e = cudaMemsetAsync(ctx->d_fsync, 0,
                          fused_sync_words(ctx->fused_tiles) * sizeof(unsigned int), ctx->stream);
    if (e != cudaSuccess) {
      ctx->err = std::string("clearing the sweep flags failed: ") + cudaGetErrorString(e);
      return bail(AGENTS_ECUDA);
    }
  }
  INIT_TRY(to_device(ctx, ctx->c0, c0, ctx->nc * sizeof(float)));
  {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      ctx->err = std::string("init synchronisation failed: ") + cudaGetErrorString(e);
      return bail(AGENTS_ECUDA);
    }
  }
#undef INIT_TRY
  *out = ctx;
  return AGENTS_OK;
}

int agents_set_image(agents_ctx* ctx, const float* c0) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (!c0) return fail(ctx, AGENTS_EINVAL, "c0 is NULL");
  DeviceGuard dg(ctx->device);
  ctx->stored = false;
  return to_device(ctx, ctx->c0, c0, ctx->nc * sizeof(float));
}

int agents_forward(agents_ctx* ctx, const double* eps, float* cT_dev, int store) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (!eps) return fail(ctx, AGENTS_EINVAL, "eps is NULL");
  TRY(check_aligned(ctx, cT_dev, "cT_dev"));
  DeviceGuard dg(ctx->device);
  std::vector<double> host;
  TRY(read_control(ctx, eps, host));
  CK(cudaMemcpyAsync(ctx->d_eps, host.data(), host.size() * sizeof(double),
                     cudaMemcpyHostToDevice, ctx->stream));
  TRY(forward_sweep(ctx, ctx->d_eps, ctx->cT, store != 0));
  if (cT_dev) CK(cudaMemcpyAsync(cT_dev, ctx->cT, ctx->nc * sizeof(float),
                                 cudaMemcpyDeviceToDevice, ctx->stream));
  if (store) {
    ctx->stored = true;
    ctx->stored_eps = host;
  } else {
    ctx->stored = false;  // cT and the work buffers were overwritten
  }
  CK(cudaStreamSynchronize(ctx->stream));  // host control buffer goes out of scope
  return fused_check(ctx);
}

int agents_adjoint(agents_ctx* ctx, const double* eps, const float* v_dev, const float* mu_dev,
                   double* D_out, double* obj_out, float* lambda0_dev) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (!eps || !D_out) return fail(ctx, AGENTS_EINVAL, "eps and D_out must not be NULL");
  TRY(need(ctx, v_dev, "v_dev"));
  TRY(need(ctx, mu_dev, "mu_dev"));
  TRY(check_aligned(ctx, lambda0_dev, "lambda0_dev"));
  DeviceGuard dg(ctx->device);
  std::vector<double> host;
  TRY(read_control(ctx, eps, host));
  if (!ctx->stored || host != ctx->stored_eps)
    return fail(ctx, AGENTS_ESTATE, "agents_adjoint needs a preceding agents_forward(store=1) "
                                    "with the same control");
  float* lam0 = nullptr;
  TRY(adjoint_sweep(ctx, ctx->d_eps, v_dev, mu_dev, 0, &lam0));
  if (lambda0_dev) CK(cudaMemcpyAsync(lambda0_dev, lam0, ctx->nc * sizeof(float),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
  if (obj_out) TRY(from_device(ctx, obj_out, ctx->d_scal + 0, sizeof(double)));
  TRY(from_device(ctx, D_out, ctx->d_D, 2 * (size_t)ctx->T * sizeof(double)));
  return AGENTS_OK;
}

int agents_adjoint_from(agents_ctx* ctx, const double* eps, const float* lambdaT_dev,
                        double* D_out, float* lambda0_dev) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (!eps || !D_out) return fail(ctx, AGENTS_EINVAL, "eps and D_out must not be NULL");
  TRY(need(ctx, lambdaT_dev, "lambdaT_dev"));
  TRY(check_aligned(ctx, lambda0_dev, "lambda0_dev"));
  DeviceGuard dg(ctx->device);
  std::vector<double> host;
  TRY(read_control(ctx, eps, host));
  if (!ctx->stored || host != ctx->stored_eps)
    return fail(ctx, AGENTS_ESTATE, "agents_adjoint_from needs a preceding "
                                    "agents_forward(store=1) with the same control");
  CK(cudaMemcpyAsync(ctx->lam[0], lambdaT_dev, ctx->nc * sizeof(float),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  float* lam0 = nullptr;
  TRY(adjoint_sweep_from(ctx, ctx->d_eps, &lam0));
  if (lambda0_dev) CK(cudaMemcpyAsync(lambda0_dev, lam0, ctx->nc * sizeof(float),
                                      cudaMemcpyDeviceToDevice, ctx->stream));
  TRY(from_device(ctx, D_out, ctx->d_D, 2 * (size_t)ctx->T * sizeof(double)));
  return AGENTS_OK;
}

int agents_flow_backward(agents_ctx* ctx, const double* eps, const float* grad_cT_dev,
                         double* grad_eps_out, float* grad_c0_dev) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (!eps) return fail(ctx, AGENTS_EINVAL, "eps must not be NULL");
  TRY(need(ctx, grad_cT_dev, "grad_cT_dev"));
  TRY(check_aligned(ctx, grad_c0_dev, "grad_c0_dev"));
  DeviceGuard dg(ctx->device);
  std::vector<double> host;
  TRY(read_control(ctx, eps, host));
  if (!ctx->stored || host != ctx->stored_eps)
    return fail(ctx, AGENTS_ESTATE, "agents_flow_backward needs a preceding "
                                    "agents_forward(store=1) with the same control");
  // lambda^T = -dL/dc^T
  CK(launch_scale_f32(grad_cT_dev, -1.0f, ctx->lam[0], ctx->nc, ctx->stream));
  ++ctx->launches;
  float* lam0 = nullptr;
  TRY(adjoint_sweep_from(ctx, ctx->d_eps, &lam0));
  if (grad_c0_dev) {  // dL/dc^0 = -lambda^0
    CK(launch_scale_f32(lam0, -1.0f, grad_c0_dev, ctx->nc, ctx->stream));
    ++ctx->launches;
  }
  if (grad_eps_out) {  // dL/deps^n = -dt D^n, reduced from the same partials
    CK(launch_reduce_rows(ctx->d_part_adj, ctx->nb_adj, 2, ctx->T, -ctx->p.dt / (2.0 * ctx->M),
                          ctx->d_trial[0], ctx->stream));
    ++ctx->launches;
    TRY(from_device(ctx, grad_eps_out, ctx->d_trial[0], 2 * (size_t)ctx->T * sizeof(double)));
  }
  return AGENTS_OK;
}

int agents_objective(agents_ctx* ctx, const float* c_dev, const float* v_dev,
                     const float* mu_dev, double* obj_out, float* lambda_dev) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  TRY(need(ctx, c_dev, "c_dev"));
  TRY(need(ctx, v_dev, "v_dev"));
  TRY(need(ctx, mu_dev, "mu_dev"));
  TRY(check_aligned(ctx, lambda_dev, "lambda_dev"));
  DeviceGuard dg(ctx->device);
  TRY(objective(ctx, c_dev, v_dev, mu_dev, lambda_dev, 1));
  if (obj_out) TRY(from_device(ctx, obj_out, ctx->d_scal + 1, sizeof(double)));
  return AGENTS_OK;
}

int pd_tv_step(agents_ctx* ctx, const float* c_dev, const float* mu_dev, float* v_dev) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  TRY(need(ctx, c_dev, "c_dev"));
  TRY(need(ctx, mu_dev, "mu_dev"));
  TRY(need(ctx, v_dev, "v_dev"));
  DeviceGuard dg(ctx->device);
  CK(launch_pd_tv_step(c_dev, mu_dev, v_dev, ctx->tg, ctx->stream));
  return AGENTS_OK;
}

int alm_update(agents_ctx* ctx, const float* c_dev, const float* c_prev_dev, const float* v_dev,
               const float* v_prev_dev, float* mu_dev, double* stats) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  TRY(need(ctx, c_dev, "c_dev"));
  TRY(need(ctx, v_dev, "v_dev"));
  TRY(need(ctx, mu_dev, "mu_dev"));
  TRY(check_aligned(ctx, c_prev_dev, "c_prev_dev"));
  TRY(check_aligned(ctx, v_prev_dev, "v_prev_dev"));
  DeviceGuard dg(ctx->device);
  double* d_stats = (stats && is_device_ptr(stats)) ? stats : nullptr;
  double* h_stats = (stats && !d_stats) ? stats : nullptr;
  return alm(ctx, c_dev, c_prev_dev, v_dev, v_prev_dev, mu_dev, h_stats, d_stats);
}

int agents_solve_log(const agents_ctx* ctx, agents_iter_record* out, int32_t capacity,
                     int32_t* count) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (count) *count = (int32_t)ctx->log.size();
  if (out && capacity > 0) {
    const size_t n = std::min((size_t)capacity, ctx->log.size());
    std::memcpy(out, ctx->log.data(), n * sizeof(agents_iter_record));
  }
  return AGENTS_OK;
}

int agents_solve_outer_log(const agents_ctx* ctx, agents_outer_record* out, int32_t capacity,
                           int32_t* count) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (count) *count = (int32_t)ctx->outer_log.size();
  if (out && capacity > 0) {
    const size_t n = std::min((size_t)capacity, ctx->outer_log.size());
    std::memcpy(out, ctx->outer_log.data(), n * sizeof(agents_outer_record));
  }
  return AGENTS_OK;
}

int agents_labels(agents_ctx* ctx, const float* c_dev, float threshold, int32_t* labels_out,
                  int32_t* count_out) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  TRY(need(ctx, c_dev, "c_dev"));
  if (!labels_out) return fail(ctx, AGENTS_EINVAL, "labels_out is NULL");
  DeviceGuard dg(ctx->device);
  CK(launch_labels(c_dev, ctx->p.height, ctx->p.width, ctx->C, threshold, label_loop_cap(),
                   ctx->d_labels, ctx->d_lstat, ctx->d_lstat + 1, ctx->stream));
  int32_t hs[2];
  CK(cudaMemcpyAsync(hs, ctx->d_lstat, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hs[1] != 0) return fail(ctx, AGENTS_ETIMEOUT, "label union-find exceeded its loop bound");
  if (count_out) *count_out = hs[0];
  TRY(from_device(ctx, labels_out, ctx->d_labels, (size_t)ctx->N * sizeof(int32_t)));
  return AGENTS_OK;
}

int dal_solve(agents_ctx* ctx, const agents_solve_opts* opts, double* eps_io, float* c_out,
              agents_solve_info* info) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (!opts || !eps_io) return fail(ctx, AGENTS_EINVAL, "opts and eps_io must not be NULL");
  const agents_solve_opts o = *opts;
  TRY(validate_opts(ctx, o));
  DeviceGuard dg(ctx->device);
  TRY(ensure_solve_buffers(ctx));
  const int64_t launches0 = ctx->launches;
  const int T = ctx->T;
  agents_solve_info inf{};
  std::vector<double> eps_h;
  TRY(read_control(ctx, eps_io, eps_h));
  ctx->log.clear();
  CK(cudaMemcpyAsync(ctx->d_eps, eps_h.data(), eps_h.size() * sizeof(double),
                     cudaMemcpyHostToDevice, ctx->stream));
  // v = mu = 0: L~(c, 0, 0) = dx dy sum [rho/2 |G c|^2 + alpha/2 |c - c0|^2]
  CK(cudaMemsetAsync(ctx->s_v, 0, ctx->nv * sizeof(float), ctx->stream));
  CK(cudaMemsetAsync(ctx->s_mu, 0, ctx->nv * sizeof(float), ctx->stream));
  ctx->stored = false;
  ctx->traj_ok = false;
  double sigma = o.sigma0;
  std::vector<double> Dh(2 * (size_t)T);
  int status = AGENTS_OK;
  for (int it = 0; it < o.k_in; ++it) {
    bool ended = false;
    status = dal_iteration(ctx, o, ctx->s_v, ctx->s_mu, 1, sigma, inf, Dh, eps_h, ended);
    if (status != AGENTS_OK || ended) break;
    const agents_iter_record& r = ctx->log.back();
    inf.final_obj = r.L;
    inf.final_res = r.L0 != 0.0 ? std::fabs(r.L - r.L0) / std::fabs(r.L0) : 0.0;
    if (o.tol > 0.0 && inf.final_res < o.tol) break;   // relative cost change below eta
  }
  ctx->stored = false;
  TRY(from_device(ctx, eps_io, ctx->d_eps, 2 * (size_t)T * sizeof(double)));
  if (c_out) {
    TRY(final_state(ctx, ctx->s_c, inf.forward_steps));
    TRY(from_device(ctx, c_out, ctx->s_c, ctx->nc * sizeof(float)));
  }
  ctx->traj_ok = false;
  CK(cudaStreamSynchronize(ctx->stream));
  inf.final_sigma = sigma;
  inf.kernel_launches = ctx->launches - launches0;
  if (info) *info = inf;
  if (status == AGENTS_EDIVERGED) return fail(ctx, status, "DAL diverged (NaN/Inf)");
  return status;
}

int solve(agents_ctx* ctx, const agents_solve_opts* opts, double* eps_io, float* mu_io,
          float* v_out, float* c_out, int32_t* labels_out, agents_solve_info* info) {
  if (!ctx) return fail(nullptr, AGENTS_EINVAL, "ctx is NULL");
  if (!opts || !eps_io || !mu_io) return fail(ctx, AGENTS_EINVAL, "opts, eps_io, mu_io must not be NULL");
  const agents_solve_opts o = *opts;
  TRY(validate_opts(ctx, o));
  DeviceGuard dg(ctx->device);
  TRY(ensure_solve_buffers(ctx));
  const int64_t launches0 = ctx->launches;
  const int T = ctx->T;
  agents_solve_info inf{};
  auto count_fwd = [&]() { inf.forward_steps += T; };

  std::vector<double> eps_h;
  TRY(read_control(ctx, eps_io, eps_h));
  ctx->log.clear();
  ctx->outer_log.clear();
  NvtxRange nr("solve");
  CK(cudaMemcpyAsync(ctx->d_eps, eps_h.data(), eps_h.size() * sizeof(double),
                     cudaMemcpyHostToDevice, ctx->stream));
  TRY(to_device(ctx, ctx->s_mu, mu_io, ctx->nv * sizeof(float)));
  ctx->stored = false;
  ctx->traj_ok = false;

  double sigma = o.sigma0;
  float *c = ctx->s_c, *cn = ctx->s_cn, *v = ctx->s_v, *vn = ctx->s_vn, *mu = ctx->s_mu;
  // c^(0) = c(T; eps^(0)),  v^(0) = argmin_v L(c^(0), v, mu^(0))
  if (ctx->reuse) {   // stored sweep: the first DAL iteration reuses it
    TRY(forward_sweep(ctx, ctx->d_eps, ctx->cT, true));
    ctx->traj_ok = true;
    CK(cudaMemcpyAsync(c, ctx->cT, ctx->nc * sizeof(float), cudaMemcpyDeviceToDevice,
                       ctx->stream));
  } else {
    TRY(forward_sweep(ctx, ctx->d_eps, c, false));
  }
  count_fwd();
  CK(launch_pd_tv_step(c, mu, v, ctx->tg, ctx->stream));
  ++ctx->launches;
  TRY(objective(ctx, c, v, mu, nullptr, 2));
  inf.tv_sweeps += 2;
  double L_prev;
  TRY(fetch_scalar(ctx, 2, &L_prev));
  int status = AGENTS_OK;
  std::vector<double> Dh(2 * (size_t)T);

  for (int j = 1; j <= o.k_out && status == AGENTS_OK; ++j) {
    const int inner0 = inf.inner_done;
    // ---- eps-step: k_in iterations of Algorithm 1 on L~(c(T; eps), v, mu)
    for (int it = 0; it < o.k_in; ++it) {
      bool ended = false;
      const int st = dal_iteration(ctx, o, v, mu, j, sigma, inf, Dh, eps_h, ended);
      if (st != AGENTS_OK) { status = st; break; }
      if (ended) break;
    }
    if (status != AGENTS_OK) break;
    // ---- c^(j), v^(j), mu^(j)
    TRY(final_state(ctx, cn, inf.forward_steps));
    CK(launch_pd_tv_step(cn, mu, vn, ctx->tg, ctx->stream));
    ++ctx->launches;
    double st[5];
    TRY(alm(ctx, cn, c, vn, v, mu, st, nullptr));
    TRY(objective(ctx, cn, vn, mu, nullptr, 2));
    inf.tv_sweeps += 3;
    double L_new;
    TRY(fetch_scalar(ctx, 2, &L_new));
    std::swap(c, cn);
    std::swap(v, vn);
    inf.outer_done = j;
    if (!std::isfinite(L_new) || !std::isfinite(st[0]) || !std::isfinite(st[1])) {
      status = AGENTS_EDIVERGED;
      break;
    }
    const double dL = L_prev != 0.0 ? std::fabs(L_new - L_prev) / std::fabs(L_prev) : 0.0;
    inf.final_res = std::max(st[3], dL);
    inf.final_obj = L_new;
    inf.final_gap = st[2];
    ctx->outer_log.push_back(agents_outer_record{j, inf.inner_done - inner0, L_new, st[4], st[0],
                                                 st[1], st[2], st[3], inf.final_res, sigma});
    L_prev = L_new;
    if (o.tol > 0.0 && inf.final_res < o.tol) break;
  }
  ctx->stored = false;
  ctx->traj_ok = false;
  // outputs
  TRY(from_device(ctx, eps_io, ctx->d_eps, 2 * (size_t)T * sizeof(double)));
  TRY(from_device(ctx, mu_io, mu, ctx->nv * sizeof(float)));
  if (v_out) TRY(from_device(ctx, v_out, v, ctx->nv * sizeof(float)));
  if (c_out) TRY(from_device(ctx, c_out, c, ctx->nc * sizeof(float)));
  int32_t lstat[2] = {0, 0};  // {count, status} of the label union-find
  if (labels_out) {
    CK(launch_labels(c, ctx->p.height, ctx->p.width, ctx->C, 0.02f, label_loop_cap(),
                     ctx->d_labels, ctx->d_lstat, ctx->d_lstat + 1, ctx->stream));
    ctx->launches += 3;
    TRY(from_device(ctx, labels_out, ctx->d_labels, (size_t)ctx->N * sizeof(int32_t)));
    CK(cudaMemcpyAsync(lstat, ctx->d_lstat, sizeof(lstat), cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  inf.final_sigma = sigma;
  inf.kernel_launches = ctx->launches - launches0;
  if (info) *info = inf;
  if (status == AGENTS_EDIVERGED) return fail(ctx, status, "solve diverged (NaN/Inf)");
  if (status == AGENTS_OK && lstat[1] != 0)
    return fail(ctx, AGENTS_ETIMEOUT, "label union-find exceeded its loop bound");
  return status;
}

}  // extern "C"
