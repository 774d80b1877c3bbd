// agents_solve_batch: Algorithm 2 (with Algorithm 1 inside) for many images of uneven size,
// channel count and window radius at once.
//
// Every sweep step is one persistent launch per (R, C) class that walks a job list of
// (image, tile) pairs over all images of the class; the TV kernels do the same per channel
// count.  The Armijo search of every image runs as a small state machine on the device
// (prepare -> [control step, trial sweep, objective, decide]* -> accept), so the launch
// sequences of one DAL sweep, one Armijo round and one multiplier step are static: each
// is captured once as a CUDA graph and replayed.  The host synchronises once per Armijo
// round (for all images together) to learn whether any image still searches.  Images
// whose epsilon-step or whole solve has ended are skipped by every kernel (their jobs
// exit at once).  The per-pixel arithmetic and the decision logic are those of solve(),
// so with the default tile shape each image's result is bitwise that of solve().
//
// An autotuner picks the tile shape of each (R, C) class by timing one Euler step of the
// class with every shape; choices are cached per (R, C, size bucket) for the process.
#include "agents.h"
#include "common.cuh"
#include "ctx_internal.h"
#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

using namespace agents;

namespace {

struct BatchState {
  double L0, g2, tau, best_tau, best_L, sigma;
  double L_prev, res, obj, gap;
  int phase;      // 0 idle, 1 first trial, 2 growing, 3 shrinking
  int ntr, found;
  int eps_active, outer_active, diverged;
  int outer_done, inner_done, trials, stalls, stationary;
  long long fwd, adj, tv;
};

struct BatchCtl {
  double* eps;        // control, [T][2]
  double* trial;      // trial control
  double* best;       // last passing trial control
  const double* D;    // D^n, [T][2]
  const double* scal; // [0] L0 (terminal), [1] trial L, [2] outer L, [8..12] ALM raw sums
  double lo[2], hi[2];
  double dt, rho, gamma, cell;
};

struct Counters {
  int trial_active, eps_active, outer_active, pad;
};

enum { kPhaseIdle = 0, kPhaseFirst = 1, kPhaseGrow = 2, kPhaseShrink = 3 };

// ---------------------------------------------------------------- state machine kernels
__global__ void batch_init_kernel(BatchState* st, const BatchCtl* ctl, int n, double sigma0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  BatchState s{};
  s.sigma = sigma0;
  s.outer_active = 1;
  s.eps_active = 1;
  s.L_prev = ctl[i].scal[2];
  s.fwd = 0;
  st[i] = s;
}

// Start an epsilon-step: every image still in the solve becomes eps-active.
__global__ void batch_begin_eps_kernel(BatchState* st, int* eps_active, Counters* cnt, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  st[i].eps_active = st[i].outer_active;
  eps_active[i] = st[i].eps_active;
  if (st[i].eps_active) atomicAdd(&cnt->eps_active, 1);
}

// After the stored sweep, the terminal objective and the reverse sweep: stationarity test
// and the first trial step (same arithmetic as dal_iteration in agents.cu).
__global__ void batch_prepare_kernel(BatchState* st, const BatchCtl* ctl, int* eps_active,
                                     int* trial_active, Counters* cnt, int n, int T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  trial_active[i] = 0;
  BatchState& s = st[i];
  if (!eps_active[i]) return;
  const BatchCtl& c = ctl[i];
  s.fwd += T;
  s.adj += T;
  s.tv += 1;
  s.inner_done += 1;
  s.L0 = c.scal[0];
  if (!isfinite(s.L0)) {
    s.diverged = 1;
    s.eps_active = s.outer_active = 0;
    eps_active[i] = 0;
    return;
  }
  double g2 = 0.0;
  bool any_free = false;
  for (int k = 0; k < 2 * T; ++k) {
    const int m = k & 1;
    const double d = c.D[k], e = c.eps[k];
    if (d != 0.0 && (e < c.hi[m] || d < 0.0) && (e > c.lo[m] || d > 0.0)) {
      any_free = true;
      g2 += d * d;
    }
  }
  s.g2 = g2 * c.dt;
  if (!isfinite(s.g2)) {
    s.diverged = 1;
    s.eps_active = s.outer_active = 0;
    eps_active[i] = 0;
    return;
  }
  if (!any_free) {
    s.stationary += 1;
    s.eps_active = 0;
    eps_active[i] = 0;
    return;
  }
  s.phase = kPhaseFirst;
  s.tau = s.sigma;
  s.ntr = 0;
  s.found = 0;
  trial_active[i] = 1;
  atomicAdd(&cnt->trial_active, 1);
}

// trial = Pi_E(eps + tau D) for every searching image (one block per image).
__global__ void batch_control_kernel(const BatchState* st, const BatchCtl* ctl,
                                     const int* trial_active, int T) {
  const int i = blockIdx.x;
  if (!trial_active[i]) return;
  const BatchCtl& c = ctl[i];
  const double tau = st[i].tau;
  for (int k = threadIdx.x; k < 2 * T; k += blockDim.x) {
    const int m = k & 1;
    const double e = fma(tau, c.D[k], c.eps[k]);
    c.trial[k] = fmin(fmax(e, c.lo[m]), c.hi[m]);
  }
}

// Armijo test of the trial just evaluated; the two-way search of solve() as a state
// machine.  A passing trial's control is kept in ctl.best (one block per image).
__global__ void batch_decide_kernel(BatchState* st, const BatchCtl* ctl, int* trial_active,
                                    Counters* cnt, int T, double ls_b, double ls_c, int max_ls) {
  const int i = blockIdx.x;
  __shared__ int keep;
  if (threadIdx.x == 0) {
    keep = 0;
    if (trial_active[i]) {
      BatchState& s = st[i];
      const double L = ctl[i].scal[1];
      s.fwd += T;
      s.tv += 1;
      s.trials += 1;
      s.ntr += 1;
      if (!isfinite(L)) {
        s.diverged = 1;
        s.phase = kPhaseIdle;
        s.eps_active = s.outer_active = 0;
      } else {
        const bool ok = (L < s.L0) && (L <= s.L0 - ls_c * s.tau * s.g2);
        if (ok) {
          s.found = 1;
          s.best_tau = s.tau;
          s.best_L = L;
          keep = 1;
        }
        if (s.phase == kPhaseFirst) {
          if (ok) { s.phase = kPhaseGrow; s.tau = s.tau / ls_b; }
          else { s.phase = kPhaseShrink; s.tau = s.tau * ls_b; }
        } else if (s.phase == kPhaseGrow) {
          if (ok) s.tau = s.tau / ls_b;
          else s.phase = kPhaseIdle;
        } else if (s.phase == kPhaseShrink) {
          if (ok) s.phase = kPhaseIdle;
          else s.tau = s.tau * ls_b;
        }
        if (s.ntr >= max_ls) s.phase = kPhaseIdle;
      }
      trial_active[i] = s.phase != kPhaseIdle;
      if (trial_active[i]) atomicAdd(&cnt->trial_active, 1);
    }
  }
  __syncthreads();
  if (keep) {
    const BatchCtl& c = ctl[i];
    for (int k = threadIdx.x; k < 2 * T; k += blockDim.x) c.best[k] = c.trial[k];
  }
}

// End of a DAL iteration: adopt the best trial, or end the epsilon-step (stall).
__global__ void batch_accept_kernel(BatchState* st, const BatchCtl* ctl, int* eps_active,
                                    Counters* cnt, int T) {
  const int i = blockIdx.x;
  __shared__ int adopt;
  if (threadIdx.x == 0) {
    adopt = 0;
    BatchState& s = st[i];
    if (eps_active[i] && s.eps_active) {
      if (s.found) {
        adopt = 1;
        s.sigma = s.best_tau;
      } else {
        s.stalls += 1;
        s.eps_active = 0;
      }
    }
    eps_active[i] = s.eps_active;
    if (s.eps_active) atomicAdd(&cnt->eps_active, 1);
  }
  __syncthreads();
  if (adopt) {
    const BatchCtl& c = ctl[i];
    for (int k = threadIdx.x; k < 2 * T; k += blockDim.x) c.eps[k] = c.best[k];
  }
}

// End of a multiplier step: residuals, objective, tolerance test.
__global__ void batch_outer_kernel(BatchState* st, const BatchCtl* ctl, int* outer_active,
                                   Counters* cnt, int n, int j, int T, double tol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  BatchState& s = st[i];
  if (!outer_active[i]) return;
  const BatchCtl& c = ctl[i];
  s.fwd += T;
  s.tv += 3;
  const double* raw = c.scal + 8;
  const double r0 = sqrt(raw[0]), r1 = c.rho * sqrt(raw[1]);
  const double rel = raw[3] > 0.0 ? sqrt(raw[2] / raw[3]) : 0.0;
  const double L_new = c.scal[2];
  s.outer_done = j;
  if (!isfinite(L_new) || !isfinite(r0) || !isfinite(r1)) {
    s.diverged = 1;
    s.outer_active = 0;
  } else {
    const double dL = s.L_prev != 0.0 ? fabs(L_new - s.L_prev) / fabs(s.L_prev) : 0.0;
    s.res = fmax(rel, dL);
    s.obj = L_new;
    s.gap = c.gamma * c.cell * raw[0];
    s.L_prev = L_new;
    if (tol > 0.0 && s.res < tol) s.outer_active = 0;
  }
  outer_active[i] = s.outer_active;
  if (s.outer_active) atomicAdd(&cnt->outer_active, 1);
}

// dst_i <- src_i for the active images (blockIdx.y = image).
struct CopySeg {
  const float* src;
  float* dst;
  size_t count;
};
__global__ void batch_copy_kernel(const CopySeg* segs, const int* active) {
  const int i = blockIdx.y;
  if (!active[i]) return;
  const CopySeg sg = segs[i];
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < sg.count;
       k += (size_t)gridDim.x * blockDim.x)
    sg.dst[k] = sg.src[k];
}

// ---------------------------------------------------------------- host side
// Owning device buffer; move-only, so a moved-from buffer never frees the memory.
template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      if (p) cudaFree(p);
      p = o.p; n = o.n;
      o.p = nullptr; o.n = 0;
    }
    return *this;
  }
  cudaError_t alloc(size_t count) {
    if (p) { cudaFree(p); p = nullptr; }
    n = count ? count : 1;
    return cudaMalloc(&p, n * sizeof(T));
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

struct SweepClass {
  int R, C, shape;
  std::vector<BatchJob> jobs;
  DevBuf<BatchJob> d_jobs;
};

struct TvClass {
  int C;
  std::vector<BatchJob> jobs;
  DevBuf<BatchJob> d_jobs;
};

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, int> g_tuned;   // (R, C, log2 pixels) -> shape

int size_bucket(long long pixels) {
  int b = 0;
  while (pixels > 1) { pixels >>= 1; ++b; }
  return b;
}

std::vector<BatchJob> sweep_jobs(const std::vector<agents_ctx*>& ctxs, const std::vector<int>& ids,
                                 int shape, bool tiled, int R, int C) {
  std::vector<BatchJob> jobs;
  const int tw = tiled ? batch_tile_w(shape) : 32;
  const int th = tiled ? batch_tile_h(shape) : untiled_tile_h(R, C);
  for (int i : ids) {
    const int W = ctxs[i]->p.width, H = ctxs[i]->p.height;
    for (int ty = 0; ty < (H + th - 1) / th; ++ty)
      for (int tx = 0; tx < (W + tw - 1) / tw; ++tx) jobs.push_back(BatchJob{i, tx, ty});
  }
  return jobs;
}

#define BCK(call)                                                                     \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_);           \
      return ctx_fail(ctxs[0], e_ == cudaErrorMemoryAllocation ? AGENTS_ENOMEM : AGENTS_ECUDA, \
                      m_.c_str());                                                    \
    }                                                                                 \
  } while (0)

}  // namespace

extern "C" int agents_solve_batch(int32_t n, agents_ctx* const* ctx_list,
                                  const agents_solve_opts* opts, int32_t autotune,
                                  int32_t use_graph, double* const* eps_io, float* const* mu_io,
                                  float* const* c_out, agents_solve_info* infos) {
  if (n < 1 || !ctx_list || !opts || !eps_io || !mu_io)
    return ctx_fail(nullptr, AGENTS_EINVAL, "need n >= 1 and non-NULL contexts, opts, eps_io, mu_io");
  std::vector<agents_ctx*> ctxs(ctx_list, ctx_list + n);
  for (auto* c : ctxs)
    if (!c) return ctx_fail(nullptr, AGENTS_EINVAL, "a context is NULL");
  const agents_solve_opts o = *opts;
  if (o.k_out < 0 || o.k_in < 0 || o.max_ls < 1 || !(o.sigma0 > 0) ||
      !(o.ls_b > 0 && o.ls_b < 1) || !(o.ls_c > 0 && o.ls_c < 1) || !(o.tol >= 0))
    return ctx_fail(ctxs[0], AGENTS_EINVAL, "invalid solve options");
  const int T = ctxs[0]->T;
  for (auto* c : ctxs) {
    if (c->T != T) return ctx_fail(ctxs[0], AGENTS_EINVAL, "all contexts need the same nsteps");
    if (c->ckpt_every != 0)
      return ctx_fail(ctxs[0], AGENTS_EINVAL, "batched solve needs traj_mode 0 (full store)");
    if (c->device != ctxs[0]->device)
      return ctx_fail(ctxs[0], AGENTS_EINVAL, "all contexts must live on one device");
  }
  // The caller's current device is restored on every return path.
  struct RestoreDevice {
    int prev = -1;
    ~RestoreDevice() {
      if (prev >= 0) cudaSetDevice(prev);
    }
  } restore;
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  cudaGetLastError();   // a launch below reports only its own error
  if (prev_dev != ctxs[0]->device) {
    cudaSetDevice(ctxs[0]->device);
    restore.prev = prev_dev;
  }
  // A stream of the batch's own (graph capture is not allowed on the legacy default
  // stream), ordered after the work already queued on the contexts' stream.
  struct OwnStream {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    ~OwnStream() {
      if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
      if (ev) cudaEventDestroy(ev);
    }
  } own;
  BCK(cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking));
  BCK(cudaEventCreateWithFlags(&own.ev, cudaEventDisableTiming));
  BCK(cudaEventRecord(own.ev, ctxs[0]->stream));
  BCK(cudaStreamWaitEvent(own.s, own.ev, 0));
  cudaStream_t s = own.s;

  // ---- per-image buffers and inputs
  for (int i = 0; i < n; ++i) {
    agents_ctx* c = ctxs[i];
    {  // the solve workspaces (solve() allocates the same ones), each on its own
      float** bufs[6] = {&c->s_c, &c->s_cn, &c->s_trial_c, &c->s_v, &c->s_vn, &c->s_mu};
      const size_t sizes[6] = {c->nc, c->nc, c->nc, c->nv, c->nv, c->nv};
      for (int k = 0; k < 6; ++k) {
        if (*bufs[k]) continue;
        void* p = nullptr;
        const int st = ctx_alloc(c, &p, sizes[k] * sizeof(float));
        if (st != AGENTS_OK) {
          if (c != ctxs[0]) ctx_fail(ctxs[0], st, c->err.c_str());
          return st;
        }
        *bufs[k] = static_cast<float*>(p);
      }
    }
    cudaPointerAttributes a;
    const bool eps_dev = cudaPointerGetAttributes(&a, eps_io[i]) == cudaSuccess &&
                         (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    BCK(cudaMemcpyAsync(c->d_eps, eps_io[i], 2 * (size_t)T * sizeof(double),
                        eps_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    const bool mu_dev = cudaPointerGetAttributes(&a, mu_io[i]) == cudaSuccess &&
                        (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    BCK(cudaMemcpyAsync(c->s_mu, mu_io[i], c->nv * sizeof(float),
                        mu_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    c->stored = false;
  }

  // ---- classes
  std::map<std::pair<int, int>, std::vector<int>> by_rc;
  std::map<int, std::vector<int>> by_c;
  for (int i = 0; i < n; ++i) {
    by_rc[{ctxs[i]->p.radius, ctxs[i]->C}].push_back(i);
    by_c[ctxs[i]->C].push_back(i);
  }

  // ---- device tables
  std::vector<BatchSweepImg> h_imgs(n);
  std::vector<BatchCtl> h_ctl(n);
  DevBuf<BatchSweepImg> d_imgs;
  DevBuf<BatchCtl> d_ctl;
  DevBuf<BatchState> d_state;
  DevBuf<int> d_eps_active, d_trial_active, d_outer_active, d_all;
  DevBuf<Counters> d_cnt;
  DevBuf<CopySeg> d_copy_c, d_copy_v;
  BCK(d_imgs.alloc(n));
  BCK(d_ctl.alloc(n));
  BCK(d_state.alloc(n));
  BCK(d_eps_active.alloc(n));
  BCK(d_trial_active.alloc(n));
  BCK(d_outer_active.alloc(n));
  BCK(d_all.alloc(n));
  BCK(d_cnt.alloc(1));
  BCK(d_copy_c.alloc(n));
  BCK(d_copy_v.alloc(n));
  Counters* h_cnt = nullptr;
  BCK(cudaMallocHost(&h_cnt, sizeof(Counters)));
  struct HostFree {
    Counters* p;
    ~HostFree() { if (p) cudaFreeHost(p); }
  } hf{h_cnt};

  // sweep classes with tile shapes (autotuned or the default 0)
  std::vector<SweepClass> sweeps;
  for (auto& kv : by_rc) {
    SweepClass sc;
    sc.R = kv.first.first;
    sc.C = kv.first.second;
    sc.shape = 0;
    sweeps.push_back(std::move(sc));
  }
  // part_adj per image sized for the largest tile count over all shapes
  std::vector<DevBuf<double>> part_adj(n);
  for (int i = 0; i < n; ++i) {
    const int W = ctxs[i]->p.width, H = ctxs[i]->p.height;
    const long long most = (long long)((W + 31) / 32) * ((H + 3) / 4);   // smallest tiles
    BCK(part_adj[i].alloc((size_t)T * most * 2));
  }
  auto fill_imgs = [&](const std::vector<SweepClass>& cls) {
    for (const auto& sc : cls) {
      const bool tiled = batch_tiled(sc.R, sc.C);
      const int tw = tiled ? batch_tile_w(sc.shape) : 32;
      const int th = tiled ? batch_tile_h(sc.shape) : untiled_tile_h(sc.R, sc.C);
      for (int i : by_rc[{sc.R, sc.C}]) {
        agents_ctx* c = ctxs[i];
        BatchSweepImg& im = h_imgs[i];
        im.g = c->sg;
        im.nsteps = T;
        im.c0 = c->c0;
        im.traj = c->traj;
        im.work0 = c->work[0];
        im.work1 = c->work[1];
        im.cT = c->cT;
        im.trial_c = c->s_trial_c;
        im.lam0 = c->lam[0];
        im.lam1 = c->lam[1];
        im.eps = c->d_eps;
        im.trial_eps = c->d_trial[0];
        im.part_adj = part_adj[i].p;
        im.ntiles = ((c->p.width + tw - 1) / tw) * ((c->p.height + th - 1) / th);
      }
    }
  };
  for (int i = 0; i < n; ++i) {
    agents_ctx* c = ctxs[i];
    BatchCtl& k = h_ctl[i];
    k.eps = c->d_eps;
    k.trial = c->d_trial[0];
    k.best = c->d_trial[1];
    k.D = c->d_D;
    k.scal = c->d_scal;
    for (int m = 0; m < 2; ++m) { k.lo[m] = c->p.eps_lo[m]; k.hi[m] = c->p.eps_hi[m]; }
    k.dt = c->p.dt;
    k.rho = c->p.rho;
    k.gamma = c->p.gamma;
    k.cell = c->tg.cell;
  }
  std::vector<int> ones(n, 1);
  BCK(cudaMemcpyAsync(d_all.p, ones.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(d_eps_active.p, ones.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(d_outer_active.p, ones.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(d_ctl.p, h_ctl.data(), n * sizeof(BatchCtl), cudaMemcpyHostToDevice, s));

  // ---- autotune: time one Euler step of each class with each shape
  for (auto& sc : sweeps) {
    const std::vector<int>& ids = by_rc[{sc.R, sc.C}];
    if (!autotune || !batch_tiled(sc.R, sc.C)) continue;
    long long pix = 0;
    for (int i : ids) pix += (long long)ctxs[i]->p.width * ctxs[i]->p.height;
    const auto key = std::make_tuple(sc.R, sc.C, size_bucket(pix));
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      auto it = g_tuned.find(key);
      if (it != g_tuned.end()) { sc.shape = it->second; continue; }
    }
    float best_ms = 1e30f;
    int best_shape = 0;
    struct Events {  // destroyed on every return path
      cudaEvent_t a = nullptr, b = nullptr;
      ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
      }
    } ev;
    BCK(cudaEventCreate(&ev.a));
    BCK(cudaEventCreate(&ev.b));
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    for (int shape = 0; shape < kNumShapes; ++shape) {
      sc.shape = shape;
      fill_imgs(sweeps);
      BCK(cudaMemcpyAsync(d_imgs.p, h_imgs.data(), n * sizeof(BatchSweepImg),
                          cudaMemcpyHostToDevice, s));
      std::vector<BatchJob> jobs = sweep_jobs(ctxs, ids, shape, true, sc.R, sc.C);
      DevBuf<BatchJob> dj;
      BCK(dj.alloc(jobs.size()));
      BCK(cudaMemcpyAsync(dj.p, jobs.data(), jobs.size() * sizeof(BatchJob), cudaMemcpyHostToDevice, s));
      BCK(launch_forward_batch(d_imgs.p, dj.p, (int)jobs.size(), d_all.p, 0, kSweepStore,
                               sc.R, sc.C, shape, s));   // warm
      BCK(cudaEventRecord(e0, s));
      for (int rep = 0; rep < 3; ++rep)
        BCK(launch_forward_batch(d_imgs.p, dj.p, (int)jobs.size(), d_all.p, 0, kSweepStore,
                                 sc.R, sc.C, shape, s));
      BCK(cudaEventRecord(e1, s));
      BCK(cudaEventSynchronize(e1));
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) { best_ms = ms; best_shape = shape; }
    }
    sc.shape = best_shape;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[key] = best_shape;
  }
  fill_imgs(sweeps);
  BCK(cudaMemcpyAsync(d_imgs.p, h_imgs.data(), n * sizeof(BatchSweepImg), cudaMemcpyHostToDevice, s));
  for (auto& sc : sweeps) {
    sc.jobs = sweep_jobs(ctxs, by_rc[{sc.R, sc.C}], sc.shape, batch_tiled(sc.R, sc.C), sc.R,
                         sc.C);
    BCK(sc.d_jobs.alloc(sc.jobs.size()));
    BCK(cudaMemcpyAsync(sc.d_jobs.p, sc.jobs.data(), sc.jobs.size() * sizeof(BatchJob),
                        cudaMemcpyHostToDevice, s));
  }
  std::vector<TvClass> tvs;
  for (auto& kv : by_c) {
    TvClass tc;
    tc.C = kv.first;
    const int bw = tv_block_w(), bh = tv_block_h();
    for (int i : kv.second) {
      const int W = ctxs[i]->p.width, H = ctxs[i]->p.height;
      for (int by = 0; by < (H + bh - 1) / bh; ++by)
        for (int bx = 0; bx < (W + bw - 1) / bw; ++bx) tc.jobs.push_back(BatchJob{i, bx, by});
    }
    BCK(tc.d_jobs.alloc(tc.jobs.size()));
    BCK(cudaMemcpyAsync(tc.d_jobs.p, tc.jobs.data(), tc.jobs.size() * sizeof(BatchJob),
                        cudaMemcpyHostToDevice, s));
    tvs.push_back(std::move(tc));
  }

  // TV argument tables and reduction segments for each role
  enum { kTerm, kTrial, kPd, kAlm, kOuter, kRoles };
  std::vector<DevBuf<BatchTvArgs>> d_tv(kRoles);
  const int bw = tv_block_w();
  for (int role = 0; role < kRoles; ++role) {
    std::vector<BatchTvArgs> h(n);
    for (int i = 0; i < n; ++i) {
      agents_ctx* c = ctxs[i];
      BatchTvArgs& a = h[i];
      std::memset(&a, 0, sizeof(a));
      a.g = c->tg;
      a.c0 = c->c0;
      a.partial = c->d_part_tv;
      a.tiles_x = (c->p.width + bw - 1) / bw;
      switch (role) {
        case kTerm: a.c = c->cT; a.v = c->s_v; a.mu = c->s_mu; a.lam = c->lam[0]; break;
        case kTrial: a.c = c->s_trial_c; a.v = c->s_v; a.mu = c->s_mu; break;
        case kPd: a.c = c->cT; a.mu = c->s_mu; a.v_out = c->s_vn; break;
        case kAlm: a.c = c->cT; a.c_prev = c->s_c; a.v = c->s_vn; a.v_prev = c->s_v;
                   a.mu_io = c->s_mu; break;
        case kOuter: a.c = c->cT; a.v = c->s_vn; a.mu = c->s_mu; break;
      }
    }
    BCK(d_tv[role].alloc(n));
    BCK(cudaMemcpyAsync(d_tv[role].p, h.data(), n * sizeof(BatchTvArgs), cudaMemcpyHostToDevice, s));
  }
  // reductions: terminal -> scal[0], trial -> scal[1], outer -> scal[2], alm -> scal[8..12], D
  std::vector<DevBuf<ReduceSeg>> d_red(5);
  for (int r = 0; r < 5; ++r) {
    std::vector<ReduceSeg> h(n);
    for (int i = 0; i < n; ++i) {
      agents_ctx* c = ctxs[i];
      ReduceSeg& g = h[i];
      g.partial = c->d_part_tv;
      g.nblocks = c->nb_tv;
      g.scale = 1.0;
      if (r == 0) g.out = c->d_scal + 0;
      if (r == 1) g.out = c->d_scal + 1;
      if (r == 2) g.out = c->d_scal + 2;
      if (r == 3) g.out = c->d_scal + 8;
      if (r == 4) {
        g.partial = part_adj[i].p;
        g.nblocks = h_imgs[i].ntiles;
        g.scale = 1.0 / (2.0 * c->M);
        g.out = c->d_D;
      }
    }
    BCK(d_red[r].alloc(n));
    BCK(cudaMemcpyAsync(d_red[r].p, h.data(), n * sizeof(ReduceSeg), cudaMemcpyHostToDevice, s));
  }
  {
    std::vector<CopySeg> hc(n), hv(n);
    for (int i = 0; i < n; ++i) {
      hc[i] = CopySeg{ctxs[i]->cT, ctxs[i]->s_c, ctxs[i]->nc};
      hv[i] = CopySeg{ctxs[i]->s_vn, ctxs[i]->s_v, ctxs[i]->nv};
    }
    BCK(cudaMemcpyAsync(d_copy_c.p, hc.data(), n * sizeof(CopySeg), cudaMemcpyHostToDevice, s));
    BCK(cudaMemcpyAsync(d_copy_v.p, hv.data(), n * sizeof(CopySeg), cudaMemcpyHostToDevice, s));
  }
  size_t max_nv = 0;
  for (auto* c : ctxs) max_nv = std::max(max_nv, c->nv);
  const int copy_grid = (int)std::min<size_t>((max_nv + 255) / 256, 1024);
  const int ib = 128, ig = (n + ib - 1) / ib;

  // ---- launch sequences
  // A failed sweep launch names its class in the error message.
  auto sweep_fail = [&](const char* what, const SweepClass& sc, int step, cudaError_t e) -> int {
    char m[256];
    snprintf(m, sizeof(m), "%s (R=%d, C=%d, shape=%d, jobs=%zu, step=%d): %s", what, sc.R, sc.C,
             sc.shape, sc.jobs.size(), step, cudaGetErrorString(e));
    return ctx_fail(ctxs[0], AGENTS_ECUDA, m);
  };
  auto fwd = [&](const SweepClass& sc, const int* active, int step, int kind) -> int {
    const cudaError_t e = launch_forward_batch(d_imgs.p, sc.d_jobs.p, (int)sc.jobs.size(), active,
                                               step, kind, sc.R, sc.C, sc.shape, s);
    return e == cudaSuccess ? AGENTS_OK : sweep_fail("forward batch", sc, step, e);
  };
  auto seq_forward_store = [&](const int* active) -> int {
    for (int step = 0; step < T; ++step)
      for (auto& sc : sweeps) {
        const int st = fwd(sc, active, step, kSweepStore);
        if (st != AGENTS_OK) return st;
      }
    return AGENTS_OK;
  };
  // A: stored sweep, terminal objective and adjoint, reverse sweep, D, prepare
  auto seq_dal = [&]() -> int {
    BCK(cudaMemsetAsync(&d_cnt.p->trial_active, 0, sizeof(int), s));
    int st = seq_forward_store(d_eps_active.p);
    if (st != AGENTS_OK) return st;
    for (auto& tc : tvs)
      BCK(launch_objective_batch(d_tv[kTerm].p, tc.d_jobs.p, (int)tc.jobs.size(),
                                 d_eps_active.p, tc.C, true, s));
    BCK(launch_reduce_segments(d_red[0].p, n, 1, 1, s));
    for (int step = T - 1; step >= 0; --step)
      for (auto& sc : sweeps) {
        const cudaError_t e = launch_adjoint_batch(d_imgs.p, sc.d_jobs.p, (int)sc.jobs.size(),
                                                   d_eps_active.p, step, sc.R, sc.C, sc.shape, s);
        if (e != cudaSuccess) return sweep_fail("adjoint batch", sc, step, e);
      }
    BCK(launch_reduce_segments(d_red[4].p, n, 2, T, s));
    batch_prepare_kernel<<<ig, ib, 0, s>>>(d_state.p, d_ctl.p, d_eps_active.p, d_trial_active.p,
                                           d_cnt.p, n, T);
    BCK(cudaGetLastError());
    return AGENTS_OK;
  };
  // B: one Armijo round for every searching image
  auto seq_round = [&]() -> int {
    batch_control_kernel<<<n, 64, 0, s>>>(d_state.p, d_ctl.p, d_trial_active.p, T);
    BCK(cudaGetLastError());
    BCK(cudaMemsetAsync(&d_cnt.p->trial_active, 0, sizeof(int), s));
    for (int step = 0; step < T; ++step)
      for (auto& sc : sweeps) {
        const int st = fwd(sc, d_trial_active.p, step, kSweepTrial);
        if (st != AGENTS_OK) return st;
      }
    for (auto& tc : tvs)
      BCK(launch_objective_batch(d_tv[kTrial].p, tc.d_jobs.p, (int)tc.jobs.size(),
                                 d_trial_active.p, tc.C, false, s));
    BCK(launch_reduce_segments(d_red[1].p, n, 1, 1, s));
    batch_decide_kernel<<<n, 64, 0, s>>>(d_state.p, d_ctl.p, d_trial_active.p, d_cnt.p, T,
                                         o.ls_b, o.ls_c, o.max_ls);
    BCK(cudaGetLastError());
    return AGENTS_OK;
  };
  // C: one multiplier step for every image still in the solve (j is a kernel argument,
  // so this sequence is captured per multiplier step)
  auto seq_outer = [&](int j) -> int {
    int st = seq_forward_store(d_outer_active.p);
    if (st != AGENTS_OK) return st;
    for (auto& tc : tvs)
      BCK(launch_pd_tv_batch(d_tv[kPd].p, tc.d_jobs.p, (int)tc.jobs.size(), d_outer_active.p,
                             tc.C, s));
    for (auto& tc : tvs)
      BCK(launch_alm_batch(d_tv[kAlm].p, tc.d_jobs.p, (int)tc.jobs.size(), d_outer_active.p,
                           tc.C, s));
    BCK(launch_reduce_segments(d_red[3].p, n, 5, 1, s));
    for (auto& tc : tvs)
      BCK(launch_objective_batch(d_tv[kOuter].p, tc.d_jobs.p, (int)tc.jobs.size(),
                                 d_outer_active.p, tc.C, false, s));
    BCK(launch_reduce_segments(d_red[2].p, n, 1, 1, s));
    BCK(cudaMemsetAsync(&d_cnt.p->outer_active, 0, sizeof(int), s));
    batch_outer_kernel<<<ig, ib, 0, s>>>(d_state.p, d_ctl.p, d_outer_active.p, d_cnt.p, n, j, T,
                                         o.tol);
    BCK(cudaGetLastError());
    batch_copy_kernel<<<dim3(copy_grid, n), 256, 0, s>>>(d_copy_c.p, d_all.p);
    batch_copy_kernel<<<dim3(copy_grid, n), 256, 0, s>>>(d_copy_v.p, d_all.p);
    BCK(cudaGetLastError());
    return AGENTS_OK;
  };

  struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    ~Graph() {
      if (x) cudaGraphExecDestroy(x);
      if (g) cudaGraphDestroy(g);
    }
  };
  Graph g_dal, g_round;
  int runs_dal = 0, runs_round = 0;
  // The first run of a sequence launches directly (one-time kernel set-up happens outside
  // any capture); later runs capture it once and replay the graph.
  auto run = [&](Graph& gr, int& runs, auto&& seq) -> int {
    if (!use_graph || runs++ == 0) return seq();
    if (!gr.x) {
      BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const int st = seq();
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(s, &g);
      if (st != AGENTS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      BCK(e);
      gr.g = g;
      BCK(cudaGraphInstantiate(&gr.x, gr.g, 0));
    }
    BCK(cudaGraphLaunch(gr.x, s));
    return AGENTS_OK;
  };
  auto read_counters = [&]() -> int {
    BCK(cudaMemcpyAsync(h_cnt, d_cnt.p, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    return AGENTS_OK;
  };

  // ---- initial iterate: c(0) = c(T; eps(0)), v(0), L~(0)
  int st = AGENTS_OK;
  BCK(cudaMemsetAsync(d_cnt.p, 0, sizeof(Counters), s));
  st = seq_forward_store(d_all.p);
  if (st != AGENTS_OK) return st;
  {
    std::vector<BatchTvArgs> h(n);
    for (int i = 0; i < n; ++i) {  // v(0) = shrink(G c(0) - mu/rho) into s_v directly
      agents_ctx* c = ctxs[i];
      std::memset(&h[i], 0, sizeof(BatchTvArgs));
      h[i].g = c->tg;
      h[i].c = c->cT;
      h[i].mu = c->s_mu;
      h[i].v_out = c->s_v;
      h[i].c0 = c->c0;
      h[i].v = c->s_v;
      h[i].partial = c->d_part_tv;
      h[i].tiles_x = (c->p.width + bw - 1) / bw;
    }
    DevBuf<BatchTvArgs> d0;
    BCK(d0.alloc(n));
    BCK(cudaMemcpyAsync(d0.p, h.data(), n * sizeof(BatchTvArgs), cudaMemcpyHostToDevice, s));
    for (auto& tc : tvs)
      BCK(launch_pd_tv_batch(d0.p, tc.d_jobs.p, (int)tc.jobs.size(), d_all.p, tc.C, s));
    for (auto& tc : tvs)
      BCK(launch_objective_batch(d0.p, tc.d_jobs.p, (int)tc.jobs.size(), d_all.p, tc.C, false, s));
    BCK(launch_reduce_segments(d_red[2].p, n, 1, 1, s));
    batch_copy_kernel<<<dim3(copy_grid, n), 256, 0, s>>>(d_copy_c.p, d_all.p);
    BCK(cudaGetLastError());
    batch_init_kernel<<<ig, ib, 0, s>>>(d_state.p, d_ctl.p, n, o.sigma0);
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(s));   // d0 is freed at the end of this scope
  }

  // ---- Algorithm 2
  for (int j = 1; j <= o.k_out; ++j) {
    BCK(cudaMemsetAsync(&d_cnt.p->eps_active, 0, sizeof(int), s));
    batch_begin_eps_kernel<<<ig, ib, 0, s>>>(d_state.p, d_eps_active.p, d_cnt.p, n);
    BCK(cudaGetLastError());
    st = read_counters();
    if (st != AGENTS_OK) return st;
    if (h_cnt->eps_active == 0) break;          // every image has finished
    for (int it = 0; it < o.k_in; ++it) {
      st = run(g_dal, runs_dal, seq_dal);
      if (st != AGENTS_OK) return st;
      st = read_counters();
      if (st != AGENTS_OK) return st;
      for (int round = 0; round < o.max_ls && h_cnt->trial_active > 0; ++round) {
        st = run(g_round, runs_round, seq_round);
        if (st != AGENTS_OK) return st;
        st = read_counters();
        if (st != AGENTS_OK) return st;
      }
      BCK(cudaMemsetAsync(&d_cnt.p->eps_active, 0, sizeof(int), s));
      batch_accept_kernel<<<n, 64, 0, s>>>(d_state.p, d_ctl.p, d_eps_active.p, d_cnt.p, T);
      BCK(cudaGetLastError());
      st = read_counters();
      if (st != AGENTS_OK) return st;
      if (h_cnt->eps_active == 0) break;
    }
    st = seq_outer(j);
    if (st != AGENTS_OK) return st;
  }

  // ---- outputs
  std::vector<BatchState> hs(n);
  BCK(cudaMemcpyAsync(hs.data(), d_state.p, n * sizeof(BatchState), cudaMemcpyDeviceToHost, s));
  BCK(cudaStreamSynchronize(s));
  int status = AGENTS_OK;
  for (int i = 0; i < n; ++i) {
    agents_ctx* c = ctxs[i];
    auto copy_out = [&](void* dst, const void* src, size_t bytes) -> int {
      cudaPointerAttributes a;
      const bool dev = cudaPointerGetAttributes(&a, dst) == cudaSuccess &&
                       (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
      cudaGetLastError();
      BCK(cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
      return AGENTS_OK;
    };
    st = copy_out(eps_io[i], c->d_eps, 2 * (size_t)T * sizeof(double));
    if (st != AGENTS_OK) return st;
    st = copy_out(mu_io[i], c->s_mu, c->nv * sizeof(float));
    if (st != AGENTS_OK) return st;
    if (c_out && c_out[i]) {
      st = copy_out(c_out[i], c->s_c, c->nc * sizeof(float));
      if (st != AGENTS_OK) return st;
    }
    if (infos) {
      agents_solve_info& inf = infos[i];
      std::memset(&inf, 0, sizeof(inf));
      inf.outer_done = hs[i].outer_done;
      inf.inner_done = hs[i].inner_done;
      inf.trials = hs[i].trials;
      inf.stalls = hs[i].stalls;
      inf.stationary = hs[i].stationary;
      inf.forward_steps = hs[i].fwd + T;   // + the initial sweep
      inf.adjoint_steps = hs[i].adj;
      inf.tv_sweeps = hs[i].tv + 2;
      inf.final_res = hs[i].res;
      inf.final_obj = hs[i].obj;
      inf.final_gap = hs[i].gap;
      inf.final_sigma = hs[i].sigma;
      inf.kernel_launches = -1;   // launches are shared by the whole batch
    }
    if (hs[i].diverged) status = AGENTS_EDIVERGED;
    c->stored = false;
  }
  BCK(cudaStreamSynchronize(s));
  if (status != AGENTS_OK) return ctx_fail(ctxs[0], status, "an image of the batch diverged");
  return AGENTS_OK;
}
