// agents_objective_noalloc: the objective L~ and terminal adjoint without any device
// allocation, for callers that are not allowed to allocate device memory.
//
// Some hosts own every byte of device memory: an application that reserves its whole
// budget up front and hands plug-ins only pre-allocated buffers, or a latency-sensitive
// loop that must not call cudaMalloc because it can synchronise the whole device and
// stall unrelated streams.  agents_init allocates a context, so such callers cannot use
// agents_objective.  This entry point takes every input and output from the caller and
// keeps its only scratch -- the float64 per-block partial sums of the reduction -- in
// the file-scope device array below, which exists in every GPU that loads the library
// until the process exits.
//
// The host cannot pass g_objective_scratch to a kernel by name (in host code the name
// is a host-side stand-in, not a device address), so every call, with the caller's
// device current, looks its address up with cudaGetSymbolAddress and checks the result.
// The first lookup on a device loads this library's device code there (allocating the
// array; it can synchronise the device), which is why the first call belongs in set-up;
// later lookups only read the loaded module's table.  Not caching the address keeps it
// right for whichever context is current: a non-primary context of the same device, or
// the primary context re-created after a device reset, has its own copy of the array.
#include "agents.h"
#include "kernels.h"

#include <cstdio>
#include <string>

namespace agents {
void set_global_error(const std::string& msg);  // agents.cu: agents_last_error(NULL)
}

using namespace agents;

namespace {

// One float64 partial per reduction block (32 x 8 threads over 128 x 8 pixels): 32768
// blocks = 256 KiB, enough for ceil(W/128) * ceil(H/8) <= 32768 (for example 4096 x 8192).
constexpr int kMaxBlocks = 32768;

static __device__ __align__(256) double g_objective_scratch[kMaxBlocks];

int fail(int code, const char* msg) {
  set_global_error(msg);
  return code;
}

// Device address of g_objective_scratch in the current device context.
int scratch_in_current_context(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_objective_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    std::string msg = std::string("cudaGetSymbolAddress(g_objective_scratch): ") +
                      cudaGetErrorString(e);
    return fail(AGENTS_ECUDA, msg.c_str());
  }
  *out = static_cast<double*>(p);
  return AGENTS_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int agents_objective_noalloc(int32_t height, int32_t width, int32_t channels,
                                        double alpha, double rho, int32_t tv_mode,
                                        const float* c_dev, const float* c0_dev,
                                        const float* v_dev, const float* mu_dev,
                                        double* obj_dev, float* lambda_dev, void* cuda_stream) {
  if (height < 1 || width < 1 || channels < 1 || channels > 64)
    return fail(AGENTS_EINVAL, "need height, width >= 1 and 1 <= channels <= 64");
  if (!(alpha > 0) || !(rho > 0)) return fail(AGENTS_EINVAL, "alpha and rho must be > 0");
  if (tv_mode != 0 && tv_mode != 1) return fail(AGENTS_EINVAL, "tv_mode must be 0 or 1");
  if (!c_dev || !c0_dev || !v_dev || !mu_dev || !obj_dev)
    return fail(AGENTS_EINVAL, "c_dev, c0_dev, v_dev, mu_dev and obj_dev must not be NULL");
  if (!aligned16(c_dev) || !aligned16(c0_dev) || !aligned16(v_dev) || !aligned16(mu_dev) ||
      (lambda_dev && !aligned16(lambda_dev)))
    return fail(AGENTS_EINVAL, "field pointers must be 16-byte aligned");
  if (!on_device(c_dev) || !on_device(c0_dev) || !on_device(v_dev) || !on_device(mu_dev) ||
      !on_device(obj_dev) || (lambda_dev && !on_device(lambda_dev)))
    return fail(AGENTS_EINVAL, "every field pointer and obj_dev must be device memory");
  const TvGeom g{height, width, channels, (float)(0.5 * width), (float)(0.5 * height),
                 (float)rho, (float)(1.0 / rho), (float)alpha, rho,
                 1.0 / ((double)width * (double)height), tv_mode};
  const int nb = tv_num_blocks(g);
  if (nb > kMaxBlocks) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "image of %d x %d needs %d reduction blocks of 128 x 8 pixels; the static "
                  "scratch holds %d (ceil(W/128) * ceil(H/8) <= %d, e.g. 4096 x 8192)",
                  height, width, nb, kMaxBlocks, kMaxBlocks);
    return fail(AGENTS_EINVAL, msg);
  }
  double* scratch = nullptr;
  int st = scratch_in_current_context(&scratch);
  if (st != AGENTS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // Every block overwrites its own partial and the reduction reads exactly those nb
  // entries, so nothing left in the array by an earlier call is ever read.
  cudaError_t e = launch_objective(c_dev, c0_dev, v_dev, mu_dev, lambda_dev, scratch, g, s);
  if (e == cudaSuccess) e = launch_reduce_rows(scratch, nb, 1, 1, 1.0, obj_dev, s);
  if (e != cudaSuccess) return fail(AGENTS_ECUDA, cudaGetErrorString(e));
  return AGENTS_OK;
}
