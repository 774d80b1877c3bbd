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
// is a host-side stand-in, not a device address), so the first call on each device,
// with that device current, looks its address up with cudaGetSymbolAddress and caches
// it; later calls on that device reuse the cached address.
#include "agents.h"
#include "kernels.h"

#include <cstdio>
#include <mutex>
#include <string>

namespace agents {
void set_global_error(const std::string& msg);  // agents.cu: agents_last_error(NULL)
}

using namespace agents;

namespace {

// One float64 partial per reduction block (32 x 8 threads over 128 x 8 pixels): 32768
// blocks = 256 KiB, enough for images of up to 33,554,432 pixels (for example 4096 x 8192).
constexpr int kMaxBlocks = 32768;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_objective_scratch[kMaxBlocks];

std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

int fail(int code, const char* msg) {
  set_global_error(msg);
  return code;
}

// Address of g_objective_scratch on the current device (looked up once per device).
int scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(AGENTS_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(AGENTS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_objective_scratch);
    if (e != cudaSuccess) {
      std::string msg = std::string("cudaGetSymbolAddress(g_objective_scratch): ") +
                        cudaGetErrorString(e);
      return fail(AGENTS_ECUDA, msg.c_str());
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
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
  if (!on_device(obj_dev)) return fail(AGENTS_EINVAL, "obj_dev must be device memory");
  const TvGeom g{height, width, channels, (float)(0.5 * width), (float)(0.5 * height),
                 (float)rho, (float)(1.0 / rho), (float)alpha, rho,
                 1.0 / ((double)width * (double)height), tv_mode};
  const int nb = tv_num_blocks(g);
  if (nb > kMaxBlocks) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "image of %d x %d needs %d reduction blocks; the static scratch holds %d "
                  "(images up to 33554432 pixels)", height, width, nb, kMaxBlocks);
    return fail(AGENTS_EINVAL, msg);
  }
  double* scratch = nullptr;
  int st = scratch_on_current_device(&scratch);
  if (st != AGENTS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // Every block overwrites its own partial and the reduction reads exactly those nb
  // entries, so nothing left in the array by an earlier call is ever read.
  cudaError_t e = launch_objective(c_dev, c0_dev, v_dev, mu_dev, lambda_dev, scratch, g, s);
  if (e == cudaSuccess) e = launch_reduce_rows(scratch, nb, 1, 1, 1.0, obj_dev, s);
  if (e != cudaSuccess) return fail(AGENTS_ECUDA, cudaGetErrorString(e));
  return AGENTS_OK;
}
