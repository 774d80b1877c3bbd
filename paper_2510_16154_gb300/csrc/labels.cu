// Cluster labels of a colour field: connected components of the 4-neighbour pixel graph
// in which two neighbours are joined when every channel differs by at most a threshold
// (the paper segments its outputs at threshold 0.02, Section 5).
//
// Union-find on the label array L (L[i] <= i always, roots satisfy L[i] = i):
//   1. L[i] = i;
//   2. every pixel unions itself with its right and lower neighbour when they are
//      joined; a union links the larger of the two roots to the smaller with atomicMin
//      and retries if another thread re-linked that root meanwhile;
//   3. L[i] = root(i).
// Because links always point to a smaller index, each root is the smallest index of its
// component, so the result is canonical (independent of thread timing).  Every loop is
// bounded by the pixel count; exceeding the bound sets *status = 1 (it cannot happen for
// a forest whose links decrease) instead of spinning.  A smaller bound can be given (a
// test hook that exercises the give-up path): the loops then stop early, every index they
// follow is still a label value in [0, n), and *status reports the give-up.
#include "common.cuh"
#include "kernels.h"

namespace agents {

__device__ __forceinline__ int find_root(const volatile int32_t* L, int a, int cap,
                                         int32_t* status) {
  for (int it = 0; it < cap; ++it) {
    const int p = L[a];
    if (p == a) return a;
    a = p;
  }
  atomicExch(status, 1);
  return a;
}

__device__ __forceinline__ void unite(int32_t* L, int a, int b, int cap, int32_t* status) {
  for (int it = 0; it < cap; ++it) {
    a = find_root(L, a, cap, status);
    b = find_root(L, b, cap, status);
    if (a == b) return;
    if (a > b) { const int t = a; a = b; b = t; }
    const int old = atomicMin(L + b, a);
    if (old == b) return;  // b was still a root and now points to a
    b = old;               // b was re-linked meanwhile: continue from its new parent
  }
  atomicExch(status, 1);
}

__device__ __forceinline__ bool joined(const float* __restrict__ c, size_t i, size_t j, int C,
                                       float thr) {
  for (int ch = 0; ch < C; ++ch)
    if (!(fabsf(c[i * C + ch] - c[j * C + ch]) <= thr)) return false;
  return true;
}

__global__ void labels_init_kernel(int32_t* L, int n, int32_t* count, int32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) L[i] = i;
  if (i == 0) { *count = 0; *status = 0; }
}

__global__ void labels_merge_kernel(const float* __restrict__ c, int H, int W, int C, float thr,
                                    int cap, int32_t* L, int32_t* status) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y * blockDim.y + threadIdx.y;
  if (q >= W || r >= H) return;
  const size_t i = (size_t)r * W + q;
  if (q + 1 < W && joined(c, i, i + 1, C, thr)) unite(L, (int)i, (int)(i + 1), cap, status);
  if (r + 1 < H && joined(c, i, i + W, C, thr)) unite(L, (int)i, (int)(i + W), cap, status);
}

__global__ void labels_flatten_kernel(int32_t* L, int n, int cap, int32_t* count,
                                      int32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int root = find_root(L, i, cap, status);
  L[i] = root;
  if (root == i) atomicAdd(count, 1);
}

cudaError_t launch_labels(const float* c, int H, int W, int C, float threshold, int loop_cap,
                          int32_t* labels, int32_t* count, int32_t* status, cudaStream_t s) {
  const int n = H * W;
  const int cap = (loop_cap > 0 && loop_cap < n) ? loop_cap : n;
  labels_init_kernel<<<(n + 255) / 256, 256, 0, s>>>(labels, n, count, status);
  dim3 block(32, 8), grid((W + 31) / 32, (H + 7) / 8);
  labels_merge_kernel<<<grid, block, 0, s>>>(c, H, W, C, threshold, cap, labels, status);
  // Roots must be final before flattening; a second kernel orders that.
  labels_flatten_kernel<<<(n + 255) / 256, 256, 0, s>>>(labels, n, cap, count, status);
  return cudaGetLastError();
}

}  // namespace agents
