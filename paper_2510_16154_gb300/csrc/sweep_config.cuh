// Tile shapes of the agent sweep kernels and the dispatch over (R, C).
#pragma once

#include "sweep.cuh"

namespace agents {

// Forward: 16 x 8 threads, 2 pixel pairs per thread -> 64 x 8 pixel tiles.
constexpr int kFwdPX = 2, kFwdBX = 16, kFwdBY = 8;
// Adjoint: 16 x 8 threads, 2 pixel pairs per thread -> 64 x 8 pixel tiles.
constexpr int kAdjPX = 2, kAdjBX = 16, kAdjBY = 8;
// Generic (any R, C) kernels: one pixel per thread.
constexpr int kGenBX = 32, kGenBY = 4;

constexpr int kMaxTiledR = 8;

inline bool tiled_shape(int R, int C) { return R >= 1 && R <= kMaxTiledR && (C == 1 || C == 3); }

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Opt a kernel into more than 48 KB of dynamic shared memory (once) and return the grid
// of a persistent launch: every resident block on every SM (computed once).
template <class K>
inline cudaError_t persistent_grid(K kern, int threads, size_t smem, int* cached, int* grid) {
  if (*cached == 0) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
      if (e != cudaSuccess) return e;
    }
    int dev = 0, nsm = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
    if (e != cudaSuccess) return e;
    *cached = nsm * (per > 0 ? per : 1);
  }
  *grid = *cached;
  return cudaSuccess;
}

// Batched tile shapes (pixel pairs per thread, threads in x and y).
#define AGENTS_BATCH_SHAPES(F, R, C)                                   \
  (shape == 0 ? F(R, C, 2, 16, 8) : shape == 1 ? F(R, C, 2, 16, 4) : F(R, C, 2, 8, 8))

// Expands F(R, C) for every tiled (R, C) and returns its value; `fallback` otherwise.
#define AGENTS_DISPATCH_RC(R_, C_, F, fallback)                           \
  do {                                                                    \
    if ((C_) == 3) {                                                      \
      switch (R_) {                                                       \
        case 1: return F(1, 3); case 2: return F(2, 3);                   \
        case 3: return F(3, 3); case 4: return F(4, 3);                   \
        case 5: return F(5, 3); case 6: return F(6, 3);                   \
        case 7: return F(7, 3); case 8: return F(8, 3);                   \
        default: break;                                                   \
      }                                                                   \
    } else if ((C_) == 1) {                                               \
      switch (R_) {                                                       \
        case 1: return F(1, 1); case 2: return F(2, 1);                   \
        case 3: return F(3, 1); case 4: return F(4, 1);                   \
        case 5: return F(5, 1); case 6: return F(6, 1);                   \
        case 7: return F(7, 1); case 8: return F(8, 1);                   \
        default: break;                                                   \
      }                                                                   \
    }                                                                     \
    return fallback;                                                      \
  } while (0)

}  // namespace agents
