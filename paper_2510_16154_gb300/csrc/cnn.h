// Internal declarations of the warm-start network's kernels (cnn_kernels.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace ws {

cudaError_t conv_forward(const float* x, const __nv_bfloat16* w16, const float* bias, float* y,
                         const float* add, float* y2, int N, int H, int W, int Cin, int Cout,
                         int relu, int up, cudaStream_t s);
cudaError_t conv_backward_data(const float* dy, const __nv_bfloat16* wt16, float* dx, int N, int H,
                               int W, int Cin, int Cout, cudaStream_t s);
size_t conv_backward_weight_workspace(int N, int H, int W, int Cin, int Cout);
cudaError_t conv_backward_weight(const float* x, const float* dy, float* dw, float* db, int N,
                                 int H, int W, int Cin, int Cout, int up, float* ws,
                                 size_t ws_bytes, cudaStream_t s);
cudaError_t transpose_weights(const float* w, __nv_bfloat16* w16, __nv_bfloat16* wt16, int Cin,
                              int Cout, cudaStream_t s);

}  // namespace ws
