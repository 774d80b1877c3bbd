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
// Tensor-core (tcgen05) form of conv_forward / conv_backward_data (cnn_tc.cu), used when
// conv_tc_applies(W, channels read, channels written): W >= 128, both channel counts
// multiples of 16 and the output count <= 128 or a multiple of 128.
bool conv_tc_applies(int W, int ci, int co);
cudaError_t conv_forward_tc(const float* x, const __nv_bfloat16* w16, const float* bias, float* y,
                            const float* add, float* y2, int N, int H, int W, int Cin, int Cout,
                            int relu, int up, cudaStream_t s);
cudaError_t conv_backward_data_tc(const float* dy, const __nv_bfloat16* wt16, float* dx, int N,
                                  int H, int W, int Cin, int Cout, cudaStream_t s);
// 1 if a tensor-core convolution gave up a bounded wait since the last call (the flag is
// cleared), 0 if not, -1 on a CUDA error.  Synchronous.
int conv_tc_take_error();
cudaError_t transpose_weights(const float* w, __nv_bfloat16* w16, __nv_bfloat16* wt16, int Cin,
                              int Cout, cudaStream_t s);

}  // namespace ws
