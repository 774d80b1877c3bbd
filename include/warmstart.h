/* Warm-start network: C ABI.
 *
 * The paper starts every solve of Algorithm 2 from the dual field mu(0) = 0 and the control
 * eps(0) = 57 (Section 5).  This network predicts both from the image, so that the solve
 * starts closer to its fixed point; the solve itself is unchanged and still decides
 * the result (the paper has no counterpart of the network).
 *
 * Architecture (levels L, base width B, widths B 2^(l-1) for l = 1..L):
 *   encoder level l: conv3x3 + ReLU, conv3x3 + ReLU, then 2x2 mean pooling before level l+1;
 *   decoder level l = L-1..1: nearest 2x upsampling, conv3x3 + ReLU to width B 2^(l-1),
 *     plus the encoder output of level l, conv3x3 + ReLU;
 *   mu head: conv3x3 to out_ch channels, no activation (out_ch = 2 C, laid out as the
 *     solve's mu: [x-components of the C channels, y-components]);
 *   control head: the mean of the level-L output over pixels, then z = A g + c with
 *     2T outputs; the control is eps = clip(exp(z), E) (z is a log-control).
 * conv3x3 is a 'same' cross-correlation with zero padding:
 *   y[n,h,w,o] = b[o] + sum_{ky,kx,i} x[n, h+ky-1, w+kx-1, i] W[o,ky,kx,i].
 *
 * Precision: convolutions run on the tensor cores with bfloat16 operands (the weights, the
 * convolution input, and in the backward pass the output gradient after the ReLU mask,
 * each rounded to nearest-even from float32) and float32 accumulation.  Biases, ReLU,
 * pooling, the control head, the loss and the optimiser are float32; master weights and
 * the Adam moments are float32.
 *
 * Flat parameter vector (float32), in this order: for every convolution enc1a, enc1b, ...,
 * encLa, encLb, dec(L-1)a, dec(L-1)b, ..., dec1a, dec1b, head: W[Cout][3][3][Cin] then
 * b[Cout]; then A[2T][B 2^(L-1)] and c[2T].
 *
 * Layouts: images and activations NHWC float32, contiguous.  Buffers are device pointers
 * unless stated otherwise.  Every function returns AGENTS_OK (0) or a negative status of
 * agents.h; ws_last_error() gives the message of the last failure on the calling thread.
 * Work is queued on the stream given at creation (cudaStream_t passed as void*; NULL = the
 * legacy default stream); functions that return host values synchronise that stream.
 */
#ifndef PAPER_2510_16154_WARMSTART_H
#define PAPER_2510_16154_WARMSTART_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- single convolutions (for checking the kernels; no state) ------------------------ */

/* y = act(conv3x3(x, W) + b) over N images of H x W.  w16: W as bfloat16 bit patterns
 * [Cout][3][3][Cin]; bias may be NULL (zero); relu != 0 applies ReLU.  If `up` is 1, x is
 * the half-resolution tensor [N][H/2][W/2][Cin] and the convolution reads its nearest 2x
 * upsampling (H and W even).  If `add` is not NULL, y2 = y + add is also written (y2 must
 * then be non-NULL).  Returns AGENTS_EINVAL on bad sizes. */
int ws_conv3x3_forward(const float* x, const uint16_t* w16, const float* bias, float* y,
                       const float* add, float* y2, int32_t N, int32_t H, int32_t W,
                       int32_t Cin, int32_t Cout, int32_t relu, int32_t up, void* stream);

/* dx = conv3x3^T(dy): dx[n,h,w,i] = sum_{ky,kx,o} dy[n, h-ky+1, w-kx+1, o] W[o,ky,kx,i] at
 * full resolution H x W.  wt16: the weights transposed to [Cin][3][3][Cout] (bfloat16);
 * see ws_transpose_weights. */
int ws_conv3x3_backward_data(const float* dy, const uint16_t* wt16, float* dx, int32_t N,
                             int32_t H, int32_t W, int32_t Cin, int32_t Cout, void* stream);

/* dW[o,ky,kx,i] = sum_{n,h,w} dy[n,h,w,o] x[n, h+ky-1, w+kx-1, i] (x read through the 2x
 * upsampling when up = 1, as in the forward) and db[o] = sum dy[...,o] (db may be NULL).
 * `workspace` holds the split-K partial sums: ws_conv3x3_backward_weight_workspace() bytes.
 * The sums are taken in a fixed order (bitwise reproducible). */
int ws_conv3x3_backward_weight(const float* x, const float* dy, float* dw, float* db,
                               int32_t N, int32_t H, int32_t W, int32_t Cin, int32_t Cout,
                               int32_t up, void* workspace, size_t workspace_bytes,
                               void* stream);
size_t ws_conv3x3_backward_weight_workspace(int32_t N, int32_t H, int32_t W, int32_t Cin,
                                            int32_t Cout);

/* w16 = bf16(w) [Cout][3][3][Cin] and, if wt16 != NULL, wt16[i][ky][kx][o] = w16[o][ky][kx][i]. */
int ws_transpose_weights(const float* w, uint16_t* w16, uint16_t* wt16, int32_t Cin,
                         int32_t Cout, void* stream);

/* ---- the network --------------------------------------------------------------------- */

typedef struct ws_net ws_net;

typedef struct ws_net_config {
  int32_t in_ch;    /* image channels */
  int32_t out_ch;   /* mu channels (2 C) */
  int32_t base;     /* width of level 1 */
  int32_t levels;   /* 2..8; H and W are padded to multiples of 2^(levels-1) */
  int32_t nsteps;   /* T: the control head has 2T outputs */
  float eps_lo[2];  /* box E for the predicted control */
  float eps_hi[2];
} ws_net_config;

/* Creates a network with all parameters zero; set them with ws_net_set_params. */
int ws_net_create(const ws_net_config* cfg, void* stream, ws_net** out);
void ws_net_destroy(ws_net* net);
int64_t ws_net_num_params(const ws_net* net);
/* Copy the flat float32 parameters in / out (host or device pointer). */
int ws_net_set_params(ws_net* net, const float* params);
int ws_net_get_params(ws_net* net, float* params);

/* Inference on N images [N][H][W][in_ch] (any H, W >= 1; padded internally by edge
 * replication to multiples of 2^(levels-1) and cropped back).  mu_out [N][H][W][out_ch]
 * (device); with project = 1 each pixel's mu is scaled into the unit ball of its group
 * (all out_ch entries: the dual ball of the coupled TV), with project = 2 each channel's
 * (x, y) pair separately (channel-wise TV); 0 leaves it raw.  eps_out [N][T][2] float64
 * (host or device, may be NULL): the clipped control.  z_out [N][2T] float32 (device, may
 * be NULL): the raw log-control. */
int ws_net_forward(ws_net* net, const float* img, int32_t N, int32_t H, int32_t W,
                   int32_t project, float* mu_out, double* eps_out, float* z_out);

/* Inference at a coarser resolution, lifted back: the f x f block means of the images
 * (H, W multiples of factor) go through ws_net_forward at H/f x W/f, and mu_out
 * [N][H][W][out_ch] (device) receives the prediction upsampled by nearest neighbour;
 * eps_out as in ws_net_forward (the control lives on the unit square and does not depend
 * on the resolution).  For images larger than those the network was trained on: the
 * prediction is made at the training resolution.  factor = 1 is ws_net_forward.  No
 * counterpart in the paper (its method has no network). */
int ws_net_forward_lifted(ws_net* net, const float* img, int32_t N, int32_t H, int32_t W,
                          int32_t factor, int32_t project, float* mu_out, double* eps_out);

/* Loss  mean((mu - mu_t)^2) + lam_eps mean((z - log_eps_t)^2)  for N images whose sides
 * are multiples of 2^(levels-1), and its gradient with respect to the flat parameters.
 * mu_t [N][H][W][out_ch] float32, log_eps_t [N][2T] float32 (device).  loss_out (host,
 * may be NULL); grad_out (host or device, num_params floats, may be NULL: the gradient
 * then stays in the network for ws_net_adam_step). */
int ws_net_loss_grad(ws_net* net, const float* img, const float* mu_t,
                     const float* log_eps_t, int32_t N, int32_t H, int32_t W, float lam_eps,
                     double* loss_out, float* grad_out);

/* One Adam step (bias-corrected, step counter kept by the network) on the gradient of
 * the last ws_net_loss_grad; refreshes the bfloat16 weight copies. */
int ws_net_adam_step(ws_net* net, float lr, float beta1, float beta2, float adam_eps,
                     float weight_decay);

/* Message of the last failure on the calling thread ("" if none). */
const char* ws_last_error(void);

/* Convolutions whose image width is at least 128 and whose channel counts are multiples
 * of 16 (the output count at most 128 or a multiple of 128) run on the tcgen05 tensor
 * cores with tensor-memory accumulators; every wait inside those kernels is bounded, and
 * a kernel that gives up writes NaN to its outputs and raises a device-side flag.
 * Returns 1 if the flag was raised since the last call (and clears it), 0 if not,
 * AGENTS_ECUDA if it could not be read.  Synchronises the device. */
int ws_tensor_core_fault_take(void);

#ifdef __cplusplus
}
#endif

#endif
