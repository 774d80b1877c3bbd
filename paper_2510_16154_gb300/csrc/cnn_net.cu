// The warm-start network (ws_net): parameters, activations, forward, loss gradient and
// Adam, over the tensor-core convolutions of cnn_kernels.cu.  The backward pass follows
// the forward in reverse: control head, mu head, decoder levels 1..L-1 (with the skip
// gradients), encoder levels L..1 (with the pooled gradients).
#include "agents.h"
#include "cnn.h"
#include "common.cuh"
#include "warmstart.h"

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace {

thread_local std::string g_ws_error;

int ws_fail(int status, const std::string& msg) {
  g_ws_error = msg;
  return status;
}

#define WCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return ws_fail(e_ == cudaErrorMemoryAllocation ? AGENTS_ENOMEM : AGENTS_ECUDA, \
                     std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

#define WTRY(expr)                   \
  do {                               \
    int st_ = (expr);                \
    if (st_ != AGENTS_OK) return st_; \
  } while (0)

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  const bool d = cudaPointerGetAttributes(&a, p) == cudaSuccess &&
                 (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  return d;
}

constexpr int kThreads = 256;
int blocks_for(size_t n) {
  const size_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < 8192 ? (b ? b : 1) : 8192);
}

// ---------------------------------------------------------------- small kernels
__global__ void avgpool2_kernel(const float* __restrict__ x, float* __restrict__ y, int N, int H,
                                int W, int C) {  // H, W: output size
  const size_t n = (size_t)N * H * W * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    size_t r = i / C;
    const int xx = (int)(r % W); r /= W;
    const int yy = (int)(r % H);
    const int img = (int)(r / H);
    const size_t W2 = 2 * (size_t)W;
    const size_t b = ((((size_t)img * 2 * H + 2 * yy) * W2) + 2 * xx) * C + c;
    y[i] = 0.25f * ((x[b] + x[b + C]) + (x[b + W2 * C] + x[b + W2 * C + C]));
  }
}

// dst (full res) += src (half res) / 4
__global__ void avgpool2_backward_acc_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                             int N, int H, int W, int C) {  // H, W: full size
  const size_t n = (size_t)N * H * W * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    size_t r = i / C;
    const int xx = (int)(r % W); r /= W;
    const int yy = (int)(r % H);
    const int img = (int)(r / H);
    const size_t s = (((size_t)img * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c;
    dst[i] += 0.25f * src[s];
  }
}

// dst (half res) (+)= sum of the 2x2 block of src (full res)
__global__ void upsample2_backward_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                          int N, int H, int W, int C, int accumulate) {  // H, W: half
  const size_t n = (size_t)N * H * W * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    size_t r = i / C;
    const int xx = (int)(r % W); r /= W;
    const int yy = (int)(r % H);
    const int img = (int)(r / H);
    const size_t W2 = 2 * (size_t)W;
    const size_t b = ((((size_t)img * 2 * H + 2 * yy) * W2) + 2 * xx) * C + c;
    const float v = (src[b] + src[b + C]) + (src[b + W2 * C] + src[b + W2 * C + C]);
    dst[i] = accumulate ? dst[i] + v : v;
  }
}

__global__ void relu_mask_kernel(float* __restrict__ g, const float* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    if (!(y[i] > 0.0f)) g[i] = 0.0f;
}

// Global mean over pixels: partial sums over pixel chunks, then a fixed-order pass.
constexpr int kGapChunks = 64;
__global__ void gap_partial_kernel(const float* __restrict__ x, int P, int C,
                                   float* __restrict__ part) {  // grid (N, kGapChunks)
  const int img = blockIdx.x, ch = blockIdx.y;
  const int per = (P + kGapChunks - 1) / kGapChunks;
  const int p0 = ch * per, p1 = min(P, p0 + per);
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float s = 0.0f;
    for (int p = p0; p < p1; ++p) s += x[((size_t)img * P + p) * C + c];
    part[((size_t)img * kGapChunks + ch) * C + c] = s;
  }
}

__global__ void gap_final_kernel(const float* __restrict__ part, int N, int P, int C,
                                 float* __restrict__ g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * C) return;
  const int img = i / C, c = i - img * C;
  float s = 0.0f;
  for (int k = 0; k < kGapChunks; ++k) s += part[((size_t)img * kGapChunks + k) * C + c];
  g[i] = s / (float)P;
}

// z[n][j] = sum_c A[j][c] g[n][c] + cvec[j]
__global__ void eps_head_kernel(const float* __restrict__ g, const float* __restrict__ A,
                                const float* __restrict__ cvec, float* __restrict__ z, int N,
                                int C, int J) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N * J) return;
  const int img = i / J, j = i - img * J;
  float s = cvec[j];
  for (int c = 0; c < C; ++c) s = fmaf(A[(size_t)j * C + c], g[(size_t)img * C + c], s);
  z[i] = s;
}

__global__ void eps_out_kernel(const float* __restrict__ z, double* __restrict__ eps, int n,
                               float lo0, float lo1, float hi0, float hi1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = i & 1;
  const double e = exp((double)z[i]);
  eps[i] = fmin(fmax(e, (double)(m ? lo1 : lo0)), (double)(m ? hi1 : hi0));
}

// Loss of the control head and its backward (one block): dz, dA, dc, dg.
__global__ void eps_head_backward_kernel(const float* __restrict__ z, const float* __restrict__ le,
                                         const float* __restrict__ g, const float* __restrict__ A,
                                         float lam, int N, int C, int J, float* __restrict__ dA,
                                         float* __restrict__ dc, float* __restrict__ dg,
                                         double* __restrict__ loss_z) {
  extern __shared__ float dz[];  // N * J
  const int nz = N * J;
  for (int i = threadIdx.x; i < nz; i += blockDim.x) dz[i] = 2.0f * lam * (z[i] - le[i]) / (float)nz;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nz; ++i) {
      const double d = (double)z[i] - (double)le[i];
      s += d * d;
    }
    *loss_z = (double)lam * s / nz;
  }
  for (int i = threadIdx.x; i < J * C; i += blockDim.x) {
    const int j = i / C, c = i - j * C;
    float s = 0.0f;
    for (int n = 0; n < N; ++n) s = fmaf(dz[n * J + j], g[(size_t)n * C + c], s);
    dA[i] = s;
  }
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    float s = 0.0f;
    for (int n = 0; n < N; ++n) s += dz[n * J + j];
    dc[j] = s;
  }
  for (int i = threadIdx.x; i < N * C; i += blockDim.x) {
    const int n = i / C, c = i - n * C;
    float s = 0.0f;
    for (int j = 0; j < J; ++j) s = fmaf(dz[n * J + j], A[(size_t)j * C + c], s);
    dg[i] = s;
  }
}

// d e_L [n, p, c] = dg[n][c] / P (the gradient of the pixel mean)
__global__ void gap_backward_kernel(const float* __restrict__ dg, float* __restrict__ dx, int N,
                                    int P, int C) {
  const size_t n = (size_t)N * P * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int img = (int)(i / ((size_t)P * C));
    dx[i] = dg[(size_t)img * C + c] / (float)P;
  }
}

// dmu = 2 (mu - mu_t) / n; per-block partial sums of (mu - mu_t)^2 in float64.
__global__ void mu_loss_kernel(const float* __restrict__ mu, const float* __restrict__ mt,
                               float* __restrict__ dmu, size_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  const float scale = 2.0f / (float)n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float d = mu[i] - mt[i];
    dmu[i] = scale * d;
    s += (double)d * (double)d;
  }
  double v[1] = {s}, tot[1];
  agents::block_sum<1>(v, red, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot[0];
}

__global__ void loss_final_kernel(const double* __restrict__ part, int nb, size_t n,
                                  const double* __restrict__ loss_z, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b];
  *out = s / (double)n + *loss_z;
}

__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2,
                            float eps, float wd, float c1, float c2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * th[i]);
  }
}

// Edge-replicating pad [N][H][W][C] -> [N][Hp][Wp][C].
__global__ void pad_kernel(const float* __restrict__ x, float* __restrict__ y, int N, int H, int W,
                           int Hp, int Wp, int C) {
  const size_t n = (size_t)N * Hp * Wp * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    size_t r = i / C;
    const int xx = (int)(r % Wp); r /= Wp;
    const int yy = (int)(r % Hp);
    const int img = (int)(r / Hp);
    const int sy = min(yy, H - 1), sx = min(xx, W - 1);
    y[i] = x[(((size_t)img * H + sy) * W + sx) * C + c];
  }
}

// Crop [N][Hp][Wp][C] -> [N][H][W][C] and project each pixel's dual onto the unit ball:
// mode 1: one ball per pixel over all C entries; mode 2: one per (x, y) channel pair.
// f x f block means of [N][H][W][C] (H, W multiples of f) -> [N][H/f][W/f][C].
__global__ void block_mean_kernel(const float* __restrict__ x, float* __restrict__ y, int N,
                                  int H, int W, int C, int f) {
  const int h = H / f, w = W / f;
  const size_t n = (size_t)N * h * w * C;
  const float inv = 1.0f / (float)(f * f);
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % C);
    size_t r = t / C;
    const int j = (int)(r % w);
    r /= w;
    const int i = (int)(r % h);
    const int b = (int)(r / h);
    const float* src = x + (((size_t)b * H + (size_t)i * f) * W + (size_t)j * f) * C + c;
    float acc = 0.0f;
    for (int u = 0; u < f; ++u)
      for (int v = 0; v < f; ++v) acc += src[((size_t)u * W + v) * C];
    y[t] = acc * inv;
  }
}

// Nearest upsampling by f: [N][h][w][C] -> [N][h f][w f][C].
__global__ void upsample_nearest_kernel(const float* __restrict__ x, float* __restrict__ y,
                                        int N, int h, int w, int C, int f) {
  const int H = h * f, W = w * f;
  const size_t n = (size_t)N * H * W * C;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % C);
    size_t r = t / C;
    const int j = (int)(r % W);
    r /= W;
    const int i = (int)(r % H);
    const int b = (int)(r / H);
    y[t] = x[(((size_t)b * h + i / f) * w + j / f) * C + c];
  }
}

__global__ void crop_project_kernel(const float* __restrict__ src, float* __restrict__ dst, int N,
                                    int H, int W, int Hp, int Wp, int C, int mode) {
  const size_t np = (size_t)N * H * W;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < np;
       i += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(i % W);
    const size_t r = i / W;
    const int yy = (int)(r % H);
    const int img = (int)(r / H);
    const float* s = src + (((size_t)img * Hp + yy) * Wp + xx) * C;
    float* d = dst + i * C;
    if (mode == 1) {
      float n2 = 0.0f;
      for (int c = 0; c < C; ++c) n2 = fmaf(s[c], s[c], n2);
      const float f = n2 > 1.0f ? rsqrtf(n2) : 1.0f;
      for (int c = 0; c < C; ++c) d[c] = s[c] * f;
    } else if (mode == 2) {
      const int h = C / 2;
      for (int c = 0; c < h; ++c) {
        const float a = s[c], b = s[h + c];
        const float n2 = fmaf(a, a, b * b);
        const float f = n2 > 1.0f ? rsqrtf(n2) : 1.0f;
        d[c] = a * f;
        d[h + c] = b * f;
      }
    } else {
      for (int c = 0; c < C; ++c) d[c] = s[c];
    }
  }
}

struct Conv {
  int cin, cout;
  size_t w_off, b_off;     // in the flat parameter vector
  __nv_bfloat16* w16 = nullptr;
  __nv_bfloat16* wt16 = nullptr;
};

}  // namespace

struct ws_net {
  ws_net_config cfg{};
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<Conv> convs;
  size_t A_off = 0, c_off = 0, nparams = 0;
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16* wbuf = nullptr;
  long long step = 0;
  bool have_grad = false;
  // activations for (N, H, W) (H, W padded); grads allocated on demand
  int aN = 0, aH = 0, aW = 0;
  bool agrad = false;
  std::vector<void*> act_allocs;
  float* xin = nullptr;                 // padded input
  std::vector<float*> P, Ea, Eb, Da, S, Db, U;   // index = level (1-based)
  std::vector<float*> dP, dEa, dEb, dS, dDb, dU;
  float *mu = nullptr, *dmu = nullptr, *gap = nullptr, *z = nullptr, *dg = nullptr;
  float* gap_part = nullptr;
  float* wsbuf = nullptr;
  size_t wsbytes = 0;
  double* d_loss = nullptr;             // [0] total, [1] control part, [2..] partials
  int nb_loss = 0;

  int width(int l) const { return cfg.base << (l - 1); }
  const Conv& conv(const char* kind, int l, char ab) const {
    // order: enc1a enc1b ... encLa encLb dec(L-1)a dec(L-1)b ... dec1a dec1b head
    const int L = cfg.levels;
    int idx;
    if (kind[0] == 'e') idx = 2 * (l - 1) + (ab == 'b');
    else if (kind[0] == 'd') idx = 2 * L + 2 * (L - 1 - l) + (ab == 'b');
    else idx = 2 * L + 2 * (L - 1);
    return convs[idx];
  }
  float* W(const Conv& c) const { return theta + c.w_off; }
  float* B(const Conv& c) const { return theta + c.b_off; }
  float* gW(const Conv& c) const { return grad + c.w_off; }
  float* gB(const Conv& c) const { return grad + c.b_off; }

  void free_acts() {
    for (void* p : act_allocs) cudaFree(p);
    act_allocs.clear();
    aN = aH = aW = 0;
    agrad = false;
  }
  ~ws_net() {
    free_acts();
    cudaFree(theta); cudaFree(grad); cudaFree(m1); cudaFree(m2); cudaFree(wbuf);
  }
  int alloc(float** p, size_t count) {
    void* q = nullptr;
    WCK(cudaMalloc(&q, (count ? count : 1) * sizeof(float)));
    act_allocs.push_back(q);
    *p = static_cast<float*>(q);
    return AGENTS_OK;
  }

  int ensure_acts(int N, int H, int W, bool grads) {
    if (N == aN && H == aH && W == aW && (!grads || agrad)) return AGENTS_OK;
    free_acts();
    const int L = cfg.levels;
    auto px = [&](int l) { return (size_t)N * (H >> (l - 1)) * (W >> (l - 1)); };
    P.assign(L + 1, nullptr); Ea.assign(L + 1, nullptr); Eb.assign(L + 1, nullptr);
    Da.assign(L + 1, nullptr); S.assign(L + 1, nullptr); Db.assign(L + 1, nullptr);
    U.assign(L + 1, nullptr);
    dP.assign(L + 1, nullptr); dEa.assign(L + 1, nullptr); dEb.assign(L + 1, nullptr);
    dS.assign(L + 1, nullptr); dDb.assign(L + 1, nullptr); dU.assign(L + 1, nullptr);
    WTRY(alloc(&xin, px(1) * cfg.in_ch));
    for (int l = 1; l <= L; ++l) {
      if (l > 1) WTRY(alloc(&P[l], px(l) * width(l - 1)));
      WTRY(alloc(&Ea[l], px(l) * width(l)));
      WTRY(alloc(&Eb[l], px(l) * width(l)));
      if (l < L) {
        WTRY(alloc(&Da[l], px(l) * width(l)));
        WTRY(alloc(&S[l], px(l) * width(l)));
        WTRY(alloc(&Db[l], px(l) * width(l)));
      }
    }
    WTRY(alloc(&mu, px(1) * cfg.out_ch));
    WTRY(alloc(&gap, (size_t)N * width(L)));
    WTRY(alloc(&gap_part, (size_t)N * kGapChunks * width(L)));
    WTRY(alloc(&z, (size_t)N * 2 * cfg.nsteps));
    if (grads) {
      for (int l = 1; l <= L; ++l) {
        if (l > 1) WTRY(alloc(&dP[l], px(l) * width(l - 1)));
        WTRY(alloc(&dEa[l], px(l) * width(l)));
        WTRY(alloc(&dEb[l], px(l) * width(l)));
        if (l < L) {
          WTRY(alloc(&dS[l], px(l) * width(l)));
          WTRY(alloc(&dDb[l], px(l) * width(l)));
          WTRY(alloc(&dU[l], px(l) * width(l + 1)));
        }
      }
      WTRY(alloc(&dmu, px(1) * cfg.out_ch));
      WTRY(alloc(&dg, (size_t)N * width(L)));
      size_t need = 0;
      for (int l = 1; l <= L; ++l) {
        const int Hl = H >> (l - 1), Wl = W >> (l - 1);
        for (const Conv* c : {&conv("e", l, 'a'), &conv("e", l, 'b')})
          need = std::max(need, ws::conv_backward_weight_workspace(N, Hl, Wl, c->cin, c->cout));
        if (l < L)
          for (const Conv* c : {&conv("d", l, 'a'), &conv("d", l, 'b')})
            need = std::max(need, ws::conv_backward_weight_workspace(N, Hl, Wl, c->cin, c->cout));
      }
      need = std::max(need, ws::conv_backward_weight_workspace(N, H, W, width(1), cfg.out_ch));
      WTRY(alloc(&wsbuf, need / sizeof(float) + 1));
      wsbytes = need;
      nb_loss = 1024;
      void* q = nullptr;
      WCK(cudaMalloc(&q, (size_t)(nb_loss + 2) * sizeof(double)));
      act_allocs.push_back(q);
      d_loss = static_cast<double*>(q);
      agrad = true;
    }
    aN = N; aH = H; aW = W;
    return AGENTS_OK;
  }

  int refresh_bf16() {
    for (Conv& c : convs) WCK(ws::transpose_weights(W(c), c.w16, c.wt16, c.cin, c.cout, stream));
    return AGENTS_OK;
  }

  // Forward over xin (padded, N x H x W); fills every saved activation, mu and z.
  int forward(int N, int H, int W) {
    const int L = cfg.levels;
    for (int l = 1; l <= L; ++l) {
      const int Hl = H >> (l - 1), Wl = W >> (l - 1);
      const float* in = xin;
      if (l > 1) {
        const size_t n = (size_t)N * Hl * Wl * width(l - 1);
        avgpool2_kernel<<<blocks_for(n), kThreads, 0, stream>>>(Eb[l - 1], P[l], N, Hl, Wl,
                                                               width(l - 1));
        WCK(cudaGetLastError());
        in = P[l];
      }
      const Conv& a = conv("e", l, 'a');
      const Conv& b = conv("e", l, 'b');
      WCK(ws::conv_forward(in, a.w16, B(a), Ea[l], nullptr, nullptr, N, Hl, Wl, a.cin, a.cout, 1, 0,
                           stream));
      WCK(ws::conv_forward(Ea[l], b.w16, B(b), Eb[l], nullptr, nullptr, N, Hl, Wl, b.cin, b.cout,
                           1, 0, stream));
    }
    const float* d = Eb[L];
    for (int l = L - 1; l >= 1; --l) {
      const int Hl = H >> (l - 1), Wl = W >> (l - 1);
      const Conv& a = conv("d", l, 'a');
      const Conv& b = conv("d", l, 'b');
      WCK(ws::conv_forward(d, a.w16, B(a), Da[l], Eb[l], S[l], N, Hl, Wl, a.cin, a.cout, 1, 1,
                           stream));
      WCK(ws::conv_forward(S[l], b.w16, B(b), Db[l], nullptr, nullptr, N, Hl, Wl, b.cin, b.cout, 1,
                           0, stream));
      d = Db[l];
    }
    const Conv& h = conv("h", 0, 0);
    WCK(ws::conv_forward(d, h.w16, B(h), mu, nullptr, nullptr, N, H, W, h.cin, h.cout, 0, 0,
                         stream));
    const int HL = H >> (L - 1), WL = W >> (L - 1), CL = width(L), J = 2 * cfg.nsteps;
    gap_partial_kernel<<<dim3(N, kGapChunks), 256, 0, stream>>>(Eb[L], HL * WL, CL, gap_part);
    gap_final_kernel<<<(N * CL + 255) / 256, 256, 0, stream>>>(gap_part, N, HL * WL, CL, gap);
    eps_head_kernel<<<(N * J + 255) / 256, 256, 0, stream>>>(gap, theta + A_off, theta + c_off, z,
                                                            N, CL, J);
    WCK(cudaGetLastError());
    return AGENTS_OK;
  }

  int relu_mask(float* g, const float* y, size_t n) {
    relu_mask_kernel<<<blocks_for(n), kThreads, 0, stream>>>(g, y, n);
    WCK(cudaGetLastError());
    return AGENTS_OK;
  }

  // dW, db of one convolution from its (masked) output gradient.
  int weight_grad(const Conv& c, const float* x, const float* dy, int N, int H, int W, int up) {
    WCK(ws::conv_backward_weight(x, dy, gW(c), gB(c), N, H, W, c.cin, c.cout, up, wsbuf, wsbytes,
                                 stream));
    return AGENTS_OK;
  }

  int backward(int N, int H, int W, const float* mu_t, const float* le_t, float lam) {
    const int L = cfg.levels;
    const size_t nmu = (size_t)N * H * W * cfg.out_ch;
    const int nb = std::min(nb_loss, blocks_for(nmu));
    mu_loss_kernel<<<nb, kThreads, 0, stream>>>(mu, mu_t, dmu, nmu, d_loss + 2);
    WCK(cudaGetLastError());
    const int HL = H >> (L - 1), WL = W >> (L - 1), CL = width(L), J = 2 * cfg.nsteps;
    eps_head_backward_kernel<<<1, 256, (size_t)N * J * sizeof(float), stream>>>(
        z, le_t, gap, theta + A_off, lam, N, CL, J, grad + A_off, grad + c_off, dg, d_loss + 1);
    loss_final_kernel<<<1, 32, 0, stream>>>(d_loss + 2, nb, nmu, d_loss + 1, d_loss);
    {
      const size_t n = (size_t)N * HL * WL * CL;
      gap_backward_kernel<<<blocks_for(n), kThreads, 0, stream>>>(dg, dEb[L], N, HL * WL, CL);
    }
    WCK(cudaGetLastError());
    // mu head (no activation)
    const Conv& h = conv("h", 0, 0);
    // (levels >= 2: the head reads the decoder output of level 1)
    WTRY(weight_grad(h, Db[1], dmu, N, H, W, 0));
    WCK(ws::conv_backward_data(dmu, h.wt16, dDb[1], N, H, W, h.cin, h.cout, stream));
    // decoder levels 1 .. L-1
    for (int l = 1; l < L; ++l) {
      const int Hl = H >> (l - 1), Wl = W >> (l - 1);
      const size_t n = (size_t)N * Hl * Wl * width(l);
      const Conv& b = conv("d", l, 'b');
      const Conv& a = conv("d", l, 'a');
      WTRY(relu_mask(dDb[l], Db[l], n));
      WTRY(weight_grad(b, S[l], dDb[l], N, Hl, Wl, 0));
      WCK(ws::conv_backward_data(dDb[l], b.wt16, dS[l], N, Hl, Wl, b.cin, b.cout, stream));
      // the skip connection carries dS to the encoder output of level l
      WCK(cudaMemcpyAsync(dEb[l], dS[l], n * sizeof(float), cudaMemcpyDeviceToDevice, stream));
      WTRY(relu_mask(dS[l], Da[l], n));
      const float* up_src = (l + 1 < L) ? Db[l + 1] : Eb[L];
      WTRY(weight_grad(a, up_src, dS[l], N, Hl, Wl, 1));
      WCK(ws::conv_backward_data(dS[l], a.wt16, dU[l], N, Hl, Wl, a.cin, a.cout, stream));
      const size_t nh = (size_t)N * (Hl / 2) * (Wl / 2) * width(l + 1);
      float* dst = (l + 1 < L) ? dDb[l + 1] : dEb[L];
      upsample2_backward_kernel<<<blocks_for(nh), kThreads, 0, stream>>>(
          dU[l], dst, N, Hl / 2, Wl / 2, width(l + 1), (l + 1 < L) ? 0 : 1);
      WCK(cudaGetLastError());
    }
    // encoder levels L .. 1
    for (int l = L; l >= 1; --l) {
      const int Hl = H >> (l - 1), Wl = W >> (l - 1);
      const size_t n = (size_t)N * Hl * Wl * width(l);
      const Conv& b = conv("e", l, 'b');
      const Conv& a = conv("e", l, 'a');
      WTRY(relu_mask(dEb[l], Eb[l], n));
      WTRY(weight_grad(b, Ea[l], dEb[l], N, Hl, Wl, 0));
      WCK(ws::conv_backward_data(dEb[l], b.wt16, dEa[l], N, Hl, Wl, b.cin, b.cout, stream));
      WTRY(relu_mask(dEa[l], Ea[l], n));
      const float* in = l > 1 ? P[l] : xin;
      WTRY(weight_grad(a, in, dEa[l], N, Hl, Wl, 0));
      if (l > 1) {
        WCK(ws::conv_backward_data(dEa[l], a.wt16, dP[l], N, Hl, Wl, a.cin, a.cout, stream));
        const size_t nf = (size_t)N * (2 * Hl) * (2 * Wl) * width(l - 1);
        avgpool2_backward_acc_kernel<<<blocks_for(nf), kThreads, 0, stream>>>(
            dP[l], dEb[l - 1], N, 2 * Hl, 2 * Wl, width(l - 1));
        WCK(cudaGetLastError());
      }
    }
    return AGENTS_OK;
  }
};

extern "C" {

const char* ws_last_error(void) { return g_ws_error.c_str(); }

int ws_conv3x3_forward(const float* x, const uint16_t* w16, const float* bias, float* y,
                       const float* add, float* y2, int32_t N, int32_t H, int32_t W, int32_t Cin,
                       int32_t Cout, int32_t relu, int32_t up, void* stream) {
  if (!x || !w16 || !y || N < 1 || H < 1 || W < 1 || Cin < 1 || Cout < 1 || (add && !y2) ||
      (up && ((H | W) & 1)) || (long long)N * H * W > 0x7fffffffLL)
    return ws_fail(AGENTS_EINVAL, "ws_conv3x3_forward: bad arguments");
  WCK(ws::conv_forward(x, reinterpret_cast<const __nv_bfloat16*>(w16), bias, y, add, y2, N, H, W,
                       Cin, Cout, relu, up, static_cast<cudaStream_t>(stream)));
  return AGENTS_OK;
}

int ws_conv3x3_backward_data(const float* dy, const uint16_t* wt16, float* dx, int32_t N,
                             int32_t H, int32_t W, int32_t Cin, int32_t Cout, void* stream) {
  if (!dy || !wt16 || !dx || N < 1 || H < 1 || W < 1 || Cin < 1 || Cout < 1 ||
      (long long)N * H * W > 0x7fffffffLL)
    return ws_fail(AGENTS_EINVAL, "ws_conv3x3_backward_data: bad arguments");
  WCK(ws::conv_backward_data(dy, reinterpret_cast<const __nv_bfloat16*>(wt16), dx, N, H, W, Cin,
                             Cout, static_cast<cudaStream_t>(stream)));
  return AGENTS_OK;
}

size_t ws_conv3x3_backward_weight_workspace(int32_t N, int32_t H, int32_t W, int32_t Cin,
                                            int32_t Cout) {
  return ws::conv_backward_weight_workspace(N, H, W, Cin, Cout);
}

int ws_conv3x3_backward_weight(const float* x, const float* dy, float* dw, float* db, int32_t N,
                               int32_t H, int32_t W, int32_t Cin, int32_t Cout, int32_t up,
                               void* workspace, size_t workspace_bytes, void* stream) {
  if (!x || !dy || !dw || !workspace || N < 1 || H < 1 || W < 1 || Cin < 1 || Cout < 1 ||
      (up && ((H | W) & 1)) || (long long)N * H * W > 0x7fffffffLL)
    return ws_fail(AGENTS_EINVAL, "ws_conv3x3_backward_weight: bad arguments");
  if (workspace_bytes < ws::conv_backward_weight_workspace(N, H, W, Cin, Cout))
    return ws_fail(AGENTS_EINVAL, "ws_conv3x3_backward_weight: workspace too small");
  WCK(ws::conv_backward_weight(x, dy, dw, db, N, H, W, Cin, Cout, up,
                               static_cast<float*>(workspace), workspace_bytes,
                               static_cast<cudaStream_t>(stream)));
  return AGENTS_OK;
}

int ws_tensor_core_fault_take(void) {
  const int r = ws::conv_tc_take_error();
  if (r < 0) return ws_fail(AGENTS_ECUDA, "ws_tensor_core_fault_take: cannot read the flag");
  return r;
}

int ws_transpose_weights(const float* w, uint16_t* w16, uint16_t* wt16, int32_t Cin, int32_t Cout,
                         void* stream) {
  if (!w || !w16 || Cin < 1 || Cout < 1)
    return ws_fail(AGENTS_EINVAL, "ws_transpose_weights: bad arguments");
  WCK(ws::transpose_weights(w, reinterpret_cast<__nv_bfloat16*>(w16),
                            reinterpret_cast<__nv_bfloat16*>(wt16), Cin, Cout,
                            static_cast<cudaStream_t>(stream)));
  return AGENTS_OK;
}

int ws_net_create(const ws_net_config* cfg, void* stream, ws_net** out) {
  if (!cfg || !out) return ws_fail(AGENTS_EINVAL, "ws_net_create: NULL argument");
  *out = nullptr;
  if (cfg->in_ch < 1 || cfg->out_ch < 1 || cfg->base < 1 || cfg->levels < 2 ||
      cfg->levels > 8 || cfg->nsteps < 1 || !(cfg->eps_lo[0] > 0) || !(cfg->eps_lo[1] > 0) ||
      !(cfg->eps_hi[0] >= cfg->eps_lo[0]) || !(cfg->eps_hi[1] >= cfg->eps_lo[1]) ||
      ((long long)cfg->base << (cfg->levels - 1)) > 4096)
    return ws_fail(AGENTS_EINVAL, "ws_net_create: invalid configuration");
  ws_net* net = new ws_net();
  net->cfg = *cfg;
  net->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&net->device);
  const int L = cfg->levels;
  size_t off = 0, nw = 0;
  auto add = [&](int cin, int cout) {
    Conv c;
    c.cin = cin;
    c.cout = cout;
    c.w_off = off;
    off += (size_t)cout * 9 * cin;
    c.b_off = off;
    off += cout;
    nw += (size_t)cout * 9 * cin;
    net->convs.push_back(c);
  };
  int cin = cfg->in_ch;
  for (int l = 1; l <= L; ++l) {
    add(cin, net->width(l));
    add(net->width(l), net->width(l));
    cin = net->width(l);
  }
  for (int l = L - 1; l >= 1; --l) {
    add(net->width(l + 1), net->width(l));
    add(net->width(l), net->width(l));
  }
  add(net->width(1), cfg->out_ch);
  net->A_off = off;
  off += (size_t)2 * cfg->nsteps * net->width(L);
  net->c_off = off;
  off += (size_t)2 * cfg->nsteps;
  net->nparams = off;
  auto fail = [&](cudaError_t e) {
    delete net;
    return ws_fail(e == cudaErrorMemoryAllocation ? AGENTS_ENOMEM : AGENTS_ECUDA,
                   std::string("ws_net_create: ") + cudaGetErrorString(e));
  };
  cudaError_t e;
  for (float** p : {&net->theta, &net->grad, &net->m1, &net->m2}) {
    if ((e = cudaMalloc(p, off * sizeof(float))) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(*p, 0, off * sizeof(float), net->stream)) != cudaSuccess) return fail(e);
  }
  if ((e = cudaMalloc(&net->wbuf, 2 * nw * sizeof(__nv_bfloat16))) != cudaSuccess) return fail(e);
  size_t k = 0;
  for (Conv& c : net->convs) {
    const size_t n = (size_t)c.cout * 9 * c.cin;
    c.w16 = net->wbuf + k;
    c.wt16 = net->wbuf + nw + k;
    k += n;
  }
  if (net->refresh_bf16() != AGENTS_OK) {
    delete net;
    return AGENTS_ECUDA;
  }
  *out = net;
  return AGENTS_OK;
}

void ws_net_destroy(ws_net* net) {
  if (!net) return;
  cudaStreamSynchronize(net->stream);
  delete net;
}

int64_t ws_net_num_params(const ws_net* net) { return net ? (int64_t)net->nparams : -1; }

int ws_net_set_params(ws_net* net, const float* params) {
  if (!net || !params) return ws_fail(AGENTS_EINVAL, "ws_net_set_params: NULL argument");
  WCK(cudaMemcpyAsync(net->theta, params, net->nparams * sizeof(float),
                      is_dev(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      net->stream));
  WCK(cudaMemsetAsync(net->m1, 0, net->nparams * sizeof(float), net->stream));
  WCK(cudaMemsetAsync(net->m2, 0, net->nparams * sizeof(float), net->stream));
  net->step = 0;
  net->have_grad = false;
  WTRY(net->refresh_bf16());
  WCK(cudaStreamSynchronize(net->stream));
  return AGENTS_OK;
}

int ws_net_get_params(ws_net* net, float* params) {
  if (!net || !params) return ws_fail(AGENTS_EINVAL, "ws_net_get_params: NULL argument");
  WCK(cudaMemcpyAsync(params, net->theta, net->nparams * sizeof(float),
                      is_dev(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                      net->stream));
  WCK(cudaStreamSynchronize(net->stream));
  return AGENTS_OK;
}

int ws_net_forward(ws_net* net, const float* img, int32_t N, int32_t H, int32_t W,
                   int32_t project, float* mu_out, double* eps_out, float* z_out) {
  if (!net || !img || N < 1 || H < 1 || W < 1 || project < 0 || project > 2 ||
      (project == 2 && (net->cfg.out_ch & 1)))
    return ws_fail(AGENTS_EINVAL, "ws_net_forward: bad arguments");
  const int q = 1 << (net->cfg.levels - 1);
  const int Hp = (H + q - 1) / q * q, Wp = (W + q - 1) / q * q;
  if ((long long)N * Hp * Wp > 0x7fffffffLL / 64)
    return ws_fail(AGENTS_EINVAL, "ws_net_forward: batch too large");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != net->device) cudaSetDevice(net->device);
  WTRY(net->ensure_acts(N, Hp, Wp, false));
  const size_t n = (size_t)N * Hp * Wp * net->cfg.in_ch;
  pad_kernel<<<blocks_for(n), kThreads, 0, net->stream>>>(img, net->xin, N, H, W, Hp, Wp,
                                                          net->cfg.in_ch);
  WCK(cudaGetLastError());
  WTRY(net->forward(N, Hp, Wp));
  if (mu_out) {
    crop_project_kernel<<<blocks_for((size_t)N * H * W), kThreads, 0, net->stream>>>(
        net->mu, mu_out, N, H, W, Hp, Wp, net->cfg.out_ch, project);
    WCK(cudaGetLastError());
  }
  const int J = 2 * net->cfg.nsteps;
  if (z_out)
    WCK(cudaMemcpyAsync(z_out, net->z, (size_t)N * J * sizeof(float), cudaMemcpyDeviceToDevice,
                        net->stream));
  if (eps_out) {
    double* d = nullptr;
    const bool dev = is_dev(eps_out);
    if (dev) {
      d = eps_out;
    } else {
      WCK(cudaMalloc(&d, (size_t)N * J * sizeof(double)));
    }
    eps_out_kernel<<<(N * J + 255) / 256, 256, 0, net->stream>>>(
        net->z, d, N * J, net->cfg.eps_lo[0], net->cfg.eps_lo[1], net->cfg.eps_hi[0],
        net->cfg.eps_hi[1]);
    cudaError_t e = cudaGetLastError();
    if (!dev) {
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(eps_out, d, (size_t)N * J * sizeof(double), cudaMemcpyDeviceToHost,
                            net->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
      cudaFree(d);
    }
    WCK(e);
  }
  if (prev >= 0 && prev != net->device) cudaSetDevice(prev);
  return AGENTS_OK;
}

int ws_net_forward_lifted(ws_net* net, const float* img, int32_t N, int32_t H, int32_t W,
                          int32_t factor, int32_t project, float* mu_out, double* eps_out) {
  if (!net || !img || !mu_out || N < 1 || factor < 1 || H < factor || W < factor ||
      H % factor || W % factor)
    return ws_fail(AGENTS_EINVAL, "ws_net_forward_lifted: bad arguments (sides must be "
                                  "multiples of factor)");
  if (factor == 1) return ws_net_forward(net, img, N, H, W, project, mu_out, eps_out, nullptr);
  const int h = H / factor, w = W / factor;
  const int ci = net->cfg.in_ch, co = net->cfg.out_ch;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != net->device) cudaSetDevice(net->device);
  float *small = nullptr, *small_mu = nullptr;
  WCK(cudaMallocAsync(&small, (size_t)N * h * w * ci * sizeof(float), net->stream));
  cudaError_t e = cudaMallocAsync(&small_mu, (size_t)N * h * w * co * sizeof(float), net->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(small, net->stream);
    return ws_fail(AGENTS_ENOMEM, "ws_net_forward_lifted: allocation failed");
  }
  block_mean_kernel<<<blocks_for((size_t)N * h * w * ci), kThreads, 0, net->stream>>>(
      img, small, N, H, W, ci, factor);
  int st = cudaGetLastError() == cudaSuccess ? AGENTS_OK : AGENTS_ECUDA;
  if (st == AGENTS_OK) st = ws_net_forward(net, small, N, h, w, project, small_mu, eps_out, nullptr);
  if (st == AGENTS_OK) {
    upsample_nearest_kernel<<<blocks_for((size_t)N * H * W * co), kThreads, 0, net->stream>>>(
        small_mu, mu_out, N, h, w, co, factor);
    if (cudaGetLastError() != cudaSuccess) st = AGENTS_ECUDA;
  }
  cudaFreeAsync(small_mu, net->stream);
  cudaFreeAsync(small, net->stream);
  if (prev >= 0 && prev != net->device) cudaSetDevice(prev);
  if (st == AGENTS_ECUDA) return ws_fail(st, "ws_net_forward_lifted: kernel launch failed");
  return st;
}

int ws_net_loss_grad(ws_net* net, const float* img, const float* mu_t, const float* log_eps_t,
                     int32_t N, int32_t H, int32_t W, float lam_eps, double* loss_out,
                     float* grad_out) {
  const int q = net ? 1 << (net->cfg.levels - 1) : 1;
  if (!net || !img || !mu_t || !log_eps_t || N < 1 || H < q || W < q || H % q || W % q ||
      !(lam_eps >= 0) || (long long)N * H * W > 0x7fffffffLL / 64)
    return ws_fail(AGENTS_EINVAL, "ws_net_loss_grad: bad arguments (sides must be multiples "
                                  "of 2^(levels-1))");
  if ((long long)N * 2 * net->cfg.nsteps * 4 > 48 * 1024)
    return ws_fail(AGENTS_EINVAL, "ws_net_loss_grad: batch too large for the control head");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != net->device) cudaSetDevice(net->device);
  WTRY(net->ensure_acts(N, H, W, true));
  WCK(cudaMemcpyAsync(net->xin, img, (size_t)N * H * W * net->cfg.in_ch * sizeof(float),
                      cudaMemcpyDeviceToDevice, net->stream));
  WTRY(net->forward(N, H, W));
  WTRY(net->backward(N, H, W, mu_t, log_eps_t, lam_eps));
  net->have_grad = true;
  if (grad_out)
    WCK(cudaMemcpyAsync(grad_out, net->grad, net->nparams * sizeof(float),
                        is_dev(grad_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        net->stream));
  if (loss_out) {
    WCK(cudaMemcpyAsync(loss_out, net->d_loss, sizeof(double), cudaMemcpyDeviceToHost,
                        net->stream));
    WCK(cudaStreamSynchronize(net->stream));
  }
  if (prev >= 0 && prev != net->device) cudaSetDevice(prev);
  return AGENTS_OK;
}

int ws_net_adam_step(ws_net* net, float lr, float beta1, float beta2, float adam_eps,
                     float weight_decay) {
  if (!net || !net->have_grad || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
      !(beta2 >= 0 && beta2 < 1) || !(adam_eps > 0) || !(weight_decay >= 0))
    return ws_fail(AGENTS_EINVAL, "ws_net_adam_step: bad arguments or no gradient");
  net->step += 1;
  const float c1 = 1.0f - (float)std::pow((double)beta1, (double)net->step);
  const float c2 = 1.0f - (float)std::pow((double)beta2, (double)net->step);
  adam_kernel<<<blocks_for(net->nparams), kThreads, 0, net->stream>>>(
      net->theta, net->grad, net->m1, net->m2, net->nparams, lr, beta1, beta2, adam_eps,
      weight_decay, c1, c2);
  WCK(cudaGetLastError());
  WTRY(net->refresh_bf16());
  return AGENTS_OK;
}

}  // extern "C"
