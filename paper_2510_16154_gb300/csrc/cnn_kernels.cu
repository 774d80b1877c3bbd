// Kernels of the warm-start network: 3x3 convolutions as implicit GEMMs on the BF16
// tensor cores (mma.sync m16n8k16, float32 accumulation) and the small float32 kernels
// around them (pooling, upsampling, control head, loss, Adam).
//
// One GEMM template serves the three convolution products:
//   forward      C[m = pixel][n = out ch]   = sum_{k = (tap, in ch)}  x(shifted pixel) W
//   backward-data C[m = pixel][n = in ch]   = sum_{k = (tap, out ch)} dy(shifted pixel) W
//   backward-weight C[m = out ch][n = (tap, in ch)] = sum_{k = pixel} dy x(shifted pixel)
// The operands are gathered from NHWC float32 tensors (zero outside the image), rounded to
// bfloat16 (nearest even) and staged in shared memory; the next K-chunk is fetched into
// registers while the current one is multiplied.  Backward-weight splits the pixel sum
// over blocks and adds the partial sums in a fixed order; its operands arrive pixel by
// pixel, so its tiles are stored k-major and transposed by ldmatrix.trans.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "cnn.h"

namespace ws {

constexpr int BM = 128, BN = 64, BK = 32, NT = 256;
constexpr int SK = BK + 8;  // shared-memory row stride (bf16): conflict-free fragment loads
// Backward-weight keeps its tiles k-major (k rows, m or n contiguous: the operands arrive
// pixel by pixel) and builds the fragments with ldmatrix.trans; the row strides keep the
// eight 16-byte rows of every 8x8 matrix in distinct banks.
constexpr int SAT = BM + 8, SBT = BN + 8;
static_assert(BK * SAT <= BM * SK && BK * SBT <= BN * SK, "k-major tiles reuse the buffers");

struct GemmArgs {
  int mode;
  int N, H, W;        // images and the convolution's (output) resolution
  int Cin, Cout;
  int up;             // conv input read through nearest 2x upsampling
  int M, Nc, K;       // GEMM sizes
  const float* x;
  const float* dy;
  const __nv_bfloat16* w;  // forward: [Cout][9 Cin]; backward-data: [Cin][9 Cout]
  const float* bias;
  const float* add;
  float* y;
  float* y2;
  int relu;
  float* out;         // backward-data: dx; backward-weight: partials [split][M][Nc]
  int k_split;        // backward-weight: pixels per split (multiple of BK)
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Four 8x8 bf16 matrices from shared memory, transposed (lane l gives the row address of
// matrix l / 8, row l % 8; each row 16 contiguous bytes).
__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t (&r)[4], const __nv_bfloat16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Address of the conv input value at logical pixel (img, yy, xx) channel ch, or nullptr
// outside the image.
__device__ __forceinline__ const float* x_at(const GemmArgs& g, int img, int yy, int xx) {
  if (yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return nullptr;
  const int Hs = g.H >> g.up, Ws = g.W >> g.up;
  return g.x + (((size_t)img * Hs + (yy >> g.up)) * Ws + (xx >> g.up)) * g.Cin;
}
__device__ __forceinline__ const float* dy_at(const GemmArgs& g, int img, int yy, int xx) {
  if (yy < 0 || yy >= g.H || xx < 0 || xx >= g.W) return nullptr;
  return g.dy + (((size_t)img * g.H + yy) * g.W + xx) * g.Cout;
}

// 8 consecutive float32 at p (16-byte aligned) or 8 zeros, packed to 4 bf16 pairs.
__device__ __forceinline__ void load8_vec(const float* p, uint32_t (&r)[4]) {
  if (p) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(p));
    const float4 v = __ldg(reinterpret_cast<const float4*>(p) + 1);
    r[0] = pack_bf16(u.x, u.y); r[1] = pack_bf16(u.z, u.w);
    r[2] = pack_bf16(v.x, v.y); r[3] = pack_bf16(v.z, v.w);
  } else {
    r[0] = r[1] = r[2] = r[3] = 0u;
  }
}

// ---- operand A for the pixel-row modes: row = pixel m, 8 consecutive k from k.
// k = tap * C + ch with C = Cin (forward) or Cout (backward-data).
__device__ __forceinline__ void load_a_pixel(const GemmArgs& g, int m, int img, int py, int px,
                                             int k, uint32_t (&r)[4]) {
  const bool fwd = g.mode == 0;
  const int C = fwd ? g.Cin : g.Cout;
  if (m >= g.M) { r[0] = r[1] = r[2] = r[3] = 0u; return; }
  if ((C & 7) == 0) {
    if (k >= g.K) { r[0] = r[1] = r[2] = r[3] = 0u; return; }
    const int tap = k / C, ch = k - tap * C;
    const int ky = tap / 3, kx = tap - 3 * (tap / 3);
    const float* base = fwd ? x_at(g, img, py + ky - 1, px + kx - 1)
                            : dy_at(g, img, py - ky + 1, px - kx + 1);
    load8_vec(base ? base + ch : nullptr, r);
    return;
  }
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int kk = k + j;
    v[j] = 0.0f;
    if (kk < g.K) {
      const int tap = kk / C, ch = kk - tap * C;
      const int ky = tap / 3, kx = tap - 3 * (tap / 3);
      const float* base = fwd ? x_at(g, img, py + ky - 1, px + kx - 1)
                              : dy_at(g, img, py - ky + 1, px - kx + 1);
      if (base) v[j] = __ldg(base + ch);
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) r[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
}

// ---- operand B for the pixel-row modes: weight row n, 8 consecutive k (bf16 in memory).
__device__ __forceinline__ void load_b_weight(const GemmArgs& g, int n, int k, uint32_t (&r)[4]) {
  if (n >= g.Nc || k >= g.K) { r[0] = r[1] = r[2] = r[3] = 0u; return; }
  const __nv_bfloat16* p = g.w + (size_t)n * g.K + k;
  if ((g.K & 7) == 0) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    r[0] = u.x; r[1] = u.y; r[2] = u.z; r[3] = u.w;
    return;
  }
  uint16_t h[8];
#pragma unroll
  for (int j = 0; j < 8; ++j)
    h[j] = (k + j < g.K) ? __bfloat16_as_ushort(p[j]) : (uint16_t)0;
#pragma unroll
  for (int j = 0; j < 4; ++j) r[j] = (uint32_t)h[2 * j] | ((uint32_t)h[2 * j + 1] << 16);
}

__device__ __forceinline__ void pixel_coords(const GemmArgs& g, int m, int& img, int& py, int& px) {
  const int hw = g.H * g.W;
  img = m / hw;
  const int rem = m - img * hw;
  py = rem / g.W;
  px = rem - py * g.W;
}

// ---- backward-weight operands: A[m = out ch][k = pixel] = dy[pixel][m],
// B[n = (tap, in ch)][k = pixel] = x[shifted pixel][in ch].  Each thread fetches 8
// consecutive m (or n) of one pixel.
__device__ __forceinline__ void load_a_dy(const GemmArgs& g, int m, int p, int kend, float (&v)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.0f;
  if (p >= kend) return;
  const float* base = g.dy + (size_t)p * g.Cout;
  if ((g.Cout & 7) == 0) {
    if (m >= g.Cout) return;
    const float4 u = __ldg(reinterpret_cast<const float4*>(base + m));
    const float4 w = __ldg(reinterpret_cast<const float4*>(base + m) + 1);
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w; v[4] = w.x; v[5] = w.y; v[6] = w.z; v[7] = w.w;
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (m + j < g.Cout) v[j] = __ldg(base + m + j);
}

__device__ __forceinline__ void load_b_x(const GemmArgs& g, int n, int p, int kend, float (&v)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.0f;
  if (p >= kend) return;
  int img, py, px;
  pixel_coords(g, p, img, py, px);
  if ((g.Cin & 7) == 0) {
    if (n >= g.Nc) return;
    const int tap = n / g.Cin, ch = n - tap * g.Cin;
    const float* base = x_at(g, img, py + tap / 3 - 1, px + tap % 3 - 1);
    if (!base) return;
    const float4 u = __ldg(reinterpret_cast<const float4*>(base + ch));
    const float4 w = __ldg(reinterpret_cast<const float4*>(base + ch) + 1);
    v[0] = u.x; v[1] = u.y; v[2] = u.z; v[3] = u.w; v[4] = w.x; v[5] = w.y; v[6] = w.z; v[7] = w.w;
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int nn = n + j;
    if (nn >= g.Nc) continue;
    const int tap = nn / g.Cin, ch = nn - tap * g.Cin;
    const float* base = x_at(g, img, py + tap / 3 - 1, px + tap % 3 - 1);
    if (base) v[j] = __ldg(base + ch);
  }
}

template <int MODE>
__global__ void __launch_bounds__(NT) igemm_kernel(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[BM * SK];
  __shared__ __align__(16) __nv_bfloat16 Bs[BN * SK];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int wm = (warp & 3) * 32, wn = (warp >> 2) * 32;
  int m0, n0, kbeg, kend;
  if (MODE == 2) {
    n0 = blockIdx.x * BN;
    m0 = blockIdx.y * BM;
    kbeg = blockIdx.z * g.k_split;
    kend = min(g.K, kbeg + g.k_split);
  } else {
    m0 = blockIdx.x * BM;
    n0 = blockIdx.y * BN;
    kbeg = 0;
    kend = g.K;
  }

  // per-thread fetch assignment
  uint32_t ra[2][4], rb[4];
  float fa[2][8], fb[8];
  int a_row = 0, a_k = 0, b_row = 0, b_k = 0, img = 0, py = 0, px = 0;
  if (MODE != 2) {
    a_row = tid >> 1;            // pixel row of the tile
    a_k = (tid & 1) * 16;        // 16 consecutive k (two groups of 8)
    b_row = tid >> 2;            // weight row
    b_k = (tid & 3) * 8;
    if (m0 + a_row < g.M) pixel_coords(g, m0 + a_row, img, py, px);
  } else {
    a_k = tid >> 3;              // pixel column of the tile (0..31)
    a_row = (tid & 7) * 16;      // 16 consecutive output channels
    b_k = tid >> 3;
    b_row = (tid & 7) * 8;       // 8 consecutive (tap, in ch)
  }

  auto fetch = [&](int k0) {
    if (MODE != 2) {
      load_a_pixel(g, m0 + a_row, img, py, px, k0 + a_k, ra[0]);
      load_a_pixel(g, m0 + a_row, img, py, px, k0 + a_k + 8, ra[1]);
      load_b_weight(g, n0 + b_row, k0 + b_k, rb);
    } else {
      load_a_dy(g, m0 + a_row, k0 + a_k, kend, fa[0]);
      load_a_dy(g, m0 + a_row + 8, k0 + a_k, kend, fa[1]);
      load_b_x(g, n0 + b_row, k0 + b_k, kend, fb);
    }
  };
  auto stash = [&]() {
    if (MODE != 2) {
      *reinterpret_cast<uint4*>(&As[a_row * SK + a_k]) = make_uint4(ra[0][0], ra[0][1], ra[0][2], ra[0][3]);
      *reinterpret_cast<uint4*>(&As[a_row * SK + a_k + 8]) = make_uint4(ra[1][0], ra[1][1], ra[1][2], ra[1][3]);
      *reinterpret_cast<uint4*>(&Bs[b_row * SK + b_k]) = make_uint4(rb[0], rb[1], rb[2], rb[3]);
    } else {  // k-major: 8 consecutive m (or n) of one pixel k as one 16-byte store
#pragma unroll
      for (int h = 0; h < 2; ++h)
        *reinterpret_cast<uint4*>(&As[a_k * SAT + a_row + 8 * h]) =
            make_uint4(pack_bf16(fa[h][0], fa[h][1]), pack_bf16(fa[h][2], fa[h][3]),
                       pack_bf16(fa[h][4], fa[h][5]), pack_bf16(fa[h][6], fa[h][7]));
      *reinterpret_cast<uint4*>(&Bs[b_k * SBT + b_row]) =
          make_uint4(pack_bf16(fb[0], fb[1]), pack_bf16(fb[2], fb[3]), pack_bf16(fb[4], fb[5]),
                     pack_bf16(fb[6], fb[7]));
    }
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

  if (kbeg < kend) fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    __syncthreads();
    stash();
    __syncthreads();
    if (k0 + BK < kend) fetch(k0 + BK);
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t a[2][4];
      if constexpr (MODE == 2) {
        // matrices (k lo, m lo), (k lo, m hi), (k hi, m lo), (k hi, m hi) = a0..a3
        const int q = lane >> 3, r = lane & 7;
#pragma unroll
        for (int i = 0; i < 2; ++i)
          ldmatrix_x4_trans(a[i], &As[(ks + ((q & 2) ? 8 : 0) + r) * SAT + wm + i * 16 +
                                      ((q & 1) ? 8 : 0)]);
#pragma unroll
        for (int jj = 0; jj < 4; jj += 2) {
          // matrices (k lo, n), (k hi, n), (k lo, n + 8), (k hi, n + 8) = b0, b1 of two blocks
          uint32_t b[4];
          ldmatrix_x4_trans(b, &Bs[(ks + ((q & 1) ? 8 : 0) + r) * SBT + wn + jj * 8 +
                                   ((q & 2) ? 8 : 0)]);
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            mma_bf16(acc[i][jj], a[i], b[0], b[1]);
            mma_bf16(acc[i][jj + 1], a[i], b[2], b[3]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int r0 = wm + i * 16 + gid, c0 = ks + tig * 2;
          a[i][0] = *reinterpret_cast<const uint32_t*>(&As[r0 * SK + c0]);
          a[i][1] = *reinterpret_cast<const uint32_t*>(&As[(r0 + 8) * SK + c0]);
          a[i][2] = *reinterpret_cast<const uint32_t*>(&As[r0 * SK + c0 + 8]);
          a[i][3] = *reinterpret_cast<const uint32_t*>(&As[(r0 + 8) * SK + c0 + 8]);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = wn + j * 8 + gid, c0 = ks + tig * 2;
          const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[n * SK + c0]);
          const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[n * SK + c0 + 8]);
#pragma unroll
          for (int i = 0; i < 2; ++i) mma_bf16(acc[i][j], a[i], b0, b1);
        }
      }
    }
  }

  // epilogue
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + i * 16 + gid + ((q & 2) ? 8 : 0);
        const int n = n0 + wn + j * 8 + tig * 2 + (q & 1);
        if (m >= g.M || n >= g.Nc) continue;
        const float v = acc[i][j][q];
        if (MODE == 0) {
          float o = v + (g.bias ? __ldg(g.bias + n) : 0.0f);
          if (g.relu) o = fmaxf(o, 0.0f);
          const size_t idx = (size_t)m * g.Cout + n;
          g.y[idx] = o;
          if (g.add) g.y2[idx] = o + __ldg(g.add + idx);
        } else if (MODE == 1) {
          g.out[(size_t)m * g.Cin + n] = v;
        } else {
          g.out[((size_t)blockIdx.z * g.M + m) * g.Nc + n] = v;
        }
      }
}

// dst[i] = sum_s partial[s][i] in order s = 0, 1, ...
__global__ void split_reduce_kernel(const float* __restrict__ part, int splits, size_t n,
                                    float* __restrict__ dst) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[(size_t)k * n + i];
    dst[i] = s;
  }
}

// Column sums of a [P][C] matrix: per-block partials over pixel ranges, then a fixed-order
// pass over the blocks.  A block's 256 threads form (lanes = 256 / C) rows of C columns
// (C <= 256; wider matrices loop over column groups): lane l sums pixels p0 + l,
// p0 + l + lanes, ... of its column, and the lanes are added in order in shared memory.
constexpr int kColBlocks = 128;
constexpr int kColThreads = 256;
__global__ void __launch_bounds__(kColThreads)
colsum_partial_kernel(const float* __restrict__ a, int P, int C, float* __restrict__ part) {
  __shared__ float red[kColThreads];
  const int per = (P + gridDim.x - 1) / gridDim.x;
  const int p0 = blockIdx.x * per, p1 = min(P, p0 + per);
  const int cw = C < kColThreads ? C : kColThreads;     // columns per group
  const int lanes = kColThreads / cw;
  const int c_in = threadIdx.x % cw, lane = threadIdx.x / cw;
  for (int c0 = 0; c0 < C; c0 += cw) {
    const int c = c0 + c_in;
    float s = 0.0f;
    if (lane < lanes && c < C)
      for (int p = p0 + lane; p < p1; p += lanes) s += a[(size_t)p * C + c];
    red[threadIdx.x] = s;
    __syncthreads();
    if (lane == 0 && c < C) {
      float t = 0.0f;
      for (int l = 0; l < lanes; ++l) t += red[l * cw + c_in];
      part[(size_t)blockIdx.x * C + c] = t;
    }
    __syncthreads();
  }
}

__global__ void colsum_final_kernel(const float* __restrict__ part, int nb, int C,
                                    float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.0f;
  for (int b = 0; b < nb; ++b) s += part[(size_t)b * C + c];
  out[c] = s;
}

__global__ void transpose_weights_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ w16,
                                         __nv_bfloat16* __restrict__ wt16, int Cin, int Cout) {
  const int n = Cout * 9 * Cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int o = i / (9 * Cin), r = i - o * 9 * Cin, tap = r / Cin, c = r - tap * Cin;
    const __nv_bfloat16 v = __float2bfloat16_rn(w[i]);
    w16[i] = v;
    if (wt16) wt16[((size_t)c * 9 + tap) * Cout + o] = v;
  }
}

// ---------------------------------------------------------------- launchers
static int grid_1d(size_t n, int threads = 256) {
  const size_t b = (n + threads - 1) / threads;
  return (int)(b < 4096 ? (b ? b : 1) : 4096);
}

cudaError_t conv_forward(const float* x, const __nv_bfloat16* w16, const float* bias, float* y,
                         const float* add, float* y2, int N, int H, int W, int Cin, int Cout,
                         int relu, int up, cudaStream_t s) {
  if (conv_tc_applies(W, Cin, Cout))
    return conv_forward_tc(x, w16, bias, y, add, y2, N, H, W, Cin, Cout, relu, up, s);
  GemmArgs g{};
  g.mode = 0;
  g.N = N; g.H = H; g.W = W; g.Cin = Cin; g.Cout = Cout; g.up = up;
  g.M = N * H * W; g.Nc = Cout; g.K = 9 * Cin;
  g.x = x; g.w = w16; g.bias = bias; g.y = y; g.add = add; g.y2 = y2; g.relu = relu;
  dim3 grid((g.M + BM - 1) / BM, (g.Nc + BN - 1) / BN);
  igemm_kernel<0><<<grid, NT, 0, s>>>(g);
  return cudaGetLastError();
}

cudaError_t conv_backward_data(const float* dy, const __nv_bfloat16* wt16, float* dx, int N, int H,
                               int W, int Cin, int Cout, cudaStream_t s) {
  if (conv_tc_applies(W, Cout, Cin))
    return conv_backward_data_tc(dy, wt16, dx, N, H, W, Cin, Cout, s);
  GemmArgs g{};
  g.mode = 1;
  g.N = N; g.H = H; g.W = W; g.Cin = Cin; g.Cout = Cout; g.up = 0;
  g.M = N * H * W; g.Nc = Cin; g.K = 9 * Cout;
  g.dy = dy; g.w = wt16; g.out = dx;
  dim3 grid((g.M + BM - 1) / BM, (g.Nc + BN - 1) / BN);
  igemm_kernel<1><<<grid, NT, 0, s>>>(g);
  return cudaGetLastError();
}

static int weight_splits(int P) {
  const int chunks = (P + BK - 1) / BK;
  int splits = chunks < 256 ? chunks : 256;
  return splits > 0 ? splits : 1;
}

size_t conv_backward_weight_workspace(int N, int H, int W, int Cin, int Cout) {
  const int P = N * H * W;
  const size_t part = (size_t)weight_splits(P) * Cout * 9 * Cin;
  return (part + (size_t)kColBlocks * Cout) * sizeof(float);
}

cudaError_t conv_backward_weight(const float* x, const float* dy, float* dw, float* db, int N,
                                 int H, int W, int Cin, int Cout, int up, float* ws,
                                 size_t ws_bytes, cudaStream_t s) {
  if (ws_bytes < conv_backward_weight_workspace(N, H, W, Cin, Cout)) return cudaErrorInvalidValue;
  GemmArgs g{};
  g.mode = 2;
  g.N = N; g.H = H; g.W = W; g.Cin = Cin; g.Cout = Cout; g.up = up;
  g.M = Cout; g.Nc = 9 * Cin; g.K = N * H * W;
  g.x = x; g.dy = dy; g.out = ws;
  const int splits = weight_splits(g.K);
  const int chunks = (g.K + BK - 1) / BK;
  g.k_split = ((chunks + splits - 1) / splits) * BK;
  const int used = (g.K + g.k_split - 1) / g.k_split;
  dim3 grid((g.Nc + BN - 1) / BN, (g.M + BM - 1) / BM, used);
  igemm_kernel<2><<<grid, NT, 0, s>>>(g);
  const size_t n = (size_t)Cout * 9 * Cin;
  split_reduce_kernel<<<grid_1d(n), 256, 0, s>>>(ws, used, n, dw);
  if (db) {
    float* part = ws + (size_t)weight_splits(g.K) * n;
    colsum_partial_kernel<<<kColBlocks, kColThreads, 0, s>>>(dy, g.K, Cout, part);
    colsum_final_kernel<<<(Cout + 255) / 256, 256, 0, s>>>(part, kColBlocks, Cout, db);
  }
  return cudaGetLastError();
}

cudaError_t transpose_weights(const float* w, __nv_bfloat16* w16, __nv_bfloat16* wt16, int Cin,
                              int Cout, cudaStream_t s) {
  transpose_weights_kernel<<<grid_1d((size_t)Cout * 9 * Cin), 256, 0, s>>>(w, w16, wt16, Cin, Cout);
  return cudaGetLastError();
}

}  // namespace ws
