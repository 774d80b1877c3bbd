// 3x3 convolutions of the warm-start network on the fifth-generation tensor cores
// (tcgen05.mma, kind::f16, bfloat16 operands, float32 accumulators in tensor memory).
//
// A CTA computes a 128-pixel segment of up to kRows (4) consecutive output rows for NT output
// channels:  Y[m][n] = sum_{tap} sum_{c} X[pixel(m) + offset(tap)][c] W[n][tap][c].
// The 3x3 taps read the same input rows at shifted columns, so the input is staged once
// per 16-channel K group as a patch of kRows + 2 rows x 130 pixels (the segment and one
// pixel either side) in the canonical K-major layout without swizzle: for each row and
// each group of 8 channels, 130 pixel slots of 16 bytes (8 bfloat16), consecutive pixels
// 16 bytes apart.  An 8-pixel core matrix is then 128 contiguous bytes, 8-pixel groups are
// 128 bytes apart (the descriptor's M stride) and the two 8-channel halves of a K step are
// one plane apart (its K stride), so the A operand of output row r and tap (ky, kx) is the
// same patch with the descriptor's start moved by r + ky row planes and kx slots: nine
// MMAs per row and K group, no im2col copy.  The weights of the K group are staged once
// for all rows as 9 taps x 2 halves x NT rows of 16 bytes (the B operand, K-major); each
// output row accumulates in its own NT columns of tensor memory.
// Three stage buffers rotate: while the tensor core works on one K group the threads
// stage the next, whose activations were fetched into registers during the group before
// (the weights go to shared memory by 16-byte asynchronous copies); a buffer is refilled
// only after the tcgen05.commit of the MMAs that read it has arrived on its mbarrier.  One thread issues the MMAs; the accumulators (128 lanes
// x NT columns of float32 per row) are read back with tcgen05.ld: warp w reads lanes
// 32 (w mod 4) .. +31 (pixels of the segment) and every other 16-column chunk, starting at
// chunk w / 4, for the bias/ReLU/skip epilogue.
// Every wait is bounded: a wait that gives up sets tc_error and the CTA writes NaN to its
// outputs instead of the accumulators, so a failure cannot pass silently.
//
// Forward:        X = x (read through nearest 2x upsampling when up = 1), W = w16
//                 [Cout][9][Cin], offset(tap) = (ky - 1, kx - 1).
// Backward-data:  X = dy, W = wt16 [Cin][9][Cout], offset(tap) = (1 - ky, 1 - kx).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "cnn.h"

namespace ws {

namespace {

constexpr int kTcM = 128;                 // pixels per CTA (MMA M)
constexpr int kTcSlots = kTcM + 2;        // patch columns x0 - 1 .. x0 + 128
constexpr int kRows = 4;                  // output rows per CTA
constexpr int kTcThreads = 256;
constexpr int kPlane = kTcSlots * 16;     // bytes of one (row, 8-channel half) patch plane
constexpr int kPatchBytes = (kRows + 2) * 2 * kPlane;
constexpr int kHeader = 128;              // mbarriers and the TMEM address
constexpr int kStages = 3;                // stage buffers (K groups in flight)
// Patch items (one pixel slot of one patch row, 16 channels) and weight items (one tap and
// output channel, 16 channels) a thread moves per K group, at most.
constexpr int kPatchItems = ((kRows + 2) * kTcSlots + kTcThreads - 1) / kTcThreads;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

__device__ int tc_error = 0;

struct TcArgs {
  int mode;            // 0 forward, 1 backward-data
  int H, W;            // output (= convolution) resolution
  int CI, CO;          // input channels (K per tap), output channels
  int up;              // forward: input read through nearest 2x upsampling
  int nt;              // output channels per CTA
  int rows;            // output rows per CTA (1..kRows)
  const float* x;      // forward: x [N][H >> up][W >> up][CI]; backward-data: dy [N][H][W][CI]
  const __nv_bfloat16* w;  // [CO][9][CI]
  const float* bias;
  const float* add;
  float* y;
  float* y2;
  int relu;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of tcgen05: start address, leading (K-direction) and
// stride (M/N-direction) byte offsets between 8 x 16-byte core matrices, all in 16-byte
// units; bit 46 set (descriptor version), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t kstride, uint32_t mstride) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kstride >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((mstride >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: float32 accumulator, bfloat16 A and B, both
// K-major, no negation, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the given phase parity of an mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive float32 columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__host__ __device__ constexpr int stage_bytes(int nt) { return kPatchBytes + 9 * 2 * nt * 16; }

// TMEM columns to allocate: a power of two >= 32 holding kRows x nt float32 columns.
__host__ __device__ constexpr int tmem_cols(int nt) {
  return kRows * nt <= 32 ? 32 : kRows * nt <= 64 ? 64 : kRows * nt <= 128 ? 128 : kRows * nt <= 256 ? 256 : 512;
}

__global__ void __launch_bounds__(kTcThreads) tc_conv_kernel(TcArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int segs = (g.W + kTcM - 1) / kTcM;
  const int rblocks = (g.H + g.rows - 1) / g.rows;
  const int seg = blockIdx.x % segs, rb = blockIdx.x / segs;   // rb = img * rblocks + row block
  const int img = rb / rblocks, py0 = (rb - img * rblocks) * g.rows;
  const int nrows = min(g.rows, g.H - py0);
  const int x0 = seg * kTcM;
  const int n0 = blockIdx.y * g.nt;
  const int nt = g.nt;
  const int stages = g.CI / 16;
  const int sbytes = stage_bytes(nt);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 32);
  uint8_t* stage0 = smem + kHeader;
  const uint32_t ncols = (uint32_t)tmem_cols(nt);

  if (tid == 0) {
    for (int b = 0; b < kStages; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bars[b])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc(kTcM, nt);

  const int Hs = g.H >> g.up, Ws = g.W >> g.up;
  const int npatch = (nrows + 2) * kTcSlots;
  // The patch of K group s (float32 activations, converted to bfloat16 on the way into
  // shared memory) is fetched into registers one group ahead: its loads are in flight
  // while the tensor core multiplies the group before.  The weights (already bfloat16)
  // go straight to shared memory with 16-byte asynchronous copies.
  float4 pf[kPatchItems][4];
  auto fetch_patch = [&](int s) {
    const int c0 = s * 16;
#pragma unroll
    for (int k = 0; k < kPatchItems; ++k) {
      const int it = tid + k * kTcThreads;
      const int rr = it / kTcSlots, sl = it - rr * kTcSlots;
      const int yy = py0 + rr - 1, xx = x0 + sl - 1;
      if (it < npatch && yy >= 0 && yy < g.H && xx >= 0 && xx < g.W) {
        const float4* p = reinterpret_cast<const float4*>(
            g.x + (((size_t)img * Hs + (yy >> g.up)) * Ws + (xx >> g.up)) * g.CI + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) pf[k][q] = __ldg(p + q);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) pf[k][q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  bool ok = true;
  int issued = 0;                                    // stages whose MMAs were committed
  if (stages > 0) fetch_patch(0);
  for (int s = 0; s < stages; ++s) {
    const int b = s % kStages;
    uint8_t* st = stage0 + b * sbytes;
    if (s >= kStages) {     // the MMAs that read this buffer (K group s - kStages) are done
      const bool mine = mbar_wait(smem_addr(&bars[b]), (uint32_t)(((s - kStages) / kStages) & 1));
      if (__syncthreads_or(!mine)) { ok = false; break; }
    }
    const int c0 = s * 16;
    // weights: 9 taps x NT rows, 16 channels each -> two 16-byte halves
    uint8_t* wb = st + kPatchBytes;
    for (int it = tid; it < 9 * nt; it += kTcThreads) {
      const int tap = it / nt, n = it - tap * nt;
      const __nv_bfloat16* p = g.w + ((size_t)(n0 + n) * 9 + tap) * g.CI + c0;
      const uint32_t d0 = smem_addr(wb + (tap * 2 + 0) * nt * 16 + n * 16);
      const uint32_t d1 = smem_addr(wb + (tap * 2 + 1) * nt * 16 + n * 16);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d0), "l"(p) : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d1), "l"(p + 8) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    // patch: nrows + 2 rows x 130 slots, 16 channels each -> two 16-byte halves
#pragma unroll
    for (int k = 0; k < kPatchItems; ++k) {
      const int it = tid + k * kTcThreads;
      if (it < npatch) {
        const int rr = it / kTcSlots, sl = it - rr * kTcSlots;
        const float4 a0 = pf[k][0], a1 = pf[k][1], a2 = pf[k][2], a3 = pf[k][3];
        const uint4 lo = make_uint4(pack2(a0.x, a0.y), pack2(a0.z, a0.w), pack2(a1.x, a1.y), pack2(a1.z, a1.w));
        const uint4 hi = make_uint4(pack2(a2.x, a2.y), pack2(a2.z, a2.w), pack2(a3.x, a3.y), pack2(a3.z, a3.w));
        *reinterpret_cast<uint4*>(st + (rr * 2 + 0) * kPlane + sl * 16) = lo;
        *reinterpret_cast<uint4*>(st + (rr * 2 + 1) * kPlane + sl * 16) = hi;
      }
    }
    if (s + 1 < stages) fetch_patch(s + 1);          // in flight during this group's MMAs
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    // make the generic-proxy stores and copies visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after_sync();
      const uint32_t pa = smem_addr(st), pw = smem_addr(wb);
#pragma unroll 1
      for (int r = 0; r < nrows; ++r) {
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
          const int ky = tap / 3, kx = tap - 3 * ky;
          const int rr = r + (g.mode == 0 ? ky : 2 - ky);
          const int sx = g.mode == 0 ? kx : 2 - kx;
          const uint64_t ad = smem_desc(pa + rr * 2 * kPlane + sx * 16, kPlane, 128);
          const uint64_t bd = smem_desc(pw + tap * 2 * nt * 16, nt * 16, 128);
          mma_f16(tmem + (uint32_t)(r * nt), ad, bd, idesc, (s > 0 || tap > 0) ? 1u : 0u);
        }
      }
      mma_commit(smem_addr(&bars[b]));
    }
    ++issued;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (ok && issued > 0) {
    const int s = issued - 1;
    const bool mine = mbar_wait(smem_addr(&bars[s % kStages]), (uint32_t)((s / kStages) & 1));
    if (__syncthreads_or(!mine)) ok = false;
  }
  fence_after_sync();

  // epilogue: thread = pixel x0 + 32 (warp mod 4) + lane, 16 accumulator columns at a time
  const int quarter = warp & 3, half = warp >> 2;
  const int px = x0 + quarter * 32 + (tid & 31);
  const bool valid = px < g.W;
  if (ok) {
    for (int r = 0; r < nrows; ++r) {
      const size_t pix = ((size_t)img * g.H + py0 + r) * g.W + px;
      for (int c = half * 16; c < nt; c += 32) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(r * nt + c), v);
        if (!valid) continue;
        float o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float a = __uint_as_float(v[i]);
          if (g.mode == 0) {
            if (g.bias) a += __ldg(g.bias + n0 + c + i);
            if (g.relu) a = fmaxf(a, 0.0f);
          }
          o[i] = a;
        }
        float* yo = g.y + pix * g.CO + n0 + c;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          reinterpret_cast<float4*>(yo)[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        if (g.mode == 0 && g.add) {
          const float4* ad = reinterpret_cast<const float4*>(g.add + pix * g.CO + n0 + c);
          float4* y2 = reinterpret_cast<float4*>(g.y2 + pix * g.CO + n0 + c);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 a = __ldg(ad + q);
            y2[q] = make_float4(o[4 * q] + a.x, o[4 * q + 1] + a.y, o[4 * q + 2] + a.z, o[4 * q + 3] + a.w);
          }
        }
      }
    }
  } else {
    if (tid == 0) atomicExch(&tc_error, 1);
    if (valid && half == 0) {
      for (int r = 0; r < nrows; ++r) {
        const size_t pix = ((size_t)img * g.H + py0 + r) * g.W + px;
        for (int c = 0; c < nt; ++c) {
          g.y[pix * g.CO + n0 + c] = __int_as_float(0x7fc00000);
          if (g.mode == 0 && g.add) g.y2[pix * g.CO + n0 + c] = __int_as_float(0x7fc00000);
        }
      }
    }
    // MMAs may still be in flight: give the last commit one more bounded wait before the
    // accumulators' columns are released.
    if (issued > 0) {
      const int s = issued - 1;
      mbar_wait(smem_addr(&bars[s % kStages]), (uint32_t)((s / kStages) & 1));
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
}

// Output channels per CTA for CO output channels, or 0 when the tensor-core kernel does
// not apply (CO must be a multiple of 16; wider layers are split into 128-channel tiles).
int tc_tile_n(int co) {
  if (co % 16 != 0) return 0;
  if (co <= 128) return co;
  return co % 128 == 0 ? 128 : 0;
}

// Shared memory of a CTA: header and min(kStages, K groups) stage buffers.  Every address a descriptor of a
// stage reaches (the start, 15 M-stride steps and one K-stride step) lies inside that
// stage: the last row's last tap ends exactly at the end of the patch, the last tap's
// weights at the end of the stage.
size_t tc_smem_bytes(int nt, int kgroups) {
  const int nbuf = kgroups < kStages ? (kgroups > 0 ? kgroups : 1) : kStages;
  return (size_t)kHeader + nbuf * (size_t)stage_bytes(nt);
}

cudaError_t launch_tc(TcArgs g, int N, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(g.nt, g.CI / 16);   // layers with fewer K groups than
                                                         // kStages use fewer buffers
  static size_t configured = 0;       // dynamic shared memory the kernel is opted into
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(tc_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  // kRows output rows per CTA: each staged weight group serves kRows x 9 MMAs.  (Fewer
  // rows on small grids, for more CTAs, measured slower: 2.70 against 2.36 ms for the
  // network at 1024 x 1024, where the deep layers' weight staging dominates.)
  const long long segs = (g.W + kTcM - 1) / kTcM;
  g.rows = kRows;
  const long long blocks = segs * N * ((g.H + g.rows - 1) / g.rows);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)blocks, g.CO / g.nt);
  tc_conv_kernel<<<grid, kTcThreads, smem, s>>>(g);
  return cudaGetLastError();
}

}  // namespace

bool conv_tc_applies(int W, int ci, int co) {
  return W >= kTcM && ci % 16 == 0 && ci >= 16 && tc_tile_n(co) > 0;
}

cudaError_t conv_forward_tc(const float* x, const __nv_bfloat16* w16, const float* bias, float* y,
                            const float* add, float* y2, int N, int H, int W, int Cin, int Cout,
                            int relu, int up, cudaStream_t s) {
  TcArgs g{};
  g.mode = 0;
  g.H = H; g.W = W; g.CI = Cin; g.CO = Cout; g.up = up; g.nt = tc_tile_n(Cout);
  g.x = x; g.w = w16; g.bias = bias; g.add = add; g.y = y; g.y2 = y2; g.relu = relu;
  return launch_tc(g, N, s);
}

cudaError_t conv_backward_data_tc(const float* dy, const __nv_bfloat16* wt16, float* dx, int N,
                                  int H, int W, int Cin, int Cout, cudaStream_t s) {
  TcArgs g{};
  g.mode = 1;
  g.H = H; g.W = W; g.CI = Cout; g.CO = Cin; g.up = 0; g.nt = tc_tile_n(Cin);
  g.x = dy; g.w = wt16; g.y = dx;
  return launch_tc(g, N, s);
}

int conv_tc_take_error() {
  int h = 0;
  if (cudaMemcpyFromSymbol(&h, tc_error, sizeof(int)) != cudaSuccess) return -1;
  if (h) {
    const int zero = 0;
    cudaMemcpyToSymbol(tc_error, &zero, sizeof(int));
  }
  return h;
}

}  // namespace ws
