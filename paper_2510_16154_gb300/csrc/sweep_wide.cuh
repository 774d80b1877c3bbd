// Agent sweep kernels for wide channel counts (hyperspectral images, C = 31): one pixel
// per thread on 32-pixel-wide tiles, every tile cell (tile pixel or halo pixel) staged in
// shared memory as one record holding all its channels (and, for the adjoint, the adjoint
// state after them), then the validity flag, padded to a stride that keeps vector loads of
// consecutive cells conflict-free.  A neighbour's record is read with 8-byte (forward) or
// 16-byte (adjoint) loads and the channel loop is unrolled in registers.  The window rows
// stream through a ring of TH + 1 tile rows in shared memory (wide_stream): the copies of
// the row the next window-row step adds (cp.async from flat, coalesced NHWC row segments)
// overlap the current step's arithmetic, and the ring is small enough for two blocks per
// SM where the whole tile with its halo allowed one.  Results are staged back through
// shared memory and stored as flat rows.  Tile height: see wide_by.
#pragma once

#include "sweep.cuh"

namespace agents {

constexpr int kWideBX = 32, kWideBY = 4;
constexpr int kWideC = 31;          // the channel count with a wide instantiation

// R <= 7 (the ring of an R = 8 tile would still fit; R = 8 is left to the generic kernel).
inline bool wide_shape(int R, int C) { return R >= 1 && R <= 7 && C == kWideC; }

// Tile height: 4 rows (128 threads).  The adjoint holds about 200 registers per thread
// (a pixel's 31 values, 31 adjoints and 31 sums, and a neighbour's record), so two blocks
// of 128 threads fit an SM's registers where one of 256 did; the row ring keeps both
// blocks' shared memory (57 KB each at R = 5) in the SM's 228 KB.
template <int R>
constexpr int wide_by() { return kWideBY; }
inline int wide_tile_h(int) { return kWideBY; }

// Record stride (floats) of a cell holding `raw` values: forward records are read with
// 8-byte loads (stride/2 odd: 16 consecutive cells hit distinct banks), adjoint records
// with 16-byte loads (stride/4 odd: 8 consecutive cells hit distinct banks).
constexpr int wide_rec2(int raw) { return ((raw + 1) / 2) % 2 ? ((raw + 1) / 2) * 2 : ((raw + 1) / 2 + 1) * 2; }
constexpr int wide_rec4(int raw) { return ((raw + 3) / 4) % 2 ? ((raw + 3) / 4) * 4 : ((raw + 3) / 4 + 1) * 4; }

template <int R, int C>
struct Wide {
  static constexpr int TW = kWideBX, TH = wide_by<R>(), NT = kWideBX * wide_by<R>();
  static constexpr int SW = TW + 2 * R, SH = TH + 2 * R, CELLS = SW * SH;
  // Channels padded to an even count CP (pad slots hold 0), so that channel pairs are
  // aligned float2 operands of the packed FFMA2 / FADD2 arithmetic.
  static constexpr int CP = (C + 1) & ~1;
  static constexpr int REC1 = wide_rec2(CP + 1);      // forward: CP values, flag
  static constexpr int REC2 = wide_rec4(2 * CP + 1);  // adjoint: CP values, CP adjoints, flag
  // The window rows stream through a ring of NR = TH + 1 tile rows (see wide_ring_row):
  // the rows one window-row step needs plus the one being fetched for the next step.
  static constexpr int NR = TH + 1;
  static constexpr size_t smem(int nf) {
    const size_t ring = (size_t)NR * SW * (nf == 1 ? REC1 : REC2) * sizeof(float);
    const size_t stage = (size_t)TW * TH * C * sizeof(float);   // wide_store
    return ring > stage ? ring : stage;
  }
};

// 4-byte asynchronous copy global -> shared: a thread issues all its copies of a tile
// without waiting on each load; a row's copies are committed as one group.
__device__ __forceinline__ void wide_cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}

// The tile's window rows are streamed: row i (0 <= i < TH + 2R, image row y0 - R + i) of
// the tile plus its halo is staged into ring slot i % NR as cell records -- values of
// field f, channel ch at slot f * CP + ch, the validity flag at slot NF * CP -- with
// asynchronous copies from the flat, coalesced NHWC row segment.  Cells outside the image
// hold 0; the flag is written only for tiles whose halo leaves the image (interior tiles
// never read it).  The caller commits the copies as one group per row.
template <class T, int R, int C, int NF>
__device__ __forceinline__ void wide_ring_row(float* __restrict__ ring,
                                              const float* __restrict__ f0,
                                              const float* __restrict__ f1, const SweepGeom& g,
                                              int x0, int y0, int i, bool border) {
  constexpr int REC = NF == 1 ? T::REC1 : T::REC2;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int gx0 = x0 - R;
  const int xa = max(0, -gx0), xb = min(T::SW, g.W - gx0);   // valid columns [xa, xb)
  const int gy = y0 - R + i;
  const bool rowok = gy >= 0 && gy < g.H;
  float* slot = ring + (size_t)(i % T::NR) * T::SW * REC;
  const int nval = (rowok && xb > xa) ? (xb - xa) * C : 0;
  const size_t base = rowok ? ((size_t)gy * g.W + (gx0 + xa)) * C : 0;
  float* row = slot + (size_t)xa * REC;
  for (int f = tid; f < nval; f += T::NT) {
    const int px = f / C, ch = f - px * C;
    wide_cp_async4(row + px * REC + ch, f0 + base + f);
    if constexpr (NF == 2) wide_cp_async4(row + px * REC + T::CP + ch, f1 + base + f);
  }
  for (int xx = tid; xx < T::SW; xx += T::NT) {
    float* cell = slot + (size_t)xx * REC;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int ch = C; ch < T::CP; ++ch) cell[f * T::CP + ch] = 0.0f;   // pad channels
    if (border) {
      const bool ok = rowok && xx >= xa && xx < xb;
      if (!ok) {
#pragma unroll 4
        for (int k = 0; k < NF * T::CP; ++k) cell[k] = 0.0f;
      }
      cell[NF * T::CP] = ok ? 1.0f : 0.0f;
    }
  }
}

__device__ __forceinline__ void wide_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// All committed groups but the most recent one have landed (this thread's copies).
__device__ __forceinline__ void wide_wait_prev() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

template <class T, int R>
__device__ __forceinline__ bool wide_border(const SweepGeom& g, int x0, int y0) {
  return (x0 - R < 0) || (y0 - R < 0) || (x0 + T::TW + R > g.W) || (y0 + T::TH + R > g.H);
}

// Drive the window-row loop of one tile: rows 0 .. TH-1 are fetched up front; before the
// step of window row dy the row the next step adds is fetched, so its copies overlap this
// step's arithmetic; step(dy, slot) then runs with every row it reads in the ring (slot:
// ring row of this thread's window row).  Barriers keep a slot from being refilled while
// a thread still reads it.
template <class T, int R, int C, int NF, class Step>
__device__ __forceinline__ void wide_stream(float* __restrict__ ring, const float* __restrict__ f0,
                                            const float* __restrict__ f1, const SweepGeom& g,
                                            int x0, int y0, bool border, Step&& step) {
  constexpr int NROWS = T::TH + 2 * R;
  for (int i = 0; i < T::TH; ++i) wide_ring_row<T, R, C, NF>(ring, f0, f1, g, x0, y0, i, border);
  wide_commit();
#pragma unroll 1
  for (int dy = -R; dy <= R; ++dy) {
    const int inext = dy + R + T::TH;                  // the row step dy + 1 adds
    if (inext < NROWS) wide_ring_row<T, R, C, NF>(ring, f0, f1, g, x0, y0, inext, border);
    wide_commit();                                     // (possibly empty) group per step
    wide_wait_prev();
    __syncthreads();
    step(dy, (dy + R + (int)threadIdx.y) % T::NR);
    __syncthreads();
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Write the tile's results (val[C] per thread) to out (NHWC) through shared memory, so
// that every tile row is stored as one flat segment.  `stage` needs TW*TH*C floats.
template <class T, int C>
__device__ __forceinline__ void wide_store(float* __restrict__ stage, const float (&val)[C],
                                           float* __restrict__ out, const SweepGeom& g, int x0,
                                           int y0) {
  __syncthreads();                                   // the tile data is no longer needed
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int ch = 0; ch < C; ++ch) stage[(ty * T::TW + tx) * C + ch] = val[ch];
  __syncthreads();
  const int tid = ty * blockDim.x + tx;
  const int ncol = min(T::TW, g.W - x0);
  for (int r = 0; r < T::TH; ++r) {
    const int gy = y0 + r;
    if (gy >= g.H) break;
    float* dst = out + ((size_t)gy * g.W + x0) * C;
    const float* src = stage + r * T::TW * C;
    for (int f = tid; f < ncol * C; f += T::NT) dst[f] = src[f];
  }
}

// The thread's own pixel: its C values of field f (0 outside the image, like the zero-filled
// records), and whether it lies in the image.
template <int C>
__device__ __forceinline__ bool wide_own(const float* __restrict__ f, const SweepGeom& g, int x0,
                                         int y0, float (&val)[C]) {
  const int gx = x0 + threadIdx.x, gy = y0 + threadIdx.y;
  const bool in = gx < g.W && gy < g.H;
  const float* src = f + ((size_t)(in ? gy : 0) * g.W + (in ? gx : 0)) * C;
#pragma unroll
  for (int ch = 0; ch < C; ++ch) val[ch] = in ? __ldg(src + ch) : 0.0f;
  return in;
}

// Forward step of the pixel at (x0 + tx, y0 + ty): c + dt/M sum_j phi(r_kj) (c_j - c_k),
// the window rows streamed through the ring (wide_stream).
template <class T, int R, int C, bool BORDER>
__device__ __forceinline__ void wide_forward_tile(float* __restrict__ sm, const float* __restrict__ src,
                                                  float* __restrict__ out, const SweepGeom& g,
                                                  float kx, float ky, float kc, int x0, int y0) {
  constexpr int REC = T::REC1, NP = T::CP / 2;   // channel pairs
  float ci[C];
  wide_own<C>(src, g, x0, y0, ci);
  float2 nci[NP], acc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    nci[q] = make_float2(-ci[2 * q], 2 * q + 1 < C ? -ci[2 * q + 1] : 0.0f);
    acc[q] = f2(0.0f);
  }
  wide_stream<T, R, C, 1>(sm, src, nullptr, g, x0, y0, BORDER, [&](int dy, int slot) {
    const float sy = fmaf(-ky, (float)(dy * dy), 1.0f);
    const int base = slot * T::SW + threadIdx.x + R;
#pragma unroll 1
    for (int dx = -R; dx <= R; ++dx) {
      const float2* rec = reinterpret_cast<const float2*>(sm + (base + dx) * REC);
      float2 d[NP];
      float2 s2a = f2(0.0f), s2b = f2(0.0f);     // four independent lanes of |d|^2
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        d[q] = __fadd2_rn(rec[q], nci[q]);
        if (q & 1) s2b = __ffma2_rn(d[q], d[q], s2b);
        else s2a = __ffma2_rn(d[q], d[q], s2a);
      }
      const float s2 = (s2a.x + s2b.x) + (s2a.y + s2b.y);
      const float t = fmaxf(fmaf(-kc, s2, fmaf(-kx, (float)(dx * dx), sy)), 0.0f);
      const float t2 = t * t;
      float ph = (t2 * t2) * fmaf(-4.0f, t, 5.0f);
      if constexpr (BORDER) ph *= rec[NP].x;            // validity flag
      const float2 ph2 = f2(ph);
#pragma unroll
      for (int q = 0; q < NP; ++q) acc[q] = __ffma2_rn(ph2, d[q], acc[q]);
    }
  });
  float val[C];
#pragma unroll
  for (int ch = 0; ch < C; ++ch)
    val[ch] = fmaf(g.scale, (ch & 1) ? acc[ch / 2].y : acc[ch / 2].x, ci[ch]);
  wide_store<T, C>(sm, val, out, g, x0, y0);
}

// Adjoint step (gather form, as adjoint_body): lam_k + dt/M sum_j [phi' eps_c delta
// (delta . dlam) + phi dlam]; the block's D partial sums go to partial[0..1].
template <class T, int R, int C, bool BORDER>
__device__ __forceinline__ void wide_adjoint_tile(float* __restrict__ sm, const float* __restrict__ c,
                                                  const float* __restrict__ lam,
                                                  float* __restrict__ out,
                                                  double* __restrict__ partial, const SweepGeom& g,
                                                  float kx, float ky, float kc, float ec, int x0,
                                                  int y0) {
  constexpr int REC = T::REC2, NP = T::CP / 2;
  float ck[C], lk[C];
  const bool own = wide_own<C>(c, g, x0, y0, ck);
  wide_own<C>(lam, g, x0, y0, lk);
  float2 nck[NP], nlk[NP], acc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const bool two = 2 * q + 1 < C;
    nck[q] = make_float2(-ck[2 * q], two ? -ck[2 * q + 1] : 0.0f);
    nlk[q] = make_float2(-lk[2 * q], two ? -lk[2 * q + 1] : 0.0f);
    acc[q] = f2(0.0f);
  }
  const float ec20 = 20.0f * ec;
  float Dx = 0.0f, Dc = 0.0f;
  wide_stream<T, R, C, 2>(sm, c, lam, g, x0, y0, BORDER, [&](int dy, int slot) {
    const float sy = fmaf(-ky, (float)(dy * dy), 1.0f);
    const float d2y = g.inv_h2 * (float)(dy * dy);
    const int base = slot * T::SW + threadIdx.x + R;
#pragma unroll 1
    for (int dx = -R; dx <= R; ++dx) {
      const float* rec = sm + (base + dx) * REC;
      const float4* r4 = reinterpret_cast<const float4*>(rec);
      float2 d[NP], dl[NP];
      float2 s2a = f2(0.0f), s2b = f2(0.0f), pa = f2(0.0f), pb = f2(0.0f);
#pragma unroll
      for (int q = 0; q < NP / 2; ++q) {              // two channel pairs per 16-byte load
        const float4 a = r4[q], b = r4[NP / 2 + q];
        d[2 * q] = __fadd2_rn(make_float2(a.x, a.y), nck[2 * q]);
        d[2 * q + 1] = __fadd2_rn(make_float2(a.z, a.w), nck[2 * q + 1]);
        dl[2 * q] = __fadd2_rn(make_float2(b.x, b.y), nlk[2 * q]);
        dl[2 * q + 1] = __fadd2_rn(make_float2(b.z, b.w), nlk[2 * q + 1]);
        s2a = __ffma2_rn(d[2 * q], d[2 * q], s2a);
        s2b = __ffma2_rn(d[2 * q + 1], d[2 * q + 1], s2b);
        pa = __ffma2_rn(d[2 * q], dl[2 * q], pa);
        pb = __ffma2_rn(d[2 * q + 1], dl[2 * q + 1], pb);
      }
      const float s2 = (s2a.x + s2b.x) + (s2a.y + s2b.y);
      const float proj = (pa.x + pb.x) + (pa.y + pb.y);
      const float t = fmaxf(fmaf(-kc, s2, fmaf(-kx, (float)(dx * dx), sy)), 0.0f);
      const float t2 = t * t, t3 = t2 * t;
      float ph = (t2 * t2) * fmaf(-4.0f, t, 5.0f);
      float dph = t3 * (t - 1.0f);                       // phi' / 20
      if constexpr (BORDER) {
        const float m = rec[2 * T::CP];                  // validity flag
        ph *= m;
        dph *= m;
      }
      const float gk = dph * proj;        // D in the paired form of adjoint_body
      const float2 coef = f2(gk * ec20), ph2 = f2(ph);
#pragma unroll
      for (int q = 0; q < NP; ++q)
        acc[q] = __ffma2_rn(ph2, dl[q], __ffma2_rn(coef, d[q], acc[q]));
      Dx = fmaf(gk, fmaf(g.inv_w2, (float)(dx * dx), d2y), Dx);
      Dc = fmaf(gk, s2, Dc);
    }
  });
  if constexpr (BORDER) {
    // a pixel outside the image has zero-filled lam_k, so its paired D terms
    // (delta . lam_j) are not zero by themselves: drop them
    if (!own) Dx = Dc = 0.0f;
  }
  __shared__ double red[2 * 32];
  double vv[2] = {-10.0 * (double)Dx, -10.0 * (double)Dc};
  double tot[2];
  block_sum<2>(vv, red, tot);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    partial[0] = tot[0];
    partial[1] = tot[1];
  }
  float val[C];
#pragma unroll
  for (int ch = 0; ch < C; ++ch)
    val[ch] = fmaf(g.scale, (ch & 1) ? acc[ch / 2].y : acc[ch / 2].x, lk[ch]);
  wide_store<T, C>(sm, val, out, g, x0, y0);
}

template <int R, int C>
__global__ void __launch_bounds__(kWideBX * wide_by<R>())
wide_forward_kernel(const float* __restrict__ c, float* __restrict__ out,
                    const double* __restrict__ eps_n, SweepGeom g) {
  using T = Wide<R, C>;
  extern __shared__ __align__(16) float wsm[];
  const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
  if (wide_border<T, R>(g, x0, y0))
    wide_forward_tile<T, R, C, true>(wsm, c, out, g, kx, ky, kc, x0, y0);
  else
    wide_forward_tile<T, R, C, false>(wsm, c, out, g, kx, ky, kc, x0, y0);
}

template <int R, int C>
__global__ void __launch_bounds__(kWideBX * wide_by<R>())
wide_adjoint_kernel(const float* __restrict__ c, const float* __restrict__ lam,
                    float* __restrict__ out, const double* __restrict__ eps_n,
                    double* __restrict__ partial, SweepGeom g) {
  using T = Wide<R, C>;
  extern __shared__ __align__(16) float wsm[];
  const int x0 = blockIdx.x * T::TW, y0 = blockIdx.y * T::TH;
  const float ex = (float)eps_n[0], ec = (float)eps_n[1];
  const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
  double* part = partial + 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
  if (wide_border<T, R>(g, x0, y0))
    wide_adjoint_tile<T, R, C, true>(wsm, c, lam, out, part, g, kx, ky, kc, ec, x0, y0);
  else
    wide_adjoint_tile<T, R, C, false>(wsm, c, lam, out, part, g, kx, ky, kc, ec, x0, y0);
}

// Batched (persistent) versions: step n of every (image, tile) job of the batch.
template <int R, int C>
__global__ void __launch_bounds__(kWideBX * wide_by<R>())
wide_forward_batch_kernel(const BatchSweepImg* __restrict__ imgs, const BatchJob* __restrict__ jobs,
                          int njobs, const int* __restrict__ active, int n, int kind) {
  using T = Wide<R, C>;
  extern __shared__ __align__(16) float wsm[];
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchSweepImg& im = imgs[job.img];
    const SweepGeom g = im.g;
    const size_t nc = (size_t)g.H * g.W * C;
    const float* src;
    float* dst;
    const double* eps_n;
    if (kind == kSweepStore) {
      src = batch_state(im, n);
      dst = n == im.nsteps - 1 ? im.cT : im.traj + (size_t)n * nc;
      eps_n = im.eps + 2 * n;
    } else {
      src = n == 0 ? im.c0 : ((n - 1) & 1 ? im.work1 : im.work0);
      dst = n == im.nsteps - 1 ? im.trial_c : (n & 1 ? im.work1 : im.work0);
      eps_n = im.trial_eps + 2 * n;
    }
    const int x0 = job.tx * T::TW, y0 = job.ty * T::TH;
    const float ex = (float)eps_n[0], ec = (float)eps_n[1];
    const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
    if (wide_border<T, R>(g, x0, y0))
      wide_forward_tile<T, R, C, true>(wsm, src, dst, g, kx, ky, kc, x0, y0);
    else
      wide_forward_tile<T, R, C, false>(wsm, src, dst, g, kx, ky, kc, x0, y0);
    __syncthreads();
  }
}

template <int R, int C>
__global__ void __launch_bounds__(kWideBX * wide_by<R>())
wide_adjoint_batch_kernel(const BatchSweepImg* __restrict__ imgs, const BatchJob* __restrict__ jobs,
                          int njobs, const int* __restrict__ active, int n) {
  using T = Wide<R, C>;
  extern __shared__ __align__(16) float wsm[];
  for (int j = blockIdx.x; j < njobs; j += gridDim.x) {
    const BatchJob job = jobs[j];
    if (!active[job.img]) continue;
    const BatchSweepImg& im = imgs[job.img];
    const SweepGeom g = im.g;
    const int li = (im.nsteps - 1 - n) & 1;
    const float* lin = li ? im.lam1 : im.lam0;
    float* lout = li ? im.lam0 : im.lam1;
    const double* eps_n = im.eps + 2 * n;
    const int x0 = job.tx * T::TW, y0 = job.ty * T::TH;
    const float ex = (float)eps_n[0], ec = (float)eps_n[1];
    const float kx = 0.5f * ex * g.inv_w2, ky = 0.5f * ex * g.inv_h2, kc = 0.5f * ec;
    const int tiles_x = (g.W + T::TW - 1) / T::TW;
    double* part = im.part_adj + ((size_t)n * im.ntiles + (size_t)job.ty * tiles_x + job.tx) * 2;
    const float* cn = batch_state(im, n);
    if (wide_border<T, R>(g, x0, y0))
      wide_adjoint_tile<T, R, C, true>(wsm, cn, lin, lout, part, g, kx, ky, kc, ec, x0, y0);
    else
      wide_adjoint_tile<T, R, C, false>(wsm, cn, lin, lout, part, g, kx, ky, kc, ec, x0, y0);
    __syncthreads();
  }
}

// Launchers (sweep_wide.cu).
cudaError_t launch_wide_forward(const float* c_in, float* c_out, const double* eps_n,
                                const SweepGeom& g, cudaStream_t s);
cudaError_t launch_wide_adjoint(const float* c_n, const float* lam_next, float* lam_out,
                                const double* eps_n, double* partial, const SweepGeom& g,
                                cudaStream_t s);
cudaError_t launch_wide_forward_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                      const int* active, int n, int kind, int R, cudaStream_t s);
cudaError_t launch_wide_adjoint_batch(const BatchSweepImg* imgs, const BatchJob* jobs, int njobs,
                                      const int* active, int n, int R, cudaStream_t s);

}  // namespace agents
