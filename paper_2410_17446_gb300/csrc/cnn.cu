// Learned GMRES initial guess: a stack of 3x3 circular convolutions on the
// transverse grid (include/prop_cnn.h).  The paper has no learned part; the
// network only supplies x0, and GMRES still converges to the same tolerance.
//
// Layout: activations NHWC bfloat16 with 16 or 32 channels; weights
// bfloat16 [9 taps][Cout][Cin] (tap t = 3 (dy+1) + (dx+1)); biases float32.
//
// Forward (and the data gradient, with flipped taps and swapped channel
// roles) is an implicit GEMM on the BF16 tensor cores: one warp owns 16
// consecutive pixels of an image row and all Cout channels; each k-step is 16
// input channels of one tap, gathered with circular wrap, and
// mma.sync.m16n8k16 accumulates in float32.  The weight gradient is a
// reduction over pixels done in float32 on the CUDA cores, per CTA, followed by
// a deterministic sum over CTAs.
#include "../../include/prop_cnn.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "tc.cuh"
#include "tma.cuh"

namespace {

// Set by a tensor-core convolution whose bounded wait for its MMAs gave up
// (read and cleared by prop_cnn_check).
__device__ int g_cnn_err;

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// y[n, y, x, co] = b[co] + sum_{t, ci} W[t, co, ci] a[n, y+dy_t, x+dx_t, ci]  (circular)
// MODE 0: store relu(y) as bf16; 1: store y as bf16; 2: store y as float32.
// active (optional): sample n is skipped when active[n * astride] != want.
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(128) k_conv(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ w,
                                              const float* __restrict__ bias, void* out, int H, int W,
                                              const int* active, int astride, int want) {
  __shared__ __align__(16) __nv_bfloat16 sw[9 * COUT * CIN];
  const int n = blockIdx.z;
  if (active && active[(long)n * astride] != want) return;
  for (int i = threadIdx.x; i < 9 * COUT * CIN / 2; i += blockDim.x)
    reinterpret_cast<uint32_t*>(sw)[i] = reinterpret_cast<const uint32_t*>(w)[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int y = blockIdx.y;
  const int x0 = (blockIdx.x * 4 + warp) * 16;
  if (x0 >= W) return;
  const __nv_bfloat16* img = in + (long)n * H * W * CIN;
  float acc[COUT / 8][4];
#pragma unroll
  for (int j = 0; j < COUT / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int dy = t / 3 - 1, dx = t % 3 - 1;
    const int yy = wrap(y + dy, H);
    const __nv_bfloat16* r0 = img + ((long)yy * W + wrap(x0 + g + dx, W)) * CIN;
    const __nv_bfloat16* r1 = img + ((long)yy * W + wrap(x0 + g + 8 + dx, W)) * CIN;
#pragma unroll
    for (int cb = 0; cb < CIN / 16; ++cb) {
      const int c = cb * 16 + tq * 2;
      const uint32_t a0 = ld_u32(r0 + c), a1 = ld_u32(r1 + c), a2 = ld_u32(r0 + c + 8), a3 = ld_u32(r1 + c + 8);
#pragma unroll
      for (int j = 0; j < COUT / 8; ++j) {
        const __nv_bfloat16* wb = sw + ((t * COUT) + j * 8 + g) * CIN + c;
        mma_bf16(acc[j], a0, a1, a2, a3, ld_u32(wb), ld_u32(wb + 8));
      }
    }
  }
#pragma unroll
  for (int j = 0; j < COUT / 8; ++j) {
    const int co = j * 8 + tq * 2;
    const float b0 = bias ? bias[co] : 0.f, b1 = bias ? bias[co + 1] : 0.f;
    float v[4] = {acc[j][0] + b0, acc[j][1] + b1, acc[j][2] + b0, acc[j][3] + b1};
    if (MODE == 0)
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = fmaxf(v[q], 0.f);
    const long p0 = ((long)n * H + y) * W + x0 + g, p1 = p0 + 8;
    if (MODE == 2) {
      float* o = reinterpret_cast<float*>(out);
      o[p0 * COUT + co] = v[0]; o[p0 * COUT + co + 1] = v[1];
      o[p1 * COUT + co] = v[2]; o[p1 * COUT + co + 1] = v[3];
    } else {
      __nv_bfloat162* o0 = reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(out) + p0 * COUT + co);
      __nv_bfloat162* o1 = reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(out) + p1 * COUT + co);
      *o0 = __floats2bfloat162_rn(v[0], v[1]);
      *o1 = __floats2bfloat162_rn(v[2], v[3]);
    }
  }
}

// The same convolution on the 5th-generation tensor cores (tcgen05).  A CTA of
// 128 threads takes 128 consecutive pixels of one sample (MMA M = 128) and all
// COUT channels (N = COUT); K runs over the 9 taps x CIN channels, 16 per MMA.
// Shared memory holds, as K-major core matrices (8 rows x 16 bytes):
//   A: 9 x CIN/8 planes of 128 pixels x 8 channels (2 KiB each), gathered with
//      the circular wrap of each tap;  B: 9 x CIN/8 planes of COUT x 8 channels.
// One thread issues the 9 CIN/16 MMAs into a 128 x COUT FP32 accumulator in
// tensor memory and commits them to an mbarrier; warp w then reads lanes
// 32 w .. 32 w + 31 (its pixels) for the bias / ReLU / store epilogue.
template <int CIN, int COUT>
constexpr size_t conv_tc_smem() { return (size_t)9 * (CIN / 8) * (128 + COUT) * 16; }

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(128) k_conv_tc(const __nv_bfloat16* __restrict__ in,
                                                 const __nv_bfloat16* __restrict__ w,
                                                 const float* __restrict__ bias, void* out, int H, int W,
                                                 const int* active, int astride, int want) {
  constexpr int NPL = CIN / 8;                  // 16-byte channel planes
  constexpr uint32_t A_PLANE = 128 * 16, B_PLANE = COUT * 16;
  extern __shared__ __align__(128) unsigned char smem_tc[];
  unsigned char* sa = smem_tc;
  unsigned char* sb = smem_tc + 9 * NPL * A_PLANE;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int n = blockIdx.y;
  if (active && active[(long)n * astride] != want) return;
  if (*reinterpret_cast<volatile const int*>(&g_cnn_err) != 0) return;   // an earlier wait gave up
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long npix = (long)H * W, p0 = (long)blockIdx.x * 128;
  const __nv_bfloat16* img = in + (long)n * npix * CIN;
  if (warp == 0) prop_tc::tmem_alloc(&tmem_base, 32);
  if (tid == 0) { prop_dev::mbar_init(&bar, 1); prop_dev::fence_mbar_init(); }
  // weights: plane (t, c8), row co = w[t][co][8 c8 .. 8 c8 + 7]
  for (int i = tid; i < 9 * NPL * COUT; i += 128) {
    const int t = i / (NPL * COUT), r = i % (NPL * COUT), c8 = r / COUT, co = r % COUT;
    *reinterpret_cast<uint4*>(sb + (size_t)i * 16) =
        *reinterpret_cast<const uint4*>(w + ((size_t)t * COUT + co) * CIN + c8 * 8);
  }
  // activations: plane (t, c8), row m = pixel p0 + m shifted by tap t (circular)
  for (int i = tid; i < 9 * 128 * NPL; i += 128) {
    const int c8 = i % NPL, m = (i / NPL) % 128, t = i / (NPL * 128);
    const long p = p0 + m;
    const int y = (int)(p / W), x = (int)(p % W);
    const int yy = wrap(y + t / 3 - 1, H), xx = wrap(x + t % 3 - 1, W);
    *reinterpret_cast<uint4*>(sa + ((size_t)(t * NPL + c8) * 128 + m) * 16) =
        *reinterpret_cast<const uint4*>(img + ((long)yy * W + xx) * CIN + c8 * 8);
  }
  prop_dev::fence_proxy_async_smem();   // the operand writes, before the tensor cores read them
  prop_tc::tc_fence_before();
  __syncthreads();
  prop_tc::tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    constexpr uint32_t idesc = prop_tc::idesc_bf16_f32(128, COUT);
    const uint32_t a0 = prop_dev::smem_u32(sa), b0 = prop_dev::smem_u32(sb);
    int k = 0;
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
      for (int kc = 0; kc < CIN / 16; ++kc, ++k) {
        const int plane = t * NPL + 2 * kc;   // two planes = 16 channels = one MMA's K
        const uint64_t a = prop_tc::smem_desc(a0 + plane * A_PLANE, A_PLANE, 128);
        const uint64_t b = prop_tc::smem_desc(b0 + plane * B_PLANE, B_PLANE, 128);
        prop_tc::mma_bf16(tmem, a, b, idesc, k > 0);
      }
    prop_tc::mma_commit(&bar);
  }
  const bool ok = prop_dev::mbar_wait(&bar, 0, &g_cnn_err);
  prop_tc::tc_fence_after();
  if (ok) {
    const long p = (long)n * npix + p0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
      float v[16];
      prop_tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        v[i] += bias ? bias[c0 + i] : 0.f;
        if (MODE == 0) v[i] = fmaxf(v[i], 0.f);
      }
      if (MODE == 2) {
        float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + p * COUT + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        uint32_t pk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
          pk[q] = *reinterpret_cast<const uint32_t*>(&h);
        }
        uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + p * COUT + c0);
        o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
    }
  }
  prop_tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    prop_tc::tc_fence_after();
    prop_tc::tmem_dealloc(tmem, 32);
  }
}

// Row-strip variant for W a multiple of 128 (every grid of the propagator's
// workloads).  A tile is 128 pixels of one image row; a CTA walks down a strip
// of consecutive rows y0 .. y1-1 at one x offset.  Input rows are staged as
// CIN/8 planes of 130 16-byte pixels (x0-1 .. x0+128, circular wrap) in a ring
// of RING row slots, so each tile loads one new row and reuses two; each tap's
// operand is a slot addressed at a plane and a one-pixel shift (descriptor
// start = plane base + 16 (dx + 1) bytes), so nothing is gathered nine times.
// Two tensor-memory accumulators let tile i's MMAs run while tile i-1's
// epilogue reads the other one back: warp 4 issues the MMAs, warps 0-3 load
// rows (two tiles ahead, by cp.async) and run the epilogue.
// Weights and biases are loaded once per CTA; tensor memory is allocated once.
template <int CIN, int COUT>
constexpr size_t conv_row_smem() {
  return (size_t)9 * (CIN / 8) * COUT * 16 + (size_t)5 * (CIN / 8) * 130 * 16;
}

__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(prop_dev::smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// grid: one CTA per (image, x tile, chunk of rows); cps chunks per strip
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(160) k_conv_tc_row(const __nv_bfloat16* __restrict__ in,
                                                     const __nv_bfloat16* __restrict__ w,
                                                     const float* __restrict__ bias, void* out, int N, int H, int W,
                                                     int cps, const int* active, int astride, int want) {
  constexpr int NPL = CIN / 8;
  constexpr int HPX = 130;                              // halo pixels per row
  constexpr int RING = 5;                               // rows i .. i+2 in use, i+3 landed or landing, i+4 loading
  constexpr uint32_t H_PLANE = HPX * 16, B_PLANE = COUT * 16;
  constexpr uint32_t ROW = NPL * H_PLANE;               // bytes of one staged row
  extern __shared__ __align__(128) unsigned char smem_row[];
  unsigned char* sb = smem_row;                         // weights
  unsigned char* sh = smem_row + 9 * NPL * B_PLANE;     // ring of staged rows
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ float sbias[COUT];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tpr = W / 128;
  const int chunk = blockIdx.x % cps, strip = blockIdx.x / cps;
  const int n = strip / tpr, x0 = (strip - n * tpr) * 128;
  const int y0 = (int)((long)chunk * H / cps), y1 = (int)((long)(chunk + 1) * H / cps);
  if (n >= N || y0 >= y1) return;
  if (active && active[(long)n * astride] != want) return;
  // an earlier wait gave up (reported by prop_cnn_check): issue nothing more
  if (*reinterpret_cast<volatile const int*>(&g_cnn_err) != 0) return;
  const int nt = y1 - y0;                               // tiles of this CTA
  const __nv_bfloat16* img = in + (long)n * H * W * CIN;
  // staged row j holds image row y0 - 1 + j (wrapped) in slot j % RING
  auto load_row = [&](int j) {
    const __nv_bfloat16* row = img + (long)wrap(y0 - 1 + j, H) * W * CIN;
    unsigned char* dst = sh + (size_t)(j % RING) * ROW;
    for (int i = tid; i < HPX * NPL; i += 128) {
      const int q = i / NPL, c8 = i % NPL;
      cp_async_16(dst + ((size_t)c8 * HPX + q) * 16, row + (long)wrap(x0 + q - 1, W) * CIN + c8 * 8);
    }
  };
  if (warp == 0) prop_tc::tmem_alloc(&tmem_base, 64);
  if (tid == 0) {
    prop_dev::mbar_init(&bar[0], 1);
    prop_dev::mbar_init(&bar[1], 1);
    prop_dev::fence_mbar_init();
  }
  const bool mma_warp = warp == 4;
  if (!mma_warp) {
    for (int i = tid; i < 9 * NPL * COUT; i += 128) {
      const int t = i / (NPL * COUT), r = i % (NPL * COUT), c8 = r / COUT, co = r % COUT;
      cp_async_16(sb + (size_t)i * 16, w + ((size_t)t * COUT + co) * CIN + c8 * 8);
    }
    for (int i = tid; i < COUT; i += 128) sbias[i] = bias ? bias[i] : 0.f;
    load_row(0);
    load_row(1);
    load_row(2);
  }
  cp_async_commit();                                    // group: weights and rows 0..2 (tile 0)
  if (nt > 1 && !mma_warp) load_row(3);
  cp_async_commit();                                    // group: row 3 (tile 1)
  prop_tc::tc_fence_before();
  __syncthreads();
  prop_tc::tc_fence_after();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = prop_tc::idesc_bf16_f32(128, COUT);
  const uint32_t b0 = prop_dev::smem_u32(sb), a0 = prop_dev::smem_u32(sh);
  bool ok = true;
  // accumulator of tile i: columns 32 (i & 1); read back, bias, activation, store
  auto epilogue = [&](int i) {
    const long p = ((long)n * H + y0 + i) * W + x0 + warp * 32 + lane;
    const uint32_t acc = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((i & 1) * 32);
#pragma unroll
    for (int c0 = 0; c0 < COUT; c0 += 16) {
      float v[16];
      prop_tc::tmem_ld16(acc + (uint32_t)c0, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        v[e] += sbias[c0 + e];
        if (MODE == 0) v[e] = fmaxf(v[e], 0.f);
      }
      if (MODE == 2) {
        float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + p * COUT + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        uint32_t pk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const __nv_bfloat162 hv = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
          pk[q] = *reinterpret_cast<const uint32_t*>(&hv);
        }
        uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(out) + p * COUT + c0);
        o[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        o[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
    }
  };
  for (int i = 0; i < nt; ++i) {
    cp_async_wait<1>();                                 // rows i .. i+2 landed (row i+3 may be in flight)
    prop_dev::fence_proxy_async_smem();
    prop_tc::tc_fence_before();
    __syncthreads();   // rows visible; accumulator (i & 1) read back by tile i-2's epilogue
    if (mma_warp) {
      if (lane == 0) {
        prop_tc::tc_fence_after();
        int kk = 0;
#pragma unroll
        for (int t = 0; t < 9; ++t)
#pragma unroll
          for (int kc = 0; kc < CIN / 16; ++kc, ++kk) {
            const int r = t / 3, dx = t % 3 - 1;
            const uint32_t slot = (uint32_t)((i + r) % RING);
            const uint64_t a = prop_tc::smem_desc(a0 + slot * ROW + (uint32_t)(2 * kc) * H_PLANE + (uint32_t)(dx + 1) * 16,
                                                  H_PLANE, 128);
            const uint64_t b = prop_tc::smem_desc(b0 + (uint32_t)(t * NPL + 2 * kc) * B_PLANE, B_PLANE, 128);
            prop_tc::mma_bf16(tmem + (uint32_t)((i & 1) * 32), a, b, idesc, kk > 0);
          }
        prop_tc::mma_commit(&bar[i & 1]);
      }
      __syncwarp();
      continue;
    }
    if (i > 0) {   // tile i-1's MMAs done: its accumulator is ready and row slot (i-1) % RING is free
      ok = ok && prop_dev::mbar_wait(&bar[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1), &g_cnn_err);
      prop_tc::tc_fence_after();
    }
    if (i + 4 < nt + 2) load_row(i + 4);               // the row tile i+2 needs last
    cp_async_commit();
    if (i > 0 && ok) epilogue(i - 1);
  }
  if (ok && !mma_warp) {
    ok = prop_dev::mbar_wait(&bar[(nt - 1) & 1], (uint32_t)(((nt - 1) >> 1) & 1), &g_cnn_err);
    prop_tc::tc_fence_after();
    if (ok) epilogue(nt - 1);
  }
  cp_async_wait<0>();
  prop_tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    prop_tc::tc_fence_after();
    prop_tc::tmem_dealloc(tmem, 64);
  }
}

// Per-CTA partial weight and bias gradients over a block of PIX pixels of one row:
// part[blk][t][co][ci] = sum_p g[p][co] a[p + d_t][ci],  part[blk][9 CO CI + co] = sum_p g[p][co].
template <int CIN, int COUT>
__global__ void __launch_bounds__(COUT * CIN / 4) k_wgrad(const __nv_bfloat16* __restrict__ g, const __nv_bfloat16* __restrict__ a,
                                                         float* part, int H, int W) {
  constexpr int PIX = 64;
  constexpr int NT = COUT * CIN / 4;
  __shared__ float sg[PIX][COUT];
  __shared__ float sa[3][PIX + 2][CIN];
  const int n = blockIdx.z, y = blockIdx.y, x0 = blockIdx.x * PIX;
  const long base = (long)n * H * W;
  for (int i = threadIdx.x; i < PIX * COUT; i += NT) {
    const int p = i / COUT, c = i % COUT;
    sg[p][c] = __bfloat162float(g[(base + (long)y * W + x0 + p) * COUT + c]);
  }
  for (int i = threadIdx.x; i < 3 * (PIX + 2) * CIN; i += NT) {
    const int r = i / ((PIX + 2) * CIN), rem = i % ((PIX + 2) * CIN), q = rem / CIN, c = rem % CIN;
    const int yy = wrap(y + r - 1, H), xx = wrap(x0 + q - 1, W);
    sa[r][q][c] = __bfloat162float(a[(base + (long)yy * W + xx) * CIN + c]);
  }
  __syncthreads();
  const int co = threadIdx.x / (CIN / 4), ci = (threadIdx.x % (CIN / 4)) * 4;
  float acc[9][4];
  float bsum = 0.f;
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
  for (int p = 0; p < PIX; ++p) {
    const float gv = sg[p][co];
    bsum += gv;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int r = t / 3, q = p + t % 3;
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[t][k] = fmaf(gv, sa[r][q][ci + k], acc[t][k]);
    }
  }
  const long blk = ((long)n * gridDim.y + y) * gridDim.x + blockIdx.x;
  float* o = part + blk * (9 * COUT * CIN + COUT);
#pragma unroll
  for (int t = 0; t < 9; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) o[(t * COUT + co) * CIN + ci + k] = acc[t][k];
  if (ci == 0) o[9 * COUT * CIN + co] = bsum;
}

// out[i] = sum over blocks of part[blk][i]  (fixed order: deterministic)
__global__ void k_reduce_parts(const float* part, long nblk, int len, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (long b = 0; b < nblk; ++b) s += part[b * len + i];
    out[i] = s;
  }
}

// Wt[t][ci][co] = W[8 - t][co][ci]: the data gradient is the forward convolution
// of the output gradient with these weights.
__global__ void k_flip_transpose(const __nv_bfloat16* w, __nv_bfloat16* wt, int cout, int cin) {
  const int total = 9 * cout * cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int t = i / (cout * cin), r = i % (cout * cin), co = r / cin, ci = r % cin;
    wt[((8 - t) * cin + ci) * cout + co] = w[i];
  }
}

// g *= [a > 0] (ReLU derivative from the stored activation), in place, bf16
__global__ void k_relu_mask(__nv_bfloat16* g, const __nv_bfloat16* a, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(a[i]) > 0.f)) g[i] = __float2bfloat16(0.f);
}

// f32 -> bf16
__global__ void k_to_bf16(const float* x, __nv_bfloat16* y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// loss = 0.5 sum_valid (out - target)^2 / npix;  grad = (out - target) / npix on the first
// `valid` of C channels, 0 on the padding; loss partials accumulated in double.
__global__ void k_mse(const float* out, const float* tgt, __nv_bfloat16* grad, long npix, int C, int valid,
                      double* loss) {
  __shared__ double red[32];
  double acc = 0.0;
  const float inv = 1.0f / (float)npix;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < npix * C; i += (long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    float d = 0.f;
    if (c < valid) d = out[i] - tgt[i];
    acc += 0.5 * (double)d * d;
    grad[i] = __float2bfloat16(d * inv);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    atomicAdd(loss, s / (double)npix);
  }
}

// Adam on float32 master parameters; writes the bf16 copy of weights (nbf16 > 0).
__global__ void k_adam(float* p, const float* grad, float* m, float* v, long n, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16* pbf16) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi; v[i] = vi;
    const float upd = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] -= upd;
    if (pbf16) pbf16[i] = __float2bfloat16(p[i]);
  }
}

int g_path = PROP_CNN_PATH_AUTO;

template <int CIN, int COUT, int MODE>
int launch_conv(const void* in, const void* w, const float* b, void* out, int N, int H, int W, const int* active,
                int astride, int want, cudaStream_t st) {
  const long npix = (long)H * W;
  if (g_path == PROP_CNN_PATH_AUTO && W % 128 == 0 && npix * N / 128 < 0x7FF00000L) {   // 32-bit strip indices
    constexpr size_t sm = conv_row_smem<CIN, COUT>();
    static int ctas_per_sm = 0;
    if (!ctas_per_sm) {
      // the whole shared-memory carveout for this kernel, so that several CTAs fit.
      // The occupancy query answers one CTA per SM for this kernel on GB300 while
      // the profiler reports three (shared memory the limit), so the CTAs that fit
      // by shared memory (at most 8; registers allow more) size the grid as well.
      int dev = 0, smem_sm = 0;
      if (cudaFuncSetAttribute(k_conv_tc_row<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
              cudaSuccess ||
          cudaFuncSetAttribute(k_conv_tc_row<CIN, COUT, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm, k_conv_tc_row<CIN, COUT, MODE>, 160, sm) !=
              cudaSuccess ||
          cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return PROP_CNN_E_CUDA;
      const int fit = smem_sm / (int)(sm + 2048);   // dynamic + static + the per-CTA reserve
      ctas_per_sm = std::max(ctas_per_sm, std::min(fit, 8));
      if (ctas_per_sm < 1) ctas_per_sm = 1;
    }
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return PROP_CNN_E_CUDA;
    // strips of 128 pixels x H rows, each cut into cps chunks of consecutive rows:
    // one wave of the CTAs that fit, or one CTA per strip when strips outnumber them
    const long strips = (long)N * (W / 128);
    const long slots = (long)ctas_per_sm * sms;
    const int cps = (int)std::max<long>(1, std::min<long>(H, slots / strips));
    k_conv_tc_row<CIN, COUT, MODE><<<(unsigned)(strips * cps), 160, sm, st>>>(
        (const __nv_bfloat16*)in, (const __nv_bfloat16*)w, b, out, N, H, W, cps, active, astride, want);
    return cudaGetLastError() == cudaSuccess ? 0 : PROP_CNN_E_CUDA;
  }
  if (g_path == PROP_CNN_PATH_AUTO && npix % 128 == 0 && npix / 128 <= 0x7FFFFFFF && N <= 65535) {
    constexpr size_t sm = conv_tc_smem<CIN, COUT>();
    static bool attr = false;
    if (!attr) {
      if (cudaFuncSetAttribute(k_conv_tc<CIN, COUT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
          cudaSuccess)
        return PROP_CNN_E_CUDA;
      attr = true;
    }
    k_conv_tc<CIN, COUT, MODE><<<dim3((unsigned)(npix / 128), N), 128, sm, st>>>(
        (const __nv_bfloat16*)in, (const __nv_bfloat16*)w, b, out, H, W, active, astride, want);
    return cudaGetLastError() == cudaSuccess ? 0 : PROP_CNN_E_CUDA;
  }
  dim3 grid((W / 16 + 3) / 4, H, N);
  k_conv<CIN, COUT, MODE><<<grid, 128, 0, st>>>((const __nv_bfloat16*)in, (const __nv_bfloat16*)w, b, out, H, W,
                                                active, astride, want);
  return cudaGetLastError() == cudaSuccess ? 0 : PROP_CNN_E_CUDA;
}

template <int CIN, int COUT>
int conv_mode(int mode, const void* in, const void* w, const float* b, void* out, int N, int H, int W,
              const int* active, int astride, int want, cudaStream_t st) {
  switch (mode) {
    case PROP_CNN_RELU_BF16: return launch_conv<CIN, COUT, 0>(in, w, b, out, N, H, W, active, astride, want, st);
    case PROP_CNN_LINEAR_BF16: return launch_conv<CIN, COUT, 1>(in, w, b, out, N, H, W, active, astride, want, st);
    case PROP_CNN_LINEAR_F32: return launch_conv<CIN, COUT, 2>(in, w, b, out, N, H, W, active, astride, want, st);
    default: return PROP_CNN_E_ARG;
  }
}

bool ok_ch(int c) { return c == 16 || c == 32; }

}  // namespace

extern "C" {

int prop_cnn_conv(int32_t cin, int32_t cout, int32_t mode, const void* d_in, const void* d_w, const float* d_bias,
                  void* d_out, int32_t N, int32_t H, int32_t W, const int32_t* d_active, int32_t active_stride,
                  int32_t active_want, void* stream) {
  if (!ok_ch(cin) || !ok_ch(cout) || N < 0 || H < 1 || W < 16 || W % 16 || !d_in || !d_w || !d_out)
    return PROP_CNN_E_ARG;
  if (N == 0) return PROP_CNN_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int* act = (const int*)d_active;
  if (cin == 16 && cout == 16) return conv_mode<16, 16>(mode, d_in, d_w, d_bias, d_out, N, H, W, act, active_stride, active_want, st);
  if (cin == 16 && cout == 32) return conv_mode<16, 32>(mode, d_in, d_w, d_bias, d_out, N, H, W, act, active_stride, active_want, st);
  if (cin == 32 && cout == 16) return conv_mode<32, 16>(mode, d_in, d_w, d_bias, d_out, N, H, W, act, active_stride, active_want, st);
  return conv_mode<32, 32>(mode, d_in, d_w, d_bias, d_out, N, H, W, act, active_stride, active_want, st);
}

int prop_cnn_set_path(int32_t path) {
  if (path != PROP_CNN_PATH_AUTO && path != PROP_CNN_PATH_MMA_SYNC) return PROP_CNN_E_ARG;
  g_path = path;
  return PROP_CNN_OK;
}

int prop_cnn_check(void* stream) {
  int e = 0;
  const int zero = 0;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
      cudaMemcpyFromSymbol(&e, g_cnn_err, sizeof(int)) != cudaSuccess ||
      (e && cudaMemcpyToSymbol(g_cnn_err, &zero, sizeof(int)) != cudaSuccess))
    return PROP_CNN_E_CUDA;
  return e ? PROP_CNN_E_TIMEOUT : PROP_CNN_OK;
}

int prop_cnn_wgrad_workspace(int32_t cin, int32_t cout, int32_t N, int32_t H, int32_t W, size_t* bytes) {
  if (!ok_ch(cin) || !ok_ch(cout) || W % 64 || !bytes) return PROP_CNN_E_ARG;
  *bytes = ((size_t)N * H * (W / 64) + 1) * (9 * cout * cin + cout) * sizeof(float);
  return PROP_CNN_OK;
}

int prop_cnn_wgrad(int32_t cin, int32_t cout, const void* d_grad, const void* d_act, int32_t N, int32_t H, int32_t W,
                   float* d_dw, float* d_db, void* d_work, size_t work_bytes, void* stream) {
  size_t need = 0;
  if (prop_cnn_wgrad_workspace(cin, cout, N, H, W, &need) || !d_grad || !d_act || !d_dw || !d_db || !d_work)
    return PROP_CNN_E_ARG;
  if (work_bytes < need) return PROP_CNN_E_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid(W / 64, H, N);
  float* part = (float*)d_work;
  const __nv_bfloat16* g = (const __nv_bfloat16*)d_grad;
  const __nv_bfloat16* a = (const __nv_bfloat16*)d_act;
  if (cin == 16 && cout == 16) k_wgrad<16, 16><<<grid, 64, 0, st>>>(g, a, part, H, W);
  else if (cin == 16 && cout == 32) k_wgrad<16, 32><<<grid, 128, 0, st>>>(g, a, part, H, W);
  else if (cin == 32 && cout == 16) k_wgrad<32, 16><<<grid, 128, 0, st>>>(g, a, part, H, W);
  else k_wgrad<32, 32><<<grid, 256, 0, st>>>(g, a, part, H, W);
  const int len = 9 * cout * cin + cout;
  const long nblk = (long)N * H * (W / 64);
  // reduce into a contiguous [9 CO CI | CO] vector placed in d_dw / d_db
  k_reduce_parts<<<(len + 255) / 256, 256, 0, st>>>(part, nblk, len, part + nblk * len);
  if (cudaMemcpyAsync(d_dw, part + nblk * len, 9 * cout * cin * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(d_db, part + nblk * len + 9 * cout * cin, cout * sizeof(float), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return PROP_CNN_E_CUDA;
  return cudaGetLastError() == cudaSuccess ? PROP_CNN_OK : PROP_CNN_E_CUDA;
}

int prop_cnn_flip_transpose(const void* d_w, void* d_wt, int32_t cout, int32_t cin, void* stream) {
  if (!d_w || !d_wt || !ok_ch(cin) || !ok_ch(cout)) return PROP_CNN_E_ARG;
  k_flip_transpose<<<(9 * cout * cin + 255) / 256, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)d_w,
                                                                                  (__nv_bfloat16*)d_wt, cout, cin);
  return cudaGetLastError() == cudaSuccess ? PROP_CNN_OK : PROP_CNN_E_CUDA;
}

int prop_cnn_relu_mask(void* d_grad, const void* d_act, int64_t n, void* stream) {
  if (!d_grad || !d_act || n < 0) return PROP_CNN_E_ARG;
  const int blocks = (int)std::min<int64_t>(4096, (n + 255) / 256);
  if (n) k_relu_mask<<<blocks, 256, 0, (cudaStream_t)stream>>>((__nv_bfloat16*)d_grad, (const __nv_bfloat16*)d_act, n);
  return cudaGetLastError() == cudaSuccess ? PROP_CNN_OK : PROP_CNN_E_CUDA;
}

int prop_cnn_to_bf16(const float* d_x, void* d_y, int64_t n, void* stream) {
  if (!d_x || !d_y || n < 0) return PROP_CNN_E_ARG;
  const int blocks = (int)std::min<int64_t>(4096, (n + 255) / 256);
  if (n) k_to_bf16<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_x, (__nv_bfloat16*)d_y, n);
  return cudaGetLastError() == cudaSuccess ? PROP_CNN_OK : PROP_CNN_E_CUDA;
}

int prop_cnn_mse(const float* d_out, const float* d_target, void* d_grad, int64_t npix, int32_t C, int32_t valid,
                 double* d_loss, void* stream) {
  if (!d_out || !d_target || !d_grad || !d_loss || npix < 0 || C < 1 || valid > C) return PROP_CNN_E_ARG;
  const int blocks = (int)std::min<int64_t>(4096, (npix * C + 255) / 256);
  if (npix) k_mse<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_out, d_target, (__nv_bfloat16*)d_grad, npix, C, valid, d_loss);
  return cudaGetLastError() == cudaSuccess ? PROP_CNN_OK : PROP_CNN_E_CUDA;
}

int prop_cnn_adam(float* d_p, const float* d_g, float* d_m, float* d_v, int64_t n, float lr, float b1, float b2,
                  float eps, int32_t step, void* d_p_bf16, void* stream) {
  if (!d_p || !d_g || !d_m || !d_v || n < 0 || step < 1) return PROP_CNN_E_ARG;
  const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
  const int blocks = (int)std::min<int64_t>(1024, (n + 255) / 256);
  if (n) k_adam<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_p, d_g, d_m, d_v, n, lr, b1, b2, eps, c1, c2,
                                                          (__nv_bfloat16*)d_p_bf16);
  return cudaGetLastError() == cudaSuccess ? PROP_CNN_OK : PROP_CNN_E_CUDA;
}

}  // extern "C"
