// Shared-memory radix FFT used by every pass of the propagator.
//
// A CTA holds NV vectors of length N in shared memory and transforms all of
// them along their length with a self-sorting (Stockham) radix sequence.  Each
// stage reads R points of every butterfly into registers, multiplies by the
// stage twiddles, does an in-register radix-R DFT, waits at a barrier, and
// writes the R outputs to their sorted positions: in place, no ping-pong
// buffer, natural order in and out.  For stage s with NS = product of the
// previous radices and M = N/R, butterfly j (k = j mod NS) reads
// x[j + t M], scales it by w_N^{t k N/(NS R)}, and writes output t to
// (j / NS) NS R + k + t NS.
//
// Layouts: COL=true is a column tile, element (v, n) at n*NV + v (v = the
// column within the tile, fastest); COL=false is NV rows with one padding
// element per 16 (index n + n/16) so that the stride-R writes of the first
// stage do not serialise on the shared-memory banks.
//
// Twiddles come from a device table w[m] = exp(-2 pi i m / N), m < N, computed
// on the host in double precision and rounded once to T.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace prop_dev {

template <typename T> struct Cx;
template <> struct Cx<float>  { using t = float2; };
template <> struct Cx<double> { using t = double2; };

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
template <typename C, typename R> __device__ __forceinline__ C scal(C a, R s) { C c; c.x = a.x * s; c.y = a.y * s; return c; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot90(C a) {
  C c;
  if (INV) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; }
  return c;
}

// cos(2 pi m / 16) for integer m, from the exact values of the 16th roots of unity.
__host__ __device__ constexpr double cos16(int m) {
  return ((m % 16 + 16) % 16) == 0 ? 1.0 :
         ((m % 16 + 16) % 16) == 1 ? 0.92387953251128675613 :
         ((m % 16 + 16) % 16) == 2 ? 0.70710678118654752440 :
         ((m % 16 + 16) % 16) == 3 ? 0.38268343236508977173 :
         ((m % 16 + 16) % 16) == 4 ? 0.0 :
         ((m % 16 + 16) % 16) == 5 ? -0.38268343236508977173 :
         ((m % 16 + 16) % 16) == 6 ? -0.70710678118654752440 :
         ((m % 16 + 16) % 16) == 7 ? -0.92387953251128675613 :
         ((m % 16 + 16) % 16) == 8 ? -1.0 :
         ((m % 16 + 16) % 16) == 9 ? -0.92387953251128675613 :
         ((m % 16 + 16) % 16) == 10 ? -0.70710678118654752440 :
         ((m % 16 + 16) % 16) == 11 ? -0.38268343236508977173 :
         ((m % 16 + 16) % 16) == 12 ? 0.0 :
         ((m % 16 + 16) % 16) == 13 ? 0.38268343236508977173 :
         ((m % 16 + 16) % 16) == 14 ? 0.70710678118654752440 : 0.92387953251128675613;
}
__host__ __device__ constexpr double sin16(int m) { return cos16(m - 4); }

// a * exp(-+ 2 pi i m / 16), sign by direction
template <int M, bool INV, typename C> __device__ __forceinline__ C tw16(C a) {
  if constexpr ((M % 16) == 0) return a;
  else if constexpr ((M % 16) == 4) return rot90<INV>(a);
  else if constexpr ((M % 16) == 8) { C c; c.x = -a.x; c.y = -a.y; return c; }
  else if constexpr ((M % 16) == 12) return rot90<!INV>(a);
  else {
    using R = decltype(a.x);
    constexpr double cr = cos16(M);
    constexpr double ci = INV ? sin16(M) : -sin16(M);
    C w; w.x = (R)cr; w.y = (R)ci;
    return cmul(a, w);
  }
}

// cos(2 pi m / 32) for integer m, from the exact values of the 32nd roots of unity
// (odd m; even m reduce to cos16).
__host__ __device__ constexpr double cos32(int m) {
  return ((m % 32 + 32) % 32) % 2 == 0 ? cos16(((m % 32 + 32) % 32) / 2) :
         ((m % 32 + 32) % 32) == 1 ? 0.98078528040323044913 :
         ((m % 32 + 32) % 32) == 3 ? 0.83146961230254523708 :
         ((m % 32 + 32) % 32) == 5 ? 0.55557023301960222474 :
         ((m % 32 + 32) % 32) == 7 ? 0.19509032201612826785 :
         ((m % 32 + 32) % 32) == 9 ? -0.19509032201612826785 :
         ((m % 32 + 32) % 32) == 11 ? -0.55557023301960222474 :
         ((m % 32 + 32) % 32) == 13 ? -0.83146961230254523708 :
         ((m % 32 + 32) % 32) == 15 ? -0.98078528040323044913 :
         ((m % 32 + 32) % 32) == 17 ? -0.98078528040323044913 :
         ((m % 32 + 32) % 32) == 19 ? -0.83146961230254523708 :
         ((m % 32 + 32) % 32) == 21 ? -0.55557023301960222474 :
         ((m % 32 + 32) % 32) == 23 ? -0.19509032201612826785 :
         ((m % 32 + 32) % 32) == 25 ? 0.19509032201612826785 :
         ((m % 32 + 32) % 32) == 27 ? 0.55557023301960222474 :
         ((m % 32 + 32) % 32) == 29 ? 0.83146961230254523708 : 0.98078528040323044913;
}
__host__ __device__ constexpr double sin32(int m) { return cos32(m - 8); }

// a * exp(-+ 2 pi i m / 32), sign by direction
template <int M, bool INV, typename C> __device__ __forceinline__ C tw32(C a) {
  if constexpr ((M % 2) == 0) return tw16<M / 2, INV>(a);
  else {
    using R = decltype(a.x);
    constexpr double cr = cos32(M);
    constexpr double ci = INV ? sin32(M) : -sin32(M);
    C w; w.x = (R)cr; w.y = (R)ci;
    return cmul(a, w);
  }
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C* x) {
  C a = x[0], b = x[1];
  x[0] = a + b; x[1] = a - b;
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C* x) {
  using R = decltype(x[0].x);
  const R h = (R)0.86602540378443864676;   // sqrt(3)/2
  C t = x[1] + x[2];
  C d = x[1] - x[2];
  C m; m.x = x[0].x - (R)0.5 * t.x; m.y = x[0].y - (R)0.5 * t.y;
  // u = d * (-i sqrt3/2) forward, (+i sqrt3/2) inverse
  C u = rot90<INV>(d); u.x *= h; u.y *= h;
  x[0] = x[0] + t;
  x[1] = m + u;
  x[2] = m - u;
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C* x) {
  C t0 = x[0] + x[2], t1 = x[0] - x[2], t2 = x[1] + x[3], t3 = rot90<INV>(x[1] - x[3]);
  x[0] = t0 + t2; x[2] = t0 - t2; x[1] = t1 + t3; x[3] = t1 - t3;
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C* x) {
  C e[4] = {x[0], x[2], x[4], x[6]};
  C o[4] = {x[1], x[3], x[5], x[7]};
  dft4<INV>(e); dft4<INV>(o);
  o[1] = tw16<2, INV>(o[1]);
  o[2] = tw16<4, INV>(o[2]);
  o[3] = tw16<6, INV>(o[3]);
#pragma unroll
  for (int k = 0; k < 4; ++k) { x[k] = e[k] + o[k]; x[k + 4] = e[k] - o[k]; }
}

// 16-point DFT as 4 x 4: inner DFT4 over n1 of x[4 n1 + n2], twiddle w16^{n2 k1},
// outer DFT4 over n2; output X[k1 + 4 k2].
template <bool INV, typename C> __device__ __forceinline__ void dft16(C* x) {
  C y[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    C a[4] = {x[n2], x[n2 + 4], x[n2 + 8], x[n2 + 12]};
    dft4<INV>(a);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = a[k1];
  }
  y[1][1] = tw16<1, INV>(y[1][1]); y[1][2] = tw16<2, INV>(y[1][2]); y[1][3] = tw16<3, INV>(y[1][3]);
  y[2][1] = tw16<2, INV>(y[2][1]); y[2][2] = tw16<4, INV>(y[2][2]); y[2][3] = tw16<6, INV>(y[2][3]);
  y[3][1] = tw16<3, INV>(y[3][1]); y[3][2] = tw16<6, INV>(y[3][2]); y[3][3] = tw16<9, INV>(y[3][3]);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C a[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
    dft4<INV>(a);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = a[k2];
  }
}

// 32-point DFT (natural order in and out): two 16-point DFTs of the even and odd
// points, then X[k] = E[k] + w32^k O[k], X[k+16] = E[k] - w32^k O[k].
template <int K, bool INV, typename C> __device__ __forceinline__ void dft32_join(C* x, const C* e, const C* o) {
  if constexpr (K < 16) {
    const C t = tw32<K, INV>(o[K]);
    x[K] = e[K] + t;
    x[K + 16] = e[K] - t;
    dft32_join<K + 1, INV>(x, e, o);
  }
}
template <bool INV, typename C> __device__ __forceinline__ void dft32(C* x) {
  C e[16], o[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) { e[k] = x[2 * k]; o[k] = x[2 * k + 1]; }
  dft16<INV>(e);
  dft16<INV>(o);
  dft32_join<0, INV>(x, e, o);
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dftR(C* x) {
  if constexpr (R == 2) dft2<INV>(x);
  else if constexpr (R == 3) dft3<INV>(x);
  else if constexpr (R == 4) dft4<INV>(x);
  else if constexpr (R == 8) dft8<INV>(x);
  else if constexpr (R == 16) dft16<INV>(x);
  else if constexpr (R == 32) dft32<INV>(x);
}

// Radix plans: product equals N, at most three stages.
template <int N> struct Plan;
template <> struct Plan<16>   { static constexpr int S = 1, R0 = 16, R1 = 1, R2 = 1; };
template <> struct Plan<32>   { static constexpr int S = 2, R0 = 4, R1 = 8, R2 = 1; };
template <> struct Plan<64>   { static constexpr int S = 2, R0 = 4, R1 = 16, R2 = 1; };
template <> struct Plan<128>  { static constexpr int S = 2, R0 = 8, R1 = 16, R2 = 1; };
template <> struct Plan<256>  { static constexpr int S = 2, R0 = 16, R1 = 16, R2 = 1; };
template <> struct Plan<384>  { static constexpr int S = 3, R0 = 3, R1 = 8, R2 = 16; };
template <> struct Plan<512>  { static constexpr int S = 3, R0 = 8, R1 = 8, R2 = 8; };
template <> struct Plan<768>  { static constexpr int S = 3, R0 = 3, R1 = 16, R2 = 16; };
template <> struct Plan<1024> { static constexpr int S = 3, R0 = 4, R1 = 16, R2 = 16; };

// shared-memory element index of (vector v, point n)
template <int N, int NV, bool COL> __device__ __forceinline__ int sidx(int v, int n) {
  if constexpr (COL) return n * NV + v;
  else return v * (N + N / 16) + n + (n >> 4);
}
template <int N, int NV, bool COL> __host__ __device__ constexpr int smem_elems() {
  return COL ? N * NV : NV * (N + N / 16);
}

template <typename C, int N, int R, int NS, bool INV, int NV, int NT, bool COL, bool TWS>
__device__ __forceinline__ void fft_stage(C* s, const C* __restrict__ tw, int tid) {
  constexpr int M = N / R;
  constexpr int NTASK = NV * M;
  constexpr int TPT = (NTASK + NT - 1) / NT;
  C r[TPT][R];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const int task = tid + q * NT;
    if ((NTASK % NT) == 0 || task < NTASK) {
      int v, j;
      if constexpr (COL) { v = task % NV; j = task / NV; } else { v = task / M; j = task % M; }
#pragma unroll
      for (int t = 0; t < R; ++t) r[q][t] = s[sidx<N, NV, COL>(v, j + t * M)];
      if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int t = 1; t < R; ++t) {
          C w = TWS ? tw[t * k * (N / (NS * R))] : __ldg(&tw[t * k * (N / (NS * R))]);
          if (INV) w.y = -w.y;
          r[q][t] = cmul(r[q][t], w);
        }
      }
      dftR<R, INV>(r[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const int task = tid + q * NT;
    if ((NTASK % NT) == 0 || task < NTASK) {
      int v, j;
      if constexpr (COL) { v = task % NV; j = task / NV; } else { v = task / M; j = task % M; }
      const int k = j % NS;
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int t = 0; t < R; ++t) s[sidx<N, NV, COL>(v, base + t * NS)] = r[q][t];
    }
  }
  __syncthreads();
}

// Full transform of the NV vectors held in s (caller synchronises before the call).
// TWS: the twiddle table tw is in shared memory (else global, read through the
// read-only cache).
template <typename C, int N, bool INV, int NV, int NT, bool COL, bool TWS = false>
__device__ __forceinline__ void fft_smem(C* s, const C* __restrict__ tw, int tid) {
  using P = Plan<N>;
  fft_stage<C, N, P::R0, 1, INV, NV, NT, COL, TWS>(s, tw, tid);
  if constexpr (P::S >= 2) fft_stage<C, N, P::R1, P::R0, INV, NV, NT, COL, TWS>(s, tw, tid);
  if constexpr (P::S >= 3) fft_stage<C, N, P::R2, P::R0 * P::R1, INV, NV, NT, COL, TWS>(s, tw, tid);
}

// ---------------------------------------------------------------------------
// Row transforms by warps: one warp transforms one N-point row (N = 32 L,
// L = 32 or 16) held in shared memory in the padded row layout, with no block
// barrier.  With n = n1 + 32 n2 and k = k2 + L k1:
//   step 1 (lane n1):  Y[n1][k2] = sum_{n2<L} x[n1 + 32 n2] w_L^{n2 k2}, times w_N^{n1 k2}
//   transpose through the row's own slots (Y[n1][k2] to slot 32 k2 + n1)
//   step 2:            X[k2 + L k1] = sum_{n1<32} Y[n1][k2] w_32^{n1 k1}
// For L = 32 lane k2 does one 32-point DFT.  For L = 16 two lanes share k2:
// lane (k2, h) takes the odd/even half k1 = h + 2 k1' by one radix-2 step,
// (Y[n] + (-1)^h Y[n + 16]) w_32^{h n}, then a 16-point DFT.
// ---------------------------------------------------------------------------
template <int N> __device__ __forceinline__ int rpad(int n) { return n + (n >> 4); }

template <int K, bool INV, typename C> __device__ __forceinline__ void half_twiddle(C* y, int h) {
  if constexpr (K < 16) {
    const C t = tw32<K, INV>(y[K]);
    y[K] = h ? t : y[K];
    half_twiddle<K + 1, INV>(y, h);
  }
}

template <typename C, int N, bool INV, bool TWS>
__device__ __forceinline__ void warp_fft_row(C* row, const C* __restrict__ tw, int lane) {
  constexpr int L = N / 32;
  static_assert(L == 32 || L == 16, "warp row transform covers N = 1024 and N = 512");
  C x[L];
#pragma unroll
  for (int n2 = 0; n2 < L; ++n2) x[n2] = row[rpad<N>(lane + 32 * n2)];
  dftR<L, INV>(x);
#pragma unroll
  for (int k2 = 1; k2 < L; ++k2) {
    C w = TWS ? tw[(lane * k2) % N] : __ldg(&tw[(lane * k2) % N]);
    if (INV) w.y = -w.y;
    x[k2] = cmul(x[k2], w);
  }
  __syncwarp();
#pragma unroll
  for (int k2 = 0; k2 < L; ++k2) row[rpad<N>(32 * k2 + lane)] = x[k2];
  __syncwarp();
  if constexpr (L == 32) {
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) x[n1] = row[rpad<N>(32 * lane + n1)];
    dft32<INV>(x);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) row[rpad<N>(lane + 32 * k1)] = x[k1];
  } else {
    const int k2 = lane & 15, h = lane >> 4;
#pragma unroll
    for (int n = 0; n < 16; ++n) {
      const C a = row[rpad<N>(32 * k2 + n)], b = row[rpad<N>(32 * k2 + n + 16)];
      x[n] = h ? a - b : a + b;
    }
    half_twiddle<0, INV>(x, h);
    dft16<INV>(x);
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) row[rpad<N>(k2 + 16 * (h + 2 * k1))] = x[k1];
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// The same two-step transform for data already in registers: lane l holds the
// points l + 32 m (m < L) of one length-N vector (N = 32 L, L = 32 or 16) and
// gets back the transform at the same positions (k = l + 32 m), so a forward
// transform, a pointwise multiply and an inverse transform chain in registers.
// `slot(s)` maps a scratch slot s < N to this warp's shared memory; the
// transpose writes slot 32 k2 + n1 and reads it back by k2.
// ---------------------------------------------------------------------------
template <typename C, int N, bool INV, typename SLOT>
__device__ __forceinline__ void warp_fft_regs(C (&x)[N / 32], const C* __restrict__ tw, int lane, SLOT slot) {
  constexpr int L = N / 32;
  static_assert(L == 32 || L == 16, "register transform covers N = 1024 and N = 512");
  dftR<L, INV>(x);
#pragma unroll
  for (int k2 = 1; k2 < L; ++k2) {
    C w = __ldg(&tw[(lane * k2) % N]);
    if (INV) w.y = -w.y;
    x[k2] = cmul(x[k2], w);
  }
  __syncwarp();
#pragma unroll
  for (int k2 = 0; k2 < L; ++k2) *slot(32 * k2 + lane) = x[k2];
  __syncwarp();
  if constexpr (L == 32) {
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) x[n1] = *slot(32 * lane + n1);
    dft32<INV>(x);      // lane k2 holds X[k2 + 32 k1] = position lane + 32 k1
  } else {
    const int k2 = lane & 15, h = lane >> 4;
#pragma unroll
    for (int n = 0; n < 16; ++n) {
      const C a = *slot(32 * k2 + n), b = *slot(32 * k2 + n + 16);
      x[n] = h ? a - b : a + b;
    }
    half_twiddle<0, INV>(x, h);
    dft16<INV>(x);      // lane (k2, h) holds X[k2 + 16 (h + 2 k1')] = position lane + 32 k1'
  }
  __syncwarp();
}

// Row transform of the NV rows held in s (padded row layout; caller synchronises
// before the call): by warps for N = 512 and 1024 when WF, else the block-wide
// Stockham.
template <typename C, int N, bool INV, int NV, int NT, bool WF = true, bool TWS = false>
__device__ __forceinline__ void fft_rows(C* s, const C* __restrict__ tw, int tid) {
  if constexpr (WF && (N == 1024 || N == 512) && NT >= 32) {
    constexpr int NW = NT / 32;
    const int warp = tid >> 5, lane = tid & 31;
    for (int r = warp; r < NV; r += NW) warp_fft_row<C, N, INV, TWS>(s + r * (N + N / 16), tw, lane);
    __syncthreads();
  } else {
    fft_smem<C, N, INV, NV, NT, false, TWS>(s, tw, tid);
  }
}

}  // namespace prop_dev
