// Device kernels of one propagation step (scalar operator).
//
// Data live in a caller-provided workspace, grouped by grid: a group is the
// set of beams that share (nx, ny, dx, dy); a "system" is one (beam, pole)
// shifted solve of Eq. (W_k_def).  Every launch covers all units of a group at
// once (grid.y = unit x component), so poles, components and beams share one
// launch.  Masked launches skip, per CTA, the systems whose GMRES state does
// not match.
//
// The three FFT passes of a 2-D transform round trip are
//   rows  (forward row DFTs, coalesced along x),
//   cols  (a tile of NV columns: column DFT, Fourier-diagonal multiply,
//          inverse column DFT, in shared memory),
//   rows  (inverse row DFTs followed by a pointwise epilogue),
// so the free-space solve (Z_fs - p I)^-1 of Sec. 4.2 -- diagonal in Fourier
// space on the periodic grid -- and the operator Z of Eq. (Z_bar_eq) share them.
#pragma once
#include <utility>
#include <cuda_bf16.h>
#include "fft.cuh"
#include "tma.cuh"

namespace prop_dev {

constexpr int MMAX = 64;   // largest GMRES restart length
constexpr int NSTRIPE = 16; // copies of each Gram-Schmidt accumulator (spreads the atomics)

enum SysStateCode { ST_DONE = 0, ST_ITER = 1, ST_CYCLE_END = 2 };

// GMRES state of one (beam, pole) system.  Complex numbers are double2.
struct SysState {
  int state, j, jend, iters, cycles, flags;   // flags: 1 = NaN seen, 2 = hit max cycles
  int used, pad_i;                            // used: iterated this step (E is meaningful)
  double beta, resid, scale, nrm_a, nrm_b, beta0;  // beta0: ||R0|| at the step start
  double z0norm2, enorm2;                     // ||z_k||^2 (free-space solve), ||e_k||^2
  double2 r0r;                                // <R0, r> of the last true-residual pass
  double2 g[MMAX + 1];             // Givens-rotated right-hand side beta e_1
  double2 sn[MMAX];
  double cs[MMAX];
  double2 H[(MMAX + 1) * MMAX];     // rotated (upper-triangular) columns, H[i + j*(MMAX+1)]
  double2 Hu[(MMAX + 1) * MMAX];    // Hessenberg columns as built (same indexing)
  double2 y[MMAX];
  double2 coef[MMAX + 1];           // coef[0]: the learned guess's scale alpha
};

template <typename T> struct GV {
  using C = typename Cx<T>::t;
  int nx, ny, ncomp, P, m, nb, nsys;
  long npts;
  C* V;          // [nsys][m+2][ncomp][npts]  Krylov basis (slot j+1 takes w = B v_j up to j = m)
  C* R0;         // [nsys][ncomp][npts]       right-hand side of the correction system
  double2* E;    // [nsys][ncomp][npts]       correction e_k, FP64
  C* Tmp;        // [nsys][ncomp][npts]       FFT intermediate
  double2* W64;  // master field.  FP64 path: complex128 [nb][ncomp][npts].  FP32 path:
                 // double-float, planar: hi plane float2 [nb][ncomp][npts], then lo plane
  C* What;       // [nb][ncomp][npts]         2-D spectrum of the field (rounded to T)
  C* Btmp;       // [nb][ncomp][npts]         beam-level FFT intermediate
  C* delta;      // [nb][npts]                (n^2 - n0^2)/n0^2
  C* basemul;    // [npts]                    (r(zeta_fs) - 1)/(nx ny)
  const T* ax;   // [(P+1)][nx][2]            -kx^2/(k0n0)^2 - Re p/2 as (hi, lo)
  const T* ay;   // [(P+1)][ny][2]            -ky^2/(k0n0)^2 - Re p/2 as (hi, lo)
  const T* pim;  // [P+1]                     -Im p (pole P is p = 0: the plain Z_fs)
  const C* twx;  // [nx] twiddles
  const C* twy;  // [ny]
  SysState* st;  // [nsys]
  double* bnorm2;       // [nb] ||w||^2 of the step's right-hand side
  int* nonhomog;        // [nb] 1 if delta != 0 somewhere
  double2* dsum;        // [nb] sum of delta over the grid: the preconditioner's constant medium is
                        //   its mean (the constant-index problem with n^2 = mean n^2)
  const double2* rk;    // [P] residues r_k
  const double* anorm;  // [2P]: bound on ||Z - p_k I|| over this grid (backward-error test), then the
                        //       per-pole tolerance factor mu_k >= 1 (error equidistribution)
  double2* part;        // [nsys][4][NSTRIPE][MMAX+1] striped accumulators of the Gram sweep,
                        //   plane 2 (j % 2) + {0: <v_i, w>, 1: <v_i, u_j> (slot MMAX: ||w||^2)}
  // vector operator (ncomp = 2) only
  C* psi;        // [nb][5][npts]  coefficients of Z - Z_fs: D1 = delta + psit_xx, D2 = delta + psit_yy,
                 //                X = psit_xy, px = psit_x, py = psit_y (psit = psi/(k0 n0)^2, psi = Log n^2)
  C* Tmp2;       // [nsys][ncomp][npts] second column-pass output (the d/dy branch)
  T kx0, ky0;    // 2 pi/(nx dx), 2 pi/(ny dy): wavenumber of FFT index 1
  double kx0d, ky0d;   // the same in FP64
  int* err;      // error word: 1 = a bounded wait for an asynchronous copy gave up, 2 = TMA alignment check failed
  const int* ulist;   // optional: grid row y works on unit ulist[y] (the compacted iterating systems)
};

// Unit and (unit, component) item of grid row y, through the optional unit list.
// -1 for an empty row of the list (the caller returns).
template <typename T> __device__ __forceinline__ int unit_of(const GV<T>& g, int y) { return g.ulist ? g.ulist[y] : y; }
template <typename T> __device__ __forceinline__ int item_of(const GV<T>& g, int y) {
  if (!g.ulist) return y;
  const int u = g.ulist[y / g.ncomp];
  return u < 0 ? -1 : u * g.ncomp + y % g.ncomp;
}

// Signed FFT frequency index of position i on an n-point grid.
__device__ __forceinline__ int ffreq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }
// i*k for a first derivative (zero at the unpaired Nyquist index), as a complex factor
template <typename C, typename T> __device__ __forceinline__ C ik_factor(int i, int n, T k0) {
  C f; f.x = 0;
  f.y = ((n % 2) == 0 && i == n / 2) ? (T)0 : (T)ffreq(i, n) * k0;
  return f;
}

// striped accumulator slot: plane 2 (j % 2) + 0 = <v_i, w>, + 1 = <v_i, u_j>
constexpr int NPLANE = 4;
__device__ __forceinline__ double2* part_at(double2* part, int s, int plane, int stripe, int i) {
  return part + (((long)s * NPLANE + plane) * NSTRIPE + stripe) * (MMAX + 1) + i;
}

// Which buffer a pass reads or writes: item (unit u, component c) lives at
// base + (u / div) * ustride + c * npts.
template <typename C> struct Buf {
  C* base;
  long ustride;
  int div;
  __device__ __forceinline__ C* at(int u, int c, long npts) const {
    return base + (long)(u / div) * ustride + (long)c * npts;
  }
};

// MUL_PREC_INV: the GMRES preconditioner (Z_fs + dbar - p)^-1, dbar = the beam's mean delta;
// MUL_POLE_INV: the free-space solve (Z_fs - p)^-1 itself.
enum MulMode { MUL_NONE = 0, MUL_TABLE = 1, MUL_POLE_INV = 2, MUL_POLE_FWD = 3, MUL_SCALE = 4,
               MUL_DY = 5, MUL_DYY = 6,   // scale * i ky,  scale * (-ky^2)
               MUL_PREC_INV = 7 };
enum EpiMode { EPI_STORE = 0, EPI_STORE64 = 1, EPI_ACCUM64 = 2, EPI_R0 = 3, EPI_ARNOLDI = 4,
               EPI_TRUERES = 5, EPI_OPERATOR = 6, EPI_ADD_E = 7 };

__device__ __forceinline__ float2 to_c(double2 a, float) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_c(double2 a, double) { return a; }
__device__ __forceinline__ float2 to_c(float2 a, float) { return a; }
__device__ __forceinline__ double2 to_d(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double2 to_d(double2 a) { return a; }

// Hint: bring the 128-byte line holding p into L2 (PTX prefetch.global.L2).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum) for the
// double-float master field of the FP32 path.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// (hi, lo) + v for one real component
__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
  float s, e;
  two_sum(hi, v, s, e);
  e += lo;
  fast_two_sum(s, e, hi, lo);
}

// block-wide sum of a double (blockDim.x threads, multiple of 32); result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
  }
  return r;
}

// Points p, p+1 (p even, 16-byte aligned) in one access: a float4 for complex
// FP32, two 16-byte accesses for complex FP64.
template <typename C> __device__ __forceinline__ void ld2(const C* base, long p, C& a, C& b) {
  if constexpr (sizeof(C) == 8) {
    const float4 q = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(base + p));
    a.x = q.x; a.y = q.y; b.x = q.z; b.y = q.w;
  } else {
    a = base[p]; b = base[p + 1];
  }
}
template <typename C> __device__ __forceinline__ void st2(C* base, long p, const C& a, const C& b) {
  if constexpr (sizeof(C) == 8) {
    *reinterpret_cast<float4*>(reinterpret_cast<float*>(base + p)) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    base[p] = a; base[p + 1] = b;
  }
}

__device__ __forceinline__ bool unit_active(const SysState* st, int mask, int u) {
  return mask < 0 || st[u].state == mask;
}

// Mean delta of a beam (the constant medium of its preconditioner), rounded to T.
template <typename T> __device__ __forceinline__ typename Cx<T>::t dbar_of(const GV<T>& g, int beam) {
  const double2 a = g.dsum[beam];
  const double inv = 1.0 / (double)g.npts;
  return to_c(make_double2(a.x * inv, a.y * inv), T());
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization is scheduled as its predecessor in the stream drains (the
// predecessor's CTAs trigger it when they exit) and waits here for the
// predecessor's completion and memory before it touches anything.  A no-op for
// a kernel launched without the attribute.  (Triggering the successor at entry
// instead let waiting CTAs hold SM slots that multi-wave predecessors needed:
// 3 % slower on the batched-scalar step.)
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

#ifndef PROP_PDL
#define PROP_PDL 1
#endif
// Host side: launch `k` with programmatic stream serialization, so that it can be
// scheduled while its predecessor drains (the kernel must begin with pdl_enter).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = PROP_PDL ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// Pass 1: forward row DFTs.  grid = (ny/NR, units*ncomp).
// ---------------------------------------------------------------------------
template <typename T, int N, int NR, int NT, typename SRC, bool WF>
__device__ __forceinline__ void rows_fwd_body(int bx, int by, int gdx, GV<T> g, Buf<SRC> src, Buf<typename Cx<T>::t> dst,
                                                 int mask, double* norm_acc) {
  pdl_enter();
  using C = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[32];
  const int item = item_of(g, (int)by);
  if (item < 0) return;
  const int u = item / g.ncomp, c = item % g.ncomp;
  if (!unit_active(g.st, mask, u)) return;
  const int row0 = bx * NR;
  const SRC* in = src.at(u, c, g.npts) + (long)row0 * N;
  T acc = 0;
  C* out = dst.at(u, c, g.npts) + (long)row0 * N;
  // 16-byte accesses (two points, same row) for complex FP32 in and out
  constexpr bool V4 = sizeof(T) == 4 && sizeof(SRC) == 8;
  const bool vec = V4 && ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
  if (vec) {
#pragma unroll
    for (int e2 = threadIdx.x; e2 < NR * N / 2; e2 += NT) {
      const int e = 2 * e2;
      C a, b;
      ld2(reinterpret_cast<const C*>(in), e, a, b);
      if (norm_acc) acc += a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y;
      s[sidx<N, NR, false>(e / N, e % N)] = a;
      s[sidx<N, NR, false>(e / N, e % N + 1)] = b;
    }
  } else {
#pragma unroll
    for (int e = threadIdx.x; e < NR * N; e += NT) {
      const int r = e / N, n = e % N;
      const C v = to_c(in[e], T());
      if (norm_acc) acc += v.x * v.x + v.y * v.y;
      s[sidx<N, NR, false>(r, n)] = v;
    }
  }
  __syncthreads();
  fft_rows<C, N, false, NR, NT, WF>(s, g.twx, threadIdx.x);
  if (vec) {
#pragma unroll
    for (int e2 = threadIdx.x; e2 < NR * N / 2; e2 += NT) {
      const int e = 2 * e2;
      st2(out, e, s[sidx<N, NR, false>(e / N, e % N)], s[sidx<N, NR, false>(e / N, e % N + 1)]);
    }
  } else {
#pragma unroll
    for (int e = threadIdx.x; e < NR * N; e += NT) out[e] = s[sidx<N, NR, false>(e / N, e % N)];
  }
  if (norm_acc) {
    const double t = block_sum((double)acc, red);
    if (threadIdx.x == 0) atomicAdd(&norm_acc[u], t);
  }
}
template <typename T, int N, int NR, int NT, typename SRC, bool WF>
__global__ void __launch_bounds__(NT) k_rows_fwd(GV<T> g, Buf<SRC> src, Buf<typename Cx<T>::t> dst,
                                                 int mask, double* norm_acc) {
  rows_fwd_body<T, N, NR, NT, SRC, WF>(blockIdx.x, blockIdx.y, gridDim.x, g, src, dst, mask, norm_acc);
}
// The warp-row variant at N = 1024 (complex FP32) with four resident CTAs per SM
// asked of the compiler: unbounded, the forward pass takes 132 registers and only
// three CTAs fit (measured: forward row pass 43.0 -> 39.7 ms per 20 batched-scalar
// steps; five or six CTAs spill and lose).
constexpr int WROWS_MINB = 4;
template <typename T, int N, int NR, int NT, typename SRC, bool WF>
__global__ void __launch_bounds__(NT, WROWS_MINB) k_rows_fwd_w(GV<T> g, Buf<SRC> src,
                                                                    Buf<typename Cx<T>::t> dst, int mask,
                                                                    double* norm_acc) {
  rows_fwd_body<T, N, NR, NT, SRC, WF>(blockIdx.x, blockIdx.y, gridDim.x, g, src, dst, mask, norm_acc);
}


// ---------------------------------------------------------------------------
// Pass 2: column tile of NV columns: [column DFT] -> multiply -> [inverse column DFT].
// grid = (nx/NV, units*ncomp).  The multiplier sees kx index i = x0 + v and ky
// index n; pole k = unit % P for system units.
// ---------------------------------------------------------------------------
// With DY the tile is 2*NV wide: columns NV..2NV-1 receive i*ky times the
// multiplied spectrum and leave through `dy` (the d/dy branch of the vector
// operator), transformed in the same shared-memory FFT.
template <typename T, int NY, int NV, int NT, bool DY>
__device__ __forceinline__ void cols_body(int bx, int by, int gdx, GV<T> g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst,
                                             int mask, int fwd, int mul, int inv, int skip_homog, int pole,
                                             T scale, Buf<typename Cx<T>::t> spec, Buf<typename Cx<T>::t> dy) {
  pdl_enter();
  using C = typename Cx<T>::t;
  constexpr int W = DY ? 2 * NV : NV;     // tile width in shared memory
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int item = item_of(g, (int)by);
  if (item < 0) return;
  const int u = item / g.ncomp, c = item % g.ncomp;
  if (!unit_active(g.st, mask, u)) return;
  if (skip_homog && !g.nonhomog[u / g.P]) return;
  const int x0 = bx * NV;
  const C* in = src.at(u, c, g.npts);
  if (mul == MUL_TABLE)   // the multiplier is read after the forward DFT: start its DRAM fetch now
    for (int n = threadIdx.x; n < NY; n += NT) prefetch_l2(g.basemul + (long)n * g.nx + x0);
#pragma unroll 8
  for (int e = threadIdx.x; e < NY * NV; e += NT) {
    const int n = e / NV, v = e % NV;
    s[n * W + v] = in[(long)n * g.nx + x0 + v];
  }
  __syncthreads();
  if (fwd) fft_smem<C, NY, false, W, NT, true>(s, g.twy, threadIdx.x);   // (DY: the extra columns are unused here)
  if (spec.base) {   // keep the 2-D spectrum as well (read again by the pole solves)
    C* sp = spec.at(u, c, g.npts);
#pragma unroll 8
    for (int e = threadIdx.x; e < NY * NV; e += NT) sp[(long)(e / NV) * g.nx + x0 + e % NV] = s[(e / NV) * W + e % NV];
  }
  if (mul != MUL_NONE) {
    const bool pm = (mul == MUL_POLE_INV || mul == MUL_POLE_FWD || mul == MUL_PREC_INV);
    const int k = pm ? (pole >= 0 ? pole : u % g.P) : 0;
    const T* ax = pm ? g.ax + (long)k * g.nx * 2 : nullptr;
    const T* ay = pm ? g.ay + (long)k * g.ny * 2 : nullptr;
    // the preconditioner's pole is p - dbar: Re shifted by +Re dbar, -Im p by +Im dbar
    C sh; sh.x = 0; sh.y = 0;
    if (mul == MUL_PREC_INV) sh = dbar_of(g, u / g.P);
    const T pim = pm ? g.pim[k] + sh.y : (T)0;
    for (int e = threadIdx.x; e < NY * NV; e += NT) {
      const int n = e / NV, v = e % NV, i = x0 + v;
      C a = s[n * W + v];
      if (mul == MUL_TABLE) {
        a = cmul(a, g.basemul[(long)n * g.nx + i]);
      } else if (mul == MUL_SCALE) {
        a.x *= scale; a.y *= scale;
      } else if (mul == MUL_DY) {
        a = cmul(a, ik_factor<C>(n, g.ny, g.ky0));
        a.x *= scale; a.y *= scale;
      } else if (mul == MUL_DYY) {
        const T k = (T)ffreq(n, g.ny) * g.ky0;
        a.x *= -k * k * scale; a.y *= -k * k * scale;
      } else {
        // Re(zeta_fs - p) = ax + ay from (hi, lo) pairs: the hi parts cancel
        // exactly near the pole (Sterbenz), the lo parts restore the rest.
        const T re = ((ax[2 * i] + ay[2 * n]) + (ax[2 * i + 1] + ay[2 * n + 1])) + sh.x;
        C f;
        if (mul != MUL_POLE_FWD) {
          const T d = scale / (re * re + pim * pim);
          f.x = re * d; f.y = -pim * d;
        } else {
          f.x = re * scale; f.y = pim * scale;
        }
        a = cmul(a, f);
      }
      s[n * W + v] = a;
      if constexpr (DY) s[n * W + NV + v] = cmul(a, ik_factor<C>(n, g.ny, g.ky0));
    }
    __syncthreads();
  }
  if (inv) fft_smem<C, NY, true, W, NT, true>(s, g.twy, threadIdx.x);
  C* out = dst.at(u, c, g.npts);
#pragma unroll 8
  for (int e = threadIdx.x; e < NY * NV; e += NT) {
    const int n = e / NV, v = e % NV;
    out[(long)n * g.nx + x0 + v] = s[n * W + v];
  }
  if constexpr (DY) {
    C* o2 = dy.at(u, c, g.npts);
#pragma unroll 8
    for (int e = threadIdx.x; e < NY * NV; e += NT) {
      const int n = e / NV, v = e % NV;
      o2[(long)n * g.nx + x0 + v] = s[n * W + NV + v];
    }
  }
}
template <typename T, int NY, int NV, int NT, bool DY>
__global__ void __launch_bounds__(NT) k_cols(GV<T> g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst,
                                             int mask, int fwd, int mul, int inv, int skip_homog, int pole,
                                             T scale, Buf<typename Cx<T>::t> spec, Buf<typename Cx<T>::t> dy) {
  cols_body<T, NY, NV, NT, DY>(blockIdx.x, blockIdx.y, gridDim.x, g, src, dst, mask, fwd, mul, inv, skip_homog, pole, scale, spec, dy);
}

// The column pass with its tiles moved by TMA: one thread issues the tensor
// loads of the whole NY x NV tile (and of the multiplier tile for MUL_TABLE)
// at entry, so every byte a CTA needs is in flight at once; the result leaves
// by TMA tensor stores.  Same arithmetic as k_cols (no d/dy branch).  Tensor
// maps view a buffer as [items][ny][nx] elements, item = unit * ncomp + c.
// DY: also the d/dy branch (i ky times the multiplied spectrum) into a second
// tile, stored through mdy; it uses the multiplier tile's room (no DY pass
// multiplies by the table).
template <typename T, int NY, int NV, int NT, bool DY>
__device__ __forceinline__ void cols_tma_body(int bx, int by, int gdx, GV<T> g, const CUtensorMap& msrc,
                                                 const CUtensorMap& mdst,
                                                 const CUtensorMap& mtab,
                                                 const CUtensorMap& mdy, int mask, int fwd, int mul,
                                                 int inv, int skip_homog, int pole, T scale,
                                                 Buf<typename Cx<T>::t> spec) {
  pdl_enter();
  using C = typename Cx<T>::t;
  constexpr int EW = sizeof(C) / 8;           // 8-byte words per element (tensor-map element size)
  constexpr int BR = tma_box_rows(NY);        // rows per TMA box
  static_assert(NY % BR == 0 && BR <= 256, "TMA boxes must tile the column");
  extern __shared__ __align__(16) unsigned char smem_tma[];
  // TMA writes shared memory at 128-byte aligned addresses: align the tile at
  // run time (the launch reserves 128 bytes of slack)
  const uint32_t pad = (128u - (smem_u32(smem_tma) & 127u)) & 127u;
  C* s = reinterpret_cast<C*>(smem_tma + pad);
  C* tws = s + NY * NV;                       // twiddles
  C* tab = tws + NY;                          // multiplier tile (MUL_TABLE), or the d/dy tile (DY)
  __shared__ __align__(8) uint64_t bar;
  const int item = item_of(g, (int)by);
  if (item < 0) return;
  const int u = item / g.ncomp, c = item % g.ncomp;
  if (!unit_active(g.st, mask, u)) return;
  if (skip_homog && !g.nonhomog[u / g.P]) return;
  // once any CTA's copy has failed the step is void: issue no further copies, so
  // the CTAs still to come return at once instead of each waiting out its bound
  if (g.err == nullptr || *reinterpret_cast<volatile const int*>(g.err) != 0) return;
  const int x0 = bx * NV;
  // self-check of the TMA alignment rules: 128-byte shared destinations, 64-byte
  // tensor maps, 16-byte x offsets; on a violation record it and do nothing
  if ((smem_u32(s) & 127u) || (smem_u32(tab) & 127u) || (reinterpret_cast<uintptr_t>(&msrc) & 63u) ||
      (reinterpret_cast<uintptr_t>(&mdst) & 63u) || (reinterpret_cast<uintptr_t>(&mtab) & 63u) ||
      (reinterpret_cast<uintptr_t>(&mdy) & 63u) ||
      ((x0 * (int)sizeof(C)) & 15) || ((BR * NV * (int)sizeof(C)) & 127)) {
    if (threadIdx.x == 0) atomicExch(g.err, 2);
    return;
  }
  if (threadIdx.x == 0) { mbar_init(&bar, 1); fence_mbar_init(); }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(&bar, (uint32_t)(NY * NV * sizeof(C) * (mul == MUL_TABLE ? 2 : 1)));
    for (int r = 0; r < NY; r += BR) {
      tma_load_3d(s + r * NV, &msrc, x0 * EW, r, item, &bar);
      if (mul == MUL_TABLE) tma_load_3d(tab + r * NV, &mtab, x0 * EW, r, 0, &bar);
    }
  }
  for (int i = threadIdx.x; i < NY; i += NT) tws[i] = g.twy[i];   // while the tiles are in flight
  // the pole's ky axis table (hi, lo pairs) into shared memory as well
  const bool pmul = (mul == MUL_POLE_INV || mul == MUL_POLE_FWD || mul == MUL_PREC_INV);
  T* ays = reinterpret_cast<T*>(DY ? tab + NY * NV : tab);   // after the d/dy tile, else in the tile's room
  if (pmul) {
    const int k = pole >= 0 ? pole : u % g.P;
    const T* ay = g.ay + (long)k * g.ny * 2;
    for (int i = threadIdx.x; i < 2 * NY; i += NT) ays[i] = ay[i];
  }
  if (!mbar_wait(&bar, 0, g.err)) { mbar_wait(&bar, 0, g.err); return; }
  __syncthreads();
  if (fwd) fft_smem<C, NY, false, NV, NT, true, true>(s, tws, threadIdx.x);
  if (spec.base) {   // keep the 2-D spectrum as well (read again by the pole solves)
    C* sp = spec.at(u, c, g.npts);
#pragma unroll 8
    for (int e = threadIdx.x; e < NY * NV; e += NT) sp[(long)(e / NV) * g.nx + x0 + e % NV] = s[e];
  }
  if (mul != MUL_NONE) {
    const bool pm = (mul == MUL_POLE_INV || mul == MUL_POLE_FWD || mul == MUL_PREC_INV);
    const int k = pm ? (pole >= 0 ? pole : u % g.P) : 0;
    const T* ax = pm ? g.ax + (long)k * g.nx * 2 : nullptr;
    const T* ay = pm ? g.ay + (long)k * g.ny * 2 : nullptr;
    // the preconditioner's pole is p - dbar: Re shifted by +Re dbar, -Im p by +Im dbar
    C sh; sh.x = 0; sh.y = 0;
    if (mul == MUL_PREC_INV) sh = dbar_of(g, u / g.P);
    const T pim = pm ? g.pim[k] + sh.y : (T)0;
    for (int e = threadIdx.x; e < NY * NV; e += NT) {
      const int n = e / NV, v = e % NV, i = x0 + v;
      C a = s[e];
      if (mul == MUL_TABLE) {
        a = cmul(a, tab[e]);
      } else if (mul == MUL_SCALE) {
        a.x *= scale; a.y *= scale;
      } else if (mul == MUL_DY) {
        a = cmul(a, ik_factor<C>(n, g.ny, g.ky0));
        a.x *= scale; a.y *= scale;
      } else if (mul == MUL_DYY) {
        const T kk = (T)ffreq(n, g.ny) * g.ky0;
        a.x *= -kk * kk * scale; a.y *= -kk * kk * scale;
      } else {   // as in k_cols: Re(zeta_fs - p) from (hi, lo) pairs (the ky table from shared memory)
        const T re = ((ax[2 * i] + ays[2 * n]) + (ax[2 * i + 1] + ays[2 * n + 1])) + sh.x;
        C f;
        if (mul != MUL_POLE_FWD) {
          const T d = scale / (re * re + pim * pim);
          f.x = re * d; f.y = -pim * d;
        } else {
          f.x = re * scale; f.y = pim * scale;
        }
        a = cmul(a, f);
      }
      s[e] = a;
      if constexpr (DY) tab[e] = cmul(a, ik_factor<C>(n, g.ny, g.ky0));
    }
    __syncthreads();
  }
  if (inv) {
    fft_smem<C, NY, true, NV, NT, true, true>(s, tws, threadIdx.x);
    if constexpr (DY) fft_smem<C, NY, true, NV, NT, true, true>(tab, tws, threadIdx.x);
  }
  fence_proxy_async_smem();   // this thread's tile writes, before the TMA store reads them
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int r = 0; r < NY; r += BR) {
      tma_store_3d(&mdst, x0 * EW, r, item, s + r * NV);
      if constexpr (DY) tma_store_3d(&mdy, x0 * EW, r, item, tab + r * NV);
    }
    bulk_commit();
    bulk_wait_read();
  }
}
template <typename T, int NY, int NV, int NT, bool DY>
__global__ void __launch_bounds__(NT) k_cols_tma(GV<T> g, const __grid_constant__ CUtensorMap msrc,
                                                 const __grid_constant__ CUtensorMap mdst,
                                                 const __grid_constant__ CUtensorMap mtab,
                                                 const __grid_constant__ CUtensorMap mdy, int mask, int fwd, int mul,
                                                 int inv, int skip_homog, int pole, T scale,
                                                 Buf<typename Cx<T>::t> spec) {
  cols_tma_body<T, NY, NV, NT, DY>(blockIdx.x, blockIdx.y, gridDim.x, g, msrc, mdst, mtab, mdy, mask, fwd, mul, inv, skip_homog, pole, scale, spec);
}

// The column pass by warps (NY = 512 or 1024): a CTA of 8 warps takes 8 adjacent
// columns (64-byte row segments, moved with 8-byte cp.async), one column per
// warp.  A warp loads its column into registers (lane l: rows l + 32 m), and the
// forward column DFT, the Fourier-diagonal multiply and the inverse column DFT
// all run in registers (warp_fft_regs), with the column's own shared memory as
// the transpose scratch.  Element (row n, column v) sits at 9 n + n/32 + v: the
// odd row stride and the skew every 32 rows keep the column reads, the
// transpose writes and the transpose reads free of bank conflicts.  Same
// arithmetic as k_cols for the modes it serves (no spectrum output, no
// multiplier table, no d/dy branch).
constexpr int CW_NV = 8;
template <int NY> __host__ __device__ constexpr int cw_elems() { return 9 * NY + NY / 32 + CW_NV; }
__device__ __forceinline__ int cw_at(int n, int v) { return 9 * n + (n >> 5) + v; }

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// complex FP32 at 512 / 1024: four / three CTAs per SM asked of the compiler (64 / 80
// registers, against 80 / 106 unbounded); FP64 keeps the counts it takes unbounded
template <typename T, int NY>
__global__ void __launch_bounds__(32 * CW_NV, sizeof(T) == 4 ? (NY == 512 ? 4 : 3) : (NY == 512 ? 2 : 1)) k_cols_warp(GV<T> g, Buf<typename Cx<T>::t> src,
                                                        Buf<typename Cx<T>::t> dst, int mask, int fwd, int mul,
                                                        int inv, int skip_homog, int pole, T scale) {
  pdl_enter();
  using C = typename Cx<T>::t;
  constexpr int NT = 32 * CW_NV, L = NY / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  const int item = item_of(g, (int)blockIdx.y);
  if (item < 0) return;
  const int u = item / g.ncomp, c = item % g.ncomp;
  if (!unit_active(g.st, mask, u)) return;
  if (skip_homog && !g.nonhomog[u / g.P]) return;
  const int x0 = blockIdx.x * CW_NV;
  const C* in = src.at(u, c, g.npts) + x0;
#pragma unroll 8
  for (int e = threadIdx.x; e < NY * CW_NV; e += NT) {
    const int n = e / CW_NV, v = e % CW_NV;
    if constexpr (sizeof(C) == 8) cp_async8(s + cw_at(n, v), in + (long)n * g.nx + v);
    else cp_async16(s + cw_at(n, v), in + (long)n * g.nx + v);
  }
  cp_async_wait_all();
  __syncthreads();
  const int v = threadIdx.x >> 5, lane = threadIdx.x & 31, i = x0 + v;
  auto slot = [&](int q) { return s + cw_at(q, v); };
  C x[L];
#pragma unroll
  for (int m = 0; m < L; ++m) x[m] = *slot(lane + 32 * m);
  if (fwd) warp_fft_regs<C, NY, false>(x, g.twy, lane, slot);
  if (mul != MUL_NONE) {
    const bool pm = (mul == MUL_POLE_INV || mul == MUL_POLE_FWD || mul == MUL_PREC_INV);
    const int k = pm ? (pole >= 0 ? pole : u % g.P) : 0;
    C sh; sh.x = 0; sh.y = 0;
    if (mul == MUL_PREC_INV) sh = dbar_of(g, u / g.P);
    T axh = 0, axl = 0, pim = 0;
    const T* ay = nullptr;
    if (pm) {
      axh = g.ax[((long)k * g.nx + i) * 2];
      axl = g.ax[((long)k * g.nx + i) * 2 + 1];
      ay = g.ay + (long)k * g.ny * 2;
      pim = g.pim[k] + sh.y;
    }
#pragma unroll
    for (int m = 0; m < L; ++m) {
      const int n = lane + 32 * m;
      C a = x[m];
      if (mul == MUL_SCALE) {
        a.x *= scale; a.y *= scale;
      } else if (mul == MUL_DY) {
        a = cmul(a, ik_factor<C>(n, g.ny, g.ky0));
        a.x *= scale; a.y *= scale;
      } else if (mul == MUL_DYY) {
        const T kk = (T)ffreq(n, g.ny) * g.ky0;
        a.x *= -kk * kk * scale; a.y *= -kk * kk * scale;
      } else {   // Re(zeta_fs - p) from (hi, lo) pairs, as in k_cols
        const T re = ((axh + __ldg(&ay[2 * n])) + (axl + __ldg(&ay[2 * n + 1]))) + sh.x;
        C f;
        if (mul != MUL_POLE_FWD) {
          const T d = scale / (re * re + pim * pim);
          f.x = re * d; f.y = -pim * d;
        } else {
          f.x = re * scale; f.y = pim * scale;
        }
        a = cmul(a, f);
      }
      x[m] = a;
    }
  }
  if (inv) warp_fft_regs<C, NY, true>(x, g.twy, lane, slot);
#pragma unroll
  for (int m = 0; m < L; ++m) *slot(lane + 32 * m) = x[m];
  __syncthreads();
  C* out = dst.at(u, c, g.npts) + x0;
#pragma unroll 8
  for (int e = threadIdx.x; e < NY * CW_NV; e += NT) {
    const int n = e / CW_NV, vv = e % CW_NV;
    out[(long)n * g.nx + vv] = s[cw_at(n, vv)];
  }
}

// ---------------------------------------------------------------------------
// Pass 3: inverse row DFTs and the pointwise epilogue.  grid = (ny/NR, units*ncomp).
// ---------------------------------------------------------------------------
struct EpiArgs {
  int mode;
  int jj;              // Arnoldi column (EPI_ARNOLDI)
  const double2* in64; // EPI_OPERATOR input
  double2* out64;      // EPI_STORE64 / EPI_OPERATOR output
  const void* aux;     // vector operator: (Z - Z_fs) applied to the same field, complex T
  int kxsel;           // before the inverse row DFT multiply by 1 (0), i kx (1) or -kx^2 (2)
  void* fwd_out;       // EPI_ACCUM64: also write the forward row DFT of the new field (next step's pass 1)
};

// ARN: the instantiation for the EPI_ARNOLDI epilogue (kept apart so that the
// other epilogues do not carry its register footprint).
template <typename T, int N, int NR, int NT, bool ARN, bool WF>
__device__ __forceinline__ void rows_inv_body(int bx, int by, int gdx, GV<T> g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst,
                                                 int mask, int skip_homog, EpiArgs ep) {
  pdl_enter();
  using C = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[32];
  const int item = item_of(g, (int)by);
  if (item < 0) return;
  const int u = item / g.ncomp, c = item % g.ncomp;
  if (!unit_active(g.st, mask, u)) return;
  const bool sys = (ep.mode == EPI_R0 || ep.mode == EPI_ARNOLDI || ep.mode == EPI_TRUERES || ep.mode == EPI_ADD_E);
  const int beam = sys ? u / g.P : u;
  if (skip_homog && !g.nonhomog[beam]) return;
  const int row0 = bx * NR;
  const long off = (long)row0 * N;
  const C* in = src.at(u, c, g.npts) + off;
  if (ep.mode == EPI_ACCUM64) {   // the old field is read after the inverse DFT: start its DRAM fetch now
    const long uo = ((long)u * g.ncomp + c) * g.npts + off;
    const char* w0 = reinterpret_cast<const char*>(g.W64);
    if constexpr (sizeof(T) == 4) {
      const long plane = (long)g.nb * g.ncomp * g.npts * 8;
      for (int e = threadIdx.x * 16; e < NR * N; e += NT * 16) {
        prefetch_l2(w0 + (uo + e) * 8);
        prefetch_l2(w0 + plane + (uo + e) * 8);
      }
    } else {
      for (int e = threadIdx.x * 8; e < NR * N; e += NT * 8) prefetch_l2(w0 + (uo + e) * 16);
    }
  }
  if constexpr (ARN) {   // v_j and delta are read after the inverse DFT: start their DRAM fetch now
    const long vj = (((long)u * (g.m + 2) + ep.jj) * g.ncomp + c) * g.npts + off;
    const char* pv = reinterpret_cast<const char*>(g.V + vj);
    const char* pd = reinterpret_cast<const char*>(g.delta + (long)beam * g.npts + off);
    for (int b = threadIdx.x * 128; b < NR * N * (int)sizeof(C); b += NT * 128) {
      prefetch_l2(pv + b);
      prefetch_l2(pd + b);
    }
  }
  const bool in16 = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
  if (sizeof(T) == 4 && in16) {   // 16-byte loads: two points (same row, N even) per access
#pragma unroll
    for (int e2 = threadIdx.x; e2 < NR * N / 2; e2 += NT) {
      const float4 q = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(in))[e2];
      const int e = 2 * e2;
      C a, b;
      a.x = (T)q.x; a.y = (T)q.y; b.x = (T)q.z; b.y = (T)q.w;
      if (ep.kxsel == 1) { a = cmul(a, ik_factor<C>(e % N, N, g.kx0)); b = cmul(b, ik_factor<C>((e + 1) % N, N, g.kx0)); }
      else if (ep.kxsel == 2) {
        const T k0 = (T)ffreq(e % N, N) * g.kx0, k1 = (T)ffreq((e + 1) % N, N) * g.kx0;
        a.x *= -k0 * k0; a.y *= -k0 * k0; b.x *= -k1 * k1; b.y *= -k1 * k1;
      }
      s[sidx<N, NR, false>(e / N, e % N)] = a;
      s[sidx<N, NR, false>(e / N, e % N + 1)] = b;
    }
  } else {
#pragma unroll
    for (int e = threadIdx.x; e < NR * N; e += NT) {
      C a = in[e];
      if (ep.kxsel == 1) a = cmul(a, ik_factor<C>(e % N, N, g.kx0));
      else if (ep.kxsel == 2) { const T k = (T)ffreq(e % N, N) * g.kx0; a.x *= -k * k; a.y *= -k * k; }
      s[sidx<N, NR, false>(e / N, e % N)] = a;
    }
  }
  __syncthreads();
  fft_rows<C, N, true, NR, NT, WF>(s, g.twx, threadIdx.x);
  const C* dl = g.delta + (long)beam * g.npts + off;
  const long unit_off = ((long)u * g.ncomp + c) * g.npts + off;   // [unit][c][pt] arrays
  if constexpr (ARN) {
    // Arnoldi step: u = v_j (the candidate left by the last update pass),
    // z = M^-1 u from this transform with M = Z_fs + dbar - p, and
    // w = (Z - p) z = u + (delta - dbar) z stored as v_{j+1}; the inner products
    // follow in k_dcgs_gram.
    const long vj = (((long)u * (g.m + 2) + ep.jj) * g.ncomp + c) * g.npts + off;
    C* wout = g.V + vj + (long)g.ncomp * g.npts;
    const C db = dbar_of(g, beam);
#pragma unroll
    for (int e2 = threadIdx.x; e2 < NR * N / 2; e2 += NT) {   // pairs: 16-byte accesses in FP32
      const int e = 2 * e2;
      C v0, v1, d0, d1, w0, w1;
      ld2(g.V + vj, e, v0, v1);
      ld2(dl, e, d0, d1);
      d0.x -= db.x; d0.y -= db.y; d1.x -= db.x; d1.y -= db.y;
      const C z0 = cmul(d0, s[sidx<N, NR, false>(e / N, e % N)]), z1 = cmul(d1, s[sidx<N, NR, false>(e / N, e % N + 1)]);
      w0.x = v0.x + z0.x; w0.y = v0.y + z0.y; w1.x = v1.x + z1.x; w1.y = v1.y + z1.y;
      st2(wout, e, w0, w1);
    }
  } else {
  // per-thread partial sums in T (FP64 arithmetic per point is scarce on this GPU),
  // summed in FP64 across the block below
  T acc = 0, acc2 = 0, accr = 0, acci = 0;
  bool acc16 = false;   // the FP32 accumulate ran vectorised below
  if constexpr (sizeof(T) == 4) {
    const long plane = (long)g.nb * g.ncomp * g.npts;
    acc16 = ep.mode == EPI_ACCUM64 &&
            ((reinterpret_cast<uintptr_t>(reinterpret_cast<const float2*>(g.W64) + unit_off) |
              reinterpret_cast<uintptr_t>(reinterpret_cast<const float2*>(g.W64) + plane + unit_off) |
              reinterpret_cast<uintptr_t>(reinterpret_cast<float2*>(ep.out64) + unit_off) |
              reinterpret_cast<uintptr_t>(reinterpret_cast<float2*>(ep.out64) + plane + unit_off)) & 15) == 0;
    if (acc16) {   // double-float accumulate with 16-byte accesses (two points each)
      const float4* ohi = reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(g.W64) + unit_off);
      const float4* olo = reinterpret_cast<const float4*>(reinterpret_cast<const float2*>(g.W64) + plane + unit_off);
      float4* nhi = reinterpret_cast<float4*>(reinterpret_cast<float2*>(ep.out64) + unit_off);
      float4* nlo = reinterpret_cast<float4*>(reinterpret_cast<float2*>(ep.out64) + plane + unit_off);
      for (int e2 = threadIdx.x; e2 < NR * N / 2; e2 += NT) {
        const int e = 2 * e2, i0 = sidx<N, NR, false>(e / N, e % N), i1 = sidx<N, NR, false>(e / N, e % N + 1);
        const C v0 = s[i0], v1 = s[i1];
        float4 h = ohi[e2], l = olo[e2];
        df_add(h.x, l.x, v0.x); df_add(h.y, l.y, v0.y);
        df_add(h.z, l.z, v1.x); df_add(h.w, l.w, v1.y);
        nhi[e2] = h; nlo[e2] = l;
        if (ep.fwd_out) { s[i0] = make_float2(h.x, h.y); s[i1] = make_float2(h.z, h.w); }
      }
    }
  }
  for (int e = threadIdx.x; e < NR * N; e += NT) {
    if (acc16) break;   // done above
    const C val = s[sidx<N, NR, false>(e / N, e % N)];
    switch (ep.mode) {
      case EPI_STORE: dst.at(u, c, g.npts)[off + e] = val; break;
      case EPI_STORE64: ep.out64[unit_off + e] = to_d(val); break;
      case EPI_ACCUM64: {   // new field = old field + val, written beside the old one
        C nw;
        if constexpr (sizeof(T) == 4) {
          const long plane = (long)g.nb * g.ncomp * g.npts;
          const float2* ohi = reinterpret_cast<const float2*>(g.W64);
          float2* nhi = reinterpret_cast<float2*>(ep.out64);
          float2 h = ohi[unit_off + e], l = ohi[plane + unit_off + e];
          df_add(h.x, l.x, val.x);
          df_add(h.y, l.y, val.y);
          nhi[unit_off + e] = h;
          nhi[plane + unit_off + e] = l;
          nw = h;
        } else {
          double2 t = g.W64[unit_off + e];
          t.x += (double)val.x; t.y += (double)val.y;
          ep.out64[unit_off + e] = t;
          nw = t;
        }
        if (ep.fwd_out) s[sidx<N, NR, false>(e / N, e % N)] = nw;   // same element, same thread
      } break;
      case EPI_OPERATOR: {
        double2 o;
        if (g.ncomp == 2) {   // Z_fs v (this pass) + (Z - Z_fs) v (computed before into aux)
          const double2 a = to_d(reinterpret_cast<const C*>(ep.aux)[unit_off + e]);
          o.x = (double)val.x + a.x; o.y = (double)val.y + a.y;
        } else {
          const double2 v = ep.in64[unit_off + e];
          const double2 d = to_d(dl[e]);
          o.x = (double)val.x + d.x * v.x - d.y * v.y;
          o.y = (double)val.y + d.x * v.y + d.y * v.x;
        }
        ep.out64[unit_off + e] = o;
      } break;
      case EPI_ADD_E: {   // e += M^-1 V y, accumulated in FP64; ||e||^2 for the backward-error test
        double2 a = g.E[unit_off + e];
        a.x += (double)val.x; a.y += (double)val.y;
        g.E[unit_off + e] = a;
        const T ax = (T)a.x, ay = (T)a.y;
        acc += ax * ax + ay * ay;
      } break;
      case EPI_R0: {
        const C r = cmul(dl[e], val);
        C m; m.x = -r.x; m.y = -r.y;
        g.R0[unit_off + e] = m;
        acc += m.x * m.x + m.y * m.y;
        acc2 += val.x * val.x + val.y * val.y;
      } break;
      case EPI_TRUERES: {   // r = R0 - (Z - p) e in T: the same precision as the transform that formed val
        const C r0 = g.R0[unit_off + e];
        const long vb = (((long)u * (g.m + 2)) * g.ncomp + c) * g.npts + off + e;
        C r;
        if (g.ncomp == 2) {   // (Z - Z_fs) e was written into v_0 by the preceding pass
          const C a = g.V[vb];
          r.x = r0.x - val.x - a.x;
          r.y = r0.y - val.y - a.y;
        } else {
          const C ee = to_c(g.E[unit_off + e], T());
          const C de = cmul(dl[e], ee);
          r.x = r0.x - val.x - de.x;
          r.y = r0.y - val.y - de.y;
        }
        g.V[vb] = r;
        acc += r.x * r.x + r.y * r.y;
        accr += r0.x * r.x + r0.y * r.y;      // <R0, r> = sum conj(R0) r
        acci += r0.x * r.y - r0.y * r.x;
      } break;
    }
  }
  if (ep.mode == EPI_ACCUM64 && ep.fwd_out) {   // forward row DFT of the new field for the next step
    __syncthreads();
    fft_rows<C, N, false, NR, NT, WF>(s, g.twx, threadIdx.x);
    C* o = reinterpret_cast<C*>(ep.fwd_out) + unit_off;
    if (sizeof(T) == 4 && (reinterpret_cast<uintptr_t>(o) & 15) == 0) {
      for (int e2 = threadIdx.x; e2 < NR * N / 2; e2 += NT) {
        const int e = 2 * e2;
        const C a = s[sidx<N, NR, false>(e / N, e % N)], b = s[sidx<N, NR, false>(e / N, e % N + 1)];
        reinterpret_cast<float4*>(reinterpret_cast<float*>(o))[e2] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
      }
    } else {
#pragma unroll
      for (int e = threadIdx.x; e < NR * N; e += NT) o[e] = s[sidx<N, NR, false>(e / N, e % N)];
    }
  }
  if (ep.mode == EPI_R0 || ep.mode == EPI_TRUERES) {
    const double t = block_sum((double)acc, red);
    if (threadIdx.x == 0) atomicAdd(&g.st[u].nrm_a, t);
  }
  if (ep.mode == EPI_R0) {
    const double t = block_sum((double)acc2, red);
    if (threadIdx.x == 0) atomicAdd(&g.st[u].z0norm2, t);
  }
  if (ep.mode == EPI_ADD_E) {
    const double t = block_sum((double)acc, red);
    if (threadIdx.x == 0) atomicAdd(&g.st[u].enorm2, t);
  }
  if (ep.mode == EPI_TRUERES) {
    const double tr = block_sum((double)accr, red);
    const double ti = block_sum((double)acci, red);
    if (threadIdx.x == 0) { atomicAdd(&g.st[u].r0r.x, tr); atomicAdd(&g.st[u].r0r.y, ti); }
  }
  }
}
template <typename T, int N, int NR, int NT, bool ARN, bool WF>
__global__ void __launch_bounds__(NT) k_rows_inv(GV<T> g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst,
                                                 int mask, int skip_homog, EpiArgs ep) {
  rows_inv_body<T, N, NR, NT, ARN, WF>(blockIdx.x, blockIdx.y, gridDim.x, g, src, dst, mask, skip_homog, ep);
}
template <typename T, int N, int NR, int NT, bool ARN, bool WF>
__global__ void __launch_bounds__(NT, WROWS_MINB) k_rows_inv_w(GV<T> g, Buf<typename Cx<T>::t> src,
                                                                    Buf<typename Cx<T>::t> dst, int mask,
                                                                    int skip_homog, EpiArgs ep) {
  rows_inv_body<T, N, NR, NT, ARN, WF>(blockIdx.x, blockIdx.y, gridDim.x, g, src, dst, mask, skip_homog, ep);
}


// ---------------------------------------------------------------------------
// Pass 3 of the vector operator (ncomp = 2), Eq. (Z_bar_eq).  A unit's two
// components arrive as column-pass outputs A_c = colIDFT(m x_hat_c) and
// B_c = colIDFT(i ky m x_hat_c).  Six inverse row DFTs in one shared-memory
// transform give z_c, d_x z_c (from i kx A_c) and d_y z_c (from B_c); the
// epilogue applies the psi and delta terms:
//   ((Z - Z_fs) z)_1 = D1 z1 + X z2 + px d_x z1 + py d_x z2
//   ((Z - Z_fs) z)_2 = X z1 + D2 z2 + px d_y z1 + py d_y z2
// grid = (ny/NR, units).
// ---------------------------------------------------------------------------
enum VecEpi { VEPI_ARNOLDI = 0, VEPI_R0 = 1, VEPI_OPDIFF = 2 };

template <typename T, int N, int NR, int NT>
__device__ __forceinline__ void rows_inv_vec_body(int bx, int by, int gdx, GV<T> g, Buf<typename Cx<T>::t> A, Buf<typename Cx<T>::t> B,
                                                     Buf<typename Cx<T>::t> out, int mask, int skip_homog,
                                                     int mode, int jj) {
  pdl_enter();
  using C = typename Cx<T>::t;
  constexpr int NVV = 6 * NR;                 // vectors: (c, {z, dx, dy}) x NR rows
  constexpr int TPT = NR * N / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* s = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[32];
  const int u = unit_of(g, (int)by);
  if (u < 0 || !unit_active(g.st, mask, u)) return;
  const int beam = (mode == VEPI_OPDIFF && mask < 0) ? u : u / g.P;
  if (skip_homog && !g.nonhomog[beam]) return;
  const int row0 = bx * NR;
  const long off = (long)row0 * N;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const C* a = A.at(u, c, g.npts) + off;
    const C* b = B.at(u, c, g.npts) + off;
    for (int e2 = threadIdx.x; e2 < NR * N / 2; e2 += NT) {   // point pairs: 16-byte accesses in FP32
      const int e = 2 * e2, r = e / N, n = e % N;
      C x[2], y[2];
      ld2(a, e, x[0], x[1]);
      ld2(b, e, y[0], y[1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        s[sidx<N, NVV, false>((c * 3 + 0) * NR + r, n + h)] = x[h];
        s[sidx<N, NVV, false>((c * 3 + 1) * NR + r, n + h)] = cmul(x[h], ik_factor<C>(n + h, N, g.kx0));
        s[sidx<N, NVV, false>((c * 3 + 2) * NR + r, n + h)] = y[h];
      }
    }
  }
  __syncthreads();
  fft_rows<C, N, true, NVV, NT>(s, g.twx, threadIdx.x);
  const C* cf = g.psi + (long)beam * 5 * g.npts + off;    // D1, D2, X, px, py planes
  const long F = 2 * g.npts;
  T acc = 0, acc2 = 0;   // per-thread partials in T, FP64 across the block
  for (int e2 = threadIdx.x; e2 < NR * N / 2; e2 += NT) {   // point pairs: 16-byte accesses in FP32
    const int e = 2 * e2, r = e / N, n0 = e % N;
    C cD1[2], cD2[2], cX[2], cpx[2], cpy[2], d1v[2], d2v[2], z1v[2], z2v[2];
    ld2(cf, e, cD1[0], cD1[1]);
    ld2(cf + g.npts, e, cD2[0], cD2[1]);
    ld2(cf + 2 * g.npts, e, cX[0], cX[1]);
    ld2(cf + 3 * g.npts, e, cpx[0], cpx[1]);
    ld2(cf + 4 * g.npts, e, cpy[0], cpy[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0 + h;
      const C z1 = s[sidx<N, NVV, false>(0 * NR + r, n)], x1 = s[sidx<N, NVV, false>(1 * NR + r, n)],
              y1 = s[sidx<N, NVV, false>(2 * NR + r, n)];
      const C z2 = s[sidx<N, NVV, false>(3 * NR + r, n)], x2 = s[sidx<N, NVV, false>(4 * NR + r, n)],
              y2 = s[sidx<N, NVV, false>(5 * NR + r, n)];
      const C D1 = cD1[h], D2 = cD2[h], X = cX[h], px = cpx[h], py = cpy[h];
      C d1 = cmul(D1, z1), d2 = cmul(X, z1), t;
      t = cmul(X, z2);  d1.x += t.x; d1.y += t.y;
      t = cmul(px, x1); d1.x += t.x; d1.y += t.y;
      t = cmul(py, x2); d1.x += t.x; d1.y += t.y;
      t = cmul(D2, z2); d2.x += t.x; d2.y += t.y;
      t = cmul(px, y1); d2.x += t.x; d2.y += t.y;
      t = cmul(py, y2); d2.x += t.x; d2.y += t.y;
      d1v[h] = d1; d2v[h] = d2; z1v[h] = z1; z2v[h] = z2;
    }
    if (mode == VEPI_ARNOLDI) {   // w = u + (Z - Z_fs - dbar) z, z = M^-1 u, stored as v_{j+1}
      const long vj = ((long)u * (g.m + 2) + jj) * F + off;
      const C db = dbar_of(g, beam);
      C v1[2], v2[2], w1[2], w2[2];
      ld2(g.V + vj, e, v1[0], v1[1]);
      ld2(g.V + vj + g.npts, e, v2[0], v2[1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const C t1 = cmul(db, z1v[h]), t2 = cmul(db, z2v[h]);
        w1[h].x = v1[h].x + d1v[h].x - t1.x; w1[h].y = v1[h].y + d1v[h].y - t1.y;
        w2[h].x = v2[h].x + d2v[h].x - t2.x; w2[h].y = v2[h].y + d2v[h].y - t2.y;
      }
      st2(g.V + vj + F, e, w1[0], w1[1]);
      st2(g.V + vj + F + g.npts, e, w2[0], w2[1]);
    } else if (mode == VEPI_R0) {
      const long rb = (long)u * F + off;
      C m1[2], m2[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        m1[h].x = -d1v[h].x; m1[h].y = -d1v[h].y; m2[h].x = -d2v[h].x; m2[h].y = -d2v[h].y;
        acc += m1[h].x * m1[h].x + m1[h].y * m1[h].y + m2[h].x * m2[h].x + m2[h].y * m2[h].y;
        acc2 += z1v[h].x * z1v[h].x + z1v[h].y * z1v[h].y + z2v[h].x * z2v[h].x + z2v[h].y * z2v[h].y;
      }
      st2(g.R0 + rb, e, m1[0], m1[1]);
      st2(g.R0 + rb + g.npts, e, m2[0], m2[1]);
    } else {
      st2(out.at(u, 0, g.npts) + off, e, d1v[0], d1v[1]);
      st2(out.at(u, 1, g.npts) + off, e, d2v[0], d2v[1]);
    }
  }
  if (mode == VEPI_R0) {
    const double t = block_sum((double)acc, red);
    if (threadIdx.x == 0) atomicAdd(&g.st[u].nrm_a, t);
    const double t2 = block_sum((double)acc2, red);
    if (threadIdx.x == 0) atomicAdd(&g.st[u].z0norm2, t2);
  }
}
template <typename T, int N, int NR, int NT>
__global__ void __launch_bounds__(NT) k_rows_inv_vec(GV<T> g, Buf<typename Cx<T>::t> A, Buf<typename Cx<T>::t> B,
                                                     Buf<typename Cx<T>::t> out, int mask, int skip_homog,
                                                     int mode, int jj) {
  rows_inv_vec_body<T, N, NR, NT>(blockIdx.x, blockIdx.y, gridDim.x, g, A, B, out, mask, skip_homog, mode, jj);
}
// Complex FP32: three CTAs per SM asked of the compiler (80 registers, small
// spills; 4.5 % faster than the two that 128 registers allow).  (An explicit
// bound of 1 is not the same as none: ptxas then spends registers freely.)
template <typename T, int N, int NR, int NT>
__global__ void __launch_bounds__(NT, 3) k_rows_inv_vec_occ(GV<T> g, Buf<typename Cx<T>::t> A,
                                                            Buf<typename Cx<T>::t> B, Buf<typename Cx<T>::t> out,
                                                            int mask, int skip_homog, int mode, int jj) {
  rows_inv_vec_body<T, N, NR, NT>(blockIdx.x, blockIdx.y, gridDim.x, g, A, B, out, mask, skip_homog, mode, jj);
}

// psi coefficient planes, after psit_xx, psit_yy, psit_xy, psit_x, psit_y have
// been written into planes 0..4: planes 0, 1 become delta + psit_xx, delta + psit_yy.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_psi_combine(GV<T> g, int beam) {
  using C = typename Cx<T>::t;
  C* pl = g.psi + (long)beam * 5 * g.npts;
  const C* d = g.delta + (long)beam * g.npts;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < g.npts; p += (long)gridDim.x * NT) {
    const C a = d[p];
    C x = pl[p], y = pl[g.npts + p];
    x.x += a.x; x.y += a.y; y.x += a.x; y.y += a.y;
    pl[p] = x; pl[g.npts + p] = y;
  }
}

// ---------------------------------------------------------------------------
// Batched Krylov vector kernels.  grid = (chunks, systems): a CTA works on
// contiguous chunks of its system's ncomp*npts points (the Gram and update
// sweeps loop over several chunks; the grid rows may come from the unit list).
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ typename Cx<T>::t* vslot(const GV<T>& g, int s, int jj) {
  return g.V + ((long)s * (g.m + 2) + jj) * g.ncomp * g.npts;
}


// Sum each of V per-lane values (V a power of two <= 32) over the warp: on
// return v[0] of lane l holds the warp total of value l % V.  A butterfly halves
// the live values at each of its first log2 V levels (lane pairs exchange the
// halves they do not keep), then plain xor steps finish the sum: V - 1 + (5 -
// log2 V) shuffles in all.
template <int V, typename A> __device__ __forceinline__ void warp_transpose_reduce(A (&v)[V]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = V / 2; k >= 1; k >>= 1) {
    const bool up = (lane & k) != 0;
#pragma unroll
    for (int i = 0; i < k; ++i) {
      const A send = up ? v[i] : v[i + k];
      const A keep = up ? v[i + k] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, k);
    }
  }
#pragma unroll
  for (int o = V; o < 32; o <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}

// The inner products of iteration j of the delayed re-orthogonalisation (see
// the scheme before dcgs_control): b_i = <v_i, w>, a_i = <v_i, u> (i < j), d = <u, w>, c = <u, u>
// and ||w||^2, with u = v_j and w = v_{j+1} (w = 0 when with_w = 0: the last
// step of a cycle needs only the products with u), for every iterating system.  Each
// thread keeps EPT points of u and w in registers and takes the basis in
// groups of GVEC vectors (GVEC*EPT loads in flight); a group's 4 GVEC partial
// sums leave the warp in one transpose-reduce.  CTAs loop over chunks (about
// one wave of them); per-warp totals are kept in FP64, summed and
// added to the striped accumulators (planes 2 (j % 2) + 0, 1; slot MMAX of the
// second takes ||w||^2).
template <typename T, int NT, int EPT, int GVEC>
__device__ __forceinline__ void dcgs_gram_body(int bx, int by, int gdx, GV<T> g, int jj, int with_w) {
  pdl_enter();
  using C = typename Cx<T>::t;
  constexpr int NW = NT / 32;
  __shared__ double red[NW][4 * (MMAX + 1)];
  const int s = unit_of(g, (int)by);
  if (s < 0 || g.st[s].state != ST_ITER) return;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long L = (long)g.ncomp * g.npts;
  const C* up = vslot(g, s, jj);
  const C* wpv = vslot(g, s, jj + 1);
  for (int t = lane; t < 4 * (jj + 1); t += 32) red[wp][t] = 0.0;   // each warp owns its row
  const long nchunks = (L + NT * EPT - 1) / (NT * EPT);
  for (long chunk = bx; chunk < nchunks; chunk += gdx) {   // persistent over chunks
  const long b0 = chunk * NT * EPT + threadIdx.x;
  C uv[EPT], wv[EPT];
  T uwr = 0, uwi = 0, uu = 0, ww = 0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const long p = b0 + (long)e * NT;
    uv[e] = C{}; wv[e] = C{};
    if (p < L) { uv[e] = up[p]; if (with_w) wv[e] = wpv[p]; }
    uwr += uv[e].x * wv[e].x + uv[e].y * wv[e].y; uwi += uv[e].x * wv[e].y - uv[e].y * wv[e].x;
    uu += uv[e].x * uv[e].x + uv[e].y * uv[e].y;
    ww += wv[e].x * wv[e].x + wv[e].y * wv[e].y;
  }
  for (int g0 = 0; g0 <= jj; g0 += GVEC) {   // slots g0..g0+GVEC-1; slot jj carries (d, c, ||w||^2)
    C vv[GVEC][EPT];
#pragma unroll
    for (int k = 0; k < GVEC; ++k) {
      const C* vi = vslot(g, s, g0 + k);
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const long p = b0 + (long)e * NT;
        vv[k][e] = (g0 + k < jj && p < L) ? vi[p] : C{};
      }
    }
    T acc[4 * GVEC];
#pragma unroll
    for (int k = 0; k < GVEC; ++k) {
      T br = 0, bi = 0, ar = 0, ai = 0;
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const C a = vv[k][e], w = wv[e], x = uv[e];
        br += a.x * w.x + a.y * w.y; bi += a.x * w.y - a.y * w.x;
        ar += a.x * x.x + a.y * x.y; ai += a.x * x.y - a.y * x.x;
      }
      if (g0 + k == jj) { br = uwr; bi = uwi; ar = uu; ai = ww; }
      acc[4 * k] = br; acc[4 * k + 1] = bi; acc[4 * k + 2] = ar; acc[4 * k + 3] = ai;
    }
    warp_transpose_reduce<4 * GVEC>(acc);
    if (lane < 4 * GVEC && g0 + (lane >> 2) <= jj) red[wp][4 * g0 + lane] += (double)acc[0];
  }
  }
  __syncthreads();
  double2* pb = part_at(g.part, s, 2 * (jj & 1), bx % NSTRIPE, 0);
  double2* pa = part_at(g.part, s, 2 * (jj & 1) + 1, bx % NSTRIPE, 0);
  for (int t = threadIdx.x; t < 4 * (jj + 1); t += NT) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) v += red[w][t];
    const int i = t >> 2, comp = t & 3;
    if (comp == 0) atomicAdd(&pb[i].x, v);
    else if (comp == 1) atomicAdd(&pb[i].y, v);
    else if (comp == 2) atomicAdd(&pa[i].x, v);
    else if (i < jj) atomicAdd(&pa[i].y, v);
    else atomicAdd(&pa[MMAX].x, v);   // ||w||^2
  }
}
template <typename T, int NT, int EPT, int GVEC>
__global__ void __launch_bounds__(NT) k_dcgs_gram(GV<T> g, int jj, int with_w) {
  dcgs_gram_body<T, NT, EPT, GVEC>(blockIdx.x, blockIdx.y, gridDim.x, g, jj, with_w);
}

// v_0 *= scale (start of a cycle)
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_scale_v0(GV<T> g) {
  pdl_enter();
  using C = typename Cx<T>::t;
  const int s = blockIdx.y;
  if (g.st[s].state != ST_ITER || g.st[s].j != 0) return;
  const T sc = (T)g.st[s].scale;
  const long L = (long)g.ncomp * g.npts;
  C* w = vslot(g, s, 0);
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < L; p += (long)gridDim.x * NT) {
    C x = w[p]; x.x *= sc; x.y *= sc; w[p] = x;
  }
  if (blockIdx.x == 0)   // the cycle's Gram accumulators start from zero
    for (int i = threadIdx.x; i < NPLANE * NSTRIPE * (MMAX + 1); i += NT) part_at(g.part, s, 0, 0, 0)[i] = make_double2(0.0, 0.0);
}

// v_0 = R0 and E = 0 for the systems that start iterating (the others keep E unused).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_init_systems(GV<T> g) {
  pdl_enter();
  const int s = blockIdx.y;
  if (g.st[s].state != ST_ITER) return;
  const long L = (long)g.ncomp * g.npts;
  auto* v = vslot(g, s, 0);
  const auto* r = g.R0 + (long)s * L;
  double2* e = g.E + (long)s * L;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < L; p += (long)gridDim.x * NT) {
    v[p] = r[p];
    e[p] = make_double2(0.0, 0.0);
  }
}

// Cycle end, first half of e += M^-1 V y: Tmp = sum_{i < jend} y_i v_i for the
// systems at a cycle end (the free-space solve and the FP64 accumulation into E
// follow as an FFT round trip with the EPI_ADD_E epilogue).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_combine(GV<T> g) {
  pdl_enter();
  using C = typename Cx<T>::t;
  __shared__ C ys[MMAX];
  const int s = blockIdx.y;
  const SysState& st = g.st[s];
  if (st.state != ST_CYCLE_END) return;
  const int J = st.jend;
  for (int i = threadIdx.x; i < J; i += NT) { ys[i].x = (T)st.y[i].x; ys[i].y = (T)st.y[i].y; }
  __syncthreads();
  const long L = (long)g.ncomp * g.npts;
  C* t = g.Tmp + (long)s * L;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < L; p += (long)gridDim.x * NT) {
    C inc; inc.x = 0; inc.y = 0;
    #pragma unroll 4
    for (int i = 0; i < J; ++i) {
      const C a = cmul(ys[i], vslot(g, s, i)[p]);
      inc.x += a.x; inc.y += a.y;
    }
    t[p] = inc;
  }
}

// Wn[b] += sum_k r_k E[b, k]  (the residue sum of Eq. approx_prop, correction part).
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_residue_sum(GV<T> g, double2* Wn) {
  pdl_enter();
  const int b = blockIdx.y;
  const long L = (long)g.ncomp * g.npts;
  const long plane = (long)g.nb * L;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < L; p += (long)gridDim.x * NT) {
    double2 a;
    if constexpr (sizeof(T) == 4) {
      const float2* wh = reinterpret_cast<const float2*>(Wn);
      const float2 h = wh[(long)b * L + p], l = wh[plane + (long)b * L + p];
      a.x = (double)h.x + (double)l.x; a.y = (double)h.y + (double)l.y;
    } else {
      a = Wn[(long)b * L + p];
    }
    for (int k = 0; k < g.P; ++k) {
      if (!g.st[b * g.P + k].used) continue;
      const double2 e = g.E[((long)b * g.P + k) * L + p];
      const double2 r = g.rk[k];
      a.x += r.x * e.x - r.y * e.y;
      a.y += r.x * e.y + r.y * e.x;
    }
    if constexpr (sizeof(T) == 4) {
      float2* wh = reinterpret_cast<float2*>(Wn);
      float2 h, l;
      h.x = (float)a.x; h.y = (float)a.y;
      l.x = (float)(a.x - (double)h.x); l.y = (float)(a.y - (double)h.y);
      wh[(long)b * L + p] = h;
      wh[plane + (long)b * L + p] = l;
    } else {
      Wn[(long)b * L + p] = a;
    }
  }
}

// Field <-> complex128 staging: FP32 path splits into / joins from the
// double-float planes; FP64 path copies.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_field_io(GV<T> g, int slot, double2* stage, int to_field) {
  const long L = (long)g.ncomp * g.npts;
  const long plane = (long)g.nb * L;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < L; p += (long)gridDim.x * NT) {
    const long i = (long)slot * L + p;
    if constexpr (sizeof(T) == 4) {
      float2* w = reinterpret_cast<float2*>(g.W64);
      if (to_field) {
        const double2 a = stage[p];
        float2 h, l;
        h.x = (float)a.x; h.y = (float)a.y;
        l.x = (float)(a.x - (double)h.x); l.y = (float)(a.y - (double)h.y);
        w[i] = h; w[plane + i] = l;
      } else {
        const float2 h = w[i], l = w[plane + i];
        stage[p] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
      }
    } else {
      if (to_field) g.W64[i] = stage[p];
      else stage[p] = g.W64[i];
    }
  }
}

// ---------------------------------------------------------------------------
// E3 from Gauss's law (Sec. 2): div(n^2 E) = 0 with n^2 = n^2(x, y) in a step and
// the z-derivative of each plane wave of D taken in the reference medium,
// i kz D3^ = -i (kx D1^ + ky D2^), kz = sqrt((k0 n0)^2 - kx^2 - ky^2), Im kz >= 0.
// Working planes hold D' = (n^2/n0^2) w = (1 + delta) w.
// ---------------------------------------------------------------------------
// D'_c = (1 + delta) w_c for both components of beam `slot` into work[2][npts].
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_e3_pre(GV<T> g, int slot, typename Cx<T>::t* work) {
  using C = typename Cx<T>::t;
  const C* d = g.delta + (long)slot * g.npts;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < g.npts; p += (long)gridDim.x * NT) {
    C r = d[p];
    r.x += (T)1;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const long i = ((long)slot * 2 + c) * g.npts + p;
      C w;
      if constexpr (sizeof(T) == 4) {   // double-float field: the hi plane is the FP32 value
        w = reinterpret_cast<const float2*>(g.W64)[i];
      } else {
        w = g.W64[i];
      }
      work[(long)c * g.npts + p] = cmul(r, w);
    }
  }
}

// In Fourier space: work[0] = -(kx D1^ + ky D2^)/kz / (nx ny) (the inverse
// transform's scale folded in); kx, ky as first derivatives (Nyquist entry 0),
// kz from the full wavenumbers; a mode with kz = 0 gets 0.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_e3_spectral(GV<T> g, typename Cx<T>::t* work, double k0n0) {
  using C = typename Cx<T>::t;
  const double sc = 1.0 / (double)g.npts;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < g.npts; p += (long)gridDim.x * NT) {
    const int i = (int)(p % g.nx), n = (int)(p / g.nx);
    const double kxf = (double)ffreq(i, g.nx) * (double)g.kx0d, kyf = (double)ffreq(n, g.ny) * (double)g.ky0d;
    const double kx = ((g.nx % 2) == 0 && i == g.nx / 2) ? 0.0 : kxf;
    const double ky = ((g.ny % 2) == 0 && n == g.ny / 2) ? 0.0 : kyf;
    const double a = k0n0 * k0n0 - kxf * kxf - kyf * kyf;
    // 1/kz: kz = sqrt(a) (propagating) or i sqrt(-a) (evanescent, Im kz > 0)
    double2 ikz = make_double2(0.0, 0.0);
    if (a > 0.0) ikz.x = 1.0 / sqrt(a);
    else if (a < 0.0) ikz.y = -1.0 / sqrt(-a);
    const double2 d1 = to_d(work[p]), d2 = to_d(work[g.npts + p]);
    const double2 num = make_double2(-(kx * d1.x + ky * d2.x) * sc, -(kx * d1.y + ky * d2.y) * sc);
    work[p] = to_c(make_double2(num.x * ikz.x - num.y * ikz.y, num.x * ikz.y + num.y * ikz.x), T());
  }
}

// E3 = D3 / (1 + delta) into the complex128 stage.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_e3_post(GV<T> g, int slot, const typename Cx<T>::t* work, double2* stage) {
  using C = typename Cx<T>::t;
  const C* d = g.delta + (long)slot * g.npts;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < g.npts; p += (long)gridDim.x * NT) {
    const double2 r = to_d(d[p]);
    const double2 v = to_d(work[p]);
    const double rx = 1.0 + r.x, ry = r.y, den = rx * rx + ry * ry;
    stage[p] = make_double2((v.x * rx + v.y * ry) / den, (v.y * rx - v.x * ry) / den);
  }
}

// ---------------------------------------------------------------------------
// Classical Runge-Kutta for the pseudo-differential form dw/dz = i k0 n0 (S(Z) - I) w
// (Sec. 3.2).  The field arrays hold L = nb ncomp npts points: complex128 for FP64,
// double-float planes (hi, then lo) for FP32; the stage data are complex128.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ double2 field_get(const double2* W, long i, long L) {
  if constexpr (sizeof(T) == 4) {
    const float2 h = reinterpret_cast<const float2*>(W)[i], l = reinterpret_cast<const float2*>(W)[L + i];
    return make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
  } else {
    return W[i];
  }
}
template <typename T> __device__ __forceinline__ void field_put(double2* W, long i, long L, double2 v) {
  if constexpr (sizeof(T) == 4) {
    float2 h, l;
    h.x = (float)v.x; h.y = (float)v.y;
    l.x = (float)(v.x - (double)h.x); l.y = (float)(v.y - (double)h.y);
    reinterpret_cast<float2*>(W)[i] = h;
    reinterpret_cast<float2*>(W)[L + i] = l;
  } else {
    W[i] = v;
  }
}

// dst = field (copies of the field at the start of a step or substep)
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_rk_copy(const double2* W, double2* d0, double2* d1, long L) {
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < L; i += (long)gridDim.x * NT) {
    const double2 v = field_get<T>(W, i, L);
    d0[i] = v;
    if (d1) d1[i] = v;
  }
}
// field = src
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_rk_restore(double2* W, const double2* src, long L) {
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < L; i += (long)gridDim.x * NT) field_put<T>(W, i, L, src[i]);
}
// After a stage: Wcur holds S(Z) y, Wprev holds y.  k = i k0n0 (S y - y),
// ACC += hb k; the field becomes the next stage's input W0 + hc k, or ACC after
// the last stage.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_rk_stage(double2* Wcur, const double2* Wprev, const double2* W0, double2* ACC,
                                                 long L, double hb, double hc, double k0n0, int last) {
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < L; i += (long)gridDim.x * NT) {
    const double2 sy = field_get<T>(Wcur, i, L), y = field_get<T>(Wprev, i, L);
    const double2 kk = make_double2(-k0n0 * (sy.y - y.y), k0n0 * (sy.x - y.x));
    double2 a = ACC[i];
    a.x += hb * kk.x; a.y += hb * kk.y;
    ACC[i] = a;
    double2 nxt = a;
    if (!last) { const double2 w0 = W0[i]; nxt = make_double2(w0.x + hc * kk.x, w0.y + hc * kk.y); }
    field_put<T>(Wcur, i, L, nxt);
  }
}

// delta = (n^2 - n0^2)/n0^2 from a complex128 slab; flags a non-zero delta and
// adds its sum (of the values as rounded to T) into dsum[beam];
// with psi_out also writes psi = Log n^2 (principal branch) for the vector operator.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_medium(GV<T> g, int beam, const double2* n2, double n0sq,
                                               typename Cx<T>::t* psi_out) {
  using C = typename Cx<T>::t;
  C* d = g.delta + (long)beam * g.npts;
  __shared__ double red[32];
  int nz = 0;
  T sr = 0, si = 0;   // per-thread partials of the delta the kernels use (FP64 across the block)
  const double inv = 1.0 / n0sq;
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < g.npts; p += (long)gridDim.x * NT) {
    const double2 a = n2[p];
    double2 v; v.x = (a.x - n0sq) * inv; v.y = a.y * inv;
    const C t = to_c(v, T());
    d[p] = t;
    sr += t.x; si += t.y;
    if (psi_out) {
      const double2 lg = make_double2(0.5 * log(a.x * a.x + a.y * a.y), atan2(a.y, a.x));
      psi_out[p] = to_c(lg, T());
    }
    nz |= (t.x != (T)0 || t.y != (T)0);
  }
  const double tr = block_sum((double)sr, red);
  const double ti = block_sum((double)si, red);
  if (threadIdx.x == 0) { atomicAdd(&g.dsum[beam].x, tr); atomicAdd(&g.dsum[beam].y, ti); }
  if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(&g.nonhomog[beam], 1);
}

// ---------------------------------------------------------------------------
// GMRES cycle control (one thread per system; tiny).  The per-step control
// runs in the update kernel (dcgs_control).
// ---------------------------------------------------------------------------

// Begin a cycle for systems in state `from` (ST_DONE-initialised systems at a
// step start use from = -1): beta = ||r||; converged if beta <= tol ||w||.
// Convergence threshold: tol ||w|| (plain relative residual), or with
// backward = 1 the normwise backward-error bound tol (||w|| + ||A|| ||x_k||),
// x_k = z_k + e_k, for arithmetic whose transforms cannot resolve residuals
// below eps ||A|| ||x||.
//
// Pole k's residual reaches the step output through r_k (Z - p_k)^-1, whose size
// is about |r_k| / dist(p_k, spectrum); mu_k = max_j(that) / (that)_k gives each
// pole the same bound on its share of the field error (FP32 path only).
__device__ __forceinline__ double conv_threshold(const SysState& q, double tol, double wn, const double* anorm,
                                                 int k, int P, int backward) {
  if (!backward) return tol * wn;
  return tol * anorm[P + k] * (wn + anorm[k] * (sqrt(q.z0norm2) + sqrt(q.enorm2)));
}

static __global__ void k_begin_cycle(SysState* st, int nsys, int P, const double* bnorm2, double tol,
                              int from, int max_cycles, int first, const double* anorm, int backward) {
  pdl_enter();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    SysState& q = st[s];
    if (!first && q.state != from) continue;
    if (first) { q.iters = 0; q.cycles = 0; q.flags = 0; q.used = 0; q.enorm2 = 0.0; q.r0r = make_double2(0.0, 0.0); }
    const double beta = sqrt(q.nrm_a);
    if (first) q.beta0 = beta;
    const double wn = sqrt(bnorm2[s / P]);
    q.nrm_a = 0.0;
    q.beta = beta;
    q.resid = wn > 0 ? beta / wn : 0.0;
    if (!isfinite(beta)) { q.flags |= 1; q.state = ST_DONE; continue; }
    if (beta <= conv_threshold(q, tol, wn, anorm, s % P, P, backward)) { q.state = ST_DONE; continue; }
    if (q.cycles >= max_cycles) { q.flags |= 2; q.state = ST_DONE; continue; }
    q.cycles += 1;
    q.used = 1;
    q.state = ST_ITER;
    q.j = 0;
    q.scale = 1.0 / beta;
    for (int i = 0; i <= MMAX; ++i) q.g[i] = make_double2(0.0, 0.0);
    q.g[0] = make_double2(beta, 0.0);
    q.nrm_b = 0.0;
  }
}

__device__ __forceinline__ double2 dmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double dabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// Apply the Givens rotation (c, sn) to the pair (x, y) of one column.
__device__ __forceinline__ void givens_apply(double c, double2 sn, double2& x, double2& y) {
  const double2 a = x, b = y;
  x = make_double2(c * a.x + (sn.x * b.x - sn.y * b.y), c * a.y + (sn.x * b.y + sn.y * b.x));
  const double2 t = dmul(dconj(sn), a);
  y = make_double2(c * b.x - t.x, c * b.y - t.y);
}
// Rotation zeroing y against x; x becomes the rotated diagonal, y zero.
__device__ __forceinline__ void givens_make(double2& x, double2& y, double& c, double2& sn) {
  const double an = sqrt(dabs2(x)), hn = sqrt(dabs2(y));
  const double r = sqrt(an * an + hn * hn);
  if (hn == 0.0) { c = 1.0; sn = make_double2(0.0, 0.0); }
  else if (an == 0.0) { c = 0.0; sn = make_double2(y.x / hn, -y.y / hn); }
  else {
    c = an / r;
    // sn = (x/|x|) conj(y) / r, so that -conj(sn) x + c y = 0
    const double2 ux = make_double2(x.x / an, x.y / an);
    sn = make_double2((ux.x * y.x + ux.y * y.y) / r, (ux.y * y.x - ux.x * y.y) / r);
  }
  x = (an == 0.0) ? make_double2(hn, 0.0) : make_double2(x.x / an * r, x.y / an * r);
  y = make_double2(0.0, 0.0);
}

// Packed upper triangle of the rotated columns 0..MMAX-1: column i holds rows 0..i.
constexpr int RPACK = MMAX * (MMAX + 1) / 2;
__device__ __forceinline__ int rp(int row, int col) { return col * (col + 1) / 2 + row; }

// Back substitution R y = g over the rotated columns 0..J-1, by the whole block
// (column-oriented: after y_i is known every thread updates its rows), from a
// shared-memory copy of R; ends the cycle.  Rs must hold columns 0..J-1 packed
// and acc the right-hand side g[0..J-1].
static __device__ void end_cycle_block(SysState& q, int J, double2* Rs, double2* acc) {
  // One warp, no block barriers: lane l holds rows l and l + 32 (J <= MMAX = 64)
  // and the reciprocals of their diagonal entries; at row i the owner lane forms
  // y_i and broadcasts it, every lane updates its rows above i.
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int l = threadIdx.x;
  const double2 zero = make_double2(0.0, 0.0);
  auto rcp = [](double2 d) { const double dd = dabs2(d); return make_double2(d.x / dd, -d.y / dd); };
  double2 a0 = l < J ? acc[l] : zero, a1 = l + 32 < J ? acc[l + 32] : zero;
  const double2 r0 = l < J ? rcp(Rs[rp(l, l)]) : zero, r1 = l + 32 < J ? rcp(Rs[rp(l + 32, l + 32)]) : zero;
  for (int i = J - 1; i >= 0; --i) {
    const int owner = i & 31;
    const bool hi = i >= 32;
    const double2 mine = hi ? dmul(a1, r1) : dmul(a0, r0);   // meaningful in the owner lane
    double2 y;
    y.x = __shfl_sync(0xffffffffu, mine.x, owner);
    y.y = __shfl_sync(0xffffffffu, mine.y, owner);
    if (l == owner) { if (hi) a1 = y; else a0 = y; }
    if (l < i) { const double2 t = dmul(Rs[rp(l, i)], y); a0.x -= t.x; a0.y -= t.y; }
    if (l + 32 < i) { const double2 t = dmul(Rs[rp(l + 32, i)], y); a1.x -= t.x; a1.y -= t.y; }
  }
  if (l < J) q.y[l] = a0;
  if (l + 32 < J) q.y[l + 32] = a1;
  if (l == 0) {
    q.jend = J;
    q.enorm2 = 0.0;          // recomputed by the correction update
    q.state = ST_CYCLE_END;
  }
}

// Stage rotated columns 0..J-1 of q.H (column c <= J-1 from global, except that
// column `own` comes from `owncol`) and g[0..J-1] (g[ownrow..] overridden by
// gown[]) for end_cycle_block.
static __device__ void stage_ls(const SysState& q, int J, int own, const double2* owncol, int ownrow, const double2* gown,
                         double2* Rs, double2* acc) {
  constexpr int L = MMAX + 1;
  for (int c = 0; c < J; ++c)
    for (int r = threadIdx.x; r <= c; r += blockDim.x) Rs[rp(r, c)] = (c == own) ? owncol[r] : q.H[r + c * L];
  for (int i = threadIdx.x; i < J; i += blockDim.x) acc[i] = i >= ownrow ? gown[i - ownrow] : q.g[i];
}

// ---------------------------------------------------------------------------
// Arnoldi with delayed re-orthogonalisation (the DCGS2 scheme of Swirydowicz,
// Langou, Ananthan, Yang and Thomas, 2020, and Bielich et al., 2022), right-
// preconditioned: B = (Z - p) M^-1.  At step j, v_0..v_{j-1} are final and
// orthonormal and u = v_j is the candidate, projected once.  The Arnoldi
// epilogue forms w = B u; k_dcgs_gram the products a_i = <v_i, u>,
// b_i = <v_i, w> (i < j), c = <u, u>, d = <u, w>.  Then, with rho^2 = c - sum |a_i|^2:
//   q_j = (u - V a) / rho  re-orthogonalises u, which finalises Hessenberg
//     column j-1:  h_{i,j-1} += a_i,  h_{j,j-1} = rho;
//   B q_j = (w - V_{j+1} t) / rho,  t = Hbar a over the final columns, so the
//     first projection of B q_j gives column j:
//     h_{i,j} = (b_i - t_i)/rho (i < j),  h_{j,j} = (d - a^H b)/rho^2 - t_j/rho;
//   u_{j+1} = (I - V_{j+1} V_{j+1}^H) w / rho
//           = w/rho - sum_{i<j} (b_i/rho) v_i - ((d - a^H b)/rho^2) q_j.
// Column j-1 becomes final only at step j, so its Givens rotation and the
// convergence test for the j-column solution happen there (one operator
// application past the converged column, and at j = m only the products with
// u are formed).  Per step the basis is swept twice (products, update) instead
// of four times for classical Gram-Schmidt run twice.
//
// The FP64 control runs in one extra CTA of the update kernel, beside the
// sweep: GB300 issues FP64 at a small fraction of its FP32 rate, so its serial
// Givens chain would otherwise sit on the critical path.  It stages what it
// reads in shared memory with parallel loads and writes back in parallel.
// ---------------------------------------------------------------------------

// Control of step j for one system (one block, FP64), concurrent with the
// update sweep of the other CTAs: finalise Hessenberg column j-1 with the
// re-orthogonalisation products, rotate it (rotations 0..j-2, then a new one),
// update g and test |g[j]| -- the residual of the J = j column solution -- for
// convergence; end the cycle then (or at j = m, or when u_j vanished); else
// form column j's first projection.  Also clears the other parity's
// accumulators (last read by step j-1, next written by the Gram sweep of j+1)
// and adds this system to the iteration's counts.
struct StepArgs {
  int m, P, backward;
  double tol, breakdown;
  const double* bnorm2;
  const double* anorm;
  int* counts;   // this iteration's slot: [0] continuing, [1] ending the cycle, [2] flags
};

static __device__ void dcgs_control(SysState& q, int s, int j, const double2* bs, const double2* as, double nw,
                             double2* part, const StepArgs& A) {
  constexpr int L = MMAX + 1;
  __shared__ double2 hu[MMAX + 1], col[MMAX + 1], tt[MMAX + 1], sn_s[MMAX], gout[2], gj_s, g0_s, ahb_s;
  __shared__ double2 Rs[RPACK], acc[MMAX + 1];
  __shared__ double cs_s[MMAX], sc[6], rho_s;
  __shared__ int code_s;
  const int tid = threadIdx.x, par = j & 1;
  if (j >= 1) for (int i = tid; i < j; i += blockDim.x) hu[i] = q.Hu[i + (j - 1) * L];
  for (int i = tid; i + 1 < j; i += blockDim.x) { cs_s[i] = q.cs[i]; sn_s[i] = q.sn[i]; }
  const int k = s % A.P;
  if (tid == 32) gj_s = j >= 1 ? q.g[j - 1] : q.g[0];
  if (tid == 33) sc[0] = q.nrm_b;
  if (tid == 34) sc[1] = sqrt(A.bnorm2[s / A.P]);
  if (tid == 35) sc[2] = q.z0norm2;
  if (tid == 36) sc[3] = q.enorm2;
  if (tid == 37) sc[4] = A.anorm[k];
  if (tid == 38) sc[5] = A.anorm[A.P + k];
  // clear the other parity (slots 0..j-1 and MMAX were written by the Gram sweep of step j-1)
  for (int t2 = tid; t2 < 2 * NSTRIPE * (j + 1); t2 += blockDim.x) {
    const int pl = t2 / (NSTRIPE * (j + 1)), r = t2 % (NSTRIPE * (j + 1));
    const int stripe = r / (j + 1), i0 = r % (j + 1);
    *part_at(part, s, 2 * (1 - par) + pl, stripe, i0 < j ? i0 : MMAX) = make_double2(0.0, 0.0);
  }
  if (tid < 32) {
    double s2 = 0.0, hr = 0.0, hi = 0.0;
    for (int i = tid; i < j; i += 32) {
      s2 += dabs2(as[i]);
      hr += as[i].x * bs[i].x + as[i].y * bs[i].y;
      hi += as[i].x * bs[i].y - as[i].y * bs[i].x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
      hr += __shfl_down_sync(0xffffffffu, hr, o);
      hi += __shfl_down_sync(0xffffffffu, hi, o);
    }
    if (tid == 0) {
      const double r2 = as[j].x - s2;
      ahb_s = make_double2(hr, hi);
      rho_s = sqrt(fmax(r2, 0.0));
      // 0: go on; 1: NaN; 2: u_j vanished against the basis
      code_s = (!isfinite(r2) || !isfinite(hr) || !isfinite(hi) || !isfinite(nw)) ? 1 : (r2 > 0.0 ? 0 : 2);
    }
  }
  __syncthreads();
  int code = code_s;
  if (code == 1 || (code == 2 && j == 0)) {
    if (tid == 0) { q.flags |= 1; q.state = ST_DONE; atomicOr(&A.counts[2], 1); }
    return;
  }
  const double rho = rho_s;
  if (j >= 1) {
    for (int i = tid; i <= j; i += blockDim.x) {
      const double2 h = i < j ? make_double2(hu[i].x + as[i].x, hu[i].y + as[i].y) : make_double2(rho, 0.0);
      hu[i] = h;
      col[i] = h;
    }
    __syncthreads();
    if (tid == 0) {   // column j-1 is final: rotations 0..j-2, then rotation j-1
      for (int i = 0; i + 1 < j; ++i) givens_apply(cs_s[i], sn_s[i], col[i], col[i + 1]);
      double c; double2 sn;
      givens_make(col[j - 1], col[j], c, sn);
      cs_s[j - 1] = c; sn_s[j - 1] = sn;
      const double2 gs = gj_s;
      gout[0] = make_double2(c * gs.x, c * gs.y);
      const double2 t2 = dmul(dconj(sn), gs);
      gout[1] = make_double2(-t2.x, -t2.y);
      const double est = sqrt(dabs2(gout[1]));
      const double wn = sc[1];
      const double thr = A.backward ? A.tol * sc[5] * (wn + sc[4] * (sqrt(sc[2]) + sqrt(sc[3]))) : A.tol * wn;
      if (!isfinite(est)) code_s = 1;
      else if (code == 2 || est <= thr || j == A.m || rho <= A.breakdown * sqrt(fmax(sc[0], 0.0))) code_s = 3;
      else code_s = 0;
    }
    __syncthreads();
    code = code_s;
    if (code == 1) {
      if (tid == 0) { q.flags |= 1; q.state = ST_DONE; atomicOr(&A.counts[2], 1); }
      return;
    }
    for (int i = tid; i <= j; i += blockDim.x) { q.H[i + (j - 1) * L] = col[i]; q.Hu[i + (j - 1) * L] = hu[i]; }
    if (tid == 0) {
      q.cs[j - 1] = cs_s[j - 1]; q.sn[j - 1] = sn_s[j - 1];
      q.g[j - 1] = gout[0]; q.g[j] = gout[1];
      q.iters += 1;
      q.j = j;
    }
    if (code == 3) {
      stage_ls(q, j, j - 1, col, j - 1, gout, Rs, acc);
      end_cycle_block(q, j, Rs, acc);
      if (tid == 0) atomicAdd(&A.counts[1], 1);
      return;
    }
  } else if (tid == 0) {
    q.g[0] = make_double2(gj_s.x * rho, gj_s.y * rho);   // r = beta u_0 = beta rho q_0
  }
  // first projection of B q_j: column j (rows 0..j; row j+1 comes with step j+1)
  for (int i = tid; i <= j; i += blockDim.x) {   // t = Hbar a over the final columns 0..j-1
    double2 sum = make_double2(0.0, 0.0);
    for (int k2 = i > 0 ? i - 1 : 0; k2 < j; ++k2) {
      const double2 h = (k2 == j - 1) ? hu[i] : q.Hu[i + k2 * L];
      const double2 m2 = dmul(h, as[k2]);
      sum.x += m2.x; sum.y += m2.y;
    }
    tt[i] = sum;
  }
  const double ir = 1.0 / rho;
  const double2 ahb = ahb_s, d = bs[j];
  const double2 gj = make_double2((d.x - ahb.x) * ir * ir, (d.y - ahb.y) * ir * ir);
  for (int i = tid; i <= j; i += blockDim.x)
    q.Hu[i + j * L] = i < j ? make_double2((bs[i].x - tt[i].x) * ir, (bs[i].y - tt[i].y) * ir)
                            : make_double2(gj.x - tt[i].x * ir, gj.y - tt[i].y * ir);
  if (tid == 0) { q.nrm_b = nw * ir * ir; atomicAdd(&A.counts[0], 1); }
}

// Step j after its Gram sweep.  grid = (chunks + 1, nsys): chunk CTAs apply
//   q_j     = (u - sum_{i<j} a_i v_i) / rho                  (written over u = v_j)
//   u_{j+1} = w / rho - sum_{i<j} gamma_i v_i - gamma_j q_j  (written over w = v_{j+1})
// gamma_i = b_i / rho (i < j), gamma_j = (d - a^H b) / rho^2, with coefficients
// each CTA derives from the folded sums; the last CTA runs dcgs_control.
// The sweep takes the basis in groups of GVEC vectors (GVEC*EPT loads in flight).
// If the control ends the cycle at this step the sweep's output goes unused.
// grid.x = 1 + sweep CTAs: CTA 0 is the control, CTA x > 0 sweeps chunks
// x - 1, x - 1 + (gridDim.x - 1), ... (one coefficient prologue per CTA).
template <typename T, int NT, int EPT, int GVEC>
__device__ __forceinline__ void dcgs_step_body(int bx, int by, int gdx, GV<T> g, int jj, StepArgs A) {
  pdl_enter();
  using C = typename Cx<T>::t;
  __shared__ double2 bs[MMAX + 1], as[MMAX + 1];
  __shared__ double nw_s;
  __shared__ C ca[MMAX + 8], cg[MMAX + 8];
  __shared__ T ir_s;
  const int s = unit_of(g, (int)by), j = jj, tid = threadIdx.x;
  if (s < 0) return;
  SysState& q = g.st[s];
  if (q.state != ST_ITER) return;
  const int par = j & 1;
  for (int t2 = tid; t2 < 2 * (j + 1) + 1; t2 += NT) {   // fold the stripes (read only)
    const int plane = t2 < j + 1 ? 0 : 1;
    const int i = t2 == 2 * (j + 1) ? MMAX : (plane == 0 ? t2 : t2 - (j + 1));
    double2 x[NSTRIPE];
#pragma unroll
    for (int k = 0; k < NSTRIPE; ++k) x[k] = *part_at(g.part, s, 2 * par + plane, k, i);
    double2 sum = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < NSTRIPE; ++k) { sum.x += x[k].x; sum.y += x[k].y; }
    if (i == MMAX) nw_s = sum.x;
    else if (plane == 0) bs[i] = sum;
    else as[i] = sum;
  }
  __syncthreads();
  // the control goes first in dispatch order, so its FP64 chain overlaps the sweep
  if (bx == 0) { dcgs_control(q, s, j, bs, as, nw_s, g.part, A); return; }
  if (j == A.m) return;   // the cycle ends at this step: nothing to sweep
  // coefficients, in the working precision (the sums themselves are FP64)
  if (tid < 32) {
    T s2 = 0, hr = 0, hi = 0;
    for (int i = tid; i < j; i += 32) {
      const T ax = (T)as[i].x, ay = (T)as[i].y, br = (T)bs[i].x, bi = (T)bs[i].y;
      s2 += ax * ax + ay * ay; hr += ax * br + ay * bi; hi += ax * bi - ay * br;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
      hr += __shfl_down_sync(0xffffffffu, hr, o);
      hi += __shfl_down_sync(0xffffffffu, hi, o);
    }
    if (tid == 0) {
      const T r2 = (T)as[j].x - s2;
      const T ir = r2 > (T)0 ? (T)1 / sqrt(r2) : (T)0;
      ir_s = ir;
      cg[j].x = ((T)bs[j].x - hr) * ir * ir; cg[j].y = ((T)bs[j].y - hi) * ir * ir;
    }
  }
  __syncthreads();
  const T ir = ir_s;
  if (!(ir > (T)0)) return;   // u_j vanished: the control ends the cycle
  for (int i = tid; i < j + 8; i += NT) {
    if (i == j) continue;
    C a{}, c{};
    if (i < j) { a.x = (T)as[i].x; a.y = (T)as[i].y; c.x = (T)bs[i].x * ir; c.y = (T)bs[i].y * ir; }
    ca[i] = a; cg[i] = c;
  }
  if (tid == 0) { ca[j].x = 0; ca[j].y = 0; }
  __syncthreads();
  const long L = (long)g.ncomp * g.npts;
  C* uj = vslot(g, s, jj);
  C* wj = vslot(g, s, jj + 1);
  const long nchunks = (L + NT * EPT - 1) / (NT * EPT);
  for (long chunk = bx - 1; chunk < nchunks; chunk += gdx - 1) {   // persistent over chunks
  const long b0 = chunk * NT * EPT + tid;
  C qv[EPT], x[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const long p = b0 + (long)e * NT;
    qv[e] = C{}; x[e] = C{};
    if (p < L) { qv[e] = uj[p]; const C w = wj[p]; x[e].x = w.x * ir; x[e].y = w.y * ir; }
  }
  for (int i0 = 0; i0 < jj; i0 += GVEC) {
    C vv[GVEC][EPT];
#pragma unroll
    for (int k = 0; k < GVEC; ++k) {
      const C* v = vslot(g, s, i0 + k);
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const long p = b0 + (long)e * NT;
        vv[k][e] = (i0 + k < jj && p < L) ? v[p] : C{};
      }
    }
#pragma unroll
    for (int k = 0; k < GVEC; ++k) {
      const C a = ca[i0 + k], gm = cg[i0 + k];   // vv is zero past v_{j-1}: padded terms vanish
#pragma unroll
      for (int e = 0; e < EPT; ++e) {
        const C t1 = cmul(a, vv[k][e]), t2 = cmul(gm, vv[k][e]);
        qv[e].x -= t1.x; qv[e].y -= t1.y;
        x[e].x -= t2.x; x[e].y -= t2.y;
      }
    }
  }
  const C gj = cg[jj];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const long p = b0 + (long)e * NT;
    if (p < L) {
      C qq = qv[e]; qq.x *= ir; qq.y *= ir;
      const C t = cmul(gj, qq);
      C xx = x[e]; xx.x -= t.x; xx.y -= t.y;
      uj[p] = qq; wj[p] = xx;
    }
  }
  }
}
template <typename T, int NT, int EPT, int GVEC>
__global__ void __launch_bounds__(NT) k_dcgs_step(GV<T> g, int jj, StepArgs A) {
  dcgs_step_body<T, NT, EPT, GVEC>(blockIdx.x, blockIdx.y, gridDim.x, g, jj, A);
}

// ---------------------------------------------------------------------------
// Learned initial guess: pack the network input, unpack its output into E.
// Input channels (bf16, 16 per pixel): R0 / rms (re, im per component),
// 10 delta (re, im), Re p, Im p, zeros.  rms = ||R0|| / sqrt(ncomp npts).
// ---------------------------------------------------------------------------
constexpr int GUESS_CH = 16;
constexpr double GUESS_ACCEPT = 0.9;   // keep a guess only if it cuts ||R0|| by at least 10%

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_guess_pack(GV<T> g, __nv_bfloat16* in, const double2* poles, int only_iter,
                                                   int s0) {
  const int s = s0 + blockIdx.y;
  const SysState& q = g.st[s];
  if (only_iter && q.state != ST_ITER) return;
  const int b = s / g.P, k = s % g.P;
  const double rms = q.beta0 / sqrt((double)g.ncomp * g.npts);
  const float inv = rms > 0 ? (float)(1.0 / rms) : 0.f;
  const double2 p = poles[k];
  __nv_bfloat16* o = in + (long)blockIdx.y * g.npts * GUESS_CH;
  const long L = (long)g.ncomp * g.npts;
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < g.npts; i += (long)gridDim.x * NT) {
    float v[GUESS_CH];
#pragma unroll
    for (int c = 0; c < GUESS_CH; ++c) v[c] = 0.f;
    for (int c = 0; c < g.ncomp; ++c) {
      const auto r = g.R0[(long)s * L + (long)c * g.npts + i];
      v[2 * c] = (float)r.x * inv; v[2 * c + 1] = (float)r.y * inv;
    }
    const auto d = g.delta[(long)b * g.npts + i];
    v[2 * g.ncomp] = 10.f * (float)d.x; v[2 * g.ncomp + 1] = 10.f * (float)d.y;
    v[2 * g.ncomp + 2] = (float)p.x; v[2 * g.ncomp + 3] = (float)p.y;
#pragma unroll
    for (int c = 0; c < GUESS_CH; c += 2)
      *reinterpret_cast<__nv_bfloat162*>(o + i * GUESS_CH + c) = __floats2bfloat162_rn(v[c], v[c + 1]);
  }
}

// E = out * rms for systems still iterating; they move to ST_CYCLE_END so that the
// cycle-end true residual R0 - (Z - p) E starts GMRES from the guess.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_guess_unpack(GV<T> g, const float* out) {
  __shared__ double red[32];
  const int s = blockIdx.y;
  SysState& q = g.st[s];
  if (q.state != ST_ITER) return;
  const double rms = q.beta0 / sqrt((double)g.ncomp * g.npts);
  const float* o = out + (long)s * g.npts * GUESS_CH;
  const long L = (long)g.ncomp * g.npts;
  float nr = 0.f;
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < g.npts; i += (long)gridDim.x * NT) {
    for (int c = 0; c < g.ncomp; ++c) {
      const float fx = o[i * GUESS_CH + 2 * c], fy = o[i * GUESS_CH + 2 * c + 1];
      g.E[(long)s * L + (long)c * g.npts + i] = make_double2((double)fx * rms, (double)fy * rms);
      nr += fx * fx + fy * fy;
    }
  }
  const double t = block_sum((double)nr, red) * rms * rms;
  if (threadIdx.x == 0) atomicAdd(&q.enorm2, t);
}

// Minimal-residual scaling of the guess.  With u = A e0 = R0 - r (r the true
// residual of the guess), alpha = <u, R0>/||u||^2 minimises ||R0 - alpha u||, so
// the scaled start e0 <- alpha e0, r <- (1 - alpha) R0 + alpha r is never worse
// than x0 = 0; a guess that does not cut the residual by 10% is dropped (alpha = 0)
// so that GMRES then runs exactly as without it.  One thread per system computes
// alpha; the kernel below applies it.
static __global__ void k_guess_alpha(SysState* st, int nsys) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    SysState& q = st[s];
    if (q.state != ST_CYCLE_END) continue;
    const double b2 = q.beta0 * q.beta0, r2 = q.nrm_a;
    const double2 c = q.r0r;                                  // <R0, r>
    const double2 uR = make_double2(b2 - c.x, c.y);          // <u, R0> = ||R0||^2 - conj(<R0, r>)
    const double u2 = fmax(b2 - 2.0 * c.x + r2, 0.0);
    double2 a = make_double2(0.0, 0.0);
    if (u2 > 0.0) a = make_double2(uR.x / u2, uR.y / u2);
    double rn2 = fmax(b2 - (uR.x * uR.x + uR.y * uR.y) / (u2 > 0.0 ? u2 : 1.0), 0.0);
    if (!(rn2 <= GUESS_ACCEPT * GUESS_ACCEPT * b2)) {      // not worth it: start from x0 = 0 exactly
      a = make_double2(0.0, 0.0);
      rn2 = b2;
    }
    q.coef[0] = a;                                           // alpha, read by k_guess_apply
    q.nrm_a = rn2;
    q.enorm2 *= a.x * a.x + a.y * a.y;
    q.r0r = make_double2(0.0, 0.0);
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_guess_apply(GV<T> g) {
  using C = typename Cx<T>::t;
  const int s = blockIdx.y;
  const SysState& q = g.st[s];
  if (q.state != ST_CYCLE_END) return;
  const double2 a = q.coef[0];
  const long L = (long)g.ncomp * g.npts;
  C* v = g.V + (long)s * (g.m + 2) * L;
  const C* r0 = g.R0 + (long)s * L;
  double2* e = g.E + (long)s * L;
  const T ax = (T)a.x, ay = (T)a.y, bx = (T)(1.0 - a.x), by = (T)(-a.y);
  for (long p = (long)blockIdx.x * NT + threadIdx.x; p < L; p += (long)gridDim.x * NT) {
    const C rr = v[p], R = r0[p];
    C o;
    o.x = bx * R.x - by * R.y + ax * rr.x - ay * rr.y;
    o.y = bx * R.y + by * R.x + ax * rr.y + ay * rr.x;
    v[p] = o;
    const double2 ee = e[p];
    e[p] = make_double2(a.x * ee.x - a.y * ee.y, a.x * ee.y + a.y * ee.x);
  }
}

// After the unpack: every system that received a guess becomes a cycle end.
static __global__ void k_guess_mark(SysState* st, int nsys) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x)
    if (st[s].state == ST_ITER) { st[s].state = ST_CYCLE_END; st[s].jend = 0; }
}

// Training target: E / rms (float32, 16 channels, padding zero) of one system.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_guess_target(GV<T> g, int s, float* tgt) {
  const SysState& q = g.st[s];
  const double rms = q.beta0 / sqrt((double)g.ncomp * g.npts);
  const double inv = (rms > 0 && q.used) ? 1.0 / rms : 0.0;
  const long L = (long)g.ncomp * g.npts;
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < g.npts; i += (long)gridDim.x * NT) {
    for (int c = 0; c < GUESS_CH; ++c) tgt[i * GUESS_CH + c] = 0.f;
    for (int c = 0; c < g.ncomp; ++c) {
      const double2 e = g.E[(long)s * L + (long)c * g.npts + i];
      tgt[i * GUESS_CH + 2 * c] = (float)(e.x * inv);
      tgt[i * GUESS_CH + 2 * c + 1] = (float)(e.y * inv);
    }
  }
}

// zero the per-step accumulators of every system
static __global__ void k_step_reset(SysState* st, int nsys) {
  pdl_enter();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    st[s].z0norm2 = 0.0; st[s].nrm_a = 0.0; st[s].enorm2 = 0.0;
  }
}

// compact per-system statistics for the host
static __global__ void k_collect(const SysState* st, int nsys, int* iters, int* cycles, double* resid, int* flags) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsys; s += gridDim.x * blockDim.x) {
    iters[s] = st[s].iters; cycles[s] = st[s].cycles; resid[s] = st[s].resid; flags[s] = st[s].flags;
  }
}

// Self-test of the bounded wait: one thread announces 16 bytes of transaction
// that no copy will deliver, every thread waits, the wait gives up after its
// time limit and records the failure in *err.  No copy is ever in flight.
static __global__ void k_selftest_wait(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) { mbar_init(&bar, 1); fence_mbar_init(); }
  __syncthreads();
  if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
  mbar_wait(&bar, 0, err);
}

// Compacted list of the systems in state ST_ITER, in index order (one block of
// a multiple of 32 threads): the Arnoldi launches of a batch cover only these.
static __global__ void k_active_list(const SysState* st, int nsys, int* list) {
  pdl_enter();
  __shared__ int wsum[32], base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int s0 = 0; s0 < nsys; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    const bool a = s < nsys && st[s].state == ST_ITER;
    const unsigned m = __ballot_sync(0xffffffffu, a);
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    int off = base;
    for (int k = 0; k < w; ++k) off += wsum[k];
    if (a) list[off + __popc(m & ((1u << lane) - 1u))] = s;
    __syncthreads();
    if (threadIdx.x == 0) for (int k = 0; k < nw; ++k) base += wsum[k];
    __syncthreads();
  }
  // the rest of the list marks empty grid rows: a launch sized for more systems
  // than iterate (the host's count lags by a batch) skips them
  for (int s = base + threadIdx.x; s < nsys; s += blockDim.x) list[s] = -1;
}

// counts[0] = systems iterating, counts[1] = at a cycle end, counts[2] = flags
static __global__ void k_count(const SysState* st, int nsys, int* counts) {
  pdl_enter();
  __shared__ int c0, c1, c2;
  if (threadIdx.x == 0) { c0 = 0; c1 = 0; c2 = 0; }
  __syncthreads();
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    if (st[s].state == ST_ITER) atomicAdd(&c0, 1);
    if (st[s].state == ST_CYCLE_END) atomicAdd(&c1, 1);
    if (st[s].flags) atomicOr(&c2, st[s].flags);
  }
  __syncthreads();
  if (threadIdx.x == 0) { counts[0] = c0; counts[1] = c1; counts[2] = c2; }
}

}  // namespace prop_dev
