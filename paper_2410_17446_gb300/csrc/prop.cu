// C ABI of the propagator (include/prop.h): handle, workspace carve-up, launch
// dispatch and the z-step driver.
//
// One step, per group of equal-grid beams (Eqs. approx_prop, W_k_def):
//   w_hat = FFT2(w)                                   (shared by every pole)
//   w_new = w + IFFT2[(r(zeta_fs) - 1) w_hat]          (free-space part, Eq. approx_fs_prop)
//   for each pole k:  z_k = IFFT2[w_hat/(zeta_fs - p_k)] (the preconditioner of Sec. 4.2)
//                     solve (Z - p_k) e_k = -delta z_k by GMRES right-preconditioned
//                     with (Z_fs - p_k)^-1, x0 = 0
//   w_new += sum_k r_k e_k
// Since x_k = z_k + e_k solves (Z - p_k) x_k = w, this is r0 w + sum_k r_k x_k
// written so that rounding errors scale with the increment, not with w; the
// field itself is accumulated in FP64.
#include "../../include/prop.h"
#include "../../include/prop_cnn.h"
#include "mg.cuh"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

using namespace prop_dev;
using cplx = std::complex<double>;

namespace {

constexpr size_t ALIGN = 256;
constexpr int NET_MAX_LAYERS = 8;                                   // guess network limits
constexpr size_t NET_W_BYTES = NET_MAX_LAYERS * 9 * 32 * 32 * 2;
constexpr size_t NET_B_BYTES = NET_MAX_LAYERS * 32 * 4;
inline size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

bool supported_n(int n) {
  switch (n) {
    case 16: case 32: case 64: case 128: case 256: case 384: case 512: case 768: case 1024: return true;
    default: return false;
  }
}

int sm_count() {   // SMs of the current device (looked up once)
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
    cudaGetLastError();
  }
  return n > 0 ? n : 1;
}

// Resident CTAs per SM of a kernel launched with `nt` threads and no dynamic
// shared memory, looked up once into `cache`: the sweeps size one wave from it.
template <typename K> int resident(K kernel, int nt, int& cache) {
  if (!cache) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, nt, 0) != cudaSuccess || n < 1) n = 1;
    cudaGetLastError();
    cache = n;
  }
  return cache;
}

// Launch geometry of the FFT passes: small CTAs, so that one 1024^2 field still
// spreads over several CTAs per SM and their load / transform / store phases overlap.
template <typename T> constexpr int cols_per_cta() { return sizeof(T) == 4 ? 4 : 2; }   // 32-byte row segments
template <int N> constexpr int rows_nr() { return N <= 128 ? 16 : (N == 256 ? 8 : (N <= 512 ? 4 : 2)); }
constexpr int clamp_nt(int t) { return t < 64 ? 64 : (t > 256 ? 256 : t); }
template <int N> constexpr int rows_nt() { return clamp_nt(rows_nr<N>() * N / 16); }
// the warp row transform (N = 512, 1024): four rows a CTA, one warp per row
constexpr int WROWS = 4;
constexpr bool warp_n_c(int n) { return n == 512 || n == 1024; }

// ---------------------------------------------------------------------------
// FFT pass variants per (size, precision), process-wide: the row pass by the
// block-wide Stockham or by warps, the column pass by TMA tiles, plain loads or
// warps.  prop_set_fft_plan installs a choice (the autotuner's); every launch
// reads it.
// ---------------------------------------------------------------------------
constexpr int NSIZES = 9;
int size_index(int n) {
  switch (n) {
    case 16: return 0; case 32: return 1; case 64: return 2; case 128: return 3; case 256: return 4;
    case 384: return 5; case 512: return 6; case 768: return 7; case 1024: return 8; default: return -1;
  }
}
// [precision][launch class: 0 large, 1 small (<= PROP_FFT_SMALL_ITEMS arrays)][size]
std::atomic<int> g_plan_rows[2][2][NSIZES];
std::atomic<int> g_plan_cols[2][2][NSIZES];
bool warp_n(int n) { return n == 512 || n == 1024; }
int launch_class(long items) { return items <= PROP_FFT_SMALL_ITEMS ? 1 : 0; }
int plan_rows(int prec, int n, long items) {
  const int i = size_index(n);
  return i < 0 ? PROP_ROWS_BLOCK : g_plan_rows[prec][launch_class(items)][i].load(std::memory_order_relaxed);
}
int plan_cols(int prec, int n, long items) {
  const int i = size_index(n);
  return i < 0 ? PROP_COLS_TMA : g_plan_cols[prec][launch_class(items)][i].load(std::memory_order_relaxed);
}
template <typename T> constexpr int prec_of() { return sizeof(T) == 4 ? PROP_FP32 : PROP_FP64; }
template <typename T, int NY> constexpr int cols_nt() { return clamp_nt(NY * cols_per_cta<T>() / 16); }
constexpr int NT_VEC = 256;
constexpr int EPT_GS = 4;     // points per thread of the update sweep
constexpr int GVEC_GS = 4;    // basis vectors per load group of the update sweep
constexpr int EPT_GRAM = 4;   // points per thread of the Gram sweep
constexpr int GVEC_GRAM = 4;  // basis vectors per transpose-reduce of the Gram sweep
#ifndef PROP_SYNC_EVERY
#define PROP_SYNC_EVERY 4
#endif
constexpr int SYNC_EVERY = PROP_SYNC_EVERY;   // Arnoldi iterations launched between host reads of the GMRES state
// Arnoldi batches in flight: 1, the host reads each batch's counts before enqueuing the
// next.  (Two deep was measured on GB300: within 2 % either way before the kernels
// were launched with programmatic dependent launch, 4.5 % slower after it on the
// batched-scalar step, so the launches stay sized by exact counts.)
constexpr int PIPE_DEPTH = 1;
// The counts area: MAXG count-slot sets (one per group of a multi-group step; the
// grid-by-grid step uses set 0), each 3 ints of cycle counts and two parities of
// SYNC_EVERY step slots of 3 ints, then the asynchronous-copy error word.
constexpr int CSLOT = 3 + 2 * 3 * SYNC_EVERY;
constexpr int ERR_SLOT = MAXG * CSLOT;
constexpr int COUNT_INTS = ERR_SLOT + 1;

struct Layout {
  size_t V, R0, E, Tmp, W64a, W64b, What, Btmp, delta, basemul, ax, ay, pim, twx, twy, st, bnorm2, nonhomog, dsum,
      rk, anorm, part, psi, Tmp2, poles, act0, act1, netout, stage, iters, cycles, resid, flags, ulist, rkw0, rkacc,
      rkstart, end;
};

struct Group {
  int nx, ny;
  double dx, dy;
  std::vector<int> beams;  // global beam ids in slot order
  long npts;
  Layout off;
  int cur;                 // which of W64a / W64b holds the field
  bool medium_dirty;       // a medium was set since the homogeneity flags were read
  bool stats_zero;         // per-system statistics already record a homogeneous step
  bool carry;              // Btmp holds the forward row DFT of the current field (from the last step)
  std::vector<int> nonhomog_host;
  // TMA tensor maps of the column pass: Btmp [nb*C][ny][nx], Tmp and Tmp2 [nsys*C][ny][nx], basemul [1][ny][nx]
  bool tma, tma_dy;
  CUtensorMap tm_btmp, tm_tmp, tm_tab, tm_tmp2;
};

}  // namespace

struct prop {
  int nbeams, P, C, prec, m, max_restarts, precond, form, substeps, multigroup;
  double tol, k0, n0, dz;
  std::vector<cplx> poles, res;
  cplx r0;
  std::vector<prop_grid> grids;
  std::vector<int> beam_group, beam_slot;
  std::vector<Group> groups;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  size_t counts_off;
  size_t net_off;          // guess network: bf16 weights, then float32 biases
  int guess, net_layers;
  int net_ch[9];
  int64_t steps, total_iters;
  int last_status;
  // launch accounting and optional per-launch event timing
  int64_t launches;
  int profiling;
  struct Pending { int kind; double bytes; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  int64_t k_launches[PROP_NKINDS];
  double k_ms[PROP_NKINDS], k_bytes[PROP_NKINDS];
  // pipelined Arnoldi batches: pinned host copies of the two count-slot sets and
  // the events that mark their arrival
  int* hcounts;
  cudaEvent_t batch_ev[2];
};

namespace {

size_t elem_size(int prec) { return prec == PROP_FP64 ? sizeof(double) : sizeof(float); }

// Carve one group's buffers starting at `base`; returns the end offset.
size_t carve(Group& G, size_t base, int P, int C, int m, int prec, int guess, int form) {
  const size_t es = elem_size(prec), cs = 2 * es;
  const size_t nb = G.beams.size(), nsys = nb * P, npts = G.npts;
  Layout& L = G.off;
  size_t o = align_up(base);
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes); return r; };
  L.V = take(nsys * (m + 2) * C * npts * cs);
  L.R0 = take(nsys * C * npts * cs);
  L.E = take(nsys * C * npts * 16);
  L.Tmp = take(nsys * C * npts * cs);
  L.W64a = take(nb * C * npts * 16);
  L.W64b = take(nb * C * npts * 16);
  L.What = take(nb * C * npts * cs);
  L.Btmp = take(nb * C * npts * cs);
  L.delta = take(nb * npts * cs);
  L.basemul = take(npts * cs);
  L.ax = take((P + 1) * G.nx * 2 * es);
  L.ay = take((P + 1) * G.ny * 2 * es);
  L.pim = take((P + 1) * es);
  L.twx = take(G.nx * cs);
  L.twy = take(G.ny * cs);
  L.st = take(nsys * sizeof(SysState));
  L.bnorm2 = take(nb * sizeof(double));
  L.nonhomog = take(nb * sizeof(int));
  L.dsum = take(nb * sizeof(double2));
  L.rk = take(P * 16);
  L.anorm = take(2 * P * sizeof(double));
  L.part = take(nsys * NPLANE * NSTRIPE * (MMAX + 1) * sizeof(double2));
  L.psi = take(C == 2 ? nb * 5 * npts * cs : 0);
  L.Tmp2 = take(C == 2 ? nsys * C * npts * cs : 0);
  L.poles = take(P * 16);
  L.act0 = take(guess ? nsys * npts * 32 * 2 : 0);     // bf16 NHWC activations of the guess network
  L.act1 = take(guess ? nsys * npts * 32 * 2 : 0);
  L.netout = take(guess ? nsys * npts * 16 * 4 : 0);   // float32 output
  L.stage = take(C * npts * 16);
  L.iters = take(nsys * sizeof(int));
  L.cycles = take(nsys * sizeof(int));
  L.resid = take(nsys * sizeof(double));
  L.flags = take(nsys * sizeof(int));
  L.ulist = take(nsys * sizeof(int));
  // pseudo-differential form: the Runge-Kutta substep start, accumulator and step start
  L.rkw0 = take(form ? nb * C * npts * 16 : 0);
  L.rkacc = take(form ? nb * C * npts * 16 : 0);
  L.rkstart = take(form ? nb * C * npts * 16 : 0);
  L.end = o;
  return o;
}

template <typename T> GV<T> view(const prop* h, const Group& G) {
  using C = typename Cx<T>::t;
  char* b = h->ws;
  const Layout& L = G.off;
  GV<T> g;
  g.nx = G.nx; g.ny = G.ny; g.ncomp = h->C; g.P = h->P; g.m = h->m;
  g.nb = (int)G.beams.size(); g.nsys = g.nb * h->P; g.npts = G.npts;
  g.V = (C*)(b + L.V); g.R0 = (C*)(b + L.R0); g.E = (double2*)(b + L.E);
  g.Tmp = (C*)(b + L.Tmp);
  g.W64 = (double2*)(b + (G.cur == 0 ? L.W64a : L.W64b));
  g.What = (C*)(b + L.What); g.Btmp = (C*)(b + L.Btmp); g.delta = (C*)(b + L.delta);
  g.basemul = (C*)(b + L.basemul);
  g.ax = (const T*)(b + L.ax); g.ay = (const T*)(b + L.ay); g.pim = (const T*)(b + L.pim);
  g.twx = (const C*)(b + L.twx); g.twy = (const C*)(b + L.twy);
  g.st = (SysState*)(b + L.st); g.bnorm2 = (double*)(b + L.bnorm2); g.nonhomog = (int*)(b + L.nonhomog);
  g.dsum = (double2*)(b + L.dsum);
  g.rk = (const double2*)(b + L.rk);
  g.anorm = (const double*)(b + L.anorm);
  g.part = (double2*)(b + L.part);
  g.psi = (C*)(b + L.psi);
  g.Tmp2 = (C*)(b + L.Tmp2);
  g.err = (int*)(b + h->counts_off) + ERR_SLOT;
  g.ulist = nullptr;
  g.kx0d = 2.0 * M_PI / ((double)G.nx * G.dx);
  g.ky0d = 2.0 * M_PI / ((double)G.ny * G.dy);
  g.kx0 = (T)g.kx0d;
  g.ky0 = (T)g.ky0d;
  return g;
}

template <typename C> Buf<C> buf(C* base, long ustride, int div = 1) { Buf<C> b; b.base = base; b.ustride = ustride; b.div = div; return b; }

// ---------------------------------------------------------------------------
// TMA tensor maps (driver entry point looked up once; no link against libcuda)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    cudaGetLastError();
  }
  return fn;
}

// [items][ny][nx] complex elements of csz bytes (8 or 16), seen as 8-byte words;
// box = nv elements x tma_box_rows(ny) rows x 1 item, as k_cols_tma loads it.
bool make_col_map(CUtensorMap* m, void* base, int nx, int ny, long items, int csz, int nv) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc || (csz != 8 && csz != 16) || ((uintptr_t)base % 16) != 0 || ((long)nv * csz) % 16 != 0) return false;
  const int ew = csz / 8;
  const cuuint64_t dims[3] = {(cuuint64_t)nx * ew, (cuuint64_t)ny, (cuuint64_t)items};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * csz, (cuuint64_t)nx * ny * csz};
  const cuuint32_t box[3] = {(cuuint32_t)(nv * ew), (cuuint32_t)tma_box_rows(ny), 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Launch dispatch over the compiled sizes
// ---------------------------------------------------------------------------

// Raise the dynamic shared-memory limit of one kernel instantiation (once per process).
template <typename K> cudaError_t set_smem_once(K kernel, size_t bytes, bool& done) {
  if (done || bytes <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

template <typename T, int N, typename SRC>
cudaError_t rows_fwd_n(const GV<T>& g, Buf<SRC> src, Buf<typename Cx<T>::t> dst, int mask, double* nacc,
                       int units, cudaStream_t st) {
  using C = typename Cx<T>::t;
  if constexpr (warp_n_c(N)) {
    if (plan_rows(prec_of<T>(), N, (long)units * g.ncomp) == PROP_ROWS_WARP) {
      const size_t sm = smem_elems<N, WROWS, false>() * sizeof(C);
      auto k = (N == 1024 && sizeof(T) == 4) ? k_rows_fwd_w<T, N, WROWS, 32 * WROWS, SRC, true>
                                             : k_rows_fwd<T, N, WROWS, 32 * WROWS, SRC, true>;
      static bool attr = false;
      cudaError_t e = set_smem_once(k, sm, attr);
      if (e != cudaSuccess) return e;
      dim3 grid(g.ny / WROWS, units * g.ncomp);
      return launch_pdl(k, grid, dim3(32 * WROWS), sm, st, g, src, dst, mask, nacc);
    }
  }
  constexpr int NR = rows_nr<N>(), NT = rows_nt<N>();
  const size_t sm = smem_elems<N, NR, false>() * sizeof(C);
  auto k = k_rows_fwd<T, N, NR, NT, SRC, false>;
  static bool attr = false;
  cudaError_t e = set_smem_once(k, sm, attr);
  if (e != cudaSuccess) return e;
  dim3 grid(g.ny / NR, units * g.ncomp);
  return launch_pdl(k, grid, dim3(NT), sm, st, g, src, dst, mask, nacc);
}

template <typename T, int N>
cudaError_t rows_inv_n(const GV<T>& g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst, int mask,
                       int skip, EpiArgs ep, int units, cudaStream_t st) {
  using C = typename Cx<T>::t;
  const bool arn = ep.mode == EPI_ARNOLDI;
  if constexpr (warp_n_c(N)) {
    if (plan_rows(prec_of<T>(), N, (long)units * g.ncomp) == PROP_ROWS_WARP) {
      const size_t sm = smem_elems<N, WROWS, false>() * sizeof(C);
      auto k = (N == 1024 && sizeof(T) == 4)
                   ? (arn ? k_rows_inv_w<T, N, WROWS, 32 * WROWS, true, true> : k_rows_inv_w<T, N, WROWS, 32 * WROWS, false, true>)
                   : (arn ? k_rows_inv<T, N, WROWS, 32 * WROWS, true, true> : k_rows_inv<T, N, WROWS, 32 * WROWS, false, true>);
      static bool attr[2] = {false, false};
      cudaError_t e = set_smem_once(k, sm, attr[arn ? 1 : 0]);
      if (e != cudaSuccess) return e;
      dim3 grid(g.ny / WROWS, units * g.ncomp);
      return launch_pdl(k, grid, dim3(32 * WROWS), sm, st, g, src, dst, mask, skip, ep);
    }
  }
  constexpr int NR = rows_nr<N>(), NT = rows_nt<N>();
  const size_t sm = smem_elems<N, NR, false>() * sizeof(C);
  auto k = arn ? k_rows_inv<T, N, NR, NT, true, false> : k_rows_inv<T, N, NR, NT, false, false>;
  static bool attr[2] = {false, false};
  cudaError_t e = set_smem_once(k, sm, attr[arn ? 1 : 0]);
  if (e != cudaSuccess) return e;
  dim3 grid(g.ny / NR, units * g.ncomp);
  return launch_pdl(k, grid, dim3(NT), sm, st, g, src, dst, mask, skip, ep);
}

// Tensor maps for a column pass: source, destination and (MUL_TABLE) multiplier.
struct ColMaps { const CUtensorMap* src; const CUtensorMap* dst; const CUtensorMap* tab; const CUtensorMap* dy; };

template <typename T, int NY, bool DY>
cudaError_t cols_nd(const GV<T>& g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst, int mask, int fwd,
                    int mul, int inv, int skip, int pole, T scale, int units, cudaStream_t st,
                    Buf<typename Cx<T>::t> spec, Buf<typename Cx<T>::t> dy, ColMaps cm) {
  using C = typename Cx<T>::t;
  const int cplan = plan_cols(prec_of<T>(), NY, (long)units * g.ncomp);
  if constexpr (warp_n_c(NY) && !DY) {
    // column pass by warps: every mode but the multiplier table and the spectrum output
    if (cplan == PROP_COLS_WARP && mul != MUL_TABLE && !spec.base && g.nx % CW_NV == 0) {
      const size_t sm = (size_t)cw_elems<NY>() * sizeof(C);
      auto k = k_cols_warp<T, NY>;
      static bool attr = false;
      cudaError_t e = set_smem_once(k, sm, attr);
      if (e != cudaSuccess) return e;
      dim3 grid(g.nx / CW_NV, units * g.ncomp);
      return launch_pdl(k, grid, dim3(32 * CW_NV), sm, st, g, src, dst, mask, fwd, mul, inv, skip, pole, scale);
    }
  }
  // the TMA pass reports failed copies through g.err: it runs only with an error word
  if (cplan != PROP_COLS_PLAIN && g.err && cm.src && cm.dst && (mul != MUL_TABLE || cm.tab) &&
      (!DY || (cm.dy && mul != MUL_TABLE))) {
    // the d/dy variant transforms two tiles back: twice the threads (at most 256)
    constexpr int NV = cols_per_cta<T>(),
                  NT = DY ? (2 * cols_nt<T, NY>() > 256 ? 256 : 2 * cols_nt<T, NY>()) : cols_nt<T, NY>();
    // tile, twiddles, then the table or d/dy tile and/or the pole's ky table; 128 bytes of alignment slack
    const bool pmul = (mul == MUL_POLE_INV || mul == MUL_POLE_FWD || mul == MUL_PREC_INV);
    const size_t sm = ((size_t)NY * NV * (mul == MUL_TABLE || DY ? 2 : 1) + NY + (pmul ? NY : 0)) * sizeof(C) + 128;
    auto k = k_cols_tma<T, NY, NV, NT, DY>;
    static bool attr = false;
    if (!attr) {   // room for the largest layout
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)((2 * (size_t)NY * NV + 2 * NY) * sizeof(C) + 128));
      if (e != cudaSuccess) return e;
      attr = true;
    }
    dim3 grid(g.nx / NV, units * g.ncomp);
    return launch_pdl(k, grid, dim3(NT), sm, st, g, *cm.src, *cm.dst, cm.tab ? *cm.tab : *cm.src,
                      cm.dy ? *cm.dy : *cm.src, mask, fwd, mul, inv, skip, pole, scale, spec);
  }
  constexpr int NV = cols_per_cta<T>(), NT = cols_nt<T, NY>() * (DY ? 2 : 1) > 256 ? 256 : cols_nt<T, NY>() * (DY ? 2 : 1);
  const size_t sm = smem_elems<NY, DY ? 2 * NV : NV, true>() * sizeof(C);
  auto k = k_cols<T, NY, NV, NT, DY>;
  static bool attr = false;
  cudaError_t e = set_smem_once(k, sm, attr);
  if (e != cudaSuccess) return e;
  dim3 grid(g.nx / NV, units * g.ncomp);
  return launch_pdl(k, grid, dim3(NT), sm, st, g, src, dst, mask, fwd, mul, inv, skip, pole, scale, spec, dy);
}
template <typename T, int NY>
cudaError_t cols_n(const GV<T>& g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst, int mask, int fwd,
                   int mul, int inv, int skip, int pole, T scale, int units, cudaStream_t st,
                   Buf<typename Cx<T>::t> spec, Buf<typename Cx<T>::t> dy, ColMaps cm) {
  if (dy.base) return cols_nd<T, NY, true>(g, src, dst, mask, fwd, mul, inv, skip, pole, scale, units, st, spec, dy, cm);
  return cols_nd<T, NY, false>(g, src, dst, mask, fwd, mul, inv, skip, pole, scale, units, st, spec, dy, cm);
}

template <int N> constexpr int vrows_nr() { return rows_nr<N>() / 2; }
constexpr int pow2_floor(int x) { int p = 1; while (p * 2 <= x) p *= 2; return p; }
template <int N> constexpr int vrows_nt() { return clamp_nt(pow2_floor(6 * vrows_nr<N>() * N / 16)); }
template <typename T, int N>
cudaError_t rows_inv_vec_n(const GV<T>& g, Buf<typename Cx<T>::t> A, Buf<typename Cx<T>::t> B,
                           Buf<typename Cx<T>::t> out, int mask, int skip, int mode, int jj, int units,
                           cudaStream_t st) {
  using C = typename Cx<T>::t;
  constexpr int NR = vrows_nr<N>(), NT = vrows_nt<N>();
  static_assert((NR * N) % NT == 0, "vector epilogue needs a whole number of points per thread");
  const size_t sm = smem_elems<N, 6 * NR, false>() * sizeof(C);
  auto k = sizeof(T) == 4 ? k_rows_inv_vec_occ<T, N, NR, NT> : k_rows_inv_vec<T, N, NR, NT>;
  static bool attr = false;
  cudaError_t e = set_smem_once(k, sm, attr);
  if (e != cudaSuccess) return e;
  dim3 grid(g.ny / NR, units);
  return launch_pdl(k, grid, dim3(NT), sm, st, g, A, B, out, mask, skip, mode, jj);
}

#define PROP_SIZE_SWITCH(n, CALL)                      \
  switch (n) {                                         \
    case 16: return CALL(16);                          \
    case 32: return CALL(32);                          \
    case 64: return CALL(64);                          \
    case 128: return CALL(128);                        \
    case 256: return CALL(256);                        \
    case 384: return CALL(384);                        \
    case 512: return CALL(512);                        \
    case 768: return CALL(768);                        \
    case 1024: return CALL(1024);                      \
    default: return cudaErrorInvalidValue;             \
  }

template <typename T, typename SRC>
cudaError_t rows_fwd(const GV<T>& g, Buf<SRC> src, Buf<typename Cx<T>::t> dst, int mask, double* nacc, int units,
                     cudaStream_t st) {
#define CALL(N) rows_fwd_n<T, N, SRC>(g, src, dst, mask, nacc, units, st)
  PROP_SIZE_SWITCH(g.nx, CALL)
#undef CALL
}
template <typename T>
cudaError_t rows_inv(const GV<T>& g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst, int mask, int skip,
                     EpiArgs ep, int units, cudaStream_t st) {
#define CALL(N) rows_inv_n<T, N>(g, src, dst, mask, skip, ep, units, st)
  PROP_SIZE_SWITCH(g.nx, CALL)
#undef CALL
}
template <typename T>
cudaError_t cols(const GV<T>& g, Buf<typename Cx<T>::t> src, Buf<typename Cx<T>::t> dst, int mask, int fwd, int mul,
                 int inv, int skip, int pole, T scale, int units, cudaStream_t st,
                 Buf<typename Cx<T>::t> spec = Buf<typename Cx<T>::t>{nullptr, 0, 1},
                 Buf<typename Cx<T>::t> dy = Buf<typename Cx<T>::t>{nullptr, 0, 1},
                 ColMaps cm = ColMaps{nullptr, nullptr, nullptr, nullptr}) {
#define CALL(N) cols_n<T, N>(g, src, dst, mask, fwd, mul, inv, skip, pole, scale, units, st, spec, dy, cm)
  PROP_SIZE_SWITCH(g.ny, CALL)
#undef CALL
}
template <typename T>
cudaError_t rows_inv_vec(const GV<T>& g, Buf<typename Cx<T>::t> A, Buf<typename Cx<T>::t> B,
                         Buf<typename Cx<T>::t> out, int mask, int skip, int mode, int jj, int units,
                         cudaStream_t st) {
#define CALL(N) rows_inv_vec_n<T, N>(g, A, B, out, mask, skip, mode, jj, units, st)
  PROP_SIZE_SWITCH(g.nx, CALL)
#undef CALL
}

EpiArgs epi(int mode, int jj = 0, const double2* in64 = nullptr, double2* out64 = nullptr,
            const void* aux = nullptr, int kxsel = 0, void* fwd_out = nullptr) {
  EpiArgs e; e.mode = mode; e.jj = jj; e.in64 = in64; e.out64 = out64; e.aux = aux; e.kxsel = kxsel;
  e.fwd_out = fwd_out;
  return e;
}

int vec_blocks(long L) { return (int)std::max<long>(1, std::min<long>(2048, (L + NT_VEC * 4 - 1) / (NT_VEC * 4))); }

#define CK(...)                                      \
  do {                                               \
    cudaError_t e_ = (__VA_ARGS__);                  \
    if (e_ != cudaSuccess) return PROP_E_CUDA;       \
  } while (0)

// ---------------------------------------------------------------------------
// Host-side tables
// ---------------------------------------------------------------------------
template <typename T> void twiddles(int n, std::vector<T>& out) {
  out.resize(2 * n);
  for (int m = 0; m < n; ++m) {
    const double a = -2.0 * M_PI * (double)m / (double)n;
    out[2 * m] = (T)std::cos(a);
    out[2 * m + 1] = (T)std::sin(a);
  }
}

double kfreq(int i, int n, double d) {   // angular wavenumber of FFT index i
  const int f = (i < (n + 1) / 2) ? i : i - n;
  return 2.0 * M_PI * (double)f / ((double)n * d);
}

// -k^2/(k0n0)^2 - Re p/2 as (hi, lo) pairs for each pole and the zero pole
template <typename T> void axis_table(int n, double d, double k0n0, const std::vector<cplx>& poles, std::vector<T>& out) {
  const int P = (int)poles.size();
  out.resize((size_t)(P + 1) * n * 2);
  for (int k = 0; k <= P; ++k) {
    const double pre = k < P ? poles[k].real() : 0.0;
    for (int i = 0; i < n; ++i) {
      const double kk = kfreq(i, n, d);
      const double v = -(kk * kk) / (k0n0 * k0n0) - 0.5 * pre;
      const T hi = (T)v;
      const T lo = (T)(v - (double)hi);
      out[((size_t)k * n + i) * 2] = hi;
      out[((size_t)k * n + i) * 2 + 1] = lo;
    }
  }
}

template <typename T> int upload_group_tables(prop* h, Group& G) {
  const double k0n0 = h->k0 * h->n0;
  std::vector<T> tw;
  char* b = h->ws;
  twiddles<T>(G.nx, tw);
  CK(cudaMemcpyAsync(b + G.off.twx, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  std::vector<T> twy;
  twiddles<T>(G.ny, twy);
  CK(cudaMemcpyAsync(b + G.off.twy, twy.data(), twy.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  std::vector<T> ax, ay;
  axis_table<T>(G.nx, G.dx, k0n0, h->poles, ax);
  axis_table<T>(G.ny, G.dy, k0n0, h->poles, ay);
  CK(cudaMemcpyAsync(b + G.off.ax, ax.data(), ax.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(b + G.off.ay, ay.data(), ay.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  std::vector<T> pim(h->P + 1);
  for (int k = 0; k < h->P; ++k) pim[k] = (T)(-h->poles[k].imag());
  pim[h->P] = (T)0;
  CK(cudaMemcpyAsync(b + G.off.pim, pim.data(), pim.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  // (r(zeta_fs) - 1)/(nx ny), r evaluated in FP64 and rounded once
  std::vector<T> bm((size_t)G.npts * 2);
  const double sc = 1.0 / (double)G.npts;
  std::vector<double> kx2(G.nx), ky2(G.ny);
  for (int i = 0; i < G.nx; ++i) { const double k = kfreq(i, G.nx, G.dx); kx2[i] = k * k / (k0n0 * k0n0); }
  for (int j = 0; j < G.ny; ++j) { const double k = kfreq(j, G.ny, G.dy); ky2[j] = k * k / (k0n0 * k0n0); }
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      const cplx z(-(kx2[i] + ky2[j]), 0.0);
      cplx r = h->r0 - 1.0;
      for (int k = 0; k < h->P; ++k) r += h->res[k] / (z - h->poles[k]);
      r *= sc;
      bm[((size_t)j * G.nx + i) * 2] = (T)r.real();
      bm[((size_t)j * G.nx + i) * 2 + 1] = (T)r.imag();
    }
  CK(cudaMemcpyAsync(b + G.off.basemul, bm.data(), bm.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  // ||Z - p_k I|| <= max over the grid's free-space spectrum of |zeta - p_k| + 0.5 (|delta| <= 0.5),
  // and the per-pole tolerance factors mu_k (see conv_threshold): the spectrum is taken as the
  // segment [zeta_min - 0.5, 0.5] of the real axis.
  {
    const double kxm = M_PI / G.dx, kym = M_PI / G.dy;
    const double zmin = -(kxm * kxm + kym * kym) / (k0n0 * k0n0);
    std::vector<double> an(2 * h->P);
    std::vector<double> ratio(h->P);
    double rmax = 0.0;
    for (int k = 0; k < h->P; ++k) {
      an[k] = std::max(std::abs(cplx(zmin, 0.0) - h->poles[k]), std::abs(h->poles[k])) + 0.5;
      const double re = h->poles[k].real(), im = h->poles[k].imag();
      const double dxs = std::max(0.0, std::max((zmin - 0.5) - re, re - 0.5));
      const double dist = std::max(std::hypot(dxs, im), 1e-12);
      ratio[k] = std::abs(h->res[k]) / dist;
      rmax = std::max(rmax, ratio[k]);
    }
    for (int k = 0; k < h->P; ++k) an[h->P + k] = ratio[k] > 0 ? std::min(100.0, std::max(1.0, rmax / ratio[k])) : 100.0;
    CK(cudaMemcpyAsync(b + G.off.anorm, an.data(), an.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  std::vector<double> pl(2 * h->P);
  for (int k = 0; k < h->P; ++k) { pl[2 * k] = h->poles[k].real(); pl[2 * k + 1] = h->poles[k].imag(); }
  CK(cudaMemcpyAsync(b + G.off.poles, pl.data(), pl.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  std::vector<double> rk(2 * h->P);
  for (int k = 0; k < h->P; ++k) { rk[2 * k] = h->res[k].real(); rk[2 * k + 1] = h->res[k].imag(); }
  CK(cudaMemcpyAsync(b + G.off.rk, rk.data(), rk.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  // the host vectors must outlive the async copies
  CK(cudaStreamSynchronize(h->stream));
  return PROP_OK;
}

// ---------------------------------------------------------------------------
// Launch accounting
// ---------------------------------------------------------------------------
enum Kind { K_ROWS_FWD, K_COLS, K_ROWS_INV, K_FIELD_IO, K_GRAM, K_GS_UPDATE, K_COMBINE, K_RESIDUE, K_MEDIUM,
            K_CONTROL, K_INIT, K_SCALE, K_GUESS };
const char* kind_name(int k) {
  static const char* n[PROP_NKINDS] = {"rows_fwd", "cols", "rows_inv", "field_io", "gram", "gs_update", "combine",
                                       "residue_sum", "medium", "control", "init_systems", "scale_v0",
                                       "guess_net"};
  return n[k];
}

cudaEvent_t take_event(prop* h) {
  if (!h->pool.empty()) { cudaEvent_t e = h->pool.back(); h->pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Resolve recorded event pairs; call only after the stream has been synchronised.
// Resolve the recorded event pairs whose launches have finished (the end event has
// completed); pairs still in flight stay pending.
void resolve_pending(prop* h) {
  size_t keep = 0;
  for (size_t i = 0; i < h->pending.size(); ++i) {
    auto& p = h->pending[i];
    if (cudaEventQuery(p.b) != cudaSuccess) { h->pending[keep++] = p; continue; }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) h->k_ms[p.kind] += ms;
    h->pool.push_back(p.a);
    h->pool.push_back(p.b);
  }
  h->pending.resize(keep);
  cudaGetLastError();
}

// Counts one launch of `kind` moving `bytes` algorithmic bytes; with profiling
// on, brackets it with events on the handle's stream.
struct Prof {
  prop* h; int kind; double bytes; cudaEvent_t a;
  Prof(prop* h_, int kind_, double bytes_) : h(h_), kind(kind_), bytes(bytes_), a(nullptr) {
    h->launches += 1;
    h->k_launches[kind] += 1;
    h->k_bytes[kind] += bytes;
    if (h->profiling) { a = take_event(h); cudaEventRecord(a, h->stream); }
  }
  ~Prof() {
    if (a) {
      cudaEvent_t b = take_event(h);
      cudaEventRecord(b, h->stream);
      h->pending.push_back({kind, bytes, a, b});
    }
  }
};

// ---------------------------------------------------------------------------
// The step
// ---------------------------------------------------------------------------
// Status of the asynchronous-copy error word: 1 = a bounded wait gave up,
// 2 = a TMA kernel's alignment self-check failed (it skipped its work).
int async_status(int e) { return e == 0 ? PROP_OK : (e == 2 ? PROP_E_WORKSPACE : PROP_E_TIMEOUT); }

int* count_slots(prop* h, int slot) { return (int*)(h->ws + h->counts_off) + slot * CSLOT; }

// Profiling only: a device spin heads each run of launches that the host enqueues
// after waiting on the device, so that the GPU does not reach a launch's opening
// event before the host has submitted the launch itself; the event pairs then time
// the kernels, not the host's submission of them.  Bounded by the global timer
// and by an iteration count.
constexpr long long PROF_GATE_NS = 200000;
__global__ void k_spin(long long ns) {
  long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0; it < (1 << 24); ++it) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 >= ns) break;
  }
}
void profile_gate(prop* h) {
  if (h->profiling) k_spin<<<1, 32, 0, h->stream>>>(PROF_GATE_NS);
}

// The whole counts area (every slot set and the error word) into buf[COUNT_INTS].
int read_count_area(prop* h, int* buf) {
  if (cudaMemcpyAsync(buf, h->ws + h->counts_off, COUNT_INTS * sizeof(int), cudaMemcpyDeviceToHost, h->stream) !=
      cudaSuccess)
    return PROP_E_CUDA;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PROP_E_CUDA;
  if (!h->pending.empty()) resolve_pending(h);
  profile_gate(h);
  return async_status(buf[ERR_SLOT]);
}

int read_counts(prop* h, int* c3, int slot) {
  int buf[COUNT_INTS];
  const int rc = read_count_area(h, buf);
  if (rc == PROP_E_CUDA) return rc;
  c3[0] = buf[slot * CSLOT]; c3[1] = buf[slot * CSLOT + 1]; c3[2] = buf[slot * CSLOT + 2];
  return rc;
}

// One group's step, in parts, so that several groups can advance in lockstep:
// begin() (free-space part, right-hand sides, first count of iterating systems),
// init() (after that count is read: initial guess, v_0), arnoldi() (the Arnoldi
// steps of one GMRES cycle, this group alone), cycle_end() (solution update, true
// residual, restart; count not read) and finish() (residue sum, commit).  The
// counts go to count-slot set `slot`.
template <typename T> struct StepGroup {
  using C = typename Cx<T>::t;
  prop* h;
  Group& G;
  int slot;
  GV<T> g, ga;             // ga: the Arnoldi launches (grid rows = the listed iterating systems)
  cudaStream_t st;
  int Cn, P, nb, nsys, m;
  long F;                  // points of one field
  double cs, pts;
  T scale;
  int* counts;
  double2* Wn;             // the new field
  int tb, tg, vb, gs_blocks, gram_blocks, bw;
  double breakdown;
  ColMaps bmaps, tmaps, dmaps;
  Buf<C> none;
  int* ulist;
  int c3[3] = {0, 0, 0};   // last count read: iterating, ending their cycle, flags
  int n_inh = 0;           // beams with a non-zero delta
  bool any_used = false;   // some system runs GMRES this step
  bool done = false;       // the step needed no GMRES (homogeneous medium)

  StepGroup(prop* h_, Group& G_, int slot_) : h(h_), G(G_), slot(slot_) {
    g = view<T>(h, G);
    st = h->stream;
    Cn = h->C; P = h->P; nb = g.nb; nsys = g.nsys; m = h->m;
    F = (long)Cn * g.npts;
    cs = (double)sizeof(C); pts = (double)g.npts;
    scale = (T)(1.0 / (double)g.npts);
    counts = count_slots(h, slot);
    Wn = (double2*)(h->ws + (G.cur == 0 ? G.off.W64b : G.off.W64a));
    tb = 128; tg = (nsys + tb - 1) / tb;
    vb = vec_blocks(F);
    gs_blocks = (int)((F + NT_VEC * EPT_GS - 1) / (NT_VEC * EPT_GS));
    gram_blocks = (int)((F + NT_VEC * EPT_GRAM - 1) / (NT_VEC * EPT_GRAM));
    bw = h->prec == PROP_FP32 ? 1 : 0;
    breakdown = sizeof(T) == 4 ? 1e-6 : 1e-14;
    const ColMaps nomaps{nullptr, nullptr, nullptr, nullptr};
    bmaps = G.tma ? ColMaps{&G.tm_btmp, &G.tm_btmp, &G.tm_tab, nullptr} : nomaps;
    tmaps = G.tma ? ColMaps{&G.tm_tmp, &G.tm_tmp, nullptr, nullptr} : nomaps;
    dmaps = G.tma_dy ? ColMaps{&G.tm_tmp, &G.tm_tmp, nullptr, &G.tm_tmp2} : nomaps;
    none = Buf<C>{nullptr, 0, 1};
    ulist = (int*)(h->ws + G.off.ulist);
    ga = g;
    ga.ulist = ulist;
  }

  int begin() {
  // which beams carry a non-zero delta (read back once per medium change)
  if (G.medium_dirty) {
    G.nonhomog_host.assign(nb, 0);
    CK(cudaMemcpyAsync(G.nonhomog_host.data(), g.nonhomog, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    profile_gate(h);
    G.medium_dirty = false;
  }
  n_inh = 0;
  for (int b = 0; b < nb; ++b) n_inh += G.nonhomog_host[b] ? 1 : 0;

  // w_hat = FFT2(w); ||w||^2 per beam
  CK(cudaMemsetAsync(g.bnorm2, 0, nb * sizeof(double), st));
  if (n_inh == 0 && G.carry) {
    // homogeneous step after a homogeneous step: the previous inverse row pass already
    // left the forward row DFT of this field in Btmp
  } else if constexpr (sizeof(T) == 4) {   // the hi plane of the double-float field is the FP32 working copy
    Prof p_(h, K_ROWS_FWD, 2 * cs * pts * nb * Cn);
    CK(rows_fwd<T, float2>(g, buf((float2*)g.W64, F), buf(g.Btmp, F), -1, n_inh ? g.bnorm2 : nullptr, nb, st));
  } else {
    Prof p_(h, K_ROWS_FWD, (16 + cs) * pts * nb * Cn);
    CK(rows_fwd<T, double2>(g, buf(g.W64, F), buf(g.Btmp, F), -1, g.bnorm2, nb, st));
  }
  G.carry = false;
  // column DFT (spectrum kept when poles will need it), then the free-space part
  // Wn = w + IFFT2[(r - 1) w_hat] (Eq. approx_fs_prop), in one column pass
  { Prof p_(h, K_COLS, (n_inh ? 4 : 3) * cs * pts * nb * Cn);
    CK(cols<T>(g, buf(g.Btmp, F), buf(g.Btmp, F), -1, 1, MUL_TABLE, 1, 0, -1, (T)1, nb, st,
               n_inh ? buf(g.What, F) : none, none, bmaps)); }
  if (n_inh == 0) {   // homogeneous: the new field is final, so its row DFT for the next step is formed here
    Prof p_(h, K_ROWS_INV, (2 * cs + 32) * pts * nb * Cn);   // increment, old field, new field, next row DFT
    CK(rows_inv<T>(g, buf(g.Btmp, F), buf(g.Btmp, F), -1, 0,
                   epi(EPI_ACCUM64, 0, nullptr, Wn, nullptr, 0, g.Btmp), nb, st));
  } else {
    Prof p_(h, K_ROWS_INV, (cs + 32) * pts * nb * Cn);   // read increment, old field (16 B), write new (16 B)
    CK(rows_inv<T>(g, buf(g.Btmp, F), buf(g.Btmp, F), -1, 0, epi(EPI_ACCUM64, 0, nullptr, Wn), nb, st));
  }
  if (n_inh == 0) {           // homogeneous medium: the free-space step is exact, no correction
    if (!G.stats_zero) {      // record zero iterations for every system (once)
      Prof p_(h, K_CONTROL, 0);
      CK(launch_pdl(k_step_reset, dim3(tg), dim3(tb), 0, st, g.st, nsys));
      CK(launch_pdl(k_begin_cycle, dim3(tg), dim3(tb), 0, st, g.st, nsys, P, (const double*)g.bnorm2, h->tol, -1, h->max_restarts, 1, g.anorm, bw));
      G.stats_zero = true;
    }
    CK(cudaGetLastError());
    G.cur ^= 1;
    G.carry = true;
    done = true;
    return PROP_OK;
  }
  G.stats_zero = false;
  { Prof p_(h, K_CONTROL, 0);
    CK(launch_pdl(k_step_reset, dim3(tg), dim3(tb), 0, st, g.st, nsys)); }
  const int sys_inh = n_inh * P;
  // correction right-hand sides: R0_k = -delta * IFFT2[w_hat/(zeta - p_k)]
  if (Cn == 2) {   // vector: R0 = -(Z - Z_fs) z_k with the psi and cross-polarisation terms
    { Prof p_(h, K_COLS, 3 * cs * pts * sys_inh * Cn);
      CK(cols<T>(g, buf(g.What, F, P), buf(g.Tmp, F), -1, 0, MUL_POLE_INV, 1, 1, -1, scale, nsys, st,
                 Buf<C>{nullptr, 0, 1}, buf(g.Tmp2, F))); }
    { Prof p_(h, K_ROWS_INV, 11 * cs * pts * sys_inh);
      CK(rows_inv_vec<T>(g, buf(g.Tmp, F), buf(g.Tmp2, F), buf(g.Tmp, F), -1, 1, VEPI_R0, 0, nsys, st)); }
  } else {
    { Prof p_(h, K_COLS, 2 * cs * pts * sys_inh * Cn);
      CK(cols<T>(g, buf(g.What, F, P), buf(g.Tmp, F), -1, 0, MUL_POLE_INV, 1, 1, -1, scale, nsys, st)); }
    { Prof p_(h, K_ROWS_INV, 3 * cs * pts * sys_inh * Cn);
      CK(rows_inv<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), -1, 1, epi(EPI_R0), nsys, st)); }
  }
  { Prof p_(h, K_CONTROL, 0);
    CK(launch_pdl(k_begin_cycle, dim3(tg), dim3(tb), 0, st, g.st, nsys, P, (const double*)g.bnorm2, h->tol, -1, h->max_restarts, 1, g.anorm, bw));
    CK(launch_pdl(k_count, dim3(1), dim3(256), 0, st, (const SysState*)g.st, nsys, counts)); }
  CK(cudaGetLastError());
  return PROP_OK;
  }

  int init() {
  any_used = c3[0] > 0;
  if (any_used && h->guess == PROP_GUESS_LEARNED && h->net_layers > 0) {
    // x0 from the network: E = net(R0/rms, delta, p) * rms, then the true residual R0 - (Z - p) E
    // (the cycle-end pass) starts GMRES from it.
    const int blocks = (int)std::min<long>(1024, (g.npts + 255) / 256);
    __nv_bfloat16* a0 = (__nv_bfloat16*)(h->ws + G.off.act0);
    __nv_bfloat16* a1 = (__nv_bfloat16*)(h->ws + G.off.act1);
    float* nout = (float*)(h->ws + G.off.netout);
    { Prof p_(h, K_GUESS, (Cn * cs + cs + 32.0) * pts * c3[0]);
      k_guess_pack<T, 256><<<dim3(blocks, nsys), 256, 0, st>>>(g, a0, (const double2*)(h->ws + G.off.poles), 1, 0); }
    const char* wbase = h->ws + h->net_off;
    const float* bbase = (const float*)(h->ws + h->net_off + NET_W_BYTES);
    size_t woff = 0, boff = 0;
    for (int l = 0; l < h->net_layers; ++l) {
      const int ci = h->net_ch[l], co = h->net_ch[l + 1];
      const bool last = l == h->net_layers - 1;
      const void* in = (l % 2 == 0) ? (const void*)a0 : (const void*)a1;
      void* out = last ? (void*)nout : ((l % 2 == 0) ? (void*)a1 : (void*)a0);
      Prof p_(h, K_GUESS, (2.0 * ci + (last ? 4.0 : 2.0) * co) * pts * c3[0]);
      if (prop_cnn_conv(ci, co, last ? PROP_CNN_LINEAR_F32 : PROP_CNN_RELU_BF16, in, wbase + woff, bbase + boff, out,
                        nsys, g.ny, g.nx, (const int32_t*)g.st, (int)(sizeof(SysState) / 4), ST_ITER, st) != 0)
        return PROP_E_CUDA;
      woff += (size_t)9 * co * ci * 2;
      boff += co;
    }
    { Prof p_(h, K_GUESS, (64.0 + 16.0 * Cn) * pts * c3[0]);
      k_guess_unpack<T, 256><<<dim3(blocks, nsys), 256, 0, st>>>(g, nout);
      k_guess_mark<<<tg, tb, 0, st>>>(g.st, nsys); }
    const double endp = (double)c3[0] * Cn * pts;
    if (Cn == 2) {
      { Prof p_(h, K_ROWS_FWD, (16 + cs) * endp);
        CK(rows_fwd<T, double2>(g, buf(g.E, F), buf(g.Tmp, F), ST_CYCLE_END, nullptr, nsys, st)); }
      { Prof p_(h, K_COLS, 3 * cs * endp);
        CK(cols<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, 1, MUL_SCALE, 1, 0, -1, scale, nsys, st,
                   Buf<C>{nullptr, 0, 1}, buf(g.Tmp2, F), dmaps)); }
      { Prof p_(h, K_ROWS_INV, 5.5 * cs * endp);
        CK(rows_inv_vec<T>(g, buf(g.Tmp, F), buf(g.Tmp2, F), buf(g.V, (long)(m + 2) * F), ST_CYCLE_END, 0,
                           VEPI_OPDIFF, 0, nsys, st)); }
    }
    { Prof p_(h, K_ROWS_FWD, (16 + cs) * endp);
      CK(rows_fwd<T, double2>(g, buf(g.E, F), buf(g.Tmp, F), ST_CYCLE_END, nullptr, nsys, st)); }
    { Prof p_(h, K_COLS, 2 * cs * endp);
      CK(cols<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, 1, MUL_POLE_FWD, 1, 0, -1, scale, nsys, st, none, none,
                 tmaps)); }
    { Prof p_(h, K_ROWS_INV, (4 * cs + 16) * endp);
      CK(rows_inv<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, 0, epi(EPI_TRUERES), nsys, st)); }
    { Prof p_(h, K_CONTROL, 0);
      k_guess_alpha<<<tg, tb, 0, st>>>(g.st, nsys); }
    { Prof p_(h, K_GUESS, (4.0 * cs + 32.0) * endp);
      k_guess_apply<T, NT_VEC><<<dim3(vb, nsys), NT_VEC, 0, st>>>(g); }
    { Prof p_(h, K_CONTROL, 0);
      CK(launch_pdl(k_begin_cycle, dim3(tg), dim3(tb), 0, st, g.st, nsys, P, (const double*)g.bnorm2, h->tol, (int)ST_CYCLE_END, h->max_restarts, 0, g.anorm, bw)); }
    { Prof p_(h, K_SCALE, 2 * cs * endp);
      CK(launch_pdl(k_scale_v0<T, NT_VEC>, dim3(vb, nsys), dim3(NT_VEC), 0, st, g)); }
    { Prof p_(h, K_CONTROL, 0);
      CK(launch_pdl(k_count, dim3(1), dim3(256), 0, st, (const SysState*)g.st, nsys, counts)); }
    CK(cudaGetLastError());
    const int rc = read_counts(h, c3, slot);
    if (rc) return rc;
  } else if (any_used) {
    { Prof p_(h, K_INIT, (cs + 16) * pts * c3[0] * Cn);
      CK(launch_pdl(k_init_systems<T, NT_VEC>, dim3(vb, nsys), dim3(NT_VEC), 0, st, g)); }
    { Prof p_(h, K_SCALE, 2 * cs * pts * c3[0] * Cn);
      CK(launch_pdl(k_scale_v0<T, NT_VEC>, dim3(vb, nsys), dim3(NT_VEC), 0, st, g)); }
  }
  return PROP_OK;
  }

  int arnoldi() {
  // Steps are launched in batches of SYNC_EVERY between host reads: every
  // kernel skips systems that have left ST_ITER, so launches past a cycle end
  // are empty.  Each step's control adds its system to the step's count slot
  // (continuing, ending the cycle, flags), zeroed at the batch start; the
  // algorithmic bytes of each launch are charged from these counts exactly.
  // Step j = m only finalises column m-1: no operator application, and the
  // Gram sweep forms the products with u alone.
  // Two batches are kept in flight: batch b+1 is enqueued, sized by the last
  // count the host has seen (a superset of the iterating systems: systems only
  // leave), before the host waits for batch b's counts, so the GPU does not idle
  // while the host reads them.  Each batch has its own count slots (parity).
  struct Batch { int jj0, nb, par; };
  Batch fl[2];
  int nfl = 0, jj = 0, ended = 0, flags = 0;
  int act_est = c3[0];        // for sizing launches
  int before = c3[0];         // systems iterating at the next unprocessed step
  bool stop = false;
  auto enqueue = [&](int par) -> int {
    const int jb = jj, nb = std::min(SYNC_EVERY, m + 1 - jj);
    int* slots = counts + 3 + par * 3 * SYNC_EVERY;
    CK(cudaMemsetAsync(slots, 0, 3 * SYNC_EVERY * sizeof(int), st));
    { Prof p_(h, K_CONTROL, 0);
      CK(launch_pdl(k_active_list, dim3(1), dim3(256), 0, st, (const SysState*)g.st, nsys, ulist)); }
    const int act = std::max(act_est, 1);
    for (int j = jb; j < jb + nb; ++j) {
      const bool op = j < m;
      if (op) {
        C* Vj = g.V + (long)j * F;
        const long vs = (long)(m + 2) * F;
        { Prof p_(h, K_ROWS_FWD, 0);
          CK(rows_fwd<T, C>(ga, buf(Vj, vs), buf(g.Tmp, F), ST_ITER, nullptr, act, st)); }
        if (Cn == 2) {
          { Prof p_(h, K_COLS, 0);
            CK(cols<T>(ga, buf(g.Tmp, F), buf(g.Tmp, F), ST_ITER, 1, MUL_PREC_INV, 1, 0, -1, scale, act, st,
                       Buf<C>{nullptr, 0, 1}, buf(g.Tmp2, F), dmaps)); }
          { Prof p_(h, K_ROWS_INV, 0);
            CK(rows_inv_vec<T>(ga, buf(g.Tmp, F), buf(g.Tmp2, F), buf(g.Tmp, F), ST_ITER, 0, VEPI_ARNOLDI, j, act,
                               st)); }
        } else {
          { Prof p_(h, K_COLS, 0);
            CK(cols<T>(ga, buf(g.Tmp, F), buf(g.Tmp, F), ST_ITER, 1, MUL_PREC_INV, 1, 0, -1, scale, act, st, none,
                       none, tmaps)); }
          { Prof p_(h, K_ROWS_INV, 0);
            CK(rows_inv<T>(ga, buf(g.Tmp, F), buf(g.Tmp, F), ST_ITER, 0, epi(EPI_ARNOLDI, j), act, st)); }
        }
      }
      // sweeps: one wave of CTAs (as many as are resident at once) shared by the
      // act systems; the update sweep keeps a slot per system for its control CTA
      // (at most a quarter of the wave: the control CTAs are short)
      static int occ_gram = 0, occ_step = 0;
      const int wave_g = resident(k_dcgs_gram<T, NT_VEC, EPT_GRAM, GVEC_GRAM>, NT_VEC, occ_gram) * sm_count();
      const int wave_s = resident(k_dcgs_step<T, NT_VEC, EPT_GS, GVEC_GS>, NT_VEC, occ_step) * sm_count();
      const int cap_g = std::max(1, wave_g / act), cap = std::max(1, (wave_s - std::min(act, wave_s / 4)) / act);
      { Prof p_(h, K_GRAM, 0);
        CK(launch_pdl(k_dcgs_gram<T, NT_VEC, EPT_GRAM, GVEC_GRAM>, dim3(std::min(gram_blocks, cap_g), act),
                      dim3(NT_VEC), 0, st, ga, j, op ? 1 : 0)); }
      { Prof p_(h, K_GS_UPDATE, 0);
        StepArgs sa;
        sa.m = m; sa.P = P; sa.backward = bw; sa.tol = h->tol; sa.breakdown = breakdown;
        sa.bnorm2 = g.bnorm2; sa.anorm = g.anorm; sa.counts = slots + 3 * (j - jb);
        CK(launch_pdl(k_dcgs_step<T, NT_VEC, EPT_GS, GVEC_GS>, dim3(std::min(gs_blocks, cap) + 1, act), dim3(NT_VEC),
                      0, st, ga, j, sa)); }
      CK(cudaGetLastError());
    }
    CK(cudaMemcpyAsync(h->hcounts + par * 3 * SYNC_EVERY, slots, 3 * nb * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->batch_ev[par], st));
    fl[nfl++] = Batch{jb, nb, par};
    jj += nb;
    return PROP_OK;
  };
  int next_par = 0;
  while (true) {
    while (!stop && jj <= m && nfl < PIPE_DEPTH) {
      const int rc2 = enqueue(next_par);
      if (rc2) return rc2;
      next_par ^= 1;
    }
    if (nfl == 0) break;
    // the oldest batch's counts
    const Batch bt = fl[0];
    fl[0] = fl[1];
    --nfl;
    if (cudaEventSynchronize(h->batch_ev[bt.par]) != cudaSuccess) return PROP_E_CUDA;
    if (!h->pending.empty()) resolve_pending(h);
    profile_gate(h);
    const int* hc = h->hcounts + bt.par * 3 * SYNC_EVERY;
    for (int b2 = 0; b2 < bt.nb; ++b2) {
      const int j = bt.jj0 + b2;
      const double act = (double)before * Cn * pts;
      if (j < m) {
        h->k_bytes[K_ROWS_FWD] += 2 * cs * act;
        h->k_bytes[K_COLS] += (Cn == 2 ? 3 : 2) * cs * act;
        h->k_bytes[K_ROWS_INV] += (Cn == 2 ? 6.5 : 4.0) * cs * act;
        h->k_bytes[K_GS_UPDATE] += (j + 4.0) * cs * act;   // v_0..v_{j-1}, u, w read; q_j, u_{j+1} written
      }
      h->k_bytes[K_GRAM] += (j + (j < m ? 2.0 : 1.0)) * cs * act;   // v_0..v_{j-1}, u (and w) read
      if (j >= 1) h->total_iters += before;               // column j-1 finalised for each of them
      const int* sl = hc + 3 * b2;
      ended += sl[1];
      flags |= sl[2];
      before = sl[0];
    }
    act_est = before;
    if (before == 0) stop = true;   // any batch still in flight is empty (every launch masked)
  }
  c3[0] = 0; c3[1] = ended; c3[2] = flags;
  return PROP_OK;
  }

  int cycle_end() {
  // cycle end: e += M^-1 (V y) (Tmp = V y, then a free-space solve round trip
  // accumulating into E); true residual r = R0 - (Z - p) e
  const double endp = (double)c3[1] * Cn * pts;
  { Prof p_(h, K_COMBINE, (1 + m) * cs * endp);   // upper bound on the v_i read: J <= m
    CK(launch_pdl(k_combine<T, NT_VEC>, dim3(vb, nsys), dim3(NT_VEC), 0, st, g)); }
  { Prof p_(h, K_ROWS_FWD, 2 * cs * endp);
    CK(rows_fwd<T, C>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, nullptr, nsys, st)); }
  { Prof p_(h, K_COLS, 2 * cs * endp);
    CK(cols<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, 1, MUL_PREC_INV, 1, 0, -1, scale, nsys, st, none, none,
               tmaps)); }
  { Prof p_(h, K_ROWS_INV, (cs + 32) * endp);
    CK(rows_inv<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, 0, epi(EPI_ADD_E), nsys, st)); }
  if (Cn == 2) {   // (Z - Z_fs) e into v_0, from a derivative round trip of e
    { Prof p_(h, K_ROWS_FWD, (16 + cs) * endp);
      CK(rows_fwd<T, double2>(g, buf(g.E, F), buf(g.Tmp, F), ST_CYCLE_END, nullptr, nsys, st)); }
    { Prof p_(h, K_COLS, 3 * cs * endp);
      CK(cols<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, 1, MUL_SCALE, 1, 0, -1, scale, nsys, st,
                 Buf<C>{nullptr, 0, 1}, buf(g.Tmp2, F), dmaps)); }
    { Prof p_(h, K_ROWS_INV, 5.5 * cs * endp);
      CK(rows_inv_vec<T>(g, buf(g.Tmp, F), buf(g.Tmp2, F), buf(g.V, (long)(m + 2) * F), ST_CYCLE_END, 0,
                         VEPI_OPDIFF, 0, nsys, st)); }
  }
  { Prof p_(h, K_ROWS_FWD, (16 + cs) * endp);
    CK(rows_fwd<T, double2>(g, buf(g.E, F), buf(g.Tmp, F), ST_CYCLE_END, nullptr, nsys, st)); }
  { Prof p_(h, K_COLS, 2 * cs * endp);
    CK(cols<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, 1, MUL_POLE_FWD, 1, 0, -1, scale, nsys, st, none, none,
               tmaps)); }
  { Prof p_(h, K_ROWS_INV, (4 * cs + 16) * endp);
    CK(rows_inv<T>(g, buf(g.Tmp, F), buf(g.Tmp, F), ST_CYCLE_END, 0, epi(EPI_TRUERES), nsys, st)); }
  { Prof p_(h, K_CONTROL, 0);
    CK(launch_pdl(k_begin_cycle, dim3(tg), dim3(tb), 0, st, g.st, nsys, P, (const double*)g.bnorm2, h->tol, (int)ST_CYCLE_END, h->max_restarts, 0, g.anorm, bw)); }
  { Prof p_(h, K_SCALE, 0);
    CK(launch_pdl(k_scale_v0<T, NT_VEC>, dim3(vb, nsys), dim3(NT_VEC), 0, st, g)); }
  { Prof p_(h, K_CONTROL, 0);
    CK(launch_pdl(k_count, dim3(1), dim3(256), 0, st, (const SysState*)g.st, nsys, counts)); }
  CK(cudaGetLastError());
  return PROP_OK;
  }

  int finish() {
  if (c3[2] & 1) return PROP_E_NAN;
  if (c3[2] & 2) return PROP_E_NOCONV;
  if (any_used) {
    Prof p_(h, K_RESIDUE, (32.0 + 16.0 * P) * pts * Cn * n_inh);   // upper bound: every pole used
    CK(launch_pdl(k_residue_sum<T, NT_VEC>, dim3(vb, nb), dim3(NT_VEC), 0, st, g, Wn));
  }
  CK(cudaGetLastError());
  G.cur ^= 1;   // commit: the new field becomes current
  return PROP_OK;
  }
};

template <typename T> int step_group(prop* h, Group& G) {
  StepGroup<T> S(h, G, 0);
  int rc = S.begin();
  if (rc || S.done) return rc;
  rc = read_counts(h, S.c3, 0);
  if (rc) return rc;
  rc = S.init();
  if (rc) return rc;
  while (S.c3[0] > 0) {
    rc = S.arnoldi();
    if (rc) return rc;
    if (S.c3[1] == 0) break;
    rc = S.cycle_end();
    if (rc) return rc;
    rc = read_counts(h, S.c3, 0);
    if (rc) return rc;
    h->k_bytes[K_SCALE] += 2 * S.cs * S.pts * S.Cn * S.c3[0];
  }
  return S.finish();
}

// ---------------------------------------------------------------------------
// Multi-group step: every group of the handle in lockstep, each Arnoldi pass one
// launch over all groups (mg.cuh).  Complex FP32, 2..MAXG groups, every grid of a
// size the multi-group kernels take.  Begin, init, cycle end and finish are each
// group's own (StepGroup); their counts are read for all groups at once.
// ---------------------------------------------------------------------------
bool multigroup_ok(const prop* h) {
  if (!h->multigroup || h->prec != PROP_FP32 || h->form != PROP_FORM_EXPONENTIAL) return false;
  const int ng = (int)h->groups.size();
  if (ng < 2 || ng > MAXG) return false;
  for (const Group& G : h->groups) {
    if (!mg_size(G.nx) || !mg_size(G.ny)) return false;
    if (G.ny % mg_nr(G.nx) != 0 || G.ny % mg_nrv(G.nx) != 0) return false;
  }
  return true;
}

// The Arnoldi steps of one GMRES cycle of every live group; afterwards each live
// group's c3 = {0, systems that ended the cycle, flags}.
int arnoldi_multigroup(prop* h, std::vector<StepGroup<float>>& S, const std::vector<char>& live) {
  const int ng = (int)S.size(), m = h->m;
  cudaStream_t st = h->stream;
  int before[MAXG], ended[MAXG], flags[MAXG];
  for (int i = 0; i < ng; ++i) { before[i] = live[i] ? S[i].c3[0] : 0; ended[i] = 0; flags[i] = 0; }
  MGroups mg;
  std::memset(&mg, 0, sizeof(mg));
  int jj = 0;
  while (jj <= m) {
    int idx[MAXG], n = 0;
    for (int i = 0; i < ng; ++i)
      if (before[i] > 0) idx[n++] = i;
    if (n == 0) break;
    const int jb = jj, nbt = std::min(SYNC_EVERY, m + 1 - jj);
    mg.ng = n;
    mg.nzero = 3 * SYNC_EVERY;
    for (int k = 0; k < n; ++k) {
      StepGroup<float>& s = S[idx[k]];
      mg.g[k] = s.ga;
      const bool vec = s.Cn == 2;
      mg.tma[k] = vec ? (s.G.tma_dy ? 1 : 0) : (s.G.tma ? 1 : 0);
      mg.tm[k] = s.G.tm_tmp;
      mg.tm2[k] = s.G.tm_tmp2;
      mg.zero[k] = s.counts + 3;
      StepArgs& sa = mg.sa[k];
      sa.m = m; sa.P = s.P; sa.backward = s.bw; sa.tol = h->tol; sa.breakdown = s.breakdown;
      sa.bnorm2 = s.g.bnorm2; sa.anorm = s.g.anorm; sa.counts = nullptr;
    }
    // sweeps: the CTAs share the listed systems' points evenly.  Systems of one
    // size get one wave (as many CTAs as are resident at once; the update sweep
    // keeps a slot per system for its control CTA, at most a quarter of the
    // wave); systems of several sizes get four waves of equal CTAs, so that the
    // largest grid's CTAs do not form a tail.
    double work = 0;
    int tot = 0;
    bool uniform = true;
    for (int k = 0; k < n; ++k) {
      work += (double)before[idx[k]] * S[idx[k]].F;
      tot += before[idx[k]];
      uniform = uniform && S[idx[k]].F == S[idx[0]].F;
    }
    const int waves = uniform ? 1 : 4;
    const int wave1 = mg_resident(MG_STEP) * sm_count();
    const double wave_g = (double)mg_resident(MG_GRAM) * sm_count() * waves;
    const double wave_s = (double)(wave1 - (uniform ? std::min(tot, wave1 / 4) : 0)) * waves;
    int cap_g[MAXG], cap_s[MAXG];
    for (int k = 0; k < n; ++k) {
      const double share = (double)S[idx[k]].F / std::max(work, 1.0);
      // one wave: round down so that the CTAs fit; several: to nearest
      cap_g[k] = std::max(1, uniform ? (int)(wave_g * share) : (int)std::lround(wave_g * share));
      cap_s[k] = std::max(1, uniform ? (int)(wave_s * share) : (int)std::lround(wave_s * share));
    }
    auto layout = [&](int pass) {
      int c = 0;
      for (int k = 0; k < n; ++k) {
        mg.c0[k] = c;
        mg.gx[k] = mg_gx(pass, mg.g[k], before[idx[k]], pass == MG_STEP ? cap_s[k] : cap_g[k]);
        c += mg.gx[k] * mg_rows(pass, mg.g[k], before[idx[k]]);
      }
      mg.c0[n] = c;
    };
    { Prof p_(h, K_CONTROL, 0);
      CK(mg_launch(MG_ACTIVE, mg, 0, 0, st)); }
    for (int j = jb; j < jb + nbt; ++j) {
      const bool op = j < m;
      if (op) {
        layout(MG_ROWS_FWD);
        { Prof p_(h, K_ROWS_FWD, 0);
          CK(mg_launch(MG_ROWS_FWD, mg, j, 0, st)); }
        layout(MG_COLS);
        { Prof p_(h, K_COLS, 0);
          CK(mg_launch(MG_COLS, mg, j, 0, st)); }
        layout(MG_ROWS_INV);
        { Prof p_(h, K_ROWS_INV, 0);
          CK(mg_launch(MG_ROWS_INV, mg, j, 0, st)); }
      }
      layout(MG_GRAM);
      { Prof p_(h, K_GRAM, 0);
        CK(mg_launch(MG_GRAM, mg, j, op ? 1 : 0, st)); }
      for (int k = 0; k < n; ++k) mg.sa[k].counts = S[idx[k]].counts + 3 + 3 * (j - jb);
      layout(MG_STEP);
      { Prof p_(h, K_GS_UPDATE, 0);
        CK(mg_launch(MG_STEP, mg, j, 0, st)); }
    }
    CK(cudaMemcpyAsync(h->hcounts, h->ws + h->counts_off, COUNT_INTS * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(h->batch_ev[0], st));
    if (cudaEventSynchronize(h->batch_ev[0]) != cudaSuccess) return PROP_E_CUDA;
    if (!h->pending.empty()) resolve_pending(h);
    profile_gate(h);
    // algorithmic bytes charged from the counts, as in the grid-by-grid step
    for (int k = 0; k < n; ++k) {
      const int i = idx[k];
      const StepGroup<float>& s = S[i];
      const int* hc = h->hcounts + i * CSLOT + 3;
      const double cs = s.cs, Cn = s.Cn;
      for (int b2 = 0; b2 < nbt; ++b2) {
        const int j = jb + b2;
        const double act = (double)before[i] * Cn * s.pts;
        if (j < m) {
          h->k_bytes[K_ROWS_FWD] += 2 * cs * act;
          h->k_bytes[K_COLS] += (Cn == 2 ? 3 : 2) * cs * act;
          h->k_bytes[K_ROWS_INV] += (Cn == 2 ? 6.5 : 4.0) * cs * act;
          h->k_bytes[K_GS_UPDATE] += (j + 4.0) * cs * act;
        }
        h->k_bytes[K_GRAM] += (j + (j < m ? 2.0 : 1.0)) * cs * act;
        if (j >= 1) h->total_iters += before[i];
        const int* sl = hc + 3 * b2;
        ended[i] += sl[1];
        flags[i] |= sl[2];
        before[i] = sl[0];
      }
    }
    jj += nbt;
  }
  for (int i = 0; i < ng; ++i)
    if (live[i]) { S[i].c3[0] = 0; S[i].c3[1] = ended[i]; S[i].c3[2] = flags[i]; }
  return PROP_OK;
}

int step_multigroup(prop* h) {
  const int ng = (int)h->groups.size();
  std::vector<StepGroup<float>> S;
  S.reserve(ng);
  for (int i = 0; i < ng; ++i) S.emplace_back(h, h->groups[i], i);
  bool any = false;
  for (StepGroup<float>& s : S) {
    const int rc = s.begin();
    if (rc) return rc;
    any = any || !s.done;
  }
  if (!any) return PROP_OK;
  int buf[COUNT_INTS];
  int rc = read_count_area(h, buf);
  if (rc) return rc;
  std::vector<char> live(ng, 0);
  for (int i = 0; i < ng; ++i) {
    if (S[i].done) continue;
    for (int t = 0; t < 3; ++t) S[i].c3[t] = buf[i * CSLOT + t];
    rc = S[i].init();
    if (rc) return rc;
    live[i] = S[i].c3[0] > 0;
  }
  while (std::find(live.begin(), live.end(), 1) != live.end()) {
    rc = arnoldi_multigroup(h, S, live);
    if (rc) return rc;
    bool any_end = false;
    for (int i = 0; i < ng; ++i) {
      if (!live[i]) continue;
      if (S[i].c3[1] == 0) { live[i] = 0; continue; }
      rc = S[i].cycle_end();
      if (rc) return rc;
      any_end = true;
    }
    if (!any_end) break;
    rc = read_count_area(h, buf);
    if (rc) return rc;
    for (int i = 0; i < ng; ++i) {
      if (!live[i]) continue;
      for (int t = 0; t < 3; ++t) S[i].c3[t] = buf[i * CSLOT + t];
      h->k_bytes[K_SCALE] += 2 * S[i].cs * S[i].pts * S[i].Cn * S[i].c3[0];
      live[i] = S[i].c3[0] > 0;
    }
  }
  for (StepGroup<float>& s : S) {
    if (s.done) continue;
    rc = s.finish();
    if (rc) return rc;
  }
  return PROP_OK;
}

// Spectral derivatives of psi = Log n^2 for the vector operator (Eq. Z_bar_eq),
// scaled by (k0 n0)^-2, into the beam's coefficient planes; the beam's Btmp holds
// psi in plane 0 (written by k_medium) and What serves as scratch.
template <typename T> int psi_derivatives(prop* h, Group& G, int slot) {
  using C = typename Cx<T>::t;
  GV<T> g = view<T>(h, G);
  g.ncomp = 1;   // single planes
  cudaStream_t st = h->stream;
  const long npts = g.npts;
  C* psi = g.Btmp + (long)slot * 2 * npts;
  C* rowft = psi + npts;
  C* colout = g.What + (long)slot * 2 * npts;
  C* planes = g.psi + (long)slot * 5 * npts;
  const double k0n0 = h->k0 * h->n0;
  const T sc = (T)(1.0 / ((double)npts * k0n0 * k0n0));
  { Prof p_(h, K_MEDIUM, 2.0 * sizeof(C) * npts);
    CK(rows_fwd<T, C>(g, buf(psi, npts), buf(rowft, npts), -1, nullptr, 1, st)); }
  // plane: 0 psi_xx, 1 psi_yy, 2 psi_xy, 3 psi_x, 4 psi_y  -> (column factor, row factor)
  const int colmul[5] = {MUL_SCALE, MUL_DYY, MUL_DY, MUL_SCALE, MUL_DY};
  const int rowmul[5] = {2, 0, 1, 1, 0};
  for (int d = 0; d < 5; ++d) {
    { Prof p_(h, K_MEDIUM, 2.0 * sizeof(C) * npts);
      CK(cols<T>(g, buf(rowft, npts), buf(colout, npts), -1, 1, colmul[d], 1, 0, -1, sc, 1, st)); }
    { Prof p_(h, K_MEDIUM, 2.0 * sizeof(C) * npts);
      CK(rows_inv<T>(g, buf(colout, npts), buf(planes + (long)d * npts, npts), -1, 0,
                     epi(EPI_STORE, 0, nullptr, nullptr, nullptr, rowmul[d]), 1, st)); }
  }
  { Prof p_(h, K_MEDIUM, 6.0 * sizeof(C) * npts);
    k_psi_combine<T, 256><<<(int)std::min<long>(1024, (npts + 255) / 256), 256, 0, st>>>(view<T>(h, G), slot); }
  CK(cudaGetLastError());
  return PROP_OK;
}

// E3 of one beam from Gauss's law (prop_get_e3): D' = (1 + delta) w into the
// beam's two Btmp planes, 2-D DFT of both, the spectral combination, inverse
// DFT, division by 1 + delta into the complex128 stage.
template <typename T> int e3_impl(prop* h, Group& G, int slot) {
  using C = typename Cx<T>::t;
  GV<T> g = view<T>(h, G);
  cudaStream_t st = h->stream;
  const long npts = g.npts;
  C* work = g.Btmp + (long)slot * 2 * npts;
  double2* stage = (double2*)(h->ws + G.off.stage);
  const int blocks = (int)std::min<long>(1024, (npts + 255) / 256);
  { Prof p_(h, K_FIELD_IO, (16.0 + 3 * sizeof(C)) * npts);
    k_e3_pre<T, 256><<<blocks, 256, 0, st>>>(g, slot, work); }
  CK(cudaGetLastError());
  GV<T> g1 = g;
  g1.ncomp = 1;   // two single planes
  { Prof p_(h, K_ROWS_FWD, 4.0 * sizeof(C) * npts);
    CK(rows_fwd<T, C>(g1, buf(work, npts), buf(work, npts), -1, nullptr, 2, st)); }
  { Prof p_(h, K_COLS, 4.0 * sizeof(C) * npts);
    CK(cols<T>(g1, buf(work, npts), buf(work, npts), -1, 1, MUL_NONE, 0, 0, -1, (T)1, 2, st)); }
  { Prof p_(h, K_FIELD_IO, 3.0 * sizeof(C) * npts);
    k_e3_spectral<T, 256><<<blocks, 256, 0, st>>>(g, work, h->k0 * h->n0); }
  CK(cudaGetLastError());
  { Prof p_(h, K_COLS, 2.0 * sizeof(C) * npts);
    CK(cols<T>(g1, buf(work, npts), buf(work, npts), -1, 0, MUL_NONE, 1, 0, -1, (T)1, 1, st)); }
  { Prof p_(h, K_ROWS_INV, 2.0 * sizeof(C) * npts);
    CK(rows_inv<T>(g1, buf(work, npts), buf(work, npts), -1, 0, epi(EPI_STORE), 1, st)); }
  { Prof p_(h, K_FIELD_IO, (16.0 + 2 * sizeof(C)) * npts);
    k_e3_post<T, 256><<<blocks, 256, 0, st>>>(g, slot, work, stage); }
  CK(cudaGetLastError());
  G.carry = false;   // the beam's Btmp planes were used as scratch
  return PROP_OK;
}

int validate_opts(const prop_opts* o) {
  if (!o) return PROP_E_ARG;
  if (o->ncomp != 1 && o->ncomp != 2) return PROP_E_UNSUPPORTED;
  if (o->precision != PROP_FP32 && o->precision != PROP_FP64) return PROP_E_ARG;
  if (o->restart < 1 || o->restart > MMAX) return PROP_E_ARG;
  if (o->max_restarts < 1) return PROP_E_ARG;
  if (!(o->tol > 0.0)) return PROP_E_ARG;
  if (o->guess != PROP_GUESS_ZERO && o->guess != PROP_GUESS_LEARNED) return PROP_E_ARG;
  if (o->precond != PROP_PRECOND_FREESPACE && o->precond != PROP_PRECOND_MEAN) return PROP_E_ARG;
  if (o->form != PROP_FORM_EXPONENTIAL && o->form != PROP_FORM_PSEUDODIFF) return PROP_E_ARG;
  if (o->substeps < 0 || o->substeps > 100000) return PROP_E_ARG;
  if (o->multigroup != 0 && o->multigroup != 1) return PROP_E_ARG;
  return PROP_OK;
}

int build_groups(int nbeams, const prop_grid* grids, std::vector<Group>& groups, std::vector<int>& bg,
                 std::vector<int>& bs) {
  groups.clear();
  bg.assign(nbeams, -1);
  bs.assign(nbeams, -1);
  for (int b = 0; b < nbeams; ++b) {
    const prop_grid& gr = grids[b];
    if (!supported_n(gr.nx) || !supported_n(gr.ny)) return PROP_E_UNSUPPORTED;
    if (!(gr.dx > 0) || !(gr.dy > 0)) return PROP_E_ARG;
    int gi = -1;
    for (size_t i = 0; i < groups.size(); ++i)
      if (groups[i].nx == gr.nx && groups[i].ny == gr.ny && groups[i].dx == gr.dx && groups[i].dy == gr.dy) gi = (int)i;
    if (gi < 0) {
      Group G;
      G.nx = gr.nx; G.ny = gr.ny; G.dx = gr.dx; G.dy = gr.dy; G.npts = (long)gr.nx * gr.ny; G.cur = 0;
      G.medium_dirty = true;
      G.stats_zero = false;
      G.carry = false;
      groups.push_back(G);
      gi = (int)groups.size() - 1;
    }
    bg[b] = gi;
    bs[b] = (int)groups[gi].beams.size();
    groups[gi].beams.push_back(b);
  }
  return PROP_OK;
}

size_t total_layout(std::vector<Group>& groups, int P, int C, int m, int prec, int guess, int form,
                    size_t* counts_off, size_t* net_off) {
  size_t o = 0;
  for (Group& G : groups) o = carve(G, o, P, C, m, prec, guess, form);
  *net_off = align_up(o);
  *counts_off = align_up(*net_off + NET_W_BYTES + NET_B_BYTES);
  return *counts_off + align_up(COUNT_INTS * sizeof(int));
}

}  // namespace

// error word of prop_selftest_wait_timeout
static __device__ int g_selftest_err;

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int prop_default_opts(prop_opts* o, int32_t ncomp, int32_t precision) {
  if (!o) return PROP_E_ARG;
  o->ncomp = ncomp;
  o->precision = precision;
  o->restart = 20;
  o->max_restarts = precision == PROP_FP64 ? 50 : 200;
  o->tol = precision == PROP_FP64 ? 1e-12 : 1e-7;
  o->guess = PROP_GUESS_ZERO;
  o->precond = PROP_PRECOND_MEAN;
  o->form = PROP_FORM_EXPONENTIAL;
  o->substeps = 0;
  o->multigroup = 1;
  return PROP_OK;
}

int prop_workspace_size(int32_t nbeams, const prop_grid* grids, int32_t npoles, const prop_opts* opts, size_t* bytes) {
  if (nbeams < 1 || !grids || npoles < 1 || !bytes) return PROP_E_ARG;
  int rc = validate_opts(opts);
  if (rc) return rc;
  std::vector<Group> groups;
  std::vector<int> bg, bs;
  rc = build_groups(nbeams, grids, groups, bg, bs);
  if (rc) return rc;
  size_t co, no;
  *bytes = total_layout(groups, npoles, opts->ncomp, opts->restart, opts->precision, opts->guess, opts->form, &co,
                        &no);
  return PROP_OK;
}

int prop_create(int32_t nbeams, const prop_grid* grids, double k0, double n0, double dz, int32_t npoles,
                const double* poles, const double* residues, const double r0[2], const prop_opts* opts,
                void* d_workspace, size_t ws_bytes, void* stream, prop** out) {
  if (!out) return PROP_E_ARG;
  *out = nullptr;
  if (nbeams < 1 || !grids || npoles < 1 || !poles || !residues || !r0) return PROP_E_ARG;
  if (!(k0 > 0) || !(n0 > 0) || !(dz > 0)) return PROP_E_ARG;
  int rc = validate_opts(opts);
  if (rc) return rc;
  if (!d_workspace || ((uintptr_t)d_workspace % ALIGN) != 0) return PROP_E_WORKSPACE;
  prop* h = new (std::nothrow) prop();
  if (!h) return PROP_E_ARG;
  h->nbeams = nbeams; h->P = npoles; h->C = opts->ncomp; h->prec = opts->precision; h->m = opts->restart;
  h->max_restarts = opts->max_restarts; h->tol = opts->tol; h->precond = opts->precond;
  h->form = opts->form; h->substeps = opts->substeps; h->multigroup = opts->multigroup; h->k0 = k0; h->n0 = n0; h->dz = dz;
  h->poles.resize(npoles); h->res.resize(npoles);
  for (int k = 0; k < npoles; ++k) {
    h->poles[k] = cplx(poles[2 * k], poles[2 * k + 1]);
    h->res[k] = cplx(residues[2 * k], residues[2 * k + 1]);
  }
  h->r0 = cplx(r0[0], r0[1]);
  h->grids.assign(grids, grids + nbeams);
  rc = build_groups(nbeams, grids, h->groups, h->beam_group, h->beam_slot);
  if (rc) { delete h; return rc; }
  h->guess = opts->guess;
  h->net_layers = 0;
  if (h->form == PROP_FORM_PSEUDODIFF && h->substeps == 0) {
    // the fewest RK4 steps with h |lambda| <= 2.5, |lambda| <= k0 n0 (1 + sqrt(1.5 + |zeta_min|))
    // for lambda = i k0 n0 (S(zeta) - 1) over the grids' spectra (medium terms within 0.5)
    double lam = 0.0;
    for (int b = 0; b < nbeams; ++b) {
      const double kx = M_PI / grids[b].dx, ky = M_PI / grids[b].dy, k0n0 = k0 * n0;
      const double zmin = (kx * kx + ky * ky) / (k0n0 * k0n0);
      lam = std::max(lam, k0n0 * (1.0 + std::sqrt(1.5 + zmin)));
    }
    h->substeps = std::max(1, (int)std::ceil(dz * lam / 2.5));
  }
  const size_t need = total_layout(h->groups, h->P, h->C, h->m, h->prec, h->guess, h->form, &h->counts_off,
                                   &h->net_off);
  if (ws_bytes < need) { delete h; return PROP_E_WORKSPACE; }
  h->ws = (char*)d_workspace; h->ws_bytes = ws_bytes;
  h->stream = (cudaStream_t)stream;
  h->steps = 0; h->total_iters = 0; h->last_status = 0;
  h->launches = 0; h->profiling = 0;
  for (int k = 0; k < PROP_NKINDS; ++k) { h->k_launches[k] = 0; h->k_ms[k] = 0.0; h->k_bytes[k] = 0.0; }
  h->hcounts = nullptr;
  h->batch_ev[0] = h->batch_ev[1] = nullptr;
  if (cudaHostAlloc((void**)&h->hcounts, COUNT_INTS * sizeof(int), cudaHostAllocDefault) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->batch_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->batch_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    prop_destroy(h);
    return PROP_E_CUDA;
  }
  if (cudaMemsetAsync(h->ws, 0, need, h->stream) != cudaSuccess) { prop_destroy(h); return PROP_E_CUDA; }
  for (Group& G : h->groups) {
    rc = h->prec == PROP_FP64 ? upload_group_tables<double>(h, G) : upload_group_tables<float>(h, G);
    if (rc) { prop_destroy(h); return rc; }
    const int csz = 2 * (int)elem_size(h->prec);   // bytes per complex element
    const int nv = h->prec == PROP_FP64 ? cols_per_cta<double>() : cols_per_cta<float>();
    const long nb = (long)G.beams.size();
    G.tma = make_col_map(&G.tm_btmp, h->ws + G.off.Btmp, G.nx, G.ny, nb * h->C, csz, nv) &&
            make_col_map(&G.tm_tmp, h->ws + G.off.Tmp, G.nx, G.ny, nb * h->P * h->C, csz, nv) &&
            make_col_map(&G.tm_tab, h->ws + G.off.basemul, G.nx, G.ny, 1, csz, nv);
    G.tma_dy = G.tma && h->C == 2 &&
               make_col_map(&G.tm_tmp2, h->ws + G.off.Tmp2, G.nx, G.ny, nb * h->P * h->C, csz, nv);
  }
  *out = h;
  return PROP_OK;
}

int prop_set_medium(prop* h, int32_t beam, const void* n2) {
  if (!h || !n2 || beam < 0 || beam >= h->nbeams) return PROP_E_ARG;
  Group& G = h->groups[h->beam_group[beam]];
  const int slot = h->beam_slot[beam];
  void* stage = h->ws + G.off.stage;
  CK(cudaMemcpyAsync(stage, n2, G.npts * 16, cudaMemcpyDefault, h->stream));
  int* nh = (int*)(h->ws + G.off.nonhomog) + slot;
  CK(cudaMemsetAsync(nh, 0, sizeof(int), h->stream));
  double2* ds = (double2*)(h->ws + G.off.dsum) + slot;
  CK(cudaMemsetAsync(ds, 0, sizeof(double2), h->stream));
  const int blocks = (int)std::min<long>(1024, (G.npts + 255) / 256);
  const double n0sq = h->n0 * h->n0;
  {
    Prof p_(h, K_MEDIUM, (16.0 + 2 * elem_size(h->prec)) * G.npts);
    if (h->prec == PROP_FP64) {
      GV<double> g = view<double>(h, G);
      k_medium<double, 256><<<blocks, 256, 0, h->stream>>>(g, slot, (const double2*)stage, n0sq,
                                                           h->C == 2 ? g.Btmp + (long)slot * 2 * G.npts : nullptr);
    } else {
      GV<float> g = view<float>(h, G);
      k_medium<float, 256><<<blocks, 256, 0, h->stream>>>(g, slot, (const double2*)stage, n0sq,
                                                          h->C == 2 ? g.Btmp + (long)slot * 2 * G.npts : nullptr);
    }
  }
  CK(cudaGetLastError());
  if (h->precond == PROP_PRECOND_FREESPACE) CK(cudaMemsetAsync(ds, 0, sizeof(double2), h->stream));   // dbar = 0
  if (h->C == 2) {
    const int rc = h->prec == PROP_FP64 ? psi_derivatives<double>(h, G, slot) : psi_derivatives<float>(h, G, slot);
    if (rc) return rc;
  }
  G.medium_dirty = true;
  G.carry = false;        // the vector psi pipeline uses the beam scratch that holds the carried row DFT
  return PROP_OK;
}

static int field_io(prop* h, Group& G, int slot, int to_field) {
  const long F = (long)h->C * G.npts;
  const int blocks = (int)std::min<long>(2048, (F + 255) / 256);
  double2* stage = (double2*)(h->ws + G.off.stage);
  Prof p_(h, K_FIELD_IO, 32.0 * F);
  if (h->prec == PROP_FP64) k_field_io<double, 256><<<blocks, 256, 0, h->stream>>>(view<double>(h, G), slot, stage, to_field);
  else k_field_io<float, 256><<<blocks, 256, 0, h->stream>>>(view<float>(h, G), slot, stage, to_field);
  CK(cudaGetLastError());
  return PROP_OK;
}

int prop_set_field(prop* h, int32_t beam, const void* w) {
  if (!h || !w || beam < 0 || beam >= h->nbeams) return PROP_E_ARG;
  Group& G = h->groups[h->beam_group[beam]];
  const long F = (long)h->C * G.npts;
  CK(cudaMemcpyAsync(h->ws + G.off.stage, w, F * 16, cudaMemcpyDefault, h->stream));
  const int rc = field_io(h, G, h->beam_slot[beam], 1);
  if (rc) return rc;
  G.carry = false;
  h->steps = 0;
  return PROP_OK;
}

int prop_get_field(prop* h, int32_t beam, void* w) {
  if (!h || !w || beam < 0 || beam >= h->nbeams) return PROP_E_ARG;
  Group& G = h->groups[h->beam_group[beam]];
  const long F = (long)h->C * G.npts;
  const int rc = field_io(h, G, h->beam_slot[beam], 0);
  if (rc) return rc;
  CK(cudaMemcpyAsync(w, h->ws + G.off.stage, F * 16, cudaMemcpyDefault, h->stream));
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, w) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    CK(cudaStreamSynchronize(h->stream));
  }
  return PROP_OK;
}

}  // extern "C"

// The pseudo-differential form (Sec. 3.2): `substeps` classical Runge-Kutta steps
// of dw/dz = i k0 n0 (S(Z) - I) w per dz.  Each stage is one step_group with the
// square root's table (field := S(Z) y, the other field buffer keeps y),
// followed by k_rk_stage.  On an error the field returns to the step's start.
template <typename T> static int rk4_group(prop* h, Group& G) {
  const long L = (long)G.beams.size() * h->C * G.npts;
  double2* W0 = (double2*)(h->ws + G.off.rkw0);
  double2* ACC = (double2*)(h->ws + G.off.rkacc);
  double2* START = (double2*)(h->ws + G.off.rkstart);
  const int blocks = (int)std::min<long>(2048, (L + 255) / 256);
  const double hs = h->dz / (double)h->substeps, k0n0 = h->k0 * h->n0;
  const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}, c[4] = {0.0, 0.5, 0.5, 1.0};
  auto cur = [&]() { return (double2*)(h->ws + (G.cur == 0 ? G.off.W64a : G.off.W64b)); };
  auto prev = [&]() { return (double2*)(h->ws + (G.cur == 0 ? G.off.W64b : G.off.W64a)); };
  { Prof p_(h, K_FIELD_IO, 48.0 * L);
    k_rk_copy<T, 256><<<blocks, 256, 0, h->stream>>>(cur(), START, nullptr, L); }
  CK(cudaGetLastError());
  for (int sub = 0; sub < h->substeps; ++sub) {
    { Prof p_(h, K_FIELD_IO, 48.0 * L);
      k_rk_copy<T, 256><<<blocks, 256, 0, h->stream>>>(cur(), W0, ACC, L); }
    CK(cudaGetLastError());
    for (int s = 0; s < 4; ++s) {
      const int rc = step_group<T>(h, G);
      if (rc) {
        k_rk_restore<T, 256><<<blocks, 256, 0, h->stream>>>(cur(), START, L);
        G.carry = false;
        return rc;
      }
      { Prof p_(h, K_FIELD_IO, 96.0 * L);
        k_rk_stage<T, 256><<<blocks, 256, 0, h->stream>>>(cur(), prev(), W0, ACC, L, hs * b[s],
                                                          s < 3 ? hs * c[s + 1] : 0.0, k0n0, s == 3 ? 1 : 0); }
      CK(cudaGetLastError());
      G.carry = false;   // the field was rewritten after the row DFT the step kept
    }
  }
  return PROP_OK;
}

extern "C" {

int prop_get_e3(prop* h, int32_t beam, void* out) {
  if (!h || !out || beam < 0 || beam >= h->nbeams) return PROP_E_ARG;
  if (h->C != 2) return PROP_E_UNSUPPORTED;
  Group& G = h->groups[h->beam_group[beam]];
  const int slot = h->beam_slot[beam];
  const int rc = h->prec == PROP_FP64 ? e3_impl<double>(h, G, slot) : e3_impl<float>(h, G, slot);
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, h->ws + G.off.stage, G.npts * 16, cudaMemcpyDefault, h->stream));
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, out) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    CK(cudaStreamSynchronize(h->stream));
  }
  return PROP_OK;
}

int prop_get_substeps(prop* h, int32_t* substeps) {
  if (!h || !substeps) return PROP_E_ARG;
  *substeps = h->form == PROP_FORM_PSEUDODIFF ? h->substeps : 0;
  return PROP_OK;
}

int prop_step(prop* h) {
  if (!h) return PROP_E_ARG;
  if (multigroup_ok(h)) {
    const int rc = step_multigroup(h);
    if (rc) { h->last_status = rc; return rc; }
    h->steps += 1;
    return PROP_OK;
  }
  for (Group& G : h->groups) {
    int rc;
    if (h->form == PROP_FORM_PSEUDODIFF) rc = h->prec == PROP_FP64 ? rk4_group<double>(h, G) : rk4_group<float>(h, G);
    else rc = h->prec == PROP_FP64 ? step_group<double>(h, G) : step_group<float>(h, G);
    if (rc) { h->last_status = rc; return rc; }
  }
  h->steps += 1;
  return PROP_OK;
}

int prop_run(prop* h, int32_t nsteps, prop_medium_fn cb, void* user) {
  if (!h || nsteps < 0) return PROP_E_ARG;
  for (int s = 0; s < nsteps; ++s) {
    if (cb) {
      const int rc = cb(h, s, user);
      if (rc) return rc;
    }
    const int rc = prop_step(h);
    if (rc) return rc;
  }
  return PROP_OK;
}

static int collect(prop* h, std::vector<int>& iters, std::vector<int>& cyc, std::vector<double>& resid) {
  iters.assign((size_t)h->nbeams * h->P, 0);
  cyc.assign((size_t)h->nbeams * h->P, 0);
  resid.assign((size_t)h->nbeams * h->P, 0.0);
  for (Group& G : h->groups) {
    const int nsys = (int)G.beams.size() * h->P;
    int* di = (int*)(h->ws + G.off.iters);
    int* dc = (int*)(h->ws + G.off.cycles);
    double* dr = (double*)(h->ws + G.off.resid);
    int* df = (int*)(h->ws + G.off.flags);
    {
      Prof p_(h, K_CONTROL, 0);
      k_collect<<<(nsys + 127) / 128, 128, 0, h->stream>>>((SysState*)(h->ws + G.off.st), nsys, di, dc, dr, df);
    }
    std::vector<int> ti(nsys), tc(nsys);
    std::vector<double> tr(nsys);
    CK(cudaMemcpyAsync(ti.data(), di, nsys * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(tc.data(), dc, nsys * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(tr.data(), dr, nsys * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int s = 0; s < nsys; ++s) {
      const int b = G.beams[s / h->P], k = s % h->P;
      iters[(size_t)b * h->P + k] = ti[s];
      cyc[(size_t)b * h->P + k] = tc[s];
      resid[(size_t)b * h->P + k] = tr[s];
    }
  }
  return PROP_OK;
}

int prop_get_stats(prop* h, prop_stats* out) {
  if (!h || !out) return PROP_E_ARG;
  std::vector<int> it, cy;
  std::vector<double> rs;
  const int rc = collect(h, it, cy, rs);
  if (rc) return rc;
  out->steps = h->steps;
  out->npoles = h->P;
  out->nbeams = h->nbeams;
  out->last_iters_max = 0; out->last_cycles_max = 0; out->last_iters_sum = 0; out->last_resid_max = 0.0;
  for (size_t i = 0; i < it.size(); ++i) {
    out->last_iters_max = std::max(out->last_iters_max, it[i]);
    out->last_cycles_max = std::max(out->last_cycles_max, cy[i]);
    out->last_iters_sum += it[i];
    out->last_resid_max = std::max(out->last_resid_max, rs[i]);
  }
  out->total_iters = h->total_iters;
  out->kernel_launches = h->launches;
  return PROP_OK;
}

int prop_get_iterations(prop* h, int32_t* iters) {
  if (!h || !iters) return PROP_E_ARG;
  std::vector<int> it, cy;
  std::vector<double> rs;
  const int rc = collect(h, it, cy, rs);
  if (rc) return rc;
  std::memcpy(iters, it.data(), it.size() * sizeof(int));
  return PROP_OK;
}

int prop_selftest_wait_timeout(void* stream) {
  static int* flag = nullptr;   // device address of g_selftest_err (current device at first call)
  if (!flag && cudaGetSymbolAddress((void**)&flag, g_selftest_err) != cudaSuccess) { flag = nullptr; return PROP_E_CUDA; }
  cudaStream_t st = (cudaStream_t)stream;
  int e = 0;
  if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return PROP_E_CUDA;
  k_selftest_wait<<<1, 64, 0, st>>>(flag);
  if (cudaGetLastError() != cudaSuccess) return PROP_E_CUDA;
  if (cudaMemcpyAsync(&e, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PROP_E_CUDA;
  return async_status(e);
}

const char* prop_error_string(int status) {
  switch (status) {
    case PROP_OK: return "ok";
    case PROP_E_ARG: return "invalid argument";
    case PROP_E_WORKSPACE: return "workspace missing, misaligned or too small";
    case PROP_E_CUDA: return "CUDA runtime error";
    case PROP_E_NOCONV: return "GMRES did not converge within max_restarts";
    case PROP_E_NAN: return "NaN or Inf in a residual";
    case PROP_E_UNSUPPORTED: return "unsupported grid size or mode";
    case PROP_E_SCRATCH: return "request exceeds the fixed scratch of prop_fft2_noalloc";
    case PROP_E_TIMEOUT: return "an asynchronous tile copy did not complete within its bounded wait";
    default: return "unknown status";
  }
}

void prop_destroy(prop* h) {
  if (!h) return;
  if (!h->pending.empty() || h->hcounts) cudaStreamSynchronize(h->stream);
  if (!h->pending.empty()) resolve_pending(h);
  for (cudaEvent_t e : h->pool) cudaEventDestroy(e);
  for (cudaEvent_t e : h->batch_ev)
    if (e) cudaEventDestroy(e);
  if (h->hcounts) cudaFreeHost(h->hcounts);
  cudaGetLastError();
  delete h;
}

int prop_set_profiling(prop* h, int32_t on) {
  if (!h) return PROP_E_ARG;
  if (!h->pending.empty()) { CK(cudaStreamSynchronize(h->stream)); resolve_pending(h); }
  h->profiling = on ? 1 : 0;
  if (on)
    for (int k = 0; k < PROP_NKINDS; ++k) { h->k_launches[k] = 0; h->k_ms[k] = 0.0; h->k_bytes[k] = 0.0; }
  return PROP_OK;
}

int prop_get_profile(prop* h, prop_kernel_profile* out) {
  if (!h || !out) return PROP_E_ARG;
  CK(cudaStreamSynchronize(h->stream));
  resolve_pending(h);
  for (int k = 0; k < PROP_NKINDS; ++k) {
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, kind_name(k), sizeof(out[k].name) - 1);
    out[k].launches = h->k_launches[k];
    out[k].total_ms = h->k_ms[k];
    out[k].alg_bytes = h->k_bytes[k];
  }
  return PROP_OK;
}

// ---- building blocks --------------------------------------------------------

int prop_fft2_workspace_size(int32_t nx, int32_t ny, int32_t precision, size_t* bytes) {
  if (!bytes) return PROP_E_ARG;
  if (!supported_n(nx) || !supported_n(ny)) return PROP_E_UNSUPPORTED;
  const size_t cs = 2 * elem_size(precision);
  *bytes = align_up(nx * cs) + align_up(ny * cs);
  return PROP_OK;
}

}  // extern "C"

template <typename T>
static int fft2_impl(int nx, int ny, int batch, int inverse, void* data, void* work, cudaStream_t st) {
  using C = typename Cx<T>::t;
  std::vector<T> tx, ty;
  twiddles<T>(nx, tx);
  twiddles<T>(ny, ty);
  char* w = (char*)work;
  const size_t ox = 0, oy = align_up(nx * sizeof(C));
  CK(cudaMemcpyAsync(w + ox, tx.data(), tx.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(w + oy, ty.data(), ty.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  GV<T> g;
  std::memset(&g, 0, sizeof(g));
  g.nx = nx; g.ny = ny; g.ncomp = 1; g.P = 1; g.m = 1; g.nb = batch; g.nsys = batch; g.npts = (long)nx * ny;
  g.twx = (const C*)(w + ox); g.twy = (const C*)(w + oy);
  C* d = (C*)data;
  const long F = g.npts;
  if (!inverse) {
    CK(rows_fwd<T, C>(g, buf(d, F), buf(d, F), -1, nullptr, batch, st));
    CK(cols<T>(g, buf(d, F), buf(d, F), -1, 1, MUL_NONE, 0, 0, -1, (T)1, batch, st));
  } else {
    CK(cols<T>(g, buf(d, F), buf(d, F), -1, 0, MUL_SCALE, 1, 0, -1, (T)(1.0 / (double)F), batch, st));
    CK(rows_inv<T>(g, buf(d, F), buf(d, F), -1, 0, epi(EPI_STORE), batch, st));
  }
  CK(cudaStreamSynchronize(st));   // the host twiddle vectors must outlive the copies
  return PROP_OK;
}

extern "C" {

int prop_fft2(int32_t nx, int32_t ny, int32_t batch, int32_t precision, int32_t inverse, void* d_data, void* d_work,
              size_t work_bytes, void* stream) {
  size_t need;
  int rc = prop_fft2_workspace_size(nx, ny, precision, &need);
  if (rc) return rc;
  if (batch < 0 || !d_data || !d_work) return PROP_E_ARG;
  if (work_bytes < need) return PROP_E_WORKSPACE;
  if (batch == 0) return PROP_OK;
  if (precision == PROP_FP64) return fft2_impl<double>(nx, ny, batch, inverse, d_data, d_work, (cudaStream_t)stream);
  if (precision == PROP_FP32) return fft2_impl<float>(nx, ny, batch, inverse, d_data, d_work, (cudaStream_t)stream);
  return PROP_E_ARG;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// FFT plan selection (prop_get/set_fft_plan, prop_fft_autotune)
// ---------------------------------------------------------------------------
static bool plan_valid(int n, int prec, const prop_fft_plan& p) {
  for (int r : {p.rows, p.rows_small})
    if ((r != PROP_ROWS_BLOCK && r != PROP_ROWS_WARP) || (!warp_n(n) && r == PROP_ROWS_WARP)) return false;
  for (int c : {p.cols, p.cols_small})
    if ((c != PROP_COLS_TMA && c != PROP_COLS_PLAIN && c != PROP_COLS_WARP) || (!warp_n(n) && c == PROP_COLS_WARP))
      return false;
  return prec == PROP_FP32 || prec == PROP_FP64;
}

// Times (CUDA events, best of reps) of one row round trip (forward rows, inverse
// rows) and of one column pass (forward, scale, inverse) per variant, on `batch`
// n x n arrays in the work buffer.
// Below this many bytes of data the timed runs would stay in L2: a 256 MiB write
// between them (outside the timed interval) flushes it.
constexpr size_t TUNE_FLUSH_BYTES = (size_t)256 << 20;

template <typename T>
static int autotune_impl(int n, int batch, int reps, int l2cold, char* work, cudaStream_t st, float* ms) {
  using C = typename Cx<T>::t;
  const size_t data_b = align_up((size_t)batch * n * n * sizeof(C));
  const bool flush = l2cold && (size_t)batch * n * n * sizeof(C) < TUNE_FLUSH_BYTES;
  char* flush_buf = work + data_b + align_up((size_t)n * sizeof(C)) + align_up(sizeof(int));
  std::vector<T> tw;
  twiddles<T>(n, tw);
  C* d = (C*)work;
  int* err = (int*)(work + data_b + align_up((size_t)n * sizeof(C)));   // the TMA pass's error word
  CK(cudaMemsetAsync(d, 0, (size_t)batch * n * n * sizeof(C), st));
  CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  CK(cudaMemcpyAsync(work + data_b, tw.data(), tw.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  GV<T> g;
  std::memset(&g, 0, sizeof(g));
  g.nx = n; g.ny = n; g.ncomp = 1; g.P = 1; g.m = 1; g.nb = batch; g.nsys = batch; g.npts = (long)n * n;
  g.twx = (const C*)(work + data_b); g.twy = g.twx;
  g.err = err;
  const long F = g.npts;
  const T scale = (T)(1.0 / (double)F);
  CUtensorMap tm;
  const bool tma = make_col_map(&tm, d, n, n, batch, (int)sizeof(C), cols_per_cta<T>());
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return PROP_E_CUDA;
  const int prec = prec_of<T>(), si = size_index(n), cl = launch_class(batch);
  const int rows_saved = g_plan_rows[prec][cl][si].load(), cols_saved = g_plan_cols[prec][cl][si].load();
  int rc = PROP_OK;
  auto time_it = [&](auto&& launch) -> float {
    float best = -1.f;
    for (int r = 0; r < reps + 1 && rc == PROP_OK; ++r) {   // the first run warms up
      if (flush && cudaMemsetAsync(flush_buf, r & 1, TUNE_FLUSH_BYTES, st) != cudaSuccess) { rc = PROP_E_CUDA; break; }
      if (cudaEventRecord(a, st) != cudaSuccess) { rc = PROP_E_CUDA; break; }
      if (launch() != cudaSuccess) { rc = PROP_E_CUDA; break; }
      if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) { rc = PROP_E_CUDA; break; }
      float t = 0.f;
      cudaEventElapsedTime(&t, a, b);
      if (r > 0 && (best < 0.f || t < best)) best = t;
    }
    return best;
  };
  // the whole 2-D round trip (forward rows, column pass, inverse rows) for every
  // combination of row and column variant: the passes hand their data to each
  // other through L2 as in the Arnoldi step, so they are timed together
  for (int v = 0; v < 6; ++v) ms[v] = -1.f;
  for (int rv = 0; rv < 2 && rc == PROP_OK; ++rv) {
    if (rv == PROP_ROWS_WARP && !warp_n(n)) continue;
    for (int cv = 0; cv < 3 && rc == PROP_OK; ++cv) {
      if (cv == PROP_COLS_WARP && !warp_n(n)) continue;
      if (cv == PROP_COLS_TMA && !tma) continue;
      g_plan_rows[prec][cl][si].store(rv);
      g_plan_cols[prec][cl][si].store(cv);
      const ColMaps cm = cv == PROP_COLS_TMA ? ColMaps{&tm, &tm, nullptr, nullptr} : ColMaps{nullptr, nullptr, nullptr, nullptr};
      ms[3 * rv + cv] = time_it([&]() {
        cudaError_t e = rows_fwd<T, C>(g, buf(d, F), buf(d, F), -1, nullptr, batch, st);
        if (e == cudaSuccess)
          e = cols<T>(g, buf(d, F), buf(d, F), -1, 1, MUL_SCALE, 1, 0, -1, scale, batch, st, Buf<C>{nullptr, 0, 1},
                      Buf<C>{nullptr, 0, 1}, cm);
        return e != cudaSuccess ? e : rows_inv<T>(g, buf(d, F), buf(d, F), -1, 0, epi(EPI_STORE), batch, st);
      });
    }
  }
  g_plan_rows[prec][cl][si].store(rows_saved);
  g_plan_cols[prec][cl][si].store(cols_saved);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc == PROP_OK) {
    int e = 0;
    if (cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PROP_E_CUDA;
    rc = async_status(e);
  }
  return rc;
}

extern "C" {

int prop_get_fft_plan(int32_t n, int32_t precision, prop_fft_plan* out) {
  if (!out || (precision != PROP_FP32 && precision != PROP_FP64)) return PROP_E_ARG;
  if (size_index(n) < 0) return PROP_E_UNSUPPORTED;
  out->rows = plan_rows(precision, n, PROP_FFT_SMALL_ITEMS + 1);
  out->cols = plan_cols(precision, n, PROP_FFT_SMALL_ITEMS + 1);
  out->rows_small = plan_rows(precision, n, 1);
  out->cols_small = plan_cols(precision, n, 1);
  return PROP_OK;
}

int prop_set_fft_plan(int32_t n, int32_t precision, const prop_fft_plan* plan) {
  if (!plan) return PROP_E_ARG;
  if (size_index(n) < 0) return PROP_E_UNSUPPORTED;
  if (!plan_valid(n, precision, *plan)) return PROP_E_UNSUPPORTED;
  g_plan_rows[precision][0][size_index(n)].store(plan->rows);
  g_plan_cols[precision][0][size_index(n)].store(plan->cols);
  g_plan_rows[precision][1][size_index(n)].store(plan->rows_small);
  g_plan_cols[precision][1][size_index(n)].store(plan->cols_small);
  return PROP_OK;
}

int prop_fft_autotune_workspace_size(int32_t n, int32_t precision, int32_t batch, size_t* bytes) {
  if (!bytes || batch < 1 || (precision != PROP_FP32 && precision != PROP_FP64)) return PROP_E_ARG;
  if (size_index(n) < 0) return PROP_E_UNSUPPORTED;
  const size_t cs = 2 * elem_size(precision);
  const size_t data = (size_t)batch * n * n * cs;
  *bytes = align_up(data) + align_up((size_t)n * cs) + align_up(sizeof(int)) + (data < TUNE_FLUSH_BYTES ? TUNE_FLUSH_BYTES : 0);
  return PROP_OK;
}

int prop_fft_autotune(int32_t n, int32_t precision, int32_t batch, int32_t reps, int32_t l2cold, void* d_work,
                      size_t work_bytes, void* stream, prop_fft_plan* best, float* ms) {
  size_t need;
  int rc = prop_fft_autotune_workspace_size(n, precision, batch, &need);
  if (rc) return rc;
  if (!d_work || !best || !ms || reps < 1 || ((uintptr_t)d_work % ALIGN) != 0) return PROP_E_ARG;
  if (work_bytes < need) return PROP_E_WORKSPACE;
  rc = precision == PROP_FP64 ? autotune_impl<double>(n, batch, reps, l2cold, (char*)d_work, (cudaStream_t)stream, ms)
                              : autotune_impl<float>(n, batch, reps, l2cold, (char*)d_work, (cudaStream_t)stream, ms);
  if (rc) return rc;
  // a combination replaces the default (block rows with TMA columns, else plain columns)
  // only when it is faster by more than TUNE_MARGIN: closer timings are within the
  // run-to-run spread
  constexpr float TUNE_MARGIN = 0.05f;
  const int dflt = ms[PROP_COLS_TMA] >= 0.f ? PROP_COLS_TMA : PROP_COLS_PLAIN;   // row variant block
  int bv = dflt;
  for (int v = 0; v < 6; ++v)
    if (ms[v] >= 0.f && ms[v] < (1.f - TUNE_MARGIN) * ms[dflt] && ms[v] < ms[bv]) bv = v;
  best->rows = bv / 3;
  best->cols = bv % 3;
  best->rows_small = best->rows;   // the fastest at this batch, for either launch class
  best->cols_small = best->cols;
  return PROP_OK;
}

}  // extern "C"

template <typename T> static int apply_impl(prop* h, int beam, int pole, const void* v, void* out, bool op) {
  using C = typename Cx<T>::t;
  Group& G = h->groups[h->beam_group[beam]];
  G.carry = false;        // Btmp is used as scratch here
  const int slot = h->beam_slot[beam];
  GV<T> g = view<T>(h, G);
  const long F = (long)h->C * g.npts;
  g.delta += (long)slot * g.npts;
  C* scratch = g.Btmp + (long)slot * F;
  const T scale = (T)(1.0 / (double)g.npts);
  cudaStream_t st = h->stream;
  C* diff = nullptr;
  if (op && h->C == 2) {   // (Z - Z_fs) v from a derivative round trip, kept for the final epilogue
    g.psi += (long)slot * 5 * g.npts;
    C* bscr = g.What + (long)slot * F;
    diff = g.Tmp + (long)slot * h->P * F;
    CK(rows_fwd<T, double2>(g, buf((double2*)v, F), buf(scratch, F), -1, nullptr, 1, st));
    CK(cols<T>(g, buf(scratch, F), buf(scratch, F), -1, 1, MUL_SCALE, 1, 0, -1, scale, 1, st, Buf<C>{nullptr, 0, 1},
               buf(bscr, F)));
    CK(rows_inv_vec<T>(g, buf(scratch, F), buf(bscr, F), buf(diff, F), -1, 0, VEPI_OPDIFF, 0, 1, st));
  }
  CK(rows_fwd<T, double2>(g, buf((double2*)v, F), buf(scratch, F), -1, nullptr, 1, st));
  CK(cols<T>(g, buf(scratch, F), buf(scratch, F), -1, 1, op ? MUL_POLE_FWD : MUL_POLE_INV, 1, 0,
             op ? h->P : pole, scale, 1, st));
  CK(rows_inv<T>(g, buf(scratch, F), buf(scratch, F), -1, 0,
                 op ? epi(EPI_OPERATOR, 0, (const double2*)v, (double2*)out, diff)
                    : epi(EPI_STORE64, 0, nullptr, (double2*)out),
                 1, st));
  return PROP_OK;
}

extern "C" {

int prop_set_guess_net(prop* h, int32_t nlayers, const int32_t* channels, const uint16_t* weights_bf16,
                       const float* biases) {
  if (!h || nlayers < 1 || nlayers > NET_MAX_LAYERS || !channels || !weights_bf16 || !biases) return PROP_E_ARG;
  if (h->guess != PROP_GUESS_LEARNED) return PROP_E_ARG;
  if (channels[0] != PROP_GUESS_CHANNELS || channels[nlayers] != PROP_GUESS_CHANNELS) return PROP_E_ARG;
  size_t wb = 0, bb = 0;
  for (int l = 0; l <= nlayers; ++l)
    if (channels[l] != 16 && channels[l] != 32) return PROP_E_ARG;
  for (int l = 0; l < nlayers; ++l) { wb += (size_t)9 * channels[l + 1] * channels[l] * 2; bb += channels[l + 1] * 4; }
  CK(cudaMemcpyAsync(h->ws + h->net_off, weights_bf16, wb, cudaMemcpyDefault, h->stream));
  CK(cudaMemcpyAsync(h->ws + h->net_off + NET_W_BYTES, biases, bb, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->net_layers = nlayers;
  for (int l = 0; l <= nlayers; ++l) h->net_ch[l] = channels[l];
  return PROP_OK;
}

int prop_get_net_io(prop* h, int32_t beam, int32_t pole, void* d_in_bf16, float* d_target) {
  if (!h || !d_in_bf16 || !d_target || beam < 0 || beam >= h->nbeams || pole < 0 || pole >= h->P) return PROP_E_ARG;
  Group& G = h->groups[h->beam_group[beam]];
  const int s = h->beam_slot[beam] * h->P + pole;
  const int blocks = (int)std::min<long>(1024, (G.npts + 255) / 256);
  Prof p_(h, K_GUESS, 0);
  if (h->prec == PROP_FP64) {
    GV<double> g = view<double>(h, G);
    k_guess_pack<double, 256><<<dim3(blocks, 1), 256, 0, h->stream>>>(g, (__nv_bfloat16*)d_in_bf16,
                                                                     (const double2*)(h->ws + G.off.poles), 0, s);
    k_guess_target<double, 256><<<blocks, 256, 0, h->stream>>>(g, s, d_target);
  } else {
    GV<float> g = view<float>(h, G);
    k_guess_pack<float, 256><<<dim3(blocks, 1), 256, 0, h->stream>>>(g, (__nv_bfloat16*)d_in_bf16,
                                                                    (const double2*)(h->ws + G.off.poles), 0, s);
    k_guess_target<float, 256><<<blocks, 256, 0, h->stream>>>(g, s, d_target);
  }
  CK(cudaGetLastError());
  return PROP_OK;
}

int prop_get_correction(prop* h, int32_t beam, int32_t pole, void* out) {
  if (!h || !out || beam < 0 || beam >= h->nbeams || pole < 0 || pole >= h->P) return PROP_E_ARG;
  Group& G = h->groups[h->beam_group[beam]];
  const long F = (long)h->C * G.npts;
  const int s = h->beam_slot[beam] * h->P + pole;
  SysState* st = (SysState*)(h->ws + G.off.st) + s;
  int used = 0;
  CK(cudaMemcpyAsync(&used, &st->used, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (!used || G.stats_zero) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, out) == cudaSuccess && at.type == cudaMemoryTypeDevice) {
      CK(cudaMemsetAsync(out, 0, F * 16, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    } else {
      cudaGetLastError();
      std::memset(out, 0, F * 16);
    }
    return PROP_OK;
  }
  CK(cudaMemcpyAsync(out, h->ws + G.off.E + (size_t)s * F * 16, F * 16, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return PROP_OK;
}

int prop_apply_freespace_inverse(prop* h, int32_t beam, int32_t pole, const void* d_v, void* d_out) {
  if (!h || !d_v || !d_out || beam < 0 || beam >= h->nbeams || pole < 0 || pole >= h->P) return PROP_E_ARG;
  return h->prec == PROP_FP64 ? apply_impl<double>(h, beam, pole, d_v, d_out, false)
                              : apply_impl<float>(h, beam, pole, d_v, d_out, false);
}

int prop_apply_operator(prop* h, int32_t beam, const void* d_v, void* d_out) {
  if (!h || !d_v || !d_out || beam < 0 || beam >= h->nbeams) return PROP_E_ARG;
  return h->prec == PROP_FP64 ? apply_impl<double>(h, beam, 0, d_v, d_out, true)
                              : apply_impl<float>(h, beam, 0, d_v, d_out, true);
}

}  // extern "C"

// ===========================================================================
// prop_fft2_noalloc: the batched 2-D DFT without any device allocation.
// Its twiddle tables live in a fixed file-scope array instead of caller
// memory.  Host code cannot use the array's name as a device address (it is a
// host-side stand-in), so the address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
// ===========================================================================
namespace {

static __device__ __align__(256) unsigned char g_fft2_noalloc_scratch[PROP_FFT2_NOALLOC_SCRATCH_BYTES];

// Every supported request fits: the largest, 1024 + 1024 complex128 twiddles
// with the second table 256-byte aligned, needs exactly the array's 32 KiB.
static_assert(PROP_FFT2_NOALLOC_SCRATCH_BYTES >= 2 * 1024 * 16, "scratch must hold the largest twiddle tables");

constexpr int NOALLOC_MAX_DEVICES = 64;
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
std::once_flag g_noalloc_once[NOALLOC_MAX_DEVICES];

// Device address of the scratch array on the current device, looked up once per
// device (std::call_once: host threads calling at the same time see one lookup).
int noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return PROP_E_CUDA;
  std::call_once(g_noalloc_once[dev], [dev] {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fft2_noalloc_scratch) == cudaSuccess && p) g_noalloc_ptr[dev] = p;
    else cudaGetLastError();
  });
  if (!g_noalloc_ptr[dev]) return PROP_E_CUDA;
  *out = g_noalloc_ptr[dev];
  return PROP_OK;
}

// w[m] = exp(-2 pi i m / n), evaluated in double and rounded once to T
template <typename T> __global__ void k_twiddle_table(typename Cx<T>::t* tw, int n) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)m / (double)n, &sn, &cs);
    tw[m].x = (T)cs;
    tw[m].y = (T)sn;
  }
}

template <typename T>
int fft2_noalloc_impl(int nx, int ny, int batch, int inverse, void* data, cudaStream_t st) {
  using C = typename Cx<T>::t;
  const size_t ox = 0, oy = align_up(nx * sizeof(C));
  if (oy + ny * sizeof(C) > PROP_FFT2_NOALLOC_SCRATCH_BYTES) return PROP_E_SCRATCH;
  void* scratch = nullptr;
  const int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  char* w = (char*)scratch;
  k_twiddle_table<T><<<(nx + 255) / 256, 256, 0, st>>>((C*)(w + ox), nx);
  k_twiddle_table<T><<<(ny + 255) / 256, 256, 0, st>>>((C*)(w + oy), ny);
  CK(cudaGetLastError());
  GV<T> g;
  std::memset(&g, 0, sizeof(g));
  g.nx = nx; g.ny = ny; g.ncomp = 1; g.P = 1; g.m = 1; g.nb = batch; g.nsys = batch; g.npts = (long)nx * ny;
  g.twx = (const C*)(w + ox); g.twy = (const C*)(w + oy);
  C* d = (C*)data;
  const long F = g.npts;
  if (!inverse) {
    CK(rows_fwd<T, C>(g, buf(d, F), buf(d, F), -1, nullptr, batch, st));
    CK(cols<T>(g, buf(d, F), buf(d, F), -1, 1, MUL_NONE, 0, 0, -1, (T)1, batch, st));
  } else {
    CK(cols<T>(g, buf(d, F), buf(d, F), -1, 0, MUL_SCALE, 1, 0, -1, (T)(1.0 / (double)F), batch, st));
    CK(rows_inv<T>(g, buf(d, F), buf(d, F), -1, 0, epi(EPI_STORE), batch, st));
  }
  return PROP_OK;
}

}  // namespace

extern "C" int prop_fft2_noalloc(int32_t nx, int32_t ny, int32_t batch, int32_t precision, int32_t inverse,
                                 void* d_data, void* stream) {
  if (!supported_n(nx) || !supported_n(ny)) return PROP_E_UNSUPPORTED;
  if (batch < 0 || !d_data) return PROP_E_ARG;
  if (batch == 0) return PROP_OK;
  if (precision == PROP_FP64) return fft2_noalloc_impl<double>(nx, ny, batch, inverse, d_data, (cudaStream_t)stream);
  if (precision == PROP_FP32) return fft2_noalloc_impl<float>(nx, ny, batch, inverse, d_data, (cudaStream_t)stream);
  return PROP_E_ARG;
}
