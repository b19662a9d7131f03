// Multi-group Arnoldi passes (mg.cuh): one launch per pass for all grid sizes.
#include "mg.cuh"

namespace prop_dev {

namespace {

constexpr int EPT_GS_MG = 4, GVEC_GS_MG = 4, EPT_GRAM_MG = 4, GVEC_GRAM_MG = 4;   // as the single-group sweeps

// The group that owns CTA c, and the CTA's (x, y) within the group's grid.
struct MgCta { int gi, bx, by; };
__device__ __forceinline__ MgCta mg_cta(const MGroups& mg, int c) {
  int i = 0;
  while (i + 1 < mg.ng && c >= mg.c0[i + 1]) ++i;
  const int l = c - mg.c0[i];
  return MgCta{i, l % mg.gx[i], l / mg.gx[i]};
}

#define MG_SWITCH(n, BODY)   \
  switch (n) {               \
    case 128: BODY(128) break;   \
    case 256: BODY(256) break;   \
    case 384: BODY(384) break;   \
    case 512: BODY(512) break;   \
    case 768: BODY(768) break;   \
    case 1024: BODY(1024) break; \
    default: break;              \
  }

// Minimum resident CTAs per SM asked of the compiler for the FFT passes: the
// switch over six grid sizes would otherwise allocate registers for the largest
// body and leave two CTAs of 256 threads per SM (the vector column pass, with
// its second tile, keeps two).
constexpr int MG_ROWS_MINB = 3, MG_COLS_MINB = 4;

// forward row DFTs of v_jj into Tmp
__global__ void __launch_bounds__(MG_NT, MG_ROWS_MINB) k_mg_rows_fwd(const __grid_constant__ MGroups mg, int jj) {
  const MgCta t = mg_cta(mg, blockIdx.x);
  const GV<float>& g = mg.g[t.gi];
  const long F = (long)g.ncomp * g.npts;
  const Buf<float2> src{g.V + (long)jj * F, (long)(g.m + 2) * F, 1}, dst{g.Tmp, F, 1};
#define BODY(N) rows_fwd_body<float, N, mg_nr(N), MG_NT, float2, false>(t.bx, t.by, mg.gx[t.gi], g, src, dst, \
                                                                          ST_ITER, nullptr);
  MG_SWITCH(g.nx, BODY)
#undef BODY
}

// column pass: column DFT, preconditioner multiply, inverse column DFT, by TMA
// tiles (every group has tensor maps) or plain loads; the vector operator also
// forms the d/dy branch into Tmp2
template <bool DY, bool TMA>
__global__ void __launch_bounds__(MG_NT, DY ? 2 : MG_COLS_MINB) k_mg_cols(const __grid_constant__ MGroups mg) {
  const MgCta t = mg_cta(mg, blockIdx.x);
  const GV<float>& g = mg.g[t.gi];
  const long F = (long)g.ncomp * g.npts;
  const float scale = (float)(1.0 / (double)g.npts);
  const Buf<float2> tmp{g.Tmp, F, 1}, none{nullptr, 0, 1}, dy{DY ? g.Tmp2 : nullptr, F, 1};
  if constexpr (TMA) {
    const CUtensorMap& m = mg.tm[t.gi];
#define BODY(N) cols_tma_body<float, N, MG_NV, MG_NT, DY>(t.bx, t.by, mg.gx[t.gi], g, m, m, m, DY ? mg.tm2[t.gi] : m, \
                                                          ST_ITER, 1, MUL_PREC_INV, 1, 0, -1, scale, none);
    MG_SWITCH(g.ny, BODY)
#undef BODY
  } else {
#define BODY(N) cols_body<float, N, MG_NV, MG_NT, DY>(t.bx, t.by, mg.gx[t.gi], g, tmp, tmp, ST_ITER, 1, MUL_PREC_INV, \
                                                      1, 0, -1, scale, none, dy);
    MG_SWITCH(g.ny, BODY)
#undef BODY
  }
}

// inverse row DFTs and the Arnoldi epilogue w = u + (delta - dbar) z into v_{jj+1}
__global__ void __launch_bounds__(MG_NT, MG_ROWS_MINB) k_mg_rows_inv(const __grid_constant__ MGroups mg, int jj) {
  const MgCta t = mg_cta(mg, blockIdx.x);
  const GV<float>& g = mg.g[t.gi];
  const long F = (long)g.ncomp * g.npts;
  const Buf<float2> tmp{g.Tmp, F, 1};
  EpiArgs ep{};
  ep.mode = EPI_ARNOLDI;
  ep.jj = jj;
#define BODY(N) rows_inv_body<float, N, mg_nr(N), MG_NT, true, false>(t.bx, t.by, mg.gx[t.gi], g, tmp, tmp, ST_ITER, \
                                                                       0, ep);
  MG_SWITCH(g.nx, BODY)
#undef BODY
}

// vector operator: six inverse row DFTs and the psi / cross-polarisation epilogue
// (two CTAs per SM asked of the compiler: unbounded it takes 164 registers, one)
__global__ void __launch_bounds__(MG_NT, 2) k_mg_rows_inv_vec(const __grid_constant__ MGroups mg, int jj) {
  const MgCta t = mg_cta(mg, blockIdx.x);
  const GV<float>& g = mg.g[t.gi];
  const long F = (long)g.ncomp * g.npts;
  const Buf<float2> a{g.Tmp, F, 1}, b{g.Tmp2, F, 1};
#define BODY(N) rows_inv_vec_body<float, N, mg_nrv(N), MG_NT>(t.bx, t.by, mg.gx[t.gi], g, a, b, a, ST_ITER, 0, \
                                                              VEPI_ARNOLDI, jj);
  MG_SWITCH(g.nx, BODY)
#undef BODY
}

__global__ void __launch_bounds__(MG_NT) k_mg_gram(const __grid_constant__ MGroups mg, int jj, int with_w) {
  const MgCta t = mg_cta(mg, blockIdx.x);
  dcgs_gram_body<float, MG_NT, EPT_GRAM_MG, GVEC_GRAM_MG>(t.bx, t.by, mg.gx[t.gi], mg.g[t.gi], jj, with_w);
}

__global__ void __launch_bounds__(MG_NT, 3) k_mg_step(const __grid_constant__ MGroups mg, int jj) {
  const MgCta t = mg_cta(mg, blockIdx.x);
  dcgs_step_body<float, MG_NT, EPT_GS_MG, GVEC_GS_MG>(t.bx, t.by, mg.gx[t.gi], mg.g[t.gi], jj, mg.sa[t.gi]);
}

// the list of iterating systems of every group (one CTA a group), padded with -1,
// and the group's count slots of the coming batch zeroed
__global__ void __launch_bounds__(MG_NT) k_mg_active(const __grid_constant__ MGroups mg) {
  pdl_enter();
  const GV<float>& g = mg.g[blockIdx.x];
  int* list = const_cast<int*>(g.ulist);
  for (int i = threadIdx.x; i < mg.nzero; i += blockDim.x) mg.zero[blockIdx.x][i] = 0;
  __shared__ int wsum[32], base;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int s0 = 0; s0 < g.nsys; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    const bool a = s < g.nsys && g.st[s].state == ST_ITER;
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
  for (int s = base + threadIdx.x; s < g.nsys; s += blockDim.x) list[s] = -1;
}

size_t smem_of(int pass, const MGroups& mg, bool tma_all) {
  size_t sm = 0;
  for (int i = 0; i < mg.ng; ++i) {
    const GV<float>& g = mg.g[i];
    const bool dy = g.ncomp == 2;
    size_t b = 0;
    if (pass == MG_ROWS_FWD || (pass == MG_ROWS_INV && !dy)) b = (size_t)mg_nr(g.nx) * (g.nx + g.nx / 16) * 8;
    else if (pass == MG_ROWS_INV) b = (size_t)6 * mg_nrv(g.nx) * (g.nx + g.nx / 16) * 8;
    else if (pass == MG_COLS)
      b = tma_all ? ((size_t)g.ny * MG_NV * (dy ? 2 : 1) + 2 * (size_t)g.ny) * 8 + 128
                  : (size_t)g.ny * MG_NV * (dy ? 2 : 1) * 8;
    sm = b > sm ? b : sm;
  }
  return sm;
}

}  // namespace

int mg_rows(int pass, const GV<float>& g, int act) {
  switch (pass) {
    case MG_ROWS_FWD: case MG_COLS: return act * g.ncomp;
    case MG_ROWS_INV: return g.ncomp == 2 ? act : act * g.ncomp;
    default: return act;
  }
}

int mg_gx(int pass, const GV<float>& g, int act, int cap) {
  const long F = (long)g.ncomp * g.npts;
  switch (pass) {
    case MG_ROWS_FWD: return g.ny / mg_nr(g.nx);
    case MG_ROWS_INV: return g.ncomp == 2 ? g.ny / mg_nrv(g.nx) : g.ny / mg_nr(g.nx);
    case MG_COLS: return g.nx / MG_NV;
    case MG_GRAM: {
      const int b = (int)((F + MG_NT * EPT_GRAM_MG - 1) / (MG_NT * EPT_GRAM_MG));
      return b < cap ? b : cap;
    }
    case MG_STEP: {
      const int b = (int)((F + MG_NT * EPT_GS_MG - 1) / (MG_NT * EPT_GS_MG));
      return (b < cap ? b : cap) + 1;   // + the control CTA (x = 0)
    }
    default: return 1;
  }
}

int mg_resident(int pass) {
  static int occ[2] = {0, 0};
  const int i = pass == MG_STEP ? 1 : 0;
  if (!occ[i]) {
    int n = 0;
    const cudaError_t e = i ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mg_step, MG_NT, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mg_gram, MG_NT, 0);
    if (e != cudaSuccess || n < 1) n = 1;
    cudaGetLastError();
    occ[i] = n;
  }
  return occ[i];
}

cudaError_t mg_launch(int pass, const MGroups& mg, int jj, int with_w, cudaStream_t st) {
  const int ctas = pass == MG_ACTIVE ? mg.ng : mg.c0[mg.ng];
  if (ctas <= 0) return cudaSuccess;
  bool tma_all = true;
  for (int i = 0; i < mg.ng; ++i) tma_all = tma_all && mg.tma[i] != 0;
  const size_t sm = smem_of(pass, mg, tma_all);
  const bool vec = mg.g[0].ncomp == 2;
  static bool attr[7] = {false, false, false, false, false, false, false};
  auto raise = [&](auto k, int slot) -> cudaError_t {   // room for the largest pass of any size mix
    if (attr[slot]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    if (e == cudaSuccess) attr[slot] = true;
    return e;
  };
  cudaError_t e = cudaSuccess;
  switch (pass) {
    case MG_ROWS_FWD:
      e = raise(k_mg_rows_fwd, 0);
      if (e == cudaSuccess) e = launch_pdl(k_mg_rows_fwd, dim3(ctas), dim3(MG_NT), sm, st, mg, jj);
      break;
    case MG_COLS:
#define COLS(DY, TMA, SLOT)                                                  \
      e = raise(k_mg_cols<DY, TMA>, SLOT);                                   \
      if (e == cudaSuccess) e = launch_pdl(k_mg_cols<DY, TMA>, dim3(ctas), dim3(MG_NT), sm, st, mg);
      if (vec) {
        if (tma_all) { COLS(true, true, 1) } else { COLS(true, false, 2) }
      } else {
        if (tma_all) { COLS(false, true, 3) } else { COLS(false, false, 4) }
      }
#undef COLS
      break;
    case MG_ROWS_INV:
      if (vec) {
        e = raise(k_mg_rows_inv_vec, 5);
        if (e == cudaSuccess) e = launch_pdl(k_mg_rows_inv_vec, dim3(ctas), dim3(MG_NT), sm, st, mg, jj);
      } else {
        e = raise(k_mg_rows_inv, 6);
        if (e == cudaSuccess) e = launch_pdl(k_mg_rows_inv, dim3(ctas), dim3(MG_NT), sm, st, mg, jj);
      }
      break;
    case MG_GRAM: e = launch_pdl(k_mg_gram, dim3(ctas), dim3(MG_NT), 0, st, mg, jj, with_w); break;
    case MG_STEP: e = launch_pdl(k_mg_step, dim3(ctas), dim3(MG_NT), 0, st, mg, jj); break;
    case MG_ACTIVE: e = launch_pdl(k_mg_active, dim3(ctas), dim3(MG_NT), 0, st, mg); break;
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace prop_dev
