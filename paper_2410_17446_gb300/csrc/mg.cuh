// One launch per kernel kind for beams of different grid sizes.
//
// A handle groups its beams by grid; the Arnoldi step of every group runs in
// lockstep, and each of its five passes (forward rows, column pass, inverse rows
// with the Arnoldi epilogue, Gram sweep, update sweep) is one launch over all
// groups: the 1-D grid is cut into one CTA range per group, and a CTA runs its
// group's code for that grid size (the size-templated pass bodies of
// kernels.cuh, selected by a switch), so no CTA is launched without work.
// Every multi-group kernel has 256 threads; the row passes take mg_nr(N) rows a
// CTA (4096 points, or 3072 for the radix-3 sizes).  Complex FP32 only; sizes
// 128 ... 1024.
#pragma once
#include "kernels.cuh"

namespace prop_dev {

constexpr int MAXG = 8;      // grid sizes one launch can carry
constexpr int MG_NT = 256;   // threads of every multi-group CTA
constexpr int MG_NV = 4;     // columns of a column tile (32-byte rows)

__host__ __device__ constexpr int mg_nr(int n) { return n == 384 ? 8 : (n == 768 ? 4 : 4096 / n); }
__host__ __device__ constexpr int mg_nrv(int n) { return mg_nr(n) / 4 > 0 ? mg_nr(n) / 4 : 1; }
__host__ __device__ constexpr bool mg_size(int n) {
  return n == 128 || n == 256 || n == 384 || n == 512 || n == 768 || n == 1024;
}

// Everything one multi-group launch needs, passed by value (a __grid_constant__
// kernel parameter): per group its Arnoldi view (with its list of iterating
// systems), its CTA range and x extent, the update sweep's arguments and the
// column tensor maps.
struct MGroups {
  CUtensorMap tm[MAXG];    // Tmp  [nsys*ncomp][ny][nx], 4-column boxes
  CUtensorMap tm2[MAXG];   // Tmp2 (the vector operator's d/dy branch)
  GV<float> g[MAXG];
  StepArgs sa[MAXG];
  int c0[MAXG + 1];        // group i owns CTAs [c0[i], c0[i+1]) of the 1-D grid,
  int gx[MAXG];            // gx[i] CTAs per row: CTA c is (x, y) = ((c - c0) % gx, (c - c0) / gx)
  int tma[MAXG];           // 1: the tensor maps of group i are valid
  int* zero[MAXG];         // MG_ACTIVE also zeroes nzero ints at zero[i] (the batch's count slots)
  int nzero;
  int ng;
};

enum MgPass { MG_ROWS_FWD = 0, MG_COLS = 1, MG_ROWS_INV = 2, MG_GRAM = 3, MG_STEP = 4, MG_ACTIVE = 5 };

// Launch one pass over all groups; `mg` must hold the CTA ranges and x extents
// of this pass (from mg_gx and mg_rows).  Returns a CUDA error code.
cudaError_t mg_launch(int pass, const MGroups& mg, int jj, int with_w, cudaStream_t st);

// x extent and rows of group g's part of a pass with `act` listed systems; `cap`
// bounds the CTAs a system gets in the two sweeps.
int mg_gx(int pass, const GV<float>& g, int act, int cap);
int mg_rows(int pass, const GV<float>& g, int act);

// Resident CTAs per SM of the pass's kernel (MG_GRAM, MG_STEP), looked up once.
int mg_resident(int pass);

}  // namespace prop_dev
