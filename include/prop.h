/*
 * prop.h -- C ABI of the GB300 one-way vector Helmholtz propagator.
 *
 * The library advances the transverse envelope w = (w1[, w2]) of the electric
 * field by steps of dz with the exponential one-way propagator of Keefe et al.
 * (arXiv 2410.17446), Sec. 2:
 *
 *   w(z+dz) = r0 w(z) + sum_k r_k (Z - p_k I)^-1 w(z)          Eqs. (approx_prop), (W_k_def)
 *
 * where r(zeta) = r0 + sum_k r_k/(zeta - p_k) approximates
 * exp(iK(-1 + sqrt(1 + zeta))), K = k0 n0 dz (Eq. expop_prop; partial
 * fractions of Eq. pf_expan_eq with the factor e^{-iK} of Eq. Wk_define
 * folded into r0 and r_k), and Z is the operator matrix of Eq. (Z_bar_eq).
 * Each shifted system is solved by restarted GMRES, right-preconditioned by the
 * free-space solve (Z_fs - p_k I)^-1 of Sec. 4.2 (Eqs. Z_bar_fs_def,
 * fs_sylvester), which on the periodic pseudo-spectral grid used here is
 * diagonal in Fourier space.
 *
 * Discretisation: nx x ny periodic grid, x fastest, spectral derivatives; the
 * absorbing border is part of the caller's complex n^2 (Im n^2 > 0 absorbs).
 * Supported sizes: nx, ny in {16, 32, 64, 128, 256, 384, 512, 768, 1024}.
 *
 * Memory and ownership.  The caller owns all device memory: it passes one
 * device workspace of at least prop_workspace_size() bytes to prop_create and
 * keeps it alive until prop_destroy.  The library itself allocates no device
 * memory.  The handle (host memory) is allocated by prop_create.  Field and
 * medium buffers passed to set/get calls may be host or device pointers
 * (unified addressing); the data is copied, so the caller may reuse its buffer
 * once the call returns.  All calls are asynchronous on the handle's stream
 * except where stated.
 *
 * Errors.  Every call returns a status (PROP_OK = 0).  Argument errors leave
 * the handle unchanged.  PROP_E_NOCONV leaves the field at the last completed
 * step.  No C++ exception crosses this interface.  A handle is not thread-safe.
 */
#ifndef PROP_H
#define PROP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum prop_status {
  PROP_OK = 0,
  PROP_E_ARG = 1,          /* invalid argument (size, pointer, option)           */
  PROP_E_WORKSPACE = 2,    /* workspace missing, misaligned or too small          */
  PROP_E_CUDA = 3,         /* a CUDA runtime call failed                          */
  PROP_E_NOCONV = 4,       /* GMRES hit max_restarts without reaching tol         */
  PROP_E_NAN = 5,          /* a residual norm became NaN or Inf                   */
  PROP_E_UNSUPPORTED = 6,  /* grid size / mode not compiled into this library     */
  PROP_E_SCRATCH = 7,      /* request exceeds the fixed scratch of prop_fft2_noalloc */
  PROP_E_TIMEOUT = 8       /* an asynchronous tile copy did not complete within its
                              bounded wait; the kernel skipped its work (results of
                              the affected step are invalid)                        */
};

enum prop_precision {
  PROP_FP64 = 0,           /* all arithmetic in complex FP64                      */
  PROP_FP32 = 1            /* transforms and Krylov basis in complex FP32; Givens,
                              least squares, residual norms, the solution and the
                              field accumulated in FP64                           */
};

typedef struct prop_grid {
  int32_t nx, ny;          /* cells, border included                              */
  double dx, dy;           /* cell size, same length unit as 2 pi / k0            */
} prop_grid;

typedef struct prop_opts {
  int32_t ncomp;           /* 1: scalar (psi terms dropped, Sec. 2); 2: (w1, w2)  */
  int32_t precision;       /* enum prop_precision                                 */
  int32_t restart;         /* GMRES restart length m, 1..64 (default 20)          */
  int32_t max_restarts;    /* cycles per solve before PROP_E_NOCONV (default 50 FP64, 200 FP32) */
  double tol;              /* FP64: stop when ||w - (Z - p_k) x_k|| <= tol ||w||.  FP32: when it is
                              <= tol mu_k (||w|| + ||Z - p_k|| ||x_k||), the normwise backward error,
                              with mu_k >= 1 equalising each pole's share of the field error */
  int32_t guess;           /* PROP_GUESS_ZERO (x0 = 0) or PROP_GUESS_LEARNED (x0 from the network
                              installed by prop_set_guess_net; reserves activation memory)      */
  int32_t precond;         /* GMRES right preconditioner (Sec. 4.2; the answer does not depend on it):
                              PROP_PRECOND_FREESPACE: (Z_fs - p_k I)^-1, the n = n0 problem of
                              Eq. Z_bar_fs_def; PROP_PRECOND_MEAN (default): (Z_fs + dbar - p_k I)^-1,
                              the constant-index problem with n^2 = mean of n^2 over the beam's grid
                              (dbar = mean delta), which carries the absorbing border's mean loss,
                              as the paper's preconditioner carries its PML.  Both are diagonal in
                              Fourier space. */
  int32_t form;            /* PROP_FORM_EXPONENTIAL: prop_step applies r(Z) (Eq. approx_prop).
                              PROP_FORM_PSEUDODIFF: the table is the partial-fraction form of a
                              square root S(zeta) ~ sqrt(1 + zeta) (Sec. 3.2, Eq. pf_sqrt_exp: s0 =
                              c_alpha + sum wt_j, poles -(1 + i alpha sigma_j), residues
                              -i alpha wt_j (1 + sigma_j)) and prop_step advances dw/dz =
                              i k0 n0 (S(Z) - I) w (Eqs. eq_barZfactor2, eq:ApproxPropagator_W) by dz
                              with `substeps` classical Runge-Kutta steps; each stage applies S(Z)
                              by the same shifted solves (Eq. eq:Auxiliary_W).  The paper names no
                              z-integrator; RK4 is this library's choice. */
  int32_t substeps;        /* RK4 steps per dz for PROP_FORM_PSEUDODIFF; 0 = the fewest with
                              h k0 n0 (1 + sqrt(1.5 + |zeta_min|)) <= 2.5 on every grid, zeta_min =
                              -((pi/dx)^2 + (pi/dy)^2)/(k0 n0)^2 (inside RK4's stability region on
                              the operator's spectrum) */
  int32_t multigroup;      /* 1 (default): when a handle holds 2..8 grids, every one of size 128,
                              256, 384, 512, 768 or 1024 (complex FP32, PROP_FORM_EXPONENTIAL),
                              prop_step advances all of them in lockstep and each Arnoldi pass is
                              one kernel launch over every grid; 0: grid by grid.  The results
                              are the same either way. */
} prop_opts;

enum prop_precond { PROP_PRECOND_FREESPACE = 0, PROP_PRECOND_MEAN = 1 };
enum prop_form { PROP_FORM_EXPONENTIAL = 0, PROP_FORM_PSEUDODIFF = 1 };

enum prop_guess { PROP_GUESS_ZERO = 0, PROP_GUESS_LEARNED = 1 };
#define PROP_GUESS_CHANNELS 16   /* padded input / output width of the guess network */

typedef struct prop_stats {
  int64_t steps;           /* steps completed since prop_create / prop_set_field  */
  int32_t npoles, nbeams;
  int32_t last_iters_max;  /* max over (beam, pole) of Arnoldi steps, last step   */
  int32_t last_cycles_max; /* max over (beam, pole) of restart cycles, last step  */
  int64_t last_iters_sum;  /* sum over (beam, pole) of Arnoldi steps, last step   */
  double last_resid_max;   /* max relative true residual, last step               */
  int64_t total_iters;     /* Arnoldi steps summed over all steps                 */
  int64_t kernel_launches; /* kernels this handle has launched since prop_create  */
} prop_stats;

/* Per kernel kind: launches, device time (CUDA events recorded on the handle's
 * stream around each launch while profiling is on) and the algorithmic bytes
 * those launches had to move (each input read once, each output written once). */
typedef struct prop_kernel_profile {
  char name[24];
  int64_t launches;
  double total_ms;
  double alg_bytes;
} prop_kernel_profile;

#define PROP_NKINDS 13

typedef struct prop prop; /* opaque handle */

/* Fill *o with the defaults for `precision` (tol 1e-12 FP64, 1e-7 FP32; restart 20;
 * PROP_GUESS_ZERO; PROP_PRECOND_MEAN; PROP_FORM_EXPONENTIAL, substeps 0). */
int prop_default_opts(prop_opts* o, int32_t ncomp, int32_t precision);

/* Bytes of device workspace prop_create needs for these beams and options.
 * grids[nbeams]: one grid per independent beam. */
int prop_workspace_size(int32_t nbeams, const prop_grid* grids, int32_t npoles,
                        const prop_opts* opts, size_t* bytes);

/* Create a propagator for nbeams independent beams sharing (k0, n0, dz) and one
 * pole table.  poles[2*npoles], residues[2*npoles]: (re, im) pairs, host
 * memory; r0[2]: the constant term.  d_workspace: 256-byte aligned device
 * memory of ws_bytes >= prop_workspace_size().  stream: a cudaStream_t (NULL =
 * legacy default stream).  On success *out holds the handle; the medium of
 * every beam starts as n^2 = n0^2 (homogeneous) and every field as zero. */
int prop_create(int32_t nbeams, const prop_grid* grids, double k0, double n0, double dz,
                int32_t npoles, const double* poles, const double* residues, const double r0[2],
                const prop_opts* opts, void* d_workspace, size_t ws_bytes, void* stream,
                prop** out);

/* Set the medium of one beam from complex128 n^2[ny][nx] (host or device).
 * Z is rebuilt from it (Sec. 2: n and psi are updated between steps):
 * delta = (n^2 - n0^2)/n0^2 and, for ncomp = 2, psi = Log n^2 with its
 * spectral derivatives psi_x, psi_y, psi_xx, psi_yy, psi_xy scaled by (k0 n0)^-2. */
int prop_set_medium(prop* h, int32_t beam, const void* n2);

/* Set / get the field of one beam: complex128 [ncomp][ny][nx], host or device.
 * prop_get_field synchronises the stream when dst is host memory. */
int prop_set_field(prop* h, int32_t beam, const void* w);
int prop_get_field(prop* h, int32_t beam, void* w);

/* The longitudinal component E3 of one beam's current field (envelope, same
 * exp(i k0 n0 z) factor as w), recovered from Gauss's law div(n^2 E) = 0 (Sec. 2:
 * within a step n^2 = n^2(x, y), so E3 follows from (w1, w2) and the current
 * medium).  The z-derivative of each plane-wave component of D = n^2 E is taken
 * in the reference medium, i kz D3^ = -i (kx D1^ + ky D2^) with
 * kz = sqrt((k0 n0)^2 - kx^2 - ky^2), Im kz >= 0 (Eq. exp_prop_planewave), and
 * E3 = D3 / n^2; exact for a homogeneous medium.  kx, ky are first-derivative
 * symbols (Nyquist entry 0); a mode with kz = 0 exactly gets 0.  Vector handles
 * only (PROP_E_UNSUPPORTED otherwise).  out: complex128 [ny][nx], host or device
 * (synchronises for host memory).  Uses the beam's FFT scratch between steps. */
int prop_get_e3(prop* h, int32_t beam, void* out);

/* Runge-Kutta steps per dz of a PROP_FORM_PSEUDODIFF handle (the automatic
 * choice when opts.substeps was 0); 0 for the exponential form. */
int prop_get_substeps(prop* h, int32_t* substeps);

/* Advance every beam by dz (one z-step, Eq. approx_prop). */
int prop_step(prop* h);

/* Callback run before step s (0-based within this call); it may call
 * prop_set_medium.  Returning non-zero stops the run with that status. */
typedef int (*prop_medium_fn)(prop* h, int32_t step, void* user);

/* nsteps calls of (cb, prop_step). cb may be NULL. */
int prop_run(prop* h, int32_t nsteps, prop_medium_fn cb, void* user);

/* Statistics of the last step (synchronises the stream). */
int prop_get_stats(prop* h, prop_stats* out);

/* Per-(beam, pole) Arnoldi step counts of the last step, iters[nbeams*npoles]
 * (host memory; synchronises the stream). */
int prop_get_iterations(prop* h, int32_t* iters);

/* Turn per-launch event timing on (1) or off (0); turning it on clears the totals. */
int prop_set_profiling(prop* h, int32_t on);

/* Copy the PROP_NKINDS per-kind totals into out[PROP_NKINDS] (synchronises). */
int prop_get_profile(prop* h, prop_kernel_profile* out);

const char* prop_error_string(int status);

/* Self-test of the failure path of the asynchronous tile copies (the paper has
 * no counterpart).  Launches one CTA that waits on an mbarrier whose copy never
 * comes; the bounded wait gives up after about one second and sets an error
 * word.  Returns PROP_E_TIMEOUT when the bound works (the expected result),
 * PROP_OK if the wait somehow completed, PROP_E_CUDA on a runtime error.  No
 * copy is ever in flight and the CUDA context stays usable.  Synchronises the
 * stream; stream may be NULL (the default stream). */
int prop_selftest_wait_timeout(void* stream);

/* Release the handle (host memory only; the workspace stays the caller's). */
void prop_destroy(prop* h);

/* ---- building blocks, exposed for tests and tools ---------------------- */

/* In-place batched 2-D DFT of `batch` complex [ny][nx] arrays on the device:
 * forward X[ky,kx] = sum w[y,x] e^{-2 pi i (kx x/nx + ky y/ny)}, inverse with
 * e^{+...} and a 1/(nx ny) factor.  precision selects complex64/complex128
 * data.  d_work: device scratch of prop_fft2_workspace_size() bytes. */
int prop_fft2_workspace_size(int32_t nx, int32_t ny, int32_t precision, size_t* bytes);
int prop_fft2(int32_t nx, int32_t ny, int32_t batch, int32_t precision, int32_t inverse,
              void* d_data, void* d_work, size_t work_bytes, void* stream);

/* ---- FFT plans and their autotuner (the paper has no counterpart) ------ *
 * Each FFT pass has variants with the same arithmetic: the row pass by a
 * block-wide shared-memory Stockham transform or by warps (one row per warp,
 * N = 512 and 1024 only); the column pass by TMA tiles of 32-byte rows, by
 * plain loads, or by warps (one column per warp in registers, N = 512 and 1024
 * only).  The choice is process-wide per (size, precision) and read at every
 * launch, so it applies to every handle; set it between steps, not while work
 * of another thread is being enqueued.  Defaults: PROP_ROWS_BLOCK,
 * PROP_COLS_TMA. */
enum prop_fft_rows { PROP_ROWS_BLOCK = 0, PROP_ROWS_WARP = 1 };
enum prop_fft_cols { PROP_COLS_TMA = 0, PROP_COLS_PLAIN = 1, PROP_COLS_WARP = 2 };
/* rows, cols: launches of more than PROP_FFT_SMALL_ITEMS arrays; *_small: launches of
 * at most that many (the late Arnoldi steps, when few systems still iterate). */
#define PROP_FFT_SMALL_ITEMS 2
typedef struct prop_fft_plan { int32_t rows, cols, rows_small, cols_small; } prop_fft_plan;

/* Current plan for size n (a supported size) and precision. */
int prop_get_fft_plan(int32_t n, int32_t precision, prop_fft_plan* out);
/* Install a plan; PROP_E_UNSUPPORTED if a variant does not exist for n. */
int prop_set_fft_plan(int32_t n, int32_t precision, const prop_fft_plan* plan);
/* Device bytes prop_fft_autotune needs for `batch` n x n arrays (plus 256 MiB to
 * flush L2 between timed runs when the arrays are smaller than that). */
int prop_fft_autotune_workspace_size(int32_t n, int32_t precision, int32_t batch, size_t* bytes);
/* Time every combination of row and column variant on `batch` n x n arrays in
 * d_work (256-byte aligned, contents overwritten): one 2-D round trip (forward
 * rows, column pass with a scale, inverse rows) per combination, best of `reps`
 * runs after one warm-up, CUDA events on `stream`.  l2cold = 1: L2 is flushed
 * before each run when the data would fit in it; 0: the data stay in L2 between
 * runs.  ms[6] receives the times in ms, index 3 rows + cols (rows: block, warp;
 * cols: TMA, plain, warp; -1 where a variant does not exist), and *best the
 * fastest (in both the large and the small fields); a combination replaces the
 * default (block rows with TMA columns, else plain) only when more than 5 %
 * faster.  Installs nothing (call prop_set_fft_plan) and leaves the current plan
 * unchanged.  Synchronises the stream. */
int prop_fft_autotune(int32_t n, int32_t precision, int32_t batch, int32_t reps, int32_t l2cold, void* d_work,
                      size_t work_bytes, void* stream, prop_fft_plan* best, float* ms);

/* Install the initial-guess network (include/prop_cnn.h) for PROP_GUESS_LEARNED.
 * The paper has no learned part: GMRES still runs to the same tolerance, the
 * network only sets x0 of each correction system (Z - p_k) e_k = R0_k.
 * channels[nlayers + 1]: widths 16 or 32, first and last 16
 * (PROP_GUESS_CHANNELS).  weights: bfloat16 bits, layers concatenated, each
 * [9][c_out][c_in]; biases: float32, concatenated.  Host or device memory.
 * Input channels per pixel: R0_k / rms(R0_k) (re, im per component), then
 * 10 delta (re, im), then Re p_k, Im p_k, zero padding; output channels:
 * e_k / rms(R0_k) (re, im per component), rest ignored.  At most 8 layers. */
int prop_set_guess_net(prop* h, int32_t nlayers, const int32_t* channels, const uint16_t* weights_bf16,
                       const float* biases);

/* Training pair of the last step for (beam, pole): the network input above
 * (bfloat16 [ny][nx][16]) and the target e_k / rms(R0_k) (float32 [ny][nx][16],
 * padding zero).  Device pointers. */
int prop_get_net_io(prop* h, int32_t beam, int32_t pole, void* d_in_bf16, float* d_target);

/* prop_fft2 for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant.  Some callers cannot call
 * cudaMalloc or take memory from an allocator, for instance a plugin whose host
 * application owns every device allocation, or a program that must run inside
 * a fixed device-memory budget decided in advance.  They pass only the data;
 * the twiddle tables that prop_fft2 keeps in d_work live here in a file-scope
 * __device__ array of PROP_FFT2_NOALLOC_SCRATCH_BYTES (32 KiB), which every GPU
 * that loads this library holds until the process exits.  A call needs
 * (nx + ny) complex twiddles of the chosen precision; every supported size fits
 * (1024 + 1024 complex128 twiddles fill the array exactly), so PROP_E_SCRATCH
 * only guards a build with larger sizes.  Nothing is allocated: no cudaMalloc,
 * cudaFree or allocating library routine is called.  The first call on each
 * device looks up the array's device address with that device current
 * (cudaGetSymbolAddress, once per device even when host threads call at the
 * same time); make that first call before any stream capture.  Each device has
 * its own copy of the array; calls on one device share it, and each call
 * rewrites the part it uses, so calls that overlap on the same device
 * (different streams, or host threads without ordering) race on that memory:
 * serialise them.  Calls on different devices do not interfere. */
#define PROP_FFT2_NOALLOC_SCRATCH_BYTES 32768
int prop_fft2_noalloc(int32_t nx, int32_t ny, int32_t batch, int32_t precision, int32_t inverse,
                      void* d_data, void* stream);

/* out = (Z_fs - p_k I)^-1 v for beam `beam`, pole k (Sec. 4.2.1): the free-space
 * preconditioner.  v, out: device complex128 [ncomp][ny][nx]. */
int prop_apply_freespace_inverse(prop* h, int32_t beam, int32_t pole, const void* d_v, void* d_out);

/* Copy the correction e_k of the last step for (beam, pole k): the solution of
 * (Z - p_k I) x_k = w of Eq. (W_k_def) is x_k = (Z_fs - p_k I)^-1 w + e_k, with
 * w the field before that step.  out: complex128 [ncomp][ny][nx], host or
 * device (synchronises for host memory).  e_k is zero when the solve needed
 * no correction (e.g. a homogeneous medium). */
int prop_get_correction(prop* h, int32_t beam, int32_t pole, void* out);

/* out = Z v for beam `beam` with its current medium (Eq. Z_bar_eq).
 * v, out: device complex128 [ncomp][ny][nx]. */
int prop_apply_operator(prop* h, int32_t beam, const void* d_v, void* d_out);

#ifdef __cplusplus
}
#endif

#endif /* PROP_H */
