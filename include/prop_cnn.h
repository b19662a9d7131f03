/*
 * prop_cnn.h -- C ABI of the learned GMRES initial-guess network.
 *
 * The paper has no learned component: every shifted system of Eq. (W_k_def)
 * is solved by GMRES to the same tolerance whatever x0 is.  This network only
 * proposes x0 for the correction systems (Z - p_k) e_k = R0_k that prop_step
 * solves; prop_set_guess_net (prop.h) installs it.
 *
 * Network: L layers of 3x3 convolutions with circular padding on the
 * transverse grid, ReLU between layers:
 *   y[n, y, x, co] = b[co] + sum_{t, ci} W[t, co, ci] a[n, y + dy_t, x + dx_t, ci]
 * with tap t = 3 (dy + 1) + (dx + 1).  Activations are NHWC bfloat16 with 16 or
 * 32 channels; weights bfloat16 [9][Cout][Cin]; biases float32.  Convolutions
 * run on the BF16 tensor cores and accumulate in float32: tcgen05 MMAs with
 * the accumulator in tensor memory (strips of 128-pixel row tiles, two accumulators, when
 * W is a multiple of 128; 128-pixel tiles when H W is), else warp-level
 * mma.sync.
 *
 * All pointers are device pointers; calls are asynchronous on `stream` and
 * return PROP_CNN_OK (0) or an error code.  Grids need W a multiple of 16
 * (64 for the weight gradient).
 */
#ifndef PROP_CNN_H
#define PROP_CNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { PROP_CNN_OK = 0, PROP_CNN_E_ARG = 1, PROP_CNN_E_CUDA = 3, PROP_CNN_E_TIMEOUT = 4 };
enum { PROP_CNN_PATH_AUTO = 0, PROP_CNN_PATH_MMA_SYNC = 1 };

/* Convolution kernel choice for this process (default PROP_CNN_PATH_AUTO:
 * tcgen05 where the tiles fit; PROP_CNN_PATH_MMA_SYNC: always warp-level
 * mma.sync).  Both give the same sums up to float32 rounding order. */
int prop_cnn_set_path(int32_t path);

/* Synchronises `stream`; PROP_CNN_E_TIMEOUT if a tensor-core convolution since
 * the last call gave up its bounded wait for its MMAs (its output is then
 * undefined; the flag is cleared), else PROP_CNN_OK. */
int prop_cnn_check(void* stream);
enum { PROP_CNN_RELU_BF16 = 0, PROP_CNN_LINEAR_BF16 = 1, PROP_CNN_LINEAR_F32 = 2 };

/* One convolution layer over N images of H x W.  mode: store relu(y) as bf16,
 * y as bf16, or y as float32.  d_active (optional): image n is skipped when
 * d_active[n * active_stride] != active_want (its output is left untouched). */
int prop_cnn_conv(int32_t cin, int32_t cout, int32_t mode, const void* d_in, const void* d_w, const float* d_bias,
                  void* d_out, int32_t N, int32_t H, int32_t W, const int32_t* d_active, int32_t active_stride,
                  int32_t active_want, void* stream);

/* Weight and bias gradients of one layer, float32:
 * dw[t, co, ci] = sum_{n,p} g[n, p, co] a[n, p + d_t, ci],  db[co] = sum_{n,p} g[n, p, co],
 * with g the gradient at the layer's output (bf16) and a its input (bf16).
 * d_work: scratch of prop_cnn_wgrad_workspace() bytes.  Deterministic. */
int prop_cnn_wgrad_workspace(int32_t cin, int32_t cout, int32_t N, int32_t H, int32_t W, size_t* bytes);
int prop_cnn_wgrad(int32_t cin, int32_t cout, const void* d_grad, const void* d_act, int32_t N, int32_t H, int32_t W,
                   float* d_dw, float* d_db, void* d_work, size_t work_bytes, void* stream);

/* wt[8 - t][ci][co] = w[t][co][ci]: the data gradient of a layer is
 * prop_cnn_conv(cout, cin, ..., grad, wt, no bias, ...). */
int prop_cnn_flip_transpose(const void* d_w, void* d_wt, int32_t cout, int32_t cin, void* stream);

/* grad[i] = 0 where act[i] <= 0 (ReLU derivative from the stored activation), bf16, in place. */
int prop_cnn_relu_mask(void* d_grad, const void* d_act, int64_t n, void* stream);

/* float32 -> bfloat16 (round to nearest even). */
int prop_cnn_to_bf16(const float* d_x, void* d_y, int64_t n, void* stream);

/* Mean-squared error over the first `valid` of C channels, per pixel:
 * *d_loss += 0.5 sum (out - target)^2 / npix; d_grad (bf16) = (out - target)/npix, 0 on padding. */
int prop_cnn_mse(const float* d_out, const float* d_target, void* d_grad, int64_t npix, int32_t C, int32_t valid,
                 double* d_loss, void* stream);

/* Adam step (bias-corrected, step >= 1) on float32 parameters; also writes a
 * bf16 copy to d_p_bf16 when it is not NULL. */
int prop_cnn_adam(float* d_p, const float* d_g, float* d_m, float* d_v, int64_t n, float lr, float b1, float b2,
                  float eps, int32_t step, void* d_p_bf16, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PROP_CNN_H */
