/*
 * unet_bf16.h -- C ABI of the warm-start U-Net kernels (sm_103a).
 *
 * The paper has no learned component; this surrogate serves the batched
 * sweeps: from a channel's wall mask, electric-force level and fill fraction
 * it predicts the steady density and velocity, which initialise the lattice
 * Boltzmann run (lbm_set_field with LBM_RHO_U_PHYS); the method then runs on
 * to convergence, so the surrogate's error never reaches the converged result.
 *
 * Conventions: activations are BF16, channels-last (NHWC: element (b, y, x, c)
 * at ((b * h + y) * w + x) * ct + c). A tensor argument is a "view": a pointer
 * to its first channel and ct, the channels per pixel of the buffer it lives
 * in, so a view may be a channel range of a larger buffer (a concatenation).
 * BF16 tensors are passed as void*, FP32 as float*. 3x3 convolutions pad
 * circularly in x and with zeros in y. All sums accumulate in FP32. Every call
 * enqueues on `stream` (a cudaStream_t) and returns 0 on success, -1 for
 * unsupported sizes or misaligned views (see each call), or a CUDA error code.
 */
#ifndef UNET_BF16_H
#define UNET_BF16_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Output-channel tile (128, 64 or 32) the convolution uses for `channels`
 * output channels, and the number of BF16 elements of a packed weight
 * operand (transpose = 0: forward, co output channels; transpose = 1: input
 * gradient, ci output channels). */
int unet_conv_ntile(int channels);
size_t unet_conv_pack_elems(int co, int ci, int transpose);

/* Pack FP32 master weights w [co][ci][3][3] into the tensor-core operand of
 * unet_conv3x3: transpose = 0 for the forward convolution (output channels
 * co), transpose = 1 for the gradient w.r.t. its input (the kernel
 * transposed and flipped; output channels ci). The output count must be a
 * multiple of 32; `out` holds unet_conv_pack_elems(co, ci, transpose)
 * elements. */
int unet_conv_pack(const float *w, int co, int ci, int transpose, void *out, void *stream);

/* Several unet_conv_pack calls in one launch. jobs (device memory, int64)
 * holds njobs records of 5 values: the address of w, co, ci, transpose and
 * the address of out (each as for unet_conv_pack, co or ci a multiple of 32
 * as the packing needs); max_elems bounds the largest record's
 * unet_conv_pack_elems (it sizes the grid). Returns -1 for a NULL table,
 * njobs outside 1 .. 65535 or max_elems < 1. */
int unet_conv_pack_many(const long long *jobs, int njobs, long max_elems, void *stream);

/* 3x3 convolution on the tensor cores (tcgen05.mma, FP32 accumulation in
 * tensor memory): y[b, p, o] = act(bias[o] + sum_{tap, i} W[o][i](tap)
 * x[b, p + off(tap), i]) with W the packed operand `wt`; bias may be NULL,
 * act = ReLU if relu != 0. With the transpose = 1 packing of a layer's
 * weights, x = dy and y = dx, this is that layer's gradient w.r.t. its input.
 * Requires wd % 32 == 0, h % 4 == 0, cout % 32 == 0, ct_in and ct_out
 * multiples of 8, 16-byte aligned views, and cin a multiple of 16, or
 * cin < 16 in a view of at least 16 readable channels whose channels >= cin
 * are zero. */
int unet_conv3x3(const void *x, int ct_in, int cin, const void *wt, const float *bias, void *y, int ct_out,
                 int cout, int n, int h, int wd, int relu, void *stream);

/* Gradients w.r.t. the weights and bias of unet_conv3x3 (forward packing),
 * ACCUMULATED into FP32 dw [co][ci][3][3] and db [co] (db may be NULL, e.g.
 * when unet_relu_bwd already accumulated it): dw += sum_{b, p}
 * dy[b, p, o] x[b, p + off(tap), i] (tensor cores), db += sum dy. Requires
 * wd % 16 == 0, co % 8 == 0, ct_x and ct_dy multiples of 8, 16-byte aligned
 * views; x must have at least 8 readable channels when ci < 8. */
int unet_conv3x3_bwd_weight(const void *x, int ct_x, int ci, const void *dy, int ct_dy, int co, float *dw,
                            float *db, int n, int h, int wd, void *stream);

/* Sticky error flag of the tensor-core kernels (nonzero after an mbarrier
 * wait timed out); reset != 0 clears it. Synchronises the stream. */
int unet_tc_error(void *stream, int reset);

/* 1x1 output head (forward: co <= 8, ci <= 64; backward: co = 3, ci <= 256):
 * y[b, o, p] = bias[o] + sum_i w[o][i]
 * x[b, p, i], with BF16 weights w [co][ci], NHWC input view and FP32 output y
 * [n][co][hw] (NCHW); backward gives the NHWC BF16 dx and accumulates FP32
 * dw [co][ci], db [co]. */
int unet_head_fwd(const void *x, int ct, int ci, const void *w, const float *bias, float *y, int co, int n,
                  int hw, void *stream);
int unet_head_bwd(const void *x, int ct, int ci, const void *w, const float *dy, int co, int n, int hw,
                  void *dx, int ct_dx, float *dw, float *db, void *stream);

/* 2x2 average pooling of an (h, wd) image and its adjoint (accumulate != 0
 * adds into dx instead of overwriting); c channels of NHWC views. c, ctx,
 * cty multiples of 8, views 16-byte aligned, h and wd even, fewer than 2^34
 * elements; otherwise -1. */
int unet_pool2_fwd(const void *x, int ctx, void *y, int cty, int c, int n, int h, int wd, void *stream);
int unet_pool2_bwd(const void *dy, int cty, void *dx, int ctx, int c, int n, int h, int wd, int accumulate,
                   void *stream);

/* Nearest 2x upsampling of an (h, wd) image and its adjoint (c, ctx, cty
 * multiples of 8 and 16-byte aligned views; otherwise -1). */
int unet_up2_fwd(const void *x, int ctx, void *y, int cty, int c, int n, int h, int wd, void *stream);
int unet_up2_bwd(const void *dy, int cty, void *dx, int ctx, int c, int n, int h, int wd, void *stream);

/* dy *= (y > 0) for the ReLU output y, c <= 256 channels (c, cty, ctd
 * multiples of 8, 16-byte aligned views) of npix pixels;
 * with db != NULL also db[ch] += sum over pixels of the masked dy (FP32),
 * the bias gradient of the layer that produced y. */
int unet_relu_bwd(const void *y, int cty, void *dy, int ctd, int c, long npix, float *db, void *stream);

/* FP32 NCHW planes x [n][c][hw] -> BF16 NHWC y with ct channels per pixel
 * (channels c..ct-1 are zero). */
int unet_input_nhwc(const float *x, int c, int hw, int n, void *y, int ct, void *stream);

/* Weighted mean squared error over count = n*c*hw FP32 values (NCHW):
 * *loss += sum wc[ch] (pred - target)^2 / count (FP64 accumulator),
 * grad = 2 wc (pred - target) / count. */
int unet_mse(const float *pred, const float *target, const float *wc, int c, int hw, long count, float *grad,
             double *loss, void *stream);

/* One Adam step on FP32 master weights (bias-corrected with `step`);
 * w_bf16 (may be NULL) receives the BF16 compute copy. */
int unet_adam(float *w_master, void *w_bf16, const float *grad, float *m, float *v, long count, float lr,
              float beta1, float beta2, float eps, int step, float weight_decay, void *stream);

/* The same with the step's scalars read from device memory: hyper[0] = lr,
 * hyper[1] = 1 - beta1^t, hyper[2] = 1 - beta2^t (written by
 * unet_adam_hyper), so that a captured CUDA graph of training steps replays
 * with each step's values. Returns -1 if hyper is NULL. */
int unet_adam_dev(float *w_master, void *w_bf16, const float *grad, float *m, float *v, long count,
                  const float *hyper, float beta1, float beta2, float eps, float weight_decay, void *stream);

/* Advance a device-side Adam step: state (6 floats, device) holds [0] the
 * step t (start 0), [1] beta1^t and [2] beta2^t (start 1, multiplied in
 * FP32 as unet_adam does); the call increments t and writes [3] the learning
 * rate lr_schedule[t - 1] (device, n >= 1 entries, the last one beyond the
 * end), [4] 1 - beta1^t and [5] 1 - beta2^t: the hyper argument of
 * unet_adam_dev is state + 3. Returns -1 for NULL pointers or n < 1. */
int unet_adam_hyper(float *state, const float *lr_schedule, int n, float beta1, float beta2, void *stream);

/* Warm-start fields of n domains (n <= 65535) from the network output y
 * [n][3][hw] (FP32, normalised): on fluid nodes (mask [n][hw] == 0)
 * rho = clamp(y0 * rho_std + rho_mean, lo, hi) and u = (y1, y2) * u_scale;
 * 0 on solid nodes; then each domain's rho is scaled so that it sums to
 * mass[b]. out [n][3][hw] FP64 (the LBM_RHO_U_PHYS layout of each domain);
 * sums [n] FP64 scratch. */
int unet_warm_fields(const float *y, int n, int hw, const unsigned char *mask, const double *mass, float rho_mean,
                     float rho_std, float u_scale, double lo, double hi, double *out, double *sums, void *stream);

/* y = BF16(x), count elements. */
int unet_f32_to_bf16(const float *x, void *y, long count, void *stream);

#ifdef __cplusplus
}
#endif

#endif
