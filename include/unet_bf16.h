/*
 * unet_bf16.h -- C ABI of the warm-start U-Net kernels (sm_103a).
 *
 * The paper has no learned component; this surrogate serves the batched
 * sweeps: from a channel's wall mask, electric-force level and fill fraction
 * it predicts the steady density and velocity, which initialise the lattice
 * Boltzmann run (lbm_set_field with LBM_RHO_U); the method then runs on to
 * convergence, so the surrogate's error never reaches the converged result.
 *
 * Conventions: tensors are NCHW; BF16 tensors are passed as void* (bfloat16
 * values), FP32 as float*. "xbs" arguments are batch strides in elements, so
 * a tensor may be a channel range of a larger buffer (a concatenation).
 * 3x3 convolutions pad circularly in x and with zeros in y. All sums
 * accumulate in FP32. Every call enqueues on `stream` (a cudaStream_t) and
 * returns 0 on success, -1 for unsupported sizes (width and height must be
 * multiples of 32 and 4, output channels of the forward and weight-gradient
 * convolutions a multiple of 32), or a CUDA error code.
 */
#ifndef UNET_BF16_H
#define UNET_BF16_H

#ifdef __cplusplus
extern "C" {
#endif

/* y[b, o] = relu?(bias[o] + sum_{i, taps} w[o][i][ky][kx] x[b, i, y+ky-1, x+kx-1]);
 * w: BF16 [co][ci][3][3]; bias: FP32 [co] (may be NULL); y: BF16. */
int unet_conv3x3_fwd(const void *x, int ci, long xbs, const void *w, const float *bias, void *y, int co,
                     long ybs, int n, int h, int wd, int relu, void *stream);

/* Gradient w.r.t. the input of unet_conv3x3_fwd (no activation):
 * dx[b, i] = sum_{o, taps} w[o][i][ky][kx] dy[b, o, y-ky+1, x-kx+1] (BF16 out). */
int unet_conv3x3_bwd_data(const void *dy, int co, long dybs, const void *w, void *dx, int ci, long dxbs,
                          int n, int h, int wd, void *stream);

/* Gradients w.r.t. weights and bias, ACCUMULATED into FP32 dw [co][ci][3][3]
 * and db [co]: dw += sum_{b, pixels} dy x(shifted), db += sum dy. */
int unet_conv3x3_bwd_weight(const void *x, int ci, long xbs, const void *dy, int co, long dybs, float *dw,
                            float *db, int n, int h, int wd, void *stream);

/* 1x1 output head (co <= 8, ci <= 64): y[b, o, p] = bias[o] + sum_i w[o][i] x[b, i, p]
 * with FP32 output y [n][co][hw]; backward gives BF16 dx and accumulates
 * FP32 dw [co][ci], db [co]. */
int unet_head_fwd(const void *x, int ci, long xbs, const void *w, const float *bias, float *y, int co, int n,
                  int hw, void *stream);
int unet_head_bwd(const void *x, int ci, long xbs, const void *w, const float *dy, int co, int n, int hw,
                  void *dx, long dxbs, float *dw, float *db, void *stream);

/* 2x2 average pooling of an (h, wd) image and its adjoint (accumulate != 0
 * adds into dx instead of overwriting). */
int unet_pool2_fwd(const void *x, long xbs, void *y, long ybs, int c, int n, int h, int wd, void *stream);
int unet_pool2_bwd(const void *dy, long dybs, void *dx, long dxbs, int c, int n, int h, int wd, int accumulate,
                   void *stream);

/* nearest 2x upsampling of an (h, wd) image and its adjoint. */
int unet_up2_fwd(const void *x, long xbs, void *y, long ybs, int c, int n, int h, int wd, void *stream);
int unet_up2_bwd(const void *dy, long dybs, void *dx, long dxbs, int c, int n, int h, int wd, void *stream);

/* dy *= (y > 0) for the ReLU output y, chw elements per image. */
int unet_relu_bwd(const void *y, long ybs, void *dy, long dybs, int chw, int n, void *stream);

/* loss += sum_i wc[c(i)] (pred - target)^2 / count; grad = 2 wc (pred - target) / count.
 * pred, target, grad FP32 [n][c][hw]; loss: one double in device memory. */
int unet_mse(const float *pred, const float *target, const float *wc, int c, int hw, long count, float *grad,
             double *loss, void *stream);

/* Adam step `step` (>= 1) on FP32 master weights, refreshing the BF16 copy
 * (w_bf16 may be NULL). */
int unet_adam(float *w_master, void *w_bf16, const float *grad, float *m, float *v, long count, float lr,
              float beta1, float beta2, float eps, int step, float weight_decay, void *stream);

/* Round FP32 to BF16 (nearest even). */
int unet_f32_to_bf16(const float *x, void *y, long count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* UNET_BF16_H */
