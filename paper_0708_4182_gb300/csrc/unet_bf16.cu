// unet_bf16.cu -- hand-written kernels of the warm-start U-Net (sm_103a).
//
// The surrogate maps a channel's wall mask, electric-force level and fill
// fraction to its steady density and velocity, which then initialise the
// lattice Boltzmann run (the warm start). Storage is BF16 (activations and
// the compute copy of the weights); every sum accumulates in FP32; the
// optimizer keeps FP32 master weights and moments.
//
// Tensors are NCHW. A tensor "view" is (pointer, channels, batch stride in
// elements), so a layer can read or write a channel range of a larger buffer
// (the decoder's concatenations are such buffers; nothing is copied).
// Padding of the 3x3 convolutions: circular in x (the channels are periodic
// along the flow), zero in y (walls).
#include "unet_bf16.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace unet {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kT = 256;       // threads per CTA
constexpr int kTco = 32;      // output channels per CTA
constexpr int kRows = 4;      // pixel tile: 4 rows x 32 columns
constexpr int kCols = 32;
constexpr int kCk = 16;       // input channels per staged chunk

__device__ __forceinline__ float ld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ int wrapx(int x, int w) { return x < 0 ? x + w : (x >= w ? x - w : x); }

// y[b, co, :, :] = act(bias[co] + sum_ci sum_taps wt(co, ci, tap) x[b, ci, shifted])
// TW = 0: wt(o, i, ky, kx) = w[o][i][ky][kx]     (forward)
// TW = 1: wt(o, i, ky, kx) = w[i][o][2-ky][2-kx] (gradient w.r.t. the input)
// w holds [wo][wi][3][3]. One CTA: 32 output channels x (4 x 32) pixels of one
// image; each thread 4 channels x 4 consecutive pixels (16 FP32 sums).
template <int TW>
__global__ void __launch_bounds__(kT) conv3x3_kernel(const bf16* __restrict__ x, int Ci, long xbs,
                                                     const bf16* __restrict__ w, int wo, int wi,
                                                     const float* __restrict__ bias, bf16* __restrict__ y,
                                                     int Co, long ybs, int H, int W, int relu)
{
    __shared__ float sx[kCk][kRows + 2][kCols + 2];
    __shared__ float sw[kTco][kCk][9];
    const int tid = threadIdx.x;
    const int tiles_x = W / kCols;
    const int ty0 = (blockIdx.x / tiles_x) * kRows, tx0 = (blockIdx.x % tiles_x) * kCols;
    const int co0 = blockIdx.y * kTco;
    const int b = blockIdx.z;
    const int cg = tid / 32;            // channel group: channels co0 + 4cg .. +3
    const int pg = tid % 32;            // pixel group: 4 pixels
    const int pr = pg / 8, pc = (pg % 8) * 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const bf16* xb = x + b * xbs;
    for (int c0 = 0; c0 < Ci; c0 += kCk) {
        __syncthreads();
        for (int i = tid; i < kCk * (kRows + 2) * (kCols + 2); i += kT) {
            const int ci = i / ((kRows + 2) * (kCols + 2));
            const int rem = i % ((kRows + 2) * (kCols + 2));
            const int r = rem / (kCols + 2), c = rem % (kCols + 2);
            const int gy = ty0 + r - 1, gx = wrapx(tx0 + c - 1, W);
            float v = 0.f;
            if (c0 + ci < Ci && gy >= 0 && gy < H) v = ld(xb + (long)(c0 + ci) * H * W + (long)gy * W + gx);
            sx[ci][r][c] = v;
        }
        for (int i = tid; i < kTco * kCk * 9; i += kT) {
            const int o = i / (kCk * 9), rem = i % (kCk * 9);
            const int ci = rem / 9, tap = rem % 9;
            const int co = co0 + o, cc = c0 + ci;
            float v = 0.f;
            if (co < Co && cc < Ci) {
                if (TW == 0)
                    v = ld(w + ((long)co * wi + cc) * 9 + tap);
                else
                    v = ld(w + ((long)cc * wi + co) * 9 + (8 - tap));
            }
            sw[o][ci][tap] = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int ci = 0; ci < kCk; ++ci) {
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                float xv[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) xv[j] = sx[ci][pr + ky][pc + j];
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float wv = sw[cg * 4 + i][ci][ky * 3 + kx];
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(wv, xv[j + kx], acc[i][j]);
                    }
                }
            }
        }
    }
    const int gy = ty0 + pr;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int co = co0 + cg * 4 + i;
        if (co >= Co) continue;
        const float bv = bias ? bias[co] : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v = acc[i][j] + bv;
            if (relu) v = fmaxf(v, 0.f);
            y[b * ybs + (long)co * H * W + (long)gy * W + tx0 + pc + j] = __float2bfloat16_rn(v);
        }
    }
}

// dw[co][ci][tap] += sum_{b, pixels} dy[b, co, p] x[b, ci, p + tap];
// one CTA: 32 output channels x 16 input channels over `rows_per_cta` rows
// of one image; each thread 1 output channel x 2 input channels x 9 taps.
__global__ void __launch_bounds__(kT) conv3x3_wgrad_kernel(const bf16* __restrict__ x, int Ci, long xbs,
                                                           const bf16* __restrict__ dy, int Co, long dybs,
                                                           float* __restrict__ dw, int H, int W,
                                                           int rows_per_cta)
{
    __shared__ float sx[kCk][3][kCols + 2];
    __shared__ float sd[kTco][kCols];
    const int tid = threadIdx.x;
    const int co0 = blockIdx.x * kTco, c0 = blockIdx.y * kCk;
    const int row_blocks = H / rows_per_cta;
    const int b = blockIdx.z / row_blocks, r0 = (blockIdx.z % row_blocks) * rows_per_cta;
    const int o = tid / 8, ip = (tid % 8) * 2;
    float acc[2][9];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int t = 0; t < 9; ++t) acc[k][t] = 0.f;
    const bf16* xb = x + b * xbs;
    const bf16* db = dy + b * dybs;
    for (int r = r0; r < r0 + rows_per_cta; ++r) {
        for (int cx = 0; cx < W; cx += kCols) {
            __syncthreads();
            for (int i = tid; i < kCk * 3 * (kCols + 2); i += kT) {
                const int ci = i / (3 * (kCols + 2)), rem = i % (3 * (kCols + 2));
                const int ry = rem / (kCols + 2), c = rem % (kCols + 2);
                const int gy = r + ry - 1, gx = wrapx(cx + c - 1, W);
                float v = 0.f;
                if (c0 + ci < Ci && gy >= 0 && gy < H) v = ld(xb + (long)(c0 + ci) * H * W + (long)gy * W + gx);
                sx[ci][ry][c] = v;
            }
            for (int i = tid; i < kTco * kCols; i += kT) {
                const int oo = i / kCols, c = i % kCols;
                sd[oo][c] = (co0 + oo < Co) ? ld(db + (long)(co0 + oo) * H * W + (long)r * W + cx + c) : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int c = 0; c < kCols; ++c) {
                const float d = sd[o][c];
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx) acc[k][ky * 3 + kx] = fmaf(d, sx[ip + k][ky][c + kx], acc[k][ky * 3 + kx]);
            }
        }
    }
    const int co = co0 + o;
    if (co >= Co) return;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int ci = c0 + ip + k;
        if (ci >= Ci) continue;
#pragma unroll
        for (int t = 0; t < 9; ++t) atomicAdd(&dw[((long)co * Ci + ci) * 9 + t], acc[k][t]);
    }
}

// db[c] += sum over images and pixels of dy[b, c, :, :] (one CTA per channel)
__global__ void bias_grad_kernel(const bf16* __restrict__ dy, int C, long dybs, int B, int HW,
                                 float* __restrict__ db)
{
    __shared__ float red[kT];
    const int c = blockIdx.x;
    float s = 0.f;
    for (int b = 0; b < B; ++b)
        for (int i = threadIdx.x; i < HW; i += kT) s += ld(dy + b * dybs + (long)c * HW + i);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] += red[0];
}

// 1x1 head: y[b, o, p] = bias[o] + sum_i w[o][i] x[b, i, p], FP32 output
__global__ void head_fwd_kernel(const bf16* __restrict__ x, int Ci, long xbs, const bf16* __restrict__ w,
                                const float* __restrict__ bias, float* __restrict__ y, int Co, int HW, int B)
{
    const long n = (long)B * HW;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int b = int(i / HW), p = int(i % HW);
        for (int o = 0; o < Co; ++o) {
            float s = bias[o];
            for (int c = 0; c < Ci; ++c) s = fmaf(ld(w + o * Ci + c), ld(x + b * xbs + (long)c * HW + p), s);
            y[((long)b * Co + o) * HW + p] = s;
        }
    }
}

// head backward: dx[b, i, p] = sum_o w[o][i] dy[b, o, p] (BF16 out);
// dw[o][i] += sum dy x, db[o] += sum dy (FP32, atomics per CTA)
__global__ void head_bwd_kernel(const bf16* __restrict__ x, int Ci, long xbs, const bf16* __restrict__ w,
                                const float* __restrict__ dy, int Co, int HW, int B, bf16* __restrict__ dx,
                                long dxbs, float* __restrict__ dw, float* __restrict__ db)
{
    __shared__ float sdw[8 * 64];
    __shared__ float sdb[8];
    for (int i = threadIdx.x; i < Co * Ci; i += blockDim.x) sdw[i] = 0.f;
    if (threadIdx.x < Co) sdb[threadIdx.x] = 0.f;
    __syncthreads();
    const long n = (long)B * HW;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int b = int(i / HW), p = int(i % HW);
        float g[8];
        for (int o = 0; o < Co; ++o) {
            g[o] = dy[((long)b * Co + o) * HW + p];
            atomicAdd(&sdb[o], g[o]);
        }
        for (int c = 0; c < Ci; ++c) {
            const float xv = ld(x + b * xbs + (long)c * HW + p);
            float s = 0.f;
            for (int o = 0; o < Co; ++o) {
                s = fmaf(ld(w + o * Ci + c), g[o], s);
                atomicAdd(&sdw[o * Ci + c], g[o] * xv);
            }
            dx[b * dxbs + (long)c * HW + p] = __float2bfloat16_rn(s);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < Co * Ci; i += blockDim.x) atomicAdd(&dw[i], sdw[i]);
    if (threadIdx.x < Co) atomicAdd(&db[threadIdx.x], sdb[threadIdx.x]);
}

// 2x2 average pooling and its adjoint
__global__ void pool2_fwd_kernel(const bf16* __restrict__ x, long xbs, bf16* __restrict__ y, long ybs, int C,
                                 int H, int W, int B)
{
    const int h = H / 2, w = W / 2;
    const long n = (long)B * C * h * w;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int b = int(i / ((long)C * h * w));
        const long r = i % ((long)C * h * w);
        const int c = int(r / (h * w)), yy = int(r % (h * w)) / w, xx = int(r % (h * w)) % w;
        const bf16* s = x + b * xbs + (long)c * H * W + (long)(2 * yy) * W + 2 * xx;
        const float v = 0.25f * ((ld(s) + ld(s + 1)) + (ld(s + W) + ld(s + W + 1)));
        y[b * ybs + (long)c * h * w + (long)yy * w + xx] = __float2bfloat16_rn(v);
    }
}

__global__ void pool2_bwd_kernel(const bf16* __restrict__ dy, long dybs, bf16* __restrict__ dx, long dxbs,
                                 int C, int H, int W, int B, int accumulate)
{
    const long n = (long)B * C * H * W;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int b = int(i / ((long)C * H * W));
        const long r = i % ((long)C * H * W);
        const int c = int(r / (H * W)), yy = int(r % (H * W)) / W, xx = int(r % (H * W)) % W;
        float v = 0.25f * ld(dy + b * dybs + (long)c * (H / 2) * (W / 2) + (long)(yy / 2) * (W / 2) + xx / 2);
        bf16* o = dx + b * dxbs + (long)c * H * W + (long)yy * W + xx;
        if (accumulate) v += ld(o);
        *o = __float2bfloat16_rn(v);
    }
}

// nearest 2x upsampling and its adjoint (sum over the 4 copies)
__global__ void up2_fwd_kernel(const bf16* __restrict__ x, long xbs, bf16* __restrict__ y, long ybs, int C,
                               int h, int w, int B)
{
    const int H = 2 * h, W = 2 * w;
    const long n = (long)B * C * H * W;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int b = int(i / ((long)C * H * W));
        const long r = i % ((long)C * H * W);
        const int c = int(r / (H * W)), yy = int(r % (H * W)) / W, xx = int(r % (H * W)) % W;
        y[b * ybs + (long)c * H * W + (long)yy * W + xx] = x[b * xbs + (long)c * h * w + (long)(yy / 2) * w + xx / 2];
    }
}

__global__ void up2_bwd_kernel(const bf16* __restrict__ dy, long dybs, bf16* __restrict__ dx, long dxbs, int C,
                               int h, int w, int B)
{
    const int W = 2 * w;
    const long n = (long)B * C * h * w;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int b = int(i / ((long)C * h * w));
        const long r = i % ((long)C * h * w);
        const int c = int(r / (h * w)), yy = int(r % (h * w)) / w, xx = int(r % (h * w)) % w;
        const bf16* s = dy + b * dybs + (long)c * 4 * h * w + (long)(2 * yy) * W + 2 * xx;
        dx[b * dxbs + (long)c * h * w + (long)yy * w + xx] =
            __float2bfloat16_rn((ld(s) + ld(s + 1)) + (ld(s + W) + ld(s + W + 1)));
    }
}

// dy <- dy * (y > 0): gradient through a ReLU whose output is y
__global__ void relu_bwd_kernel(const bf16* __restrict__ y, long ybs, bf16* __restrict__ dy, long dybs, int CHW,
                                int B)
{
    const long n = (long)B * CHW;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int b = int(i / CHW), r = int(i % CHW);
        if (!(ld(y + b * ybs + r) > 0.f)) dy[b * dybs + r] = __float2bfloat16_rn(0.f);
    }
}

// weighted mean squared error over n = B*C*HW values, weight per channel:
// loss = sum_i wc (p - t)^2 / n; grad = 2 wc (p - t) / n (FP32)
__global__ void mse_kernel(const float* __restrict__ p, const float* __restrict__ t, const float* __restrict__ wc,
                           int C, int HW, long n, float* __restrict__ grad, double* __restrict__ loss)
{
    __shared__ double red[kT];
    double s = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int c = int((i / HW) % C);
        const float d = p[i] - t[i];
        s += double(wc[c]) * d * d;
        grad[i] = 2.f * wc[c] * d / float(n);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / double(n));
}

// Adam on FP32 master weights; writes the BF16 compute copy
__global__ void adam_kernel(float* __restrict__ wm, bf16* __restrict__ wb, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float wd)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float gi = g[i] + wd * wm[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = wm[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        wm[i] = w;
        if (wb) wb[i] = __float2bfloat16_rn(w);
    }
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, bf16* __restrict__ y, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

int blocks_for(long n) { return int(n / kT + 1 < 4096 ? n / kT + 1 : 4096); }

int status(cudaError_t e) { return e == cudaSuccess ? 0 : int(e); }

}  // namespace
}  // namespace unet

using namespace unet;

extern "C" {

int unet_conv3x3_fwd(const void* x, int ci, long xbs, const void* w, const float* bias, void* y, int co, long ybs,
                     int n, int h, int wd, int relu, void* stream)
{
    if (wd % kCols || h % kRows || co % kTco) return -1;
    dim3 grid((h / kRows) * (wd / kCols), co / kTco, n);
    conv3x3_kernel<0><<<grid, kT, 0, (cudaStream_t)stream>>>((const bf16*)x, ci, xbs, (const bf16*)w, co, ci, bias,
                                                             (bf16*)y, co, ybs, h, wd, relu);
    return status(cudaGetLastError());
}

int unet_conv3x3_bwd_data(const void* dy, int co, long dybs, const void* w, void* dx, int ci, long dxbs, int n,
                          int h, int wd, void* stream)
{
    if (wd % kCols || h % kRows) return -1;
    dim3 grid((h / kRows) * (wd / kCols), (ci + kTco - 1) / kTco, n);
    conv3x3_kernel<1><<<grid, kT, 0, (cudaStream_t)stream>>>((const bf16*)dy, co, dybs, (const bf16*)w, co, ci,
                                                             nullptr, (bf16*)dx, ci, dxbs, h, wd, 0);
    return status(cudaGetLastError());
}

int unet_conv3x3_bwd_weight(const void* x, int ci, long xbs, const void* dy, int co, long dybs, float* dw,
                            float* db, int n, int h, int wd, void* stream)
{
    if (wd % kCols || co % kTco) return -1;
    int rows = h >= 8 ? 8 : h;
    while (h % rows) --rows;
    dim3 grid(co / kTco, (ci + kCk - 1) / kCk, n * (h / rows));
    conv3x3_wgrad_kernel<<<grid, kT, 0, (cudaStream_t)stream>>>((const bf16*)x, ci, xbs, (const bf16*)dy, co, dybs,
                                                                dw, h, wd, rows);
    bias_grad_kernel<<<co, kT, 0, (cudaStream_t)stream>>>((const bf16*)dy, co, dybs, n, h * wd, db);
    return status(cudaGetLastError());
}

int unet_head_fwd(const void* x, int ci, long xbs, const void* w, const float* bias, float* y, int co, int n, int hw,
                  void* stream)
{
    if (co > 8 || ci > 64) return -1;
    head_fwd_kernel<<<blocks_for((long)n * hw), kT, 0, (cudaStream_t)stream>>>((const bf16*)x, ci, xbs,
                                                                               (const bf16*)w, bias, y, co, hw, n);
    return status(cudaGetLastError());
}

int unet_head_bwd(const void* x, int ci, long xbs, const void* w, const float* dy, int co, int n, int hw, void* dx,
                  long dxbs, float* dw, float* db, void* stream)
{
    if (co > 8 || co * ci > 512) return -1;
    head_bwd_kernel<<<blocks_for((long)n * hw) / 4 + 1, kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, ci, xbs, (const bf16*)w, dy, co, hw, n, (bf16*)dx, dxbs, dw, db);
    return status(cudaGetLastError());
}

int unet_pool2_fwd(const void* x, long xbs, void* y, long ybs, int c, int n, int h, int wd, void* stream)
{
    pool2_fwd_kernel<<<blocks_for((long)n * c * h * wd / 4), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, xbs, (bf16*)y, ybs, c, h, wd, n);
    return status(cudaGetLastError());
}

int unet_pool2_bwd(const void* dy, long dybs, void* dx, long dxbs, int c, int n, int h, int wd, int accumulate,
                   void* stream)
{
    pool2_bwd_kernel<<<blocks_for((long)n * c * h * wd), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)dy, dybs, (bf16*)dx, dxbs, c, h, wd, n, accumulate);
    return status(cudaGetLastError());
}

int unet_up2_fwd(const void* x, long xbs, void* y, long ybs, int c, int n, int h, int wd, void* stream)
{
    up2_fwd_kernel<<<blocks_for((long)n * c * h * wd * 4), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, xbs, (bf16*)y, ybs, c, h, wd, n);
    return status(cudaGetLastError());
}

int unet_up2_bwd(const void* dy, long dybs, void* dx, long dxbs, int c, int n, int h, int wd, void* stream)
{
    up2_bwd_kernel<<<blocks_for((long)n * c * h * wd), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)dy, dybs, (bf16*)dx, dxbs, c, h, wd, n);
    return status(cudaGetLastError());
}

int unet_relu_bwd(const void* y, long ybs, void* dy, long dybs, int chw, int n, void* stream)
{
    relu_bwd_kernel<<<blocks_for((long)n * chw), kT, 0, (cudaStream_t)stream>>>((const bf16*)y, ybs, (bf16*)dy,
                                                                                dybs, chw, n);
    return status(cudaGetLastError());
}

int unet_mse(const float* pred, const float* target, const float* wc, int c, int hw, long count, float* grad,
             double* loss, void* stream)
{
    mse_kernel<<<blocks_for(count) / 8 + 1, kT, 0, (cudaStream_t)stream>>>(pred, target, wc, c, hw, count, grad,
                                                                           loss);
    return status(cudaGetLastError());
}

int unet_adam(float* w_master, void* w_bf16, const float* grad, float* m, float* v, long count, float lr,
              float beta1, float beta2, float eps, int step, float weight_decay, void* stream)
{
    float c1 = 1.f, c2 = 1.f;
    for (int k = 0; k < step; ++k) {
        c1 *= beta1;
        c2 *= beta2;
    }
    adam_kernel<<<blocks_for(count), kT, 0, (cudaStream_t)stream>>>(w_master, (bf16*)w_bf16, grad, m, v, count, lr,
                                                                    beta1, beta2, eps, 1.f - c1, 1.f - c2,
                                                                    weight_decay);
    return status(cudaGetLastError());
}

int unet_f32_to_bf16(const float* x, void* y, long count, void* stream)
{
    f32_to_bf16_kernel<<<blocks_for(count), kT, 0, (cudaStream_t)stream>>>(x, (bf16*)y, count);
    return status(cudaGetLastError());
}

}  // extern "C"
