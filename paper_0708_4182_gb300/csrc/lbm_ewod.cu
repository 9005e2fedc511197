// lbm_ewod.cu -- C ABI (include/lbm_ewod.h) and the auxiliary kernels of the
// GB300 D2Q9 Shan-Chen electrowetting library. The time step itself is the
// fused kernel in lbm_step.cuh.
//
// Device workspace (caller-owned, carved here, every region 256-byte aligned):
//   A, B      two population buffers, FP32 planes [9][ny][pitch] (ping-pong)
//   mask      uint8 [ny][nx] copy of the solid mask (used by set/get only)
//   partials  kPartialStride doubles per CTA of the step grid (observables)
//   ring      kRing lbm_obs records written by the fused observables, plus
//             one scratch record for lbm_observables
//   status    int error flag raised by bounded device-side waits that gave up
//   staging   bounded buffer for host <-> device transfers of FP64 populations
#include "lbm_ewod.h"
#include "lbm_step.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <algorithm>
#include <vector>

namespace lbm {
namespace {

constexpr int kRing = 64;
constexpr int kGraphSteps = 32;  // plain steps per CUDA graph of lbm_step (even)
constexpr size_t kStagingMax = size_t(16) << 20;
constexpr int kAuxThreads = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int pitch_of(int nx) { return (nx + 31) / 32 * 32; }

struct Layout {
    size_t off_a, off_b, off_mask, off_partials, off_ring, off_status, off_staging, total;
    size_t pops_bytes, staging_bytes;
    int max_ctas;
};

bool params_valid(const lbm_params* p, const char** why)
{
    if (!p) { *why = "params is NULL"; return false; }
    if (p->nx < 1 || p->ny < 1) { *why = "nx and ny must be >= 1"; return false; }
    if (!(p->tau > 0.5) || !(p->tau < 1e6)) { *why = "tau must be > 0.5"; return false; }
    if (!(p->rho0 > 0.0)) { *why = "rho0 must be > 0"; return false; }
    if (p->green != LBM_GREEN_MC && p->green != LBM_GREEN_PRINTED) { *why = "unknown green convention"; return false; }
    if (p->normal != LBM_NORMAL_FACES && p->normal != LBM_NORMAL_UNIT) { *why = "unknown normal reading"; return false; }
    if (p->layout != LBM_LAYOUT_AUTO && p->layout != LBM_LAYOUT_PAIRS && p->layout != LBM_LAYOUT_SINGLE) {
        *why = "unknown thread layout"; return false;
    }
    if (p->storage < LBM_FP32 || p->storage > LBM_BF16_DEV) { *why = "unsupported storage"; return false; }
    if ((p->storage == LBM_FP16_DEV || p->storage == LBM_BF16_DEV) && (p->nx % 8) != 0) {
        *why = "16-bit storage needs nx to be a multiple of 8"; return false;
    }
    if (p->obs_every < 0) { *why = "obs_every must be >= 0"; return false; }
    if (p->tile_rows < 0 || (p->tile_rows != 0 && p->tile_rows < 4)) { *why = "tile_rows must be 0 or >= 4"; return false; }
    if ((p->ny + 3) / 4 > 65535) { *why = "ny too large for the step grid (ny <= 262140)"; return false; }
    const double plane = double(p->ny) * pitch_of(p->nx);
    if (9.0 * plane + 2.0 * pitch_of(p->nx) > 2147483647.0) { *why = "domain too large (9*ny*pitch must fit in int32)"; return false; }
    if (!std::isfinite(p->G) || !std::isfinite(p->G_wall) || !std::isfinite(p->rho_c) ||
        !std::isfinite(p->f_elec) || !std::isfinite(p->body_fx) || !std::isfinite(p->body_fy)) {
        *why = "non-finite model parameter"; return false;
    }
    return true;
}

// CTAs across a domain of nx columns (strips of strip_cols(storage) columns)
int ctas_x(int nx, int storage) { return (nx + strip_cols(storage) - 1) / strip_cols(storage); }

Layout layout_of(const lbm_params* p)
{
    Layout L{};
    const int pitch = pitch_of(p->nx);
    L.pops_bytes = size_t(9) * p->ny * pitch * sizeof(float);
    L.max_ctas = ctas_x(p->nx, p->storage) * ((p->ny + 3) / 4);
    size_t o = 0;
    L.off_a = o; o = align_up(o + L.pops_bytes, 256);
    L.off_b = o; o = align_up(o + L.pops_bytes, 256);
    L.off_mask = o; o = align_up(o + size_t(p->nx) * p->ny, 256);
    L.off_partials = o; o = align_up(o + size_t(L.max_ctas) * kPartialStride * sizeof(double), 256);
    L.off_ring = o; o = align_up(o + (kRing + 1) * sizeof(lbm_obs), 256);
    L.off_status = o; o = align_up(o + sizeof(int), 256);
    const size_t full = size_t(9) * p->nx * p->ny * sizeof(double);
    L.staging_bytes = full < kStagingMax ? full : kStagingMax;
    if (L.staging_bytes < size_t(9) * p->nx * sizeof(double)) L.staging_bytes = size_t(9) * p->nx * sizeof(double);
    L.off_staging = o; o = align_up(o + L.staging_bytes, 256);
    L.total = o;
    return L;
}

int auto_tile_rows(int nx, int ny, int storage, int sm_count, bool pair)
{
    // Segment height. Each CTA re-stages 4 halo rows, so taller segments waste
    // less, but several waves of CTAs (3 per SM) balance the slower seam
    // strips and hide the pipeline start of each CTA. Measured on the
    // 16384x4096 channel: 64 rows 90.8% of HBM peak, 48/96/160/192 rows
    // 88-90%, one wave of 586 rows 84%. Take 64 rows and halve it while
    // the grid has fewer than 4 waves; then even the segments out (same
    // count, heights differing by at most one row) so that no short last
    // segment pays the pipeline start and halo rows for a few rows.
    const long long slots = (long long)ctas_of(storage, true, pair) * sm_count;
    int rows = 64;
    while (rows > 4 && (long long)ctas_x(nx, storage) * ((ny + rows - 1) / rows) < 4 * slots) rows >>= 1;
    const int nseg = (ny + rows - 1) / rows;
    const int even = (ny + nseg - 1) / nseg;
    return even >= 4 ? even : rows;
}

// ---------------------------------------------------------------------------
// auxiliary kernels (set-up and read-back; not on the per-step path)

__constant__ int kEx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kEy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ int kOpp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
__constant__ double kW[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Write the solid sentinel into every plane of both buffers at solid nodes.
// Fluid nodes are left as they are: the state there is written by the next
// lbm_set_field (the spare buffer's by the next step); pitch padding is left
// untouched too.
__global__ void geometry_kernel(const uint8_t* __restrict__ mask, float* A,
                                float* B, Geom g)
{
    const int n = g.nx * g.ny;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!mask[i]) continue;
        const float v = __uint_as_float(kSolidBits);
        const int o = (i / g.nx) * g.pitch + i % g.nx;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            A[a * g.plane + o] = v;
            B[a * g.plane + o] = v;
        }
    }
}

__device__ __forceinline__ double feq_d(int a, double rho, double ux, double uy)
{
    const double eu = kEx[a] * ux + kEy[a] * uy;
    return kW[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy));
}

// The 9 equilibria f_a^eq(rho, u) of Eq. 3 in FP64, each rounded once to
// FP32: w_a rho (1 + 3 c + 4.5 c^2 - 1.5 u^2) with c = e_a . u, the
// polynomial as two FMAs around the shared 1 - 1.5 u^2 (the device has few
// FP64 units, so the set-up time follows the FP64 operation count).
__device__ __forceinline__ void feq_all_d(double rho, double ux, double uy, float* __restrict__ f, size_t plane)
{
    const double om = 1.0 - 1.5 * (ux * ux + uy * uy);
    const double w0r = kW[0] * rho, w1r = kW[1] * rho, w2r = kW[5] * rho;
    auto q = [om](double c) { return fma(c, fma(4.5, c, 3.0), om); };
    const double d5 = ux + uy, d6 = uy - ux;
    f[0] = float(w0r * om);
    f[plane] = float(w1r * q(ux));
    f[2 * plane] = float(w1r * q(uy));
    f[3 * plane] = float(w1r * q(-ux));
    f[4 * plane] = float(w1r * q(-uy));
    f[5 * plane] = float(w2r * q(d5));
    f[6 * plane] = float(w2r * q(d6));
    f[7 * plane] = float(w2r * q(-d5));
    f[8 * plane] = float(w2r * q(-d6));
}

// Initial state from (rho, ux, uy): the post-streaming populations
// f_a = f_a^eq(rho, u) of Eq. 3 (evaluated in FP64, rounded once), written
// into buffer `f` in plane layout; solid nodes get the sentinel.
__global__ void feq_kernel(const double* __restrict__ ru, const uint8_t* __restrict__ mask,
                           float* __restrict__ f, Geom g)
{
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = int(i / g.nx), x = int(i % g.nx);
        const int o = y * g.pitch + x;
        if (mask[i]) {
#pragma unroll
            for (int a = 0; a < 9; ++a) f[a * g.plane + o] = __uint_as_float(kSolidBits);
            continue;
        }
        feq_all_d(ru[i], ru[n + i], ru[2 * n + i], f + o, size_t(g.plane));
    }
}

// Initial state of a fluid at rest from its density alone (Eq. 3 at u = 0):
// f_a = w_a rho, evaluated in FP64 and rounded once (the values feq_kernel
// gives for u = 0); solid nodes get the sentinel.
__global__ void feq_rest_kernel(const double* __restrict__ rho, const uint8_t* __restrict__ mask,
                                float* __restrict__ f, Geom g)
{
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = int(i / g.nx), x = int(i % g.nx);
        const int o = y * g.pitch + x;
        const bool solid = mask[i] != 0;
        const double r = rho[i];
#pragma unroll
        for (int a = 0; a < 9; ++a) f[a * g.plane + o] = solid ? __uint_as_float(kSolidBits) : float(kW[a] * r);
    }
}

// State of a fluid at rest from an FP32 density rho [y][x] (dense, nx per
// row), directly in the storage form ST of `out`: f*_a(x) = w_a rho(s_a) with
// s_a = x + e_a, or x where that node is solid (un-streaming of f_a = w_a rho
// with the half-way bounce-back). Deviation forms: delta = sum_a w_a Delta_a,
// Delta_a = rho(s_a) - rho(x); rho* = rho(x) + delta, d_a = w_a (Delta_a -
// delta). FP32 arithmetic with the step kernel's weights. Solid nodes get the
// sentinel (plane 0; every plane in plain storage).
template <int ST>
__global__ void rest_f32_kernel(const float* __restrict__ rho, const uint8_t* __restrict__ mask,
                                float* __restrict__ out, Geom g)
{
    using T = typename StoreT<ST>::T;
    constexpr float w1 = 1.f / 9.f, w2 = 1.f / 36.f, w0 = 4.f / 9.f;
    const int n = g.nx * g.ny;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int y = i / g.nx, x = i % g.nx;
        const int o = y * g.pitch + x;
        if (mask[i]) {
            if constexpr (ST == kF32) {
#pragma unroll
                for (int a = 0; a < 9; ++a) out[a * g.plane + o] = __uint_as_float(kSolidBits);
            } else {
                out[o] = __uint_as_float(kSolidBits);
            }
            continue;
        }
        const float r = rho[i];
        float rs[9];
        rs[0] = r;
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const int xn = wrapi(x + kEx[a], g.nx), yn = wrapi(y + kEy[a], g.ny);
            const int j = yn * g.nx + xn;
            rs[a] = mask[j] ? r : rho[j];
        }
        if constexpr (ST == kF32) {
#pragma unroll
            for (int a = 0; a < 9; ++a) out[a * g.plane + o] = __fmul_rn(a == 0 ? w0 : (a <= 4 ? w1 : w2), rs[a]);
        } else {
            float dl[9];
#pragma unroll
            for (int a = 1; a < 9; ++a) dl[a] = __fsub_rn(rs[a], r);
            const float delta = fmaf(w1, __fadd_rn(__fadd_rn(dl[1], dl[3]), __fadd_rn(dl[2], dl[4])),
                                     __fmul_rn(w2, __fadd_rn(__fadd_rn(dl[5], dl[7]), __fadd_rn(dl[6], dl[8]))));
            out[o] = __fadd_rn(r, delta);
            T* od = reinterpret_cast<T*>(out + g.plane);
#pragma unroll
            for (int a = 1; a < 9; ++a)
                od[dev_index<T>(size_t(o), a, size_t(g.plane))] =
                    from_f<T>(__fmul_rn(a <= 4 ? w1 : w2, __fsub_rn(dl[a], delta)));
        }
    }
}

// plane p of buffer f <- the solid sentinel on solid nodes (other nodes untouched)
__global__ void solid_plane_kernel(const uint8_t* __restrict__ mask, float* __restrict__ f, int p, Geom g)
{
    const int n = g.nx * g.ny;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (mask[i]) f[size_t(p) * g.plane + (i / g.nx) * g.pitch + i % g.nx] = __uint_as_float(kSolidBits);
}

// Model constants in FP64 for the force-corrected initial state.
struct PhysD {
    double rho0, rho_c, f_elec, bfx, bfy;
    double g_axis, g_diag, w_axis, w_diag;
    int unit_normal;  // LBM_NORMAL_UNIT: the electric force along the unit face normal
};

__device__ __forceinline__ double psi_in(const double* __restrict__ rho, const uint8_t* __restrict__ mask,
                                         long long i, double rho0)
{
    return mask[i] ? 0.0 : rho0 * (1.0 - exp(-rho[i] / rho0));
}

// Initial state from (rho, u) with u the physical velocity (sum_a f_a e_a +
// F/2)/rho: f_a = f_a^eq(rho, u - F/(2 rho)) of Eq. 3, F the total force of
// the given density field (Eq. 5 fluid-fluid, Eq. 6 wall, the electric force
// on conductive wall-layer nodes, the body force), all in FP64.
__global__ void feq_phys_kernel(const double* __restrict__ ru, const uint8_t* __restrict__ mask,
                                float* __restrict__ f, Geom g, PhysD p)
{
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = int(i / g.nx), x = int(i % g.nx);
        const int o = y * g.pitch + x;
        if (mask[i]) {
#pragma unroll
            for (int a = 0; a < 9; ++a) f[a * g.plane + o] = __uint_as_float(kSolidBits);
            continue;
        }
        const int xe = x + 1 == g.nx ? 0 : x + 1, xw = x == 0 ? g.nx - 1 : x - 1;
        const int yn = y + 1 == g.ny ? 0 : y + 1, ys = y == 0 ? g.ny - 1 : y - 1;
        const long long rn = (long long)yn * g.nx, rc = (long long)y * g.nx, rs = (long long)ys * g.nx;
        const double pE = psi_in(ru, mask, rc + xe, p.rho0), pW = psi_in(ru, mask, rc + xw, p.rho0);
        const double pN = psi_in(ru, mask, rn + x, p.rho0), pS = psi_in(ru, mask, rs + x, p.rho0);
        const double pNE = psi_in(ru, mask, rn + xe, p.rho0), pNW = psi_in(ru, mask, rn + xw, p.rho0);
        const double pSE = psi_in(ru, mask, rs + xe, p.rho0), pSW = psi_in(ru, mask, rs + xw, p.rho0);
        const double sE = mask[rc + xe] ? 1.0 : 0.0, sW = mask[rc + xw] ? 1.0 : 0.0;
        const double sN = mask[rn + x] ? 1.0 : 0.0, sS = mask[rs + x] ? 1.0 : 0.0;
        const double sNE = mask[rn + xe] ? 1.0 : 0.0, sNW = mask[rn + xw] ? 1.0 : 0.0;
        const double sSE = mask[rs + xe] ? 1.0 : 0.0, sSW = mask[rs + xw] ? 1.0 : 0.0;
        const double rho = ru[i], ux = ru[n + i], uy = ru[2 * n + i];
        const double psi = p.rho0 * (1.0 - exp(-rho / p.rho0));
        const double gx = p.g_axis * (pE - pW) + p.g_diag * ((pNE - pNW) + (pSE - pSW)) +
                          p.w_axis * (sE - sW) + p.w_diag * ((sNE - sNW) + (sSE - sSW));
        const double gy = p.g_axis * (pN - pS) + p.g_diag * ((pNE + pNW) - (pSE + pSW)) +
                          p.w_axis * (sN - sS) + p.w_diag * ((sNE + sNW) - (sSE + sSW));
        double Fx = -psi * gx + rho * p.bfx, Fy = -psi * gy + rho * p.bfy;
        if (rho >= p.rho_c) {
            const double ex = sE - sW, ey = sN - sS;
            const double len = (p.unit_normal && ex != 0.0 && ey != 0.0) ? sqrt(2.0) : 1.0;
            Fx += p.f_elec * ex / len;
            Fy += p.f_elec * ey / len;
        }
        const double vx = ux - 0.5 * Fx / rho, vy = uy - 0.5 * Fy / rho;
#pragma unroll
        for (int a = 0; a < 9; ++a) f[a * g.plane + o] = float(feq_d(a, rho, vx, vy));
    }
}

// Rows [r0, r0 + rows) of dense FP64 populations laid out [9][rows][nx]
// -> FP32 post-streaming planes of buffer `f` (pitch layout).
__global__ void pops_in_kernel(const double* __restrict__ src, float* __restrict__ f, Geom g,
                               int r0, int rows)
{
    const long long n = 9LL * rows * g.nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int a = int(i / ((long long)rows * g.nx));
        const long long rem = i % ((long long)rows * g.nx);
        const int y = r0 + int(rem / g.nx), x = int(rem % g.nx);
        f[a * g.plane + y * g.pitch + x] = float(src[i]);
    }
}

// Post-streaming f (buffer `f`) -> post-collision f* (buffer `out`), the
// inverse of the pull: f*_a(x) = f_a(x + e_a) or, next to a wall, f_opp(a)(x).
// Solid nodes of `out` get the sentinel.
__global__ void unstream_kernel(const float* __restrict__ f, const uint8_t* __restrict__ mask,
                                float* __restrict__ out, Geom g)
{
    const long long n = (long long)g.nx * g.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = int(i / g.nx), x = int(i % g.nx);
        if (mask[i]) {
            for (int a = 0; a < 9; ++a) out[a * g.plane + y * g.pitch + x] = __uint_as_float(kSolidBits);
            continue;
        }
        for (int a = 0; a < 9; ++a) {
            const int xn = wrapi(x + kEx[a], g.nx), yn = wrapi(y + kEy[a], g.ny);
            float v;
            if (mask[(long long)yn * g.nx + xn])
                v = f[kOpp[a] * g.plane + y * g.pitch + x];
            else
                v = f[a * g.plane + yn * g.pitch + xn];
            out[a * g.plane + y * g.pitch + x] = v;
        }
    }
}

// Post-streaming populations of rows [r0, r0 + rows) pulled from the f*
// buffer, written as dense FP64 [9][rows][nx] (0 on solid nodes).
__global__ void pops_out_kernel(const float* __restrict__ fs, const uint8_t* __restrict__ mask,
                                double* __restrict__ dst, Geom g, int r0, int rows)
{
    const long long n = (long long)rows * g.nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = r0 + int(i / g.nx), x = int(i % g.nx);
        const bool solid = mask[(long long)y * g.nx + x] != 0;
        for (int a = 0; a < 9; ++a) {
            double v = 0.0;
            if (!solid) {
                const int xs = wrapi(x - kEx[a], g.nx), ys = wrapi(y - kEy[a], g.ny);
                if (mask[(long long)ys * g.nx + xs])
                    v = fs[kOpp[a] * g.plane + y * g.pitch + x];
                else
                    v = fs[a * g.plane + ys * g.pitch + xs];
            }
            dst[a * n + i] = v;
        }
    }
}

// Plain post-collision planes f* (FP32) -> deviation form: plane 0 gets
// rho* = sum_a f*_a, the deviations (type T, laid out by dev_index) get
// d_a = f*_a - w_a rho* (FP64 arithmetic, one rounding each). Solid nodes get
// the sentinel.
template <typename T>
__global__ void plain_to_dev_kernel(const float* __restrict__ fs, const uint8_t* __restrict__ mask,
                                    float* __restrict__ out, Geom g)
{
    const long long n = (long long)g.nx * g.ny;
    T* od = reinterpret_cast<T*>(out + g.plane);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = int(i / g.nx), x = int(i % g.nx);
        const int o = y * g.pitch + x;
        if (mask[i]) {
            out[o] = __uint_as_float(kSolidBits);
            continue;
        }
        double r = 0.0;
        for (int a = 0; a < 9; ++a) r += fs[a * g.plane + o];
        const float r32 = float(r);
        out[o] = r32;
        for (int a = 1; a < 9; ++a)
            od[dev_index<T>(size_t(o), a, size_t(g.plane))] =
                from_f<T>(float(double(fs[a * g.plane + o]) - kW[a] * double(r32)));
    }
}

// Deviation form -> plain post-collision planes: f*_a = w_a rho* + d_a,
// f*_0 = w_0 rho* - sum_a d_a (FP64, one rounding each); solids get the sentinel.
template <typename T>
__global__ void dev_to_plain_kernel(const float* __restrict__ in, const uint8_t* __restrict__ mask,
                                    float* __restrict__ fs, Geom g)
{
    const long long n = (long long)g.nx * g.ny;
    const T* id = reinterpret_cast<const T*>(in + g.plane);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = int(i / g.nx), x = int(i % g.nx);
        const int o = y * g.pitch + x;
        if (mask[i]) {
            for (int a = 0; a < 9; ++a) fs[a * g.plane + o] = __uint_as_float(kSolidBits);
            continue;
        }
        const double r = in[o];
        double dsum = 0.0;
        for (int a = 1; a < 9; ++a) {
            const double d = to_f(id[dev_index<T>(size_t(o), a, size_t(g.plane))]);
            dsum += d;
            fs[a * g.plane + o] = float(kW[a] * r + d);
        }
        fs[o] = float(kW[0] * r - dsum);
    }
}

// Self-test of the timeout path: thread 0 waits, with the step kernel's
// bounded mbarrier wait, on a phase of an mbarrier that nothing arrives at;
// the wait gives up and raises *err.
__global__ void wait_selftest_kernel(int* err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_wait(&bar, 0, err);
    }
}

// Mean velocity profile across the channel: out[y] = (1/nx) sum_x u_x(x, y)
// from a kFields array (solid nodes hold 0), one block per row, FP64 tree sum.
__global__ void ux_profile_kernel(const double* __restrict__ fields, Geom g, double* __restrict__ out)
{
    __shared__ double red[kAuxThreads];
    const size_t nn = (size_t)g.nx * g.ny;
    for (int y = blockIdx.x; y < g.ny; y += gridDim.x) {
        double s = 0.0;
        for (int x = threadIdx.x; x < g.nx; x += kAuxThreads) s += fields[nn + (size_t)y * g.nx + x];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = kAuxThreads / 2; h > 0; h >>= 1) {
            if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[y] = red[0] / g.nx;
        __syncthreads();
    }
}

// Sum the per-CTA partials in a fixed order and write one lbm_obs record.
__global__ void finalize_obs_kernel(const double* __restrict__ partials, int nctas, double inv_nx,
                                    long long step, lbm_obs* __restrict__ rec)
{
    __shared__ double s[4][kAuxThreads];
    __shared__ double mx[kAuxThreads], mn[kAuxThreads], bd[kAuxThreads];
    const int t = threadIdx.x;
    double a[4] = {0, 0, 0, 0}, um = 0.0, rm = INFINITY, b = 0.0;
    for (int c = t; c < nctas; c += kAuxThreads) {
        const double* q = partials + (size_t)c * kPartialStride;
        for (int k = 0; k < 4; ++k) a[k] += q[k];
        um = fmax(um, q[4]);
        rm = fmin(rm, q[5]);
        b += q[6];
    }
    for (int k = 0; k < 4; ++k) s[k][t] = a[k];
    mx[t] = um;
    mn[t] = rm;
    bd[t] = b;
    __syncthreads();
    for (int h = kAuxThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            for (int k = 0; k < 4; ++k) s[k][t] += s[k][t + h];
            mx[t] = fmax(mx[t], mx[t + h]);
            mn[t] = fmin(mn[t], mn[t + h]);
            bd[t] += bd[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        rec->step = step;
        rec->mass = s[0][0];
        rec->flux_Q = s[1][0] * inv_nx;
        rec->mom_x = s[2][0];
        rec->mom_y = s[3][0];
        rec->max_u = sqrt(mx[0]);
        rec->min_rho = mn[0];
        rec->nonfinite = (long long)bd[0];
    }
}

int aux_blocks(long long n, int sm_count)
{
    long long b = (n + kAuxThreads - 1) / kAuxThreads;
    const long long cap = 32LL * sm_count;
    return int(b < 1 ? 1 : (b > cap ? cap : b));
}

// One CTA per domain: sum domain d's nctas[d] partials in a fixed order into
// rec[d]; domains with want[d] == 0 are skipped.
__global__ void finalize_batch_kernel(double* const* __restrict__ partials, const int* __restrict__ nctas,
                                      const double* __restrict__ inv_nx, const long long* __restrict__ step,
                                      const unsigned char* __restrict__ want, lbm_obs* __restrict__ rec)
{
    const int d = blockIdx.x;
    if (!want[d]) return;
    __shared__ double s[4][kAuxThreads];
    __shared__ double mx[kAuxThreads], mn[kAuxThreads], bd[kAuxThreads];
    const int t = threadIdx.x;
    double a[4] = {0, 0, 0, 0}, um = 0.0, rm = INFINITY, b = 0.0;
    for (int c = t; c < nctas[d]; c += kAuxThreads) {
        const double* q = partials[d] + (size_t)c * kPartialStride;
        for (int k = 0; k < 4; ++k) a[k] += q[k];
        um = fmax(um, q[4]);
        rm = fmin(rm, q[5]);
        b += q[6];
    }
    for (int k = 0; k < 4; ++k) s[k][t] = a[k];
    mx[t] = um;
    mn[t] = rm;
    bd[t] = b;
    __syncthreads();
    for (int h = kAuxThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            for (int k = 0; k < 4; ++k) s[k][t] += s[k][t + h];
            mx[t] = fmax(mx[t], mx[t + h]);
            mn[t] = fmin(mn[t], mn[t + h]);
            bd[t] += bd[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        lbm_obs& r = rec[d];
        r.step = step[d];
        r.mass = s[0][0];
        r.flux_Q = s[1][0] * inv_nx[d];
        r.mom_x = s[2][0];
        r.mom_y = s[3][0];
        r.max_u = sqrt(mx[0]);
        r.min_rho = mn[0];
        r.nonfinite = (long long)bd[0];
    }
}

// ---------------------------------------------------------------------------
// allocation-free observables (see lbm_observables_noalloc in lbm_ewod.h)

constexpr int kNoAllocSlots = 1024;                   // per-CTA partial slots
constexpr int kNoAllocNodesPerCta = 64 * kAuxThreads;  // nodes one CTA reduces
constexpr long long kNoAllocMaxNodes = (long long)kNoAllocSlots * kNoAllocNodesPerCta;

// Per-CTA partials followed by one lbm_obs record: 64 KB + 64 B, resident on
// every device that loads the library. Host code must not use this name as an
// address; it goes through cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots * kPartialStride + 8];

// Observables of the post-streaming populations `pops` (dense FP64
// [9][ny][nx]) on the fluid nodes of `solid`, one CTA per chunk of
// kNoAllocNodesPerCta nodes. Per node it rebuilds what the step kernel's
// observables pass sees (FP32 populations, rho, j, psi of the node and its 8
// neighbours, solid flags of the pull sources) and hands them to the same
// collide_node<kObs>. Every CTA writes its whole partial slot.
__global__ void __launch_bounds__(kAuxThreads)
    observe_dense_kernel(const double* __restrict__ pops, const uint8_t* __restrict__ solid, Geom g,
                         Phys p, double* __restrict__ partials)
{
    const long long n = (long long)g.nx * g.ny;
    const long long first = (long long)blockIdx.x * kNoAllocNodesPerCta;
    const long long last = min(first + kNoAllocNodesPerCta, n);
    ObsAcc acc;
    auto rho_at = [&](int x, int y) {
        const long long j = (long long)y * g.nx + x;
        float v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = float(pops[a * n + j]);
        return ((v[0] + (v[1] + v[3])) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
    };
    for (long long i = first + threadIdx.x; i < last; i += kAuxThreads) {
        if (solid[i]) continue;
        const int y = int(i / g.nx), x = int(i % g.nx);
        Pulled nd;
        nd.solid = false;
        float v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = float(pops[a * n + i]);
        uint32_t sb = 0;
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            const int xs = wrapi(x - kEx[a], g.nx), ys = wrapi(y - kEy[a], g.ny);
            if (solid[(long long)ys * g.nx + xs]) sb |= 1u << a;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) nd.f[a] = v[a];
        nd.sb = sb;
        nd.rho = ((v[0] + (v[1] + v[3])) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
        nd.jx = (v[1] - v[3]) + (v[5] - v[7]) + (v[8] - v[6]);
        nd.jy = (v[2] - v[4]) + (v[5] - v[7]) + (v[6] - v[8]);
        // psi of the 3x3 neighbourhood, rows y-1, y, y+1 and columns x-1, x, x+1
        float psi3[3][3];
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int xn = wrapi(x + dx, g.nx), yn = wrapi(y + dy, g.ny);
                Pulled q;
                q.solid = solid[(long long)yn * g.nx + xn] != 0;
                q.rho = q.solid ? 0.f : (dx == 0 && dy == 0 ? nd.rho : rho_at(xn, yn));
                psi3[dy + 1][dx + 1] = pseudopotential(p, q);
            }
        collide_node<kObs, true>(nd, psi3[0], psi3[1], psi3[2], 1, p, g, nullptr, nullptr, x, y, acc);
    }
    // deterministic CTA reduction into this CTA's partial slot
    __shared__ double red_d[4][kAuxThreads / 32];
    __shared__ float red_f[2][kAuxThreads / 32];
    __shared__ unsigned red_u[kAuxThreads / 32];
    double d[4] = {acc.mass.value(), acc.q.value(), acc.px.value(), acc.py.value()};
    float umax2 = acc.umax2, rmin = acc.rmin;
    unsigned bad = acc.bad;
    for (int off = 16; off > 0; off >>= 1) {
        for (int q = 0; q < 4; ++q) d[q] += __shfl_down_sync(0xffffffffu, d[q], off);
        umax2 = fmaxf(umax2, __shfl_down_sync(0xffffffffu, umax2, off));
        rmin = fminf(rmin, __shfl_down_sync(0xffffffffu, rmin, off));
        bad += __shfl_down_sync(0xffffffffu, bad, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (int q = 0; q < 4; ++q) red_d[q][w] = d[q];
        red_f[0][w] = umax2;
        red_f[1][w] = rmin;
        red_u[w] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s4[4] = {0, 0, 0, 0};
        float um = 0.f, rm = __int_as_float(0x7f800000);
        unsigned b = 0;
        for (int k = 0; k < kAuxThreads / 32; ++k) {
            for (int q = 0; q < 4; ++q) s4[q] += red_d[q][k];
            um = fmaxf(um, red_f[0][k]);
            rm = fminf(rm, red_f[1][k]);
            b += red_u[k];
        }
        double* out = partials + (size_t)blockIdx.x * kPartialStride;
        for (int q = 0; q < 4; ++q) out[q] = s4[q];
        out[4] = um;
        out[5] = rm;
        out[6] = b;
        out[7] = 0.0;
    }
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_ctx {
    lbm_params prm{};
    Layout L{};
    Geom g{};
    Phys ph{};
    cudaStream_t stream = nullptr;
    unsigned char* ws = nullptr;
    float* cur = nullptr;  // f* of the current state
    float* nxt = nullptr;
    uint8_t* mask = nullptr;
    double* partials = nullptr;
    lbm_obs* ring = nullptr;
    double* staging = nullptr;
    int* status = nullptr;
    int sm_count = 0;
    bool pair = true;  // the 32-bit forms' pair layout (false: one node per thread)
    dim3 grid;
    int64_t t = 0;
    int64_t last_obs_t = -1;
    int ring_count = 0;
    bool has_geometry = false, has_field = false;
    char err[512] = {0};
    // kGraphSteps plain steps as one CUDA graph, one per buffer holding the
    // current state (buffer A, buffer B); built on first use
    cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
    ~lbm_ctx()
    {
        for (cudaGraphExec_t e : step_graph)
            if (e) cudaGraphExecDestroy(e);
    }
};

namespace {

lbm_status fail(lbm_ctx* c, lbm_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

lbm_status check_cuda(lbm_ctx* c, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return LBM_OK;
    return fail(c, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

lbm_status check_launch(lbm_ctx* c, const char* what) { return check_cuda(c, cudaGetLastError(), what); }

Phys make_phys(const lbm_params& p)
{
    Phys h{};
    h.tau = float(p.tau);
    h.inv_tau = float(1.0 / p.tau);
    h.rho0 = float(p.rho0);
    h.inv_rho0 = float(1.0 / p.rho0);
    h.rho_c = float(p.rho_c);
    h.f_elec = float(p.f_elec);
    h.bfx = float(p.body_fx);
    h.bfy = float(p.body_fy);
    // Green-function magnitudes on axis (|e| = 1) and diagonal (|e| = sqrt 2) links
    const double ka = p.green == LBM_GREEN_PRINTED ? 2.0 : 1.0;
    const double kd = p.green == LBM_GREEN_PRINTED ? 1.0 : 0.5;
    h.g_axis = float(ka * p.G);
    h.g_diag = float(kd * p.G);
    h.w_axis = float(ka * p.G_wall);
    h.w_diag = float(kd * p.G_wall);
    // a corner's two face directions add up to length sqrt 2
    h.e_corner = p.normal == LBM_NORMAL_UNIT ? float(std::sqrt(0.5)) : 1.f;
    return h;
}

// The kernel instance: the tau = 1 specialisation unless a step relaxes
// with tau != 1 (the observing modes never relax).
template <int MODE, int ST, bool PAIR>
lbm_status launch_step_layout(lbm_ctx* c, const float* fin, float* fout, double* fields)
{
    constexpr unsigned nt = threads_of(ST, PAIR);
    constexpr size_t sm = smem_bytes<ST, PAIR>();
    bool t1 = true;
    if constexpr (MODE == kStep || MODE == kStepObs) {
        if (c->ph.tau != 1.f) {
            t1 = false;
            step_kernel<MODE, ST, false, PAIR><<<c->grid, nt, sm, c->stream>>>(fin, fout, c->g, c->ph, c->partials,
                                                                              fields, c->status);
        }
    }
    if (t1)
        step_kernel<MODE, ST, true, PAIR><<<c->grid, nt, sm, c->stream>>>(fin, fout, c->g, c->ph, c->partials,
                                                                         fields, c->status);
    return check_launch(c, "step kernel launch");
}

// The 16-bit forms have one layout (one node per thread, PAIR = false).
template <int MODE, int ST>
lbm_status launch_step_st(lbm_ctx* c, const float* fin, float* fout, double* fields)
{
    if constexpr (is16(ST))
        return launch_step_layout<MODE, ST, false>(c, fin, fout, fields);
    else if (c->pair)
        return launch_step_layout<MODE, ST, true>(c, fin, fout, fields);
    else
        return launch_step_layout<MODE, ST, false>(c, fin, fout, fields);
}

template <int MODE>
lbm_status launch_step(lbm_ctx* c, const float* fin, float* fout, double* fields)
{
    switch (c->prm.storage) {
    case LBM_FP32_DEV: return launch_step_st<MODE, kF32Dev>(c, fin, fout, fields);
    case LBM_FP16_DEV: return launch_step_st<MODE, kF16Dev>(c, fin, fout, fields);
    case LBM_BF16_DEV: return launch_step_st<MODE, kBF16Dev>(c, fin, fout, fields);
    default: return launch_step_st<MODE, kF32>(c, fin, fout, fields);
    }
}

// Step kernel (plain step, no observables) of a storage form and layout
// (the same as launch_step_st picks).
template <int ST, bool PAIR> const void* plain_step_layout(bool t1)
{
    return t1 ? reinterpret_cast<const void*>(&step_kernel<kStep, ST, true, PAIR>)
              : reinterpret_cast<const void*>(&step_kernel<kStep, ST, false, PAIR>);
}

template <int ST> const void* plain_step_ptr(bool t1, bool pair)
{
    if constexpr (is16(ST))
        return plain_step_layout<ST, false>(t1);
    else
        return pair ? plain_step_layout<ST, true>(t1) : plain_step_layout<ST, false>(t1);
}

const void* plain_step_kernel(int storage, bool t1, bool pair)
{
    switch (storage) {
    case LBM_FP32_DEV: return plain_step_ptr<kF32Dev>(t1, pair);
    case LBM_FP16_DEV: return plain_step_ptr<kF16Dev>(t1, pair);
    case LBM_BF16_DEV: return plain_step_ptr<kBF16Dev>(t1, pair);
    default: return plain_step_ptr<kF32>(t1, pair);
    }
}

size_t step_smem(int storage, bool pair)
{
    switch (storage) {
    case LBM_FP32_DEV: return pair ? smem_bytes<kF32Dev, true>() : smem_bytes<kF32Dev, false>();
    case LBM_FP16_DEV: return smem_bytes<kF16Dev, false>();
    case LBM_BF16_DEV: return smem_bytes<kBF16Dev, false>();
    default: return pair ? smem_bytes<kF32, true>() : smem_bytes<kF32, false>();
    }
}

// threads per CTA of a storage form and layout
unsigned step_threads(int storage, bool pair)
{
    return unsigned(threads_of(storage, pair && !is16(storage)));
}

// kGraphSteps (even) plain steps starting from the current buffer, as one
// explicitly built graph of kernel nodes; an even count returns the state
// to the same buffer, so the graph replays for as long as the context lives.
lbm_status step_graph(lbm_ctx* c, cudaGraphExec_t* out)
{
    const int slot = c->cur == reinterpret_cast<float*>(c->ws + c->L.off_a) ? 0 : 1;
    if (c->step_graph[slot]) {
        *out = c->step_graph[slot];
        return LBM_OK;
    }
    cudaGraph_t graph = nullptr;
    lbm_status s = check_cuda(c, cudaGraphCreate(&graph, 0), "graph create");
    if (s) return s;
    cudaGraphNode_t prev = nullptr;
    double* no_fields = nullptr;
    for (int k = 0; k < kGraphSteps && !s; ++k) {
        const float* fin = (k & 1) ? c->nxt : c->cur;
        float* fout = (k & 1) ? c->cur : c->nxt;
        void* args[] = {&fin, &fout, &c->g, &c->ph, &c->partials, &no_fields, &c->status};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(plain_step_kernel(c->prm.storage, c->ph.tau == 1.f, c->pair));
        kp.gridDim = c->grid;
        kp.blockDim = dim3(step_threads(c->prm.storage, c->pair));
        kp.sharedMemBytes = static_cast<unsigned>(step_smem(c->prm.storage, c->pair));
        kp.kernelParams = args;
        cudaGraphNode_t node;
        s = check_cuda(c, cudaGraphAddKernelNode(&node, graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp),
                       "graph node");
        prev = node;
    }
    if (!s) s = check_cuda(c, cudaGraphInstantiate(&c->step_graph[slot], graph, 0), "graph instantiate");
    cudaGraphDestroy(graph);
    if (!s) *out = c->step_graph[slot];
    return s;
}


template <int MODE, int ST, bool PAIR>
cudaError_t allow_smem_st()
{
    cudaError_t e = cudaFuncSetAttribute(step_kernel<MODE, ST, true, PAIR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes<ST, PAIR>()));
    if constexpr (MODE == kStep || MODE == kStepObs) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(step_kernel<MODE, ST, false, PAIR>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_bytes<ST, PAIR>()));
    }
    return e;
}

template <int MODE>
cudaError_t allow_smem()
{
    cudaError_t e = allow_smem_st<MODE, kF32, true>();
    if (e == cudaSuccess) e = allow_smem_st<MODE, kF32, false>();
    if (e == cudaSuccess) e = allow_smem_st<MODE, kF32Dev, true>();
    if (e == cudaSuccess) e = allow_smem_st<MODE, kF32Dev, false>();
    if (e == cudaSuccess) e = allow_smem_st<MODE, kF16Dev, false>();
    if (e == cudaSuccess) e = allow_smem_st<MODE, kBF16Dev, false>();
    return e;
}

// Convert the plain f* in c->cur to the context's deviation form (into the
// spare buffer, which becomes current). No-op for plain storage.
lbm_status plain_to_storage(lbm_ctx* c)
{
    const long long n = (long long)c->g.nx * c->g.ny;
    const int b = aux_blocks(n, c->sm_count);
    switch (c->prm.storage) {
    case LBM_FP32_DEV: plain_to_dev_kernel<float><<<b, kAuxThreads, 0, c->stream>>>(c->cur, c->mask, c->nxt, c->g); break;
    case LBM_FP16_DEV: plain_to_dev_kernel<__half><<<b, kAuxThreads, 0, c->stream>>>(c->cur, c->mask, c->nxt, c->g); break;
    case LBM_BF16_DEV: plain_to_dev_kernel<__nv_bfloat16><<<b, kAuxThreads, 0, c->stream>>>(c->cur, c->mask, c->nxt, c->g); break;
    default: return LBM_OK;
    }
    lbm_status s = check_launch(c, "storage conversion launch");
    if (s) return s;
    float* tmp = c->cur;
    c->cur = c->nxt;
    c->nxt = tmp;
    return LBM_OK;
}

// Plain f* of the current state: c->cur itself for plain storage, else a
// conversion into the spare buffer (which the next step overwrites).
lbm_status storage_to_plain(lbm_ctx* c, const float** plain)
{
    const long long n = (long long)c->g.nx * c->g.ny;
    const int b = aux_blocks(n, c->sm_count);
    switch (c->prm.storage) {
    case LBM_FP32_DEV: dev_to_plain_kernel<float><<<b, kAuxThreads, 0, c->stream>>>(c->cur, c->mask, c->nxt, c->g); break;
    case LBM_FP16_DEV: dev_to_plain_kernel<__half><<<b, kAuxThreads, 0, c->stream>>>(c->cur, c->mask, c->nxt, c->g); break;
    case LBM_BF16_DEV: dev_to_plain_kernel<__nv_bfloat16><<<b, kAuxThreads, 0, c->stream>>>(c->cur, c->mask, c->nxt, c->g); break;
    default: *plain = c->cur; return LBM_OK;
    }
    *plain = c->nxt;
    return check_launch(c, "storage conversion launch");
}

// Read and clear the device error flag (the stream must be synchronised).
lbm_status check_status(lbm_ctx* c)
{
    int flag = 0;
    lbm_status s = check_cuda(c, cudaMemcpy(&flag, c->status, sizeof(int), cudaMemcpyDeviceToHost),
                              "status download");
    if (s) return s;
    if (flag) {
        cudaMemset(c->status, 0, sizeof(int));
        return fail(c, LBM_ETIMEOUT, "a bounded device-side wait gave up (flag %d)", flag);
    }
    return LBM_OK;
}

lbm_status finalize(lbm_ctx* c, int64_t step, lbm_obs* rec)
{
    finalize_obs_kernel<<<1, kAuxThreads, 0, c->stream>>>(c->partials, int(c->grid.x * c->grid.y),
                                                          1.0 / c->prm.nx, (long long)step, rec);
    return check_launch(c, "observables finalize launch");
}

lbm_status ready(lbm_ctx* c)
{
    if (!c) return LBM_EINVAL;
    if (!c->has_geometry || !c->has_field)
        return fail(c, LBM_ESTATE, "set the geometry and a field before this call");
    return LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_workspace_bytes(const lbm_params* p)
{
    const char* why;
    if (!params_valid(p, &why)) return 0;
    return layout_of(p).total;
}

lbm_status lbm_create(const lbm_params* p, void* d_workspace, size_t bytes, void* cuda_stream,
                      lbm_ctx** out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    const char* why = "";
    if (!params_valid(p, &why)) return LBM_EINVAL;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return LBM_EINVAL;
    Layout L = layout_of(p);
    if (bytes < L.total) return LBM_ENOMEM;
    lbm_ctx* c = new (std::nothrow) lbm_ctx;
    if (!c) return LBM_ENOMEM;
    c->prm = *p;
    c->L = L;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->ws = static_cast<unsigned char*>(d_workspace);
    c->cur = reinterpret_cast<float*>(c->ws + L.off_a);
    c->nxt = reinterpret_cast<float*>(c->ws + L.off_b);
    c->mask = c->ws + L.off_mask;
    c->partials = reinterpret_cast<double*>(c->ws + L.off_partials);
    c->ring = reinterpret_cast<lbm_obs*>(c->ws + L.off_ring);
    c->staging = reinterpret_cast<double*>(c->ws + L.off_staging);
    c->status = reinterpret_cast<int*>(c->ws + L.off_status);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        allow_smem<kStep>() != cudaSuccess || allow_smem<kStepObs>() != cudaSuccess ||
        allow_smem<kObs>() != cudaSuccess || allow_smem<kFields>() != cudaSuccess ||
        cudaMemsetAsync(c->status, 0, sizeof(int), c->stream) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return LBM_ECUDA;
    }
    c->g.nx = p->nx;
    c->g.ny = p->ny;
    c->g.pitch = pitch_of(p->nx);
    c->g.plane = p->ny * c->g.pitch;
    // Thread layout of the 32-bit forms: pairs, unless the domain is too small
    // to give the GPU more than 3 CTAs per SM at the smallest segment height
    // (4 rows); there the one-node layout's twice as many threads per CTA
    // hide more latency. Measured (MLUPS, FP32 one-node / pairs): 128x64
    // 1114 / 889, 1024x256 29901 / 27499, 1024x512 34375 / 47015.
    c->pair = !is16(p->storage) &&
              (p->layout == LBM_LAYOUT_PAIRS ||
               (p->layout == LBM_LAYOUT_AUTO &&
                (long long)ctas_x(p->nx, p->storage) * ((p->ny + 3) / 4) > 3LL * c->sm_count));
    c->g.tile_rows =
        p->tile_rows ? p->tile_rows : auto_tile_rows(p->nx, p->ny, p->storage, c->sm_count, c->pair);
    c->grid = dim3(ctas_x(p->nx, p->storage), (p->ny + c->g.tile_rows - 1) / c->g.tile_rows);
    c->ph = make_phys(*p);
    *out = c;
    return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_ctx* c, const uint8_t* solid, int on_device)
{
    if (!c) return LBM_EINVAL;
    if (!solid) return fail(c, LBM_EINVAL, "solid mask is NULL");
    const size_t n = size_t(c->g.nx) * c->g.ny;
    lbm_status s = check_cuda(c, cudaMemcpyAsync(c->mask, solid, n,
                                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                                 c->stream), "mask upload");
    if (s) return s;
    geometry_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(c->mask, c->cur, c->nxt, c->g);
    if ((s = check_launch(c, "geometry kernel launch"))) return s;
    c->has_geometry = true;
    c->has_field = false;
    c->t = 0;
    c->last_obs_t = -1;
    c->ring_count = 0;
    return LBM_OK;
}

lbm_status lbm_set_field(lbm_ctx* c, int which, const double* data, int on_device)
{
    if (!c) return LBM_EINVAL;
    if (!data) return fail(c, LBM_EINVAL, "field data is NULL");
    if (!c->has_geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry must come before lbm_set_field");
    const size_t n = size_t(c->g.nx) * c->g.ny;
    lbm_status s;
    if (which == LBM_RHO_U || which == LBM_RHO_U_PHYS || which == LBM_RHO) {
        // (rho, u) -> f_eq into the current buffer -> un-streamed into the
        // spare one, which becomes current; both end with solid sentinels
        const double* src = data;
        const size_t comps = which == LBM_RHO ? 1 : 3;
        if (!on_device) {
            // (rho, ux, uy) in FP64 fits in the spare population buffer
            double* tmp = reinterpret_cast<double*>(c->nxt);
            if ((s = check_cuda(c, cudaMemcpyAsync(tmp, data, comps * n * sizeof(double), cudaMemcpyHostToDevice,
                                                   c->stream), "field upload")))
                return s;
            src = tmp;
        }
        if (which == LBM_RHO) {
            feq_rest_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(src, c->mask, c->cur, c->g);
        } else if (which == LBM_RHO_U) {
            feq_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(src, c->mask, c->cur, c->g);
        } else {
            const lbm_params& q = c->prm;
            const double ka = q.green == LBM_GREEN_PRINTED ? 2.0 : 1.0;
            const double kd = q.green == LBM_GREEN_PRINTED ? 1.0 : 0.5;
            const PhysD pd{q.rho0, q.rho_c, q.f_elec, q.body_fx, q.body_fy,
                           ka * q.G, kd * q.G, ka * q.G_wall, kd * q.G_wall, q.normal == LBM_NORMAL_UNIT};
            feq_phys_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(src, c->mask, c->cur, c->g,
                                                                                     pd);
        }
        if ((s = check_launch(c, "field kernel launch"))) return s;
        unstream_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(c->cur, c->mask, c->nxt, c->g);
        if ((s = check_launch(c, "unstream kernel launch"))) return s;
        float* tmpb = c->cur;
        c->cur = c->nxt;
        c->nxt = tmpb;
        if ((s = plain_to_storage(c))) return s;
    } else if (which == LBM_POPS) {
        const int nx = c->g.nx, ny = c->g.ny;
        const int rows_per = on_device ? ny : int(c->L.staging_bytes / (9 * size_t(nx) * sizeof(double)));
        for (int r0 = 0; r0 < ny; r0 += rows_per) {
            const int rows = (r0 + rows_per <= ny) ? rows_per : ny - r0;
            const double* src = data;
            if (!on_device) {
                for (int a = 0; a < 9; ++a) {
                    if ((s = check_cuda(c, cudaMemcpyAsync(c->staging + size_t(a) * rows * nx,
                                                           data + size_t(a) * n + size_t(r0) * nx,
                                                           size_t(rows) * nx * sizeof(double),
                                                           cudaMemcpyHostToDevice, c->stream),
                                        "population upload")))
                        return s;
                }
                src = c->staging;
            } else if (rows != ny) {
                return fail(c, LBM_EINVAL, "internal: device populations are converted in one pass");
            }
            pops_in_kernel<<<aux_blocks(9LL * rows * nx, c->sm_count), kAuxThreads, 0, c->stream>>>(src, c->nxt, c->g, r0, rows);
            if ((s = check_launch(c, "population kernel launch"))) return s;
            if (!on_device) {
                // the staging buffer is reused by the next chunk
                if ((s = check_cuda(c, cudaStreamSynchronize(c->stream), "population upload sync"))) return s;
            }
        }
        unstream_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(c->nxt, c->mask, c->cur, c->g);
        if ((s = check_launch(c, "unstream kernel launch"))) return s;
        geometry_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(c->mask, c->nxt, c->nxt, c->g);
        if ((s = check_launch(c, "geometry kernel launch"))) return s;
        if ((s = plain_to_storage(c))) return s;
    } else {
        return fail(c, LBM_EINVAL, "unknown field selector %d", which);
    }
    c->has_field = true;
    return LBM_OK;
}

lbm_status lbm_set_density_f32(lbm_ctx* c, const float* rho, int on_device)
{
    if (!c) return LBM_EINVAL;
    if (!rho) return fail(c, LBM_EINVAL, "density is NULL");
    if (!c->has_geometry) return fail(c, LBM_ESTATE, "lbm_set_geometry must come before lbm_set_density_f32");
    const size_t n = size_t(c->g.nx) * c->g.ny;
    lbm_status s;
    const float* src = rho;
    // a host density goes into the spare buffer's last plane (no form stores
    // anything there that the set-up reads), restored to sentinels below
    float* tmp = c->nxt + size_t(8) * c->g.plane;
    if (!on_device) {
        if ((s = check_cuda(c, cudaMemcpyAsync(tmp, rho, n * sizeof(float), cudaMemcpyHostToDevice, c->stream),
                            "density upload")))
            return s;
        src = tmp;
    }
    const int b = aux_blocks((long long)n, c->sm_count);
    switch (c->prm.storage) {
    case LBM_FP32_DEV: rest_f32_kernel<kF32Dev><<<b, kAuxThreads, 0, c->stream>>>(src, c->mask, c->cur, c->g); break;
    case LBM_FP16_DEV: rest_f32_kernel<kF16Dev><<<b, kAuxThreads, 0, c->stream>>>(src, c->mask, c->cur, c->g); break;
    case LBM_BF16_DEV: rest_f32_kernel<kBF16Dev><<<b, kAuxThreads, 0, c->stream>>>(src, c->mask, c->cur, c->g); break;
    default: rest_f32_kernel<kF32><<<b, kAuxThreads, 0, c->stream>>>(src, c->mask, c->cur, c->g); break;
    }
    if ((s = check_launch(c, "rest state kernel launch"))) return s;
    if (!on_device) {
        solid_plane_kernel<<<b, kAuxThreads, 0, c->stream>>>(c->mask, c->nxt, 8, c->g);
        if ((s = check_launch(c, "sentinel kernel launch"))) return s;
    }
    c->has_field = true;
    return LBM_OK;
}

lbm_status lbm_get_field(lbm_ctx* c, int which, double* out, int on_device)
{
    lbm_status s = ready(c);
    if (s) return s;
    if (!out) return fail(c, LBM_EINVAL, "output is NULL");
    const size_t n = size_t(c->g.nx) * c->g.ny;
    if (which == LBM_RHO_U) {
        double* dst = on_device ? out : reinterpret_cast<double*>(c->nxt);
        if ((s = launch_step<kFields>(c, c->cur, nullptr, dst))) return s;
        if (!on_device) {
            if ((s = check_cuda(c, cudaMemcpyAsync(out, dst, 3 * n * sizeof(double), cudaMemcpyDeviceToHost,
                                                   c->stream), "field download")))
                return s;
            if ((s = check_cuda(c, cudaStreamSynchronize(c->stream), "field download sync"))) return s;
            if ((s = check_status(c))) return s;
            geometry_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(c->mask, c->nxt, c->nxt, c->g);
            if ((s = check_launch(c, "geometry kernel launch"))) return s;
        }
        return LBM_OK;
    }
    if (which == LBM_UX_PROFILE) {
        // fields into the spare buffer (3n doubles), the profile after them
        double* fld = reinterpret_cast<double*>(c->nxt);
        double* dst = on_device ? out : fld + 3 * n;
        if ((s = launch_step<kFields>(c, c->cur, nullptr, fld))) return s;
        const int blocks = c->g.ny < 4 * c->sm_count ? c->g.ny : 4 * c->sm_count;
        ux_profile_kernel<<<blocks, kAuxThreads, 0, c->stream>>>(fld, c->g, dst);
        if ((s = check_launch(c, "profile kernel launch"))) return s;
        if (!on_device) {
            if ((s = check_cuda(c, cudaMemcpyAsync(out, dst, size_t(c->g.ny) * sizeof(double), cudaMemcpyDeviceToHost,
                                                   c->stream), "profile download")))
                return s;
            if ((s = check_cuda(c, cudaStreamSynchronize(c->stream), "profile download sync"))) return s;
            if ((s = check_status(c))) return s;
        }
        // the spare buffer served as scratch: restore its solid sentinels
        geometry_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(c->mask, c->nxt, c->nxt, c->g);
        return check_launch(c, "geometry kernel launch");
    }
    if (which != LBM_POPS) return fail(c, LBM_EINVAL, "unknown field selector %d", which);
    const int nx = c->g.nx, ny = c->g.ny;
    const float* plain = nullptr;
    if ((s = storage_to_plain(c, &plain))) return s;
    if (on_device) {
        pops_out_kernel<<<aux_blocks(n, c->sm_count), kAuxThreads, 0, c->stream>>>(plain, c->mask, out, c->g, 0, ny);
        return check_launch(c, "population kernel launch");
    }
    const int rows_per = int(c->L.staging_bytes / (9 * size_t(nx) * sizeof(double)));
    for (int r0 = 0; r0 < ny; r0 += rows_per) {
        const int rows = (r0 + rows_per <= ny) ? rows_per : ny - r0;
        pops_out_kernel<<<aux_blocks(size_t(rows) * nx, c->sm_count), kAuxThreads, 0, c->stream>>>(plain, c->mask, c->staging, c->g, r0, rows);
        if ((s = check_launch(c, "population kernel launch"))) return s;
        for (int a = 0; a < 9; ++a) {
            if ((s = check_cuda(c, cudaMemcpyAsync(out + size_t(a) * n + size_t(r0) * nx,
                                                   c->staging + size_t(a) * rows * nx,
                                                   size_t(rows) * nx * sizeof(double), cudaMemcpyDeviceToHost,
                                                   c->stream), "population download")))
                return s;
        }
        if ((s = check_cuda(c, cudaStreamSynchronize(c->stream), "population download sync"))) return s;
    }
    return check_status(c);
}

lbm_status lbm_step(lbm_ctx* c, int64_t nsteps)
{
    lbm_status s = ready(c);
    if (s) return s;
    if (nsteps < 0) return fail(c, LBM_EINVAL, "nsteps must be >= 0");
    const int K = c->prm.obs_every;
    for (int64_t k = 0; k < nsteps; ++k) {
        // whole graphs of plain steps while no fused-observables step falls inside
        if (nsteps - k >= kGraphSteps && (K == 0 || (c->t % K != 0 && c->t / K == (c->t + kGraphSteps - 1) / K))) {
            cudaGraphExec_t exec;
            if ((s = step_graph(c, &exec))) return s;
            if ((s = check_cuda(c, cudaGraphLaunch(exec, c->stream), "graph launch"))) return s;
            c->t += kGraphSteps;
            k += kGraphSteps - 1;
            continue;
        }
        if (K > 0 && c->t % K == 0) {
            if ((s = launch_step<kStepObs>(c, c->cur, c->nxt, nullptr))) return s;
            if ((s = finalize(c, c->t, c->ring + (c->ring_count % kRing)))) return s;
            c->last_obs_t = c->t;
            ++c->ring_count;
        } else {
            if ((s = launch_step<kStep>(c, c->cur, c->nxt, nullptr))) return s;
        }
        float* tmp = c->cur;
        c->cur = c->nxt;
        c->nxt = tmp;
        ++c->t;
    }
    return LBM_OK;
}

static lbm_status read_record(lbm_ctx* c, const lbm_obs* rec, lbm_obs* out)
{
    lbm_status s;
    if ((s = check_cuda(c, cudaMemcpyAsync(out, rec, sizeof(lbm_obs), cudaMemcpyDeviceToHost, c->stream),
                        "observables download")))
        return s;
    if ((s = check_cuda(c, cudaStreamSynchronize(c->stream), "observables sync"))) return s;
    if ((s = check_status(c))) return s;
    if (out->nonfinite > 0) return fail(c, LBM_ENAN, "%lld non-finite fluid nodes at step %lld",
                                        (long long)out->nonfinite, (long long)out->step);
    return LBM_OK;
}

lbm_status lbm_selftest_timeout(lbm_ctx* c)
{
    if (!c) return LBM_EINVAL;
    wait_selftest_kernel<<<1, 32, 0, c->stream>>>(c->status);
    lbm_status s = check_launch(c, "self-test kernel launch");
    if (s) return s;
    if ((s = check_cuda(c, cudaStreamSynchronize(c->stream), "self-test sync"))) return s;
    return check_status(c);
}

lbm_status lbm_observables(lbm_ctx* c, lbm_obs* out)
{
    lbm_status s = ready(c);
    if (s) return s;
    if (!out) return fail(c, LBM_EINVAL, "output is NULL");
    lbm_obs* rec = c->ring + kRing;  // scratch slot after the fused ones
    if ((s = launch_step<kObs>(c, c->cur, nullptr, nullptr))) return s;
    if ((s = finalize(c, c->t, rec))) return s;
    return read_record(c, rec, out);
}

lbm_status lbm_run_to_steady(lbm_ctx* c, double rel_tol, int64_t check_every, int64_t max_steps,
                             lbm_obs* out)
{
    lbm_status s = ready(c);
    if (s) return s;
    if (!out) return fail(c, LBM_EINVAL, "output is NULL");
    if (check_every < 1 || !(rel_tol >= 0.0) || max_steps < 0)
        return fail(c, LBM_EINVAL, "need check_every >= 1, rel_tol >= 0, max_steps >= 0");
    bool have_prev = false;
    double q_prev = 0.0;
    for (int64_t done = 0; done < max_steps;) {
        const int64_t n = (max_steps - done < check_every) ? max_steps - done : check_every;
        if ((s = lbm_step(c, n))) return s;
        done += n;
        if ((s = lbm_observables(c, out))) return s;
        const double q = out->flux_Q;
        if (have_prev && n == check_every && std::fabs(q - q_prev) <= rel_tol * std::fabs(q)) return LBM_OK;
        q_prev = q;
        have_prev = true;
    }
    return fail(c, LBM_ENOTCONV, "flux not steady after %lld steps", (long long)max_steps);
}

lbm_status lbm_obs_latest(lbm_ctx* c, lbm_obs* out)
{
    lbm_status s = ready(c);
    if (s) return s;
    if (!out) return fail(c, LBM_EINVAL, "output is NULL");
    if (c->ring_count == 0) return fail(c, LBM_ESTATE, "no fused observables recorded yet (obs_every = %d)", c->prm.obs_every);
    return read_record(c, c->ring + ((c->ring_count - 1) % kRing), out);
}

lbm_status lbm_obs_latest_async(lbm_ctx* c, lbm_obs* out)
{
    lbm_status s = ready(c);
    if (s) return s;
    if (!out) return fail(c, LBM_EINVAL, "output is NULL");
    if (c->ring_count == 0) return fail(c, LBM_ESTATE, "no fused observables recorded yet (obs_every = %d)", c->prm.obs_every);
    return check_cuda(c, cudaMemcpyAsync(out, c->ring + ((c->ring_count - 1) % kRing), sizeof(lbm_obs),
                                         cudaMemcpyDeviceToHost, c->stream),
                      "observables download");
}

int64_t lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : "null context"; }

const char* lbm_status_string(int s)
{
    switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_EINVAL: return "LBM_EINVAL";
    case LBM_ENOMEM: return "LBM_ENOMEM";
    case LBM_ECUDA: return "LBM_ECUDA";
    case LBM_ENAN: return "LBM_ENAN";
    case LBM_ETIMEOUT: return "LBM_ETIMEOUT";
    case LBM_ESTATE: return "LBM_ESTATE";
    case LBM_ENOTCONV: return "LBM_ENOTCONV";
    default: return "unknown status";
    }
}

void lbm_destroy(lbm_ctx* c) { delete c; }

// Device address of g_noalloc_scratch in the current context, looked up once
// per context (normally once per device) with that context current. The cache
// is keyed on the context's unique id, so a context that replaces an earlier
// one on the same device (after cudaDeviceReset, say) gets its own lookup and
// never a stale address. The driver calls are reached through the runtime's
// entry-point query, so the library does not link the driver library.
// Returns nullptr on failure.
static double* noalloc_scratch(cudaError_t* err)
{
    using ctx_current_fn = int (*)(void**);
    using ctx_id_fn = int (*)(void*, unsigned long long*);
    constexpr int kMaxContexts = 64;
    static std::mutex mu;
    static ctx_current_fn ctx_current = nullptr;
    static ctx_id_fn ctx_id = nullptr;
    static unsigned long long ids[kMaxContexts] = {};
    static double* addr[kMaxContexts] = {};
    static int used = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!ctx_current || !ctx_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        *err = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (*err == cudaSuccess)
            *err = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (*err != cudaSuccess) return nullptr;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            *err = cudaErrorNotSupported;
            return nullptr;
        }
        ctx_current = reinterpret_cast<ctx_current_fn>(f1);
        ctx_id = reinterpret_cast<ctx_id_fn>(f2);
    }
    void* ctx = nullptr;
    void* ptr = nullptr;
    if (ctx_current(&ctx) != 0) {
        *err = cudaErrorDeviceUninitialized;
        return nullptr;
    }
    if (!ctx) {
        // no context current yet: the runtime's lookup makes the device's
        // primary context current, then the context is known
        *err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        if (ctx_current(&ctx) != 0 || !ctx) {
            *err = cudaErrorDeviceUninitialized;
            return nullptr;
        }
    }
    unsigned long long id = 0;
    if (ctx_id(ctx, &id) != 0) {
        *err = cudaErrorDeviceUninitialized;
        return nullptr;
    }
    for (int i = 0; i < used; ++i)
        if (ids[i] == id) return addr[i];
    if (!ptr) *err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    const int slot = used < kMaxContexts ? used++ : int(id % kMaxContexts);  // reuse a slot past 64 contexts
    ids[slot] = id;
    addr[slot] = static_cast<double*>(ptr);
    return addr[slot];
}

static thread_local char g_noalloc_err[256];

lbm_status lbm_observables_noalloc(const lbm_params* p, const double* d_pops, const uint8_t* d_solid,
                                   int64_t step, void* cuda_stream, lbm_obs* out)
{
    g_noalloc_err[0] = 0;
    const char* why = "";
    if (!params_valid(p, &why)) {
        snprintf(g_noalloc_err, sizeof(g_noalloc_err), "invalid parameters: %s", why);
        return LBM_EINVAL;
    }
    if (!d_pops || !d_solid || !out) {
        snprintf(g_noalloc_err, sizeof(g_noalloc_err), "null populations, mask or output");
        return LBM_EINVAL;
    }
    const long long n = (long long)p->nx * p->ny;
    if (n > kNoAllocMaxNodes) {
        snprintf(g_noalloc_err, sizeof(g_noalloc_err),
                 "domain of %lld nodes exceeds the allocation-free limit of %lld nodes", n, kNoAllocMaxNodes);
        return LBM_EINVAL;
    }
    cudaError_t e = cudaSuccess;
    double* scratch = noalloc_scratch(&e);
    if (!scratch) {
        cudaGetLastError();
        snprintf(g_noalloc_err, sizeof(g_noalloc_err), "scratch address: %s", cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    Geom g{};
    g.nx = p->nx;
    g.ny = p->ny;
    g.pitch = p->nx;
    g.plane = p->ny * p->nx;
    g.tile_rows = 1;
    const int ctas = int((n + kNoAllocNodesPerCta - 1) / kNoAllocNodesPerCta);
    lbm_obs* rec = reinterpret_cast<lbm_obs*>(scratch + kNoAllocSlots * kPartialStride);
    observe_dense_kernel<<<ctas, kAuxThreads, 0, st>>>(d_pops, d_solid, g, make_phys(*p), scratch);
    finalize_obs_kernel<<<1, kAuxThreads, 0, st>>>(scratch, ctas, 1.0 / p->nx, (long long)step, rec);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, rec, sizeof(lbm_obs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(g_noalloc_err, sizeof(g_noalloc_err), "observables: %s", cudaGetErrorString(e));
        return LBM_ECUDA;
    }
    if (out->nonfinite > 0) {
        snprintf(g_noalloc_err, sizeof(g_noalloc_err), "%lld non-finite fluid nodes", (long long)out->nonfinite);
        return LBM_ENAN;
    }
    return LBM_OK;
}

const char* lbm_noalloc_last_error(void) { return g_noalloc_err; }

}  // extern "C"


// ===========================================================================
// Batches: many domains of different sizes stepped by one launch per step.

struct lbm_batch {
    int count = 0;
    int storage = 0;
    std::vector<lbm_ctx*> ctx;
    std::vector<unsigned char> active;   // host flags
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int tile_rows = 0;                   // 0 = each domain's own choice
    int ctas_per_sm = 3;                 // resident CTAs per SM of the persistent grid (1..max_ctas)
    int max_ctas = 3;                    // CTAs of the step kernel instance that fit on one SM
    bool tau1 = true;                    // every domain relaxes with tau = 1 (the tau = 1 kernel instance)
    bool pair = true;                    // the 32-bit forms' pair layout (false: one node per thread)
    // device tables (in the batch's own workspace region)
    DomainDev* d_dom = nullptr;
    int4* d_tiles = nullptr;
    int* d_status = nullptr;
    lbm_obs* d_rec = nullptr;
    double** d_partials = nullptr;
    int* d_nctas = nullptr;
    double* d_inv_nx = nullptr;
    long long* d_step = nullptr;
    unsigned char* d_want = nullptr;
    int max_tiles = 0;
    // host mirrors
    std::vector<DomainDev> h_dom;
    std::vector<int4> h_tiles;
    int ntiles = 0;
    bool tiles_dirty = true;
    int tiles_for_all = -1;              // 1 if h_tiles covers every domain
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_ntiles = -1, graph_grid = -1;
    char err[512] = {0};
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const char* fmt, ...)
{
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

lbm_status bcheck(lbm_batch* b, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return LBM_OK;
    return bfail(b, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct BatchLayout {
    std::vector<size_t> off;  // per-domain workspace offsets
    size_t off_dom, off_tiles, off_status, off_rec, off_ptrs, off_nctas, off_invnx, off_step, off_want, total;
    int max_tiles;
};

bool batch_layout(const lbm_params* p, int count, BatchLayout* L, const char** why)
{
    if (!p || count < 1) { *why = "need at least one domain"; return false; }
    size_t o = 0;
    L->off.resize(count);
    L->max_tiles = 0;
    for (int i = 0; i < count; ++i) {
        if (!params_valid(&p[i], why)) return false;
        if (p[i].storage != p[0].storage) { *why = "all domains of a batch share one storage form"; return false; }
        L->off[i] = o;
        o = align_up(o + layout_of(&p[i]).total, 256);
        L->max_tiles += ctas_x(p[i].nx, p[i].storage) * ((p[i].ny + 3) / 4);
    }
    L->off_dom = o; o = align_up(o + count * sizeof(DomainDev), 256);
    L->off_tiles = o; o = align_up(o + size_t(L->max_tiles) * sizeof(int4), 256);
    L->off_status = o; o = align_up(o + sizeof(int), 256);
    L->off_rec = o; o = align_up(o + count * sizeof(lbm_obs), 256);
    L->off_ptrs = o; o = align_up(o + count * sizeof(double*), 256);
    L->off_nctas = o; o = align_up(o + count * sizeof(int), 256);
    L->off_invnx = o; o = align_up(o + count * sizeof(double), 256);
    L->off_step = o; o = align_up(o + count * sizeof(long long), 256);
    L->off_want = o; o = align_up(o + count, 256);
    L->total = o;
    return true;
}

// Segment height of a domain's tiles: the requested height, evened out so
// that the ceil(ny / height) segments differ by at most one row (a 40-row
// channel at height 32 gets two segments of 20 rows, not 32 + 8: a short
// last segment pays the pipeline start and the 4 re-staged halo rows for
// few rows). The segment count is unchanged.
// Segment height of a domain of ny rows for a wanted height: the same
// segment count with heights that differ by at most one row.
int even_rows(int ny, int want)
{
    const int nseg = (ny + want - 1) / want;
    const int even = (ny + nseg - 1) / nseg;
    return even >= 4 ? even : want;
}

int domain_tile_rows(const lbm_batch* b, const lbm_ctx* c)
{
    return even_rows(c->g.ny, b->tile_rows ? b->tile_rows : c->g.tile_rows);
}

// Tiles of the active domains at the wanted tile height `rows`.
long long active_tiles(const lbm_batch* b, int rows)
{
    long long n = 0;
    for (int d = 0; d < b->count; ++d) {
        if (!b->active[d]) continue;
        const lbm_ctx* c = b->ctx[d];
        const int r = even_rows(c->g.ny, rows);
        n += (long long)ctas_x(c->g.nx, c->prm.storage) * ((c->g.ny + r - 1) / r);
    }
    return n;
}

// Tile list of the active domains (or of all domains), largest domains first
// so that the strided walk of the persistent grid ends evenly.
void build_tiles(lbm_batch* b, bool all)
{
    std::vector<int> order;
    for (int d = 0; d < b->count; ++d)
        if (all || b->active[d]) order.push_back(d);
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        return (long long)b->ctx[x]->g.nx * b->ctx[x]->g.ny > (long long)b->ctx[y]->g.nx * b->ctx[y]->g.ny;
    });
    b->h_tiles.clear();
    for (int d : order) {
        const lbm_ctx* c = b->ctx[d];
        const int rows = domain_tile_rows(b, c);
        const int tx = ctas_x(c->g.nx, c->prm.storage), ty = (c->g.ny + rows - 1) / rows;
        for (int by = 0; by < ty; ++by)
            for (int bx = 0; bx < tx; ++bx) b->h_tiles.push_back(make_int4(d, bx, by, by * tx + bx));
    }
    b->ntiles = int(b->h_tiles.size());
    b->tiles_for_all = all ? 1 : 0;
}

lbm_status upload_tables(lbm_batch* b, bool all)
{
    for (int d = 0; d < b->count; ++d) {
        lbm_ctx* c = b->ctx[d];
        DomainDev& dd = b->h_dom[d];
        dd.g = c->g;
        dd.g.tile_rows = domain_tile_rows(b, c);
        dd.p = c->ph;
        dd.buf[0] = c->cur;
        dd.buf[1] = c->nxt;
        dd.partials = c->partials;
    }
    lbm_status s = bcheck(b, cudaMemcpyAsync(b->d_dom, b->h_dom.data(), b->count * sizeof(DomainDev),
                                             cudaMemcpyHostToDevice, b->stream), "domain table upload");
    if (s) return s;
    if (b->tiles_dirty || b->tiles_for_all != (all ? 1 : 0)) {
        build_tiles(b, all);
        if (b->ntiles > 0 &&
            (s = bcheck(b, cudaMemcpyAsync(b->d_tiles, b->h_tiles.data(), b->ntiles * sizeof(int4),
                                           cudaMemcpyHostToDevice, b->stream), "tile list upload")))
            return s;
        b->tiles_dirty = false;  // tiles_for_all records which list is on the device
    }
    // pageable H2D copies return once the host buffers are consumed; the
    // kernels that read the tables follow on the same stream
    return LBM_OK;
}

// t1: every domain of the batch relaxes with tau = 1
template <int ST, bool PAIR>
const void* batch_kernel_layout(int mode, bool t1)
{
    if (mode == kObs) return reinterpret_cast<const void*>(&batch_step_kernel<kObs, ST, true, PAIR>);
    return t1 ? reinterpret_cast<const void*>(&batch_step_kernel<kStep, ST, true, PAIR>)
              : reinterpret_cast<const void*>(&batch_step_kernel<kStep, ST, false, PAIR>);
}

template <int ST>
const void* batch_kernel_ptr(int mode, bool t1, bool pair)
{
    if constexpr (is16(ST))
        return batch_kernel_layout<ST, false>(mode, t1);
    else
        return pair ? batch_kernel_layout<ST, true>(mode, t1) : batch_kernel_layout<ST, false>(mode, t1);
}

const void* batch_kernel(int storage, int mode, bool t1, bool pair)
{
    switch (storage) {
    case LBM_FP32_DEV: return batch_kernel_ptr<kF32Dev>(mode, t1, pair);
    case LBM_FP16_DEV: return batch_kernel_ptr<kF16Dev>(mode, t1, pair);
    case LBM_BF16_DEV: return batch_kernel_ptr<kBF16Dev>(mode, t1, pair);
    default: return batch_kernel_ptr<kF32>(mode, t1, pair);
    }
}

// the batch kernel's dynamic shared memory: the single-domain step's
size_t batch_smem(int storage, bool pair) { return step_smem(storage, pair); }

int batch_grid(const lbm_batch* b)
{
    const int slots = b->ctas_per_sm * b->sm_count;
    return b->ntiles < slots ? b->ntiles : slots;
}

lbm_status launch_batch(lbm_batch* b, int mode, int parity)
{
    if (b->ntiles == 0) return LBM_OK;
    int nt = b->ntiles;
    void* args[] = {&b->d_dom, &b->d_tiles, &nt, &parity, &b->d_status};
    return bcheck(b, cudaLaunchKernel(batch_kernel(b->storage, mode, b->tau1, b->pair), dim3(batch_grid(b)),
                                      dim3(step_threads(b->storage, b->pair)), args,
                                      batch_smem(b->storage, b->pair), b->stream),
                  "batch step launch");
}

// Two steps (parity 0 then 1) as one explicitly built graph; rebuilt when
// the tile list or grid changes.
lbm_status batch_graph(lbm_batch* b)
{
    const int grid = batch_grid(b);
    if (b->exec && b->graph_ntiles == b->ntiles && b->graph_grid == grid) return LBM_OK;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    lbm_status s = bcheck(b, cudaGraphCreate(&b->graph, 0), "graph create");
    if (s) return s;
    static int parities[2] = {0, 1};
    int nt = b->ntiles;
    cudaGraphNode_t prev = nullptr;
    for (int k = 0; k < 2; ++k) {
        void* args[] = {&b->d_dom, &b->d_tiles, &nt, &parities[k], &b->d_status};
        cudaKernelNodeParams kp{};
        kp.func = const_cast<void*>(batch_kernel(b->storage, kStep, b->tau1, b->pair));
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(step_threads(b->storage, b->pair));
        kp.sharedMemBytes = unsigned(batch_smem(b->storage, b->pair));
        kp.kernelParams = args;
        cudaGraphNode_t node;
        if ((s = bcheck(b, cudaGraphAddKernelNode(&node, b->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp),
                        "graph node")))
            return s;
        prev = node;
    }
    if ((s = bcheck(b, cudaGraphInstantiate(&b->exec, b->graph, 0), "graph instantiate"))) return s;
    b->graph_ntiles = b->ntiles;
    b->graph_grid = grid;
    return LBM_OK;
}

lbm_status batch_ready(lbm_batch* b)
{
    if (!b) return LBM_EINVAL;
    for (int d = 0; d < b->count; ++d)
        if (b->active[d] && (!b->ctx[d]->has_geometry || !b->ctx[d]->has_field))
            return bfail(b, LBM_ESTATE, "domain %d has no geometry or field yet", d);
    return LBM_OK;
}

lbm_status batch_check_status(lbm_batch* b)
{
    int flag = 0;
    lbm_status s = bcheck(b, cudaMemcpy(&flag, b->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status download");
    if (s) return s;
    if (flag) {
        cudaMemset(b->d_status, 0, sizeof(int));
        return bfail(b, LBM_ETIMEOUT, "a bounded device-side wait gave up (flag %d)", flag);
    }
    return LBM_OK;
}

// Observables of the domains with want[d] into rec (device) and out (host);
// the pass covers every domain (all) or only the active ones.
lbm_status batch_observe(lbm_batch* b, const std::vector<unsigned char>& want, lbm_obs* out, bool all)
{
    lbm_status s = upload_tables(b, all);
    if (s) return s;
    if ((s = launch_batch(b, kObs, 0))) return s;
    std::vector<double*> parts(b->count);
    std::vector<int> nct(b->count);
    std::vector<double> invnx(b->count);
    std::vector<long long> steps(b->count);
    for (int d = 0; d < b->count; ++d) {
        const lbm_ctx* c = b->ctx[d];
        const int rows = domain_tile_rows(b, c);
        parts[d] = c->partials;
        nct[d] = ctas_x(c->g.nx, c->prm.storage) * ((c->g.ny + rows - 1) / rows);
        invnx[d] = 1.0 / c->g.nx;
        steps[d] = c->t;
    }
    cudaStream_t st = b->stream;
    if ((s = bcheck(b, cudaMemcpyAsync(b->d_partials, parts.data(), b->count * sizeof(double*), cudaMemcpyHostToDevice, st), "upload")) ||
        (s = bcheck(b, cudaMemcpyAsync(b->d_nctas, nct.data(), b->count * sizeof(int), cudaMemcpyHostToDevice, st), "upload")) ||
        (s = bcheck(b, cudaMemcpyAsync(b->d_inv_nx, invnx.data(), b->count * sizeof(double), cudaMemcpyHostToDevice, st), "upload")) ||
        (s = bcheck(b, cudaMemcpyAsync(b->d_step, steps.data(), b->count * sizeof(long long), cudaMemcpyHostToDevice, st), "upload")) ||
        (s = bcheck(b, cudaMemcpyAsync(b->d_want, want.data(), b->count, cudaMemcpyHostToDevice, st), "upload")))
        return s;
    finalize_batch_kernel<<<b->count, kAuxThreads, 0, st>>>(b->d_partials, b->d_nctas, b->d_inv_nx, b->d_step,
                                                            b->d_want, b->d_rec);
    if ((s = bcheck(b, cudaGetLastError(), "finalize launch"))) return s;
    if ((s = bcheck(b, cudaMemcpyAsync(out, b->d_rec, b->count * sizeof(lbm_obs), cudaMemcpyDeviceToHost, st),
                    "observables download")))
        return s;
    if ((s = bcheck(b, cudaStreamSynchronize(st), "observables sync"))) return s;
    return batch_check_status(b);
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(const lbm_params* params, int32_t count)
{
    BatchLayout L;
    const char* why;
    if (!batch_layout(params, count, &L, &why)) return 0;
    return L.total;
}

lbm_status lbm_batch_create(const lbm_params* params, int32_t count, void* d_workspace, size_t bytes,
                            void* cuda_stream, lbm_batch** out)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    BatchLayout L;
    const char* why = "";
    if (!batch_layout(params, count, &L, &why)) return LBM_EINVAL;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u)) return LBM_EINVAL;
    if (bytes < L.total) return LBM_ENOMEM;
    lbm_batch* b = new (std::nothrow) lbm_batch;
    if (!b) return LBM_ENOMEM;
    unsigned char* ws = static_cast<unsigned char*>(d_workspace);
    b->count = count;
    b->storage = params[0].storage;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->ctx.assign(count, nullptr);
    b->active.assign(count, 1);
    b->h_dom.resize(count);
    for (int d = 0; d < count; ++d) {
        const size_t need = layout_of(&params[d]).total;
        lbm_status s = lbm_create(&params[d], ws + L.off[d], need, cuda_stream, &b->ctx[d]);
        if (s) {
            for (int e = 0; e < d; ++e) lbm_destroy(b->ctx[e]);
            delete b;
            return s;
        }
    }
    b->sm_count = b->ctx[0]->sm_count;
    b->d_dom = reinterpret_cast<DomainDev*>(ws + L.off_dom);
    b->d_tiles = reinterpret_cast<int4*>(ws + L.off_tiles);
    b->d_status = reinterpret_cast<int*>(ws + L.off_status);
    b->d_rec = reinterpret_cast<lbm_obs*>(ws + L.off_rec);
    b->d_partials = reinterpret_cast<double**>(ws + L.off_ptrs);
    b->d_nctas = reinterpret_cast<int*>(ws + L.off_nctas);
    b->d_inv_nx = reinterpret_cast<double*>(ws + L.off_invnx);
    b->d_step = reinterpret_cast<long long*>(ws + L.off_step);
    b->d_want = ws + L.off_want;
    b->max_tiles = L.max_tiles;
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < count; ++d)
        if (b->ctx[d]->ph.tau != 1.f) b->tau1 = false;
    // Thread layout (32-bit forms), by the rule of a single domain applied to
    // the whole batch: pairs unless all domains together give the GPU no
    // more than 3 CTAs per SM at 4-row segments; the first domain's layout
    // field may force either.
    {
        long long tiles4 = 0;
        for (int d = 0; d < count; ++d)
            tiles4 += (long long)ctas_x(params[d].nx, params[d].storage) * ((params[d].ny + 3) / 4);
        const int lay = params[0].layout;
        b->pair = !is16(b->storage) &&
                  (lay == LBM_LAYOUT_PAIRS || (lay == LBM_LAYOUT_AUTO && tiles4 > 3LL * b->sm_count));
    }
    for (int st = 0; st < 4 && e == cudaSuccess; ++st) {
        for (int pr = 0; pr < 2 && e == cudaSuccess; ++pr) {
            for (int t1 = 0; t1 < 2 && e == cudaSuccess; ++t1)
                e = cudaFuncSetAttribute(batch_kernel(st, kStep, t1 != 0, pr != 0),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(batch_smem(st, pr != 0)));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(batch_kernel(st, kObs, true, pr != 0),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(batch_smem(st, pr != 0)));
        }
    }
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &b->max_ctas, batch_kernel(b->storage, kStep, b->tau1, b->pair), step_threads(b->storage, b->pair),
            batch_smem(b->storage, b->pair));
    if (e == cudaSuccess && b->max_ctas < 1) e = cudaErrorInvalidConfiguration;
    b->ctas_per_sm = b->max_ctas;
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (int d = 0; d < count; ++d) lbm_destroy(b->ctx[d]);
        delete b;
        return LBM_ECUDA;
    }
    *out = b;
    return LBM_OK;
}

lbm_ctx* lbm_batch_domain(lbm_batch* b, int32_t i)
{
    if (!b || i < 0 || i >= b->count) return nullptr;
    return b->ctx[i];
}

lbm_status lbm_batch_set_active(lbm_batch* b, const uint8_t* active)
{
    if (!b || !active) return LBM_EINVAL;
    for (int d = 0; d < b->count; ++d) b->active[d] = active[d] ? 1 : 0;
    b->tiles_dirty = true;
    return LBM_OK;
}

lbm_status lbm_batch_set_tile_rows(lbm_batch* b, int32_t rows)
{
    if (!b) return LBM_EINVAL;
    if (rows != 0 && rows < 4) return bfail(b, LBM_EINVAL, "tile rows must be 0 or >= 4");
    b->tile_rows = rows;
    b->tiles_dirty = true;
    return LBM_OK;
}

int32_t lbm_batch_tile_rows(const lbm_batch* b) { return b ? b->tile_rows : -1; }

lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps)
{
    lbm_status s = batch_ready(b);
    if (s) return s;
    if (nsteps < 0) return bfail(b, LBM_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return LBM_OK;
    if ((s = upload_tables(b, false))) return s;
    if (b->ntiles == 0) return LBM_OK;
    if ((s = batch_graph(b))) return s;
    for (int64_t k = 0; k + 1 < nsteps; k += 2)
        if ((s = bcheck(b, cudaGraphLaunch(b->exec, b->stream), "graph launch"))) return s;
    if (nsteps & 1)
        if ((s = launch_batch(b, kStep, 0))) return s;
    for (int d = 0; d < b->count; ++d) {
        if (!b->active[d]) continue;
        lbm_ctx* c = b->ctx[d];
        c->t += nsteps;
        if (nsteps & 1) {
            float* tmp = c->cur;
            c->cur = c->nxt;
            c->nxt = tmp;
        }
    }
    return LBM_OK;
}

lbm_status lbm_batch_observables(lbm_batch* b, lbm_obs* out)
{
    if (!b || !out) return LBM_EINVAL;
    for (int d = 0; d < b->count; ++d)
        if (!b->ctx[d]->has_geometry || !b->ctx[d]->has_field)
            return bfail(b, LBM_ESTATE, "domain %d has no geometry or field yet", d);
    std::vector<unsigned char> want(b->count, 1);
    lbm_status s = batch_observe(b, want, out, true);
    if (s) return s;
    for (int d = 0; d < b->count; ++d)
        if (out[d].nonfinite > 0) return bfail(b, LBM_ENAN, "domain %d has %lld non-finite nodes", d, (long long)out[d].nonfinite);
    return LBM_OK;
}

lbm_status lbm_batch_run_to_steady(lbm_batch* b, double rel_tol, int64_t check_every, int64_t max_steps,
                                   int64_t* steps_to_steady, lbm_obs* out)
{
    lbm_status s = batch_ready(b);
    if (s) return s;
    if (!steps_to_steady || !out || check_every < 1 || !(rel_tol >= 0.0) || max_steps < 0)
        return bfail(b, LBM_EINVAL, "bad arguments");
    std::vector<double> q_prev(b->count, 0.0);
    std::vector<unsigned char> have_prev(b->count, 0);
    std::vector<unsigned char> start_active = b->active;
    for (int d = 0; d < b->count; ++d) steps_to_steady[d] = -1;
    std::vector<lbm_obs> rec(b->count);
    int first_nan = -1;
    // As domains converge and leave, the tile list shrinks and the persistent
    // grid's SMs fall idle; a lower tile height gives the remaining domains
    // more tiles. Keep at least two waves (the arithmetic does not depend on
    // the tiling), down to 8-row segments; the caller's height is restored.
    const int32_t rows_start = b->tile_rows;
    const long long slots = (long long)b->ctas_per_sm * b->sm_count;
    auto retile = [&]() {
        if (b->tile_rows <= 0) return;  // each domain's own height (already sized for it alone)
        int r = b->tile_rows;
        // down to 4 rows: with fewer than two waves of tiles a step is bound by
        // the latency of one tile's row pipeline, not by the re-staged halo
        // rows (measured on 32 small channels: 1.04 s to steady at 8 rows,
        // 0.82 s at 4)
        while (r > 4 && active_tiles(b, r) < 2 * slots) r = r / 2 < 4 ? 4 : r / 2;
        if (r != b->tile_rows) {
            b->tile_rows = r;
            b->tiles_dirty = true;
        }
    };
    retile();
    for (int64_t done = 0; done < max_steps;) {
        bool any = false;
        for (int d = 0; d < b->count; ++d) any = any || b->active[d];
        if (!any) break;
        const int64_t n = (max_steps - done < check_every) ? max_steps - done : check_every;
        if ((s = lbm_batch_step(b, n))) return s;
        done += n;
        std::vector<unsigned char> want = b->active;
        if ((s = batch_observe(b, want, rec.data(), false))) return s;
        bool changed = false;
        for (int d = 0; d < b->count; ++d) {
            if (!want[d]) continue;
            out[d] = rec[d];
            if (rec[d].nonfinite > 0) {
                // drop it; the sweep goes on with the others
                steps_to_steady[d] = -2;
                b->active[d] = 0;
                changed = true;
                if (first_nan < 0) first_nan = d;
                continue;
            }
            const double q = rec[d].flux_Q;
            if (have_prev[d] && n == check_every && std::fabs(q - q_prev[d]) <= rel_tol * std::fabs(q)) {
                steps_to_steady[d] = b->ctx[d]->t;
                b->active[d] = 0;
                changed = true;
            }
            q_prev[d] = q;
            have_prev[d] = 1;
        }
        if (changed) {
            b->tiles_dirty = true;
            retile();
        }
    }
    // restore the caller's active set and tile height
    b->active = start_active;
    b->tile_rows = rows_start;
    b->tiles_dirty = true;
    if (first_nan >= 0) return bfail(b, LBM_ENAN, "domain %d became non-finite", first_nan);
    for (int d = 0; d < b->count; ++d)
        if (start_active[d] && steps_to_steady[d] < 0) return bfail(b, LBM_ENOTCONV, "domain %d not steady", d);
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, const int32_t* candidates, int32_t n, int32_t steps, int32_t* chosen,
                              double* ms_per_step)
{
    lbm_status s = batch_ready(b);
    if (s) return s;
    if (!candidates || n < 1 || steps < 1 || !chosen) return bfail(b, LBM_EINVAL, "bad arguments");
    cudaEvent_t e0, e1;
    if ((s = bcheck(b, cudaEventCreate(&e0), "event")) || (s = bcheck(b, cudaEventCreate(&e1), "event"))) return s;
    double best = 1e300;
    int32_t pick = b->tile_rows;
    for (int i = 0; i < n; ++i) {
        if ((s = lbm_batch_set_tile_rows(b, candidates[i]))) break;
        if ((s = lbm_batch_step(b, 2))) break;  // warm-up (and graph build)
        cudaEventRecord(e0, b->stream);
        if ((s = lbm_batch_step(b, steps))) break;
        cudaEventRecord(e1, b->stream);
        if ((s = bcheck(b, cudaEventSynchronize(e1), "event sync"))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = double(ms) / steps;
        if (ms_per_step) ms_per_step[i] = per;
        if (per < best) {
            best = per;
            pick = candidates[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    *chosen = pick;
    if ((s = lbm_batch_set_tile_rows(b, pick))) return s;
    return batch_check_status(b);
}

lbm_status lbm_batch_set_ctas_per_sm(lbm_batch* b, int32_t ctas)
{
    if (!b) return LBM_EINVAL;
    if (ctas < 1 || ctas > b->max_ctas)
        return bfail(b, LBM_EINVAL, "ctas_per_sm must be 1 .. %d for this batch", b->max_ctas);
    b->ctas_per_sm = ctas;  // the graph is rebuilt when the grid changes
    return LBM_OK;
}

int32_t lbm_batch_ctas_per_sm(const lbm_batch* b) { return b ? b->ctas_per_sm : -1; }

lbm_status lbm_batch_autotune_grid(lbm_batch* b, const int32_t* rows, int32_t nrows, const int32_t* ctas,
                                   int32_t nctas, int32_t steps, int32_t* chosen_rows, int32_t* chosen_ctas,
                                   double* ms_per_step)
{
    lbm_status s = batch_ready(b);
    if (s) return s;
    if (!rows || nrows < 1 || !ctas || nctas < 1 || steps < 1 || !chosen_rows || !chosen_ctas)
        return bfail(b, LBM_EINVAL, "bad arguments");
    for (int j = 0; j < nctas; ++j)
        if (ctas[j] < 1 || ctas[j] > b->max_ctas)
            return bfail(b, LBM_EINVAL, "ctas_per_sm must be 1 .. %d for this batch", b->max_ctas);
    double best = 1e300;
    int32_t best_rows = b->tile_rows, best_ctas = b->ctas_per_sm;
    std::vector<double> ms(nrows);
    for (int j = 0; j < nctas; ++j) {
        b->ctas_per_sm = ctas[j];
        int32_t r = 0;
        if ((s = lbm_batch_autotune(b, rows, nrows, steps, &r, ms.data()))) return s;
        for (int i = 0; i < nrows; ++i) {
            if (ms_per_step) ms_per_step[j * nrows + i] = ms[i];
            if (ms[i] < best) {
                best = ms[i];
                best_rows = rows[i];
                best_ctas = ctas[j];
            }
        }
    }
    b->ctas_per_sm = best_ctas;
    *chosen_rows = best_rows;
    *chosen_ctas = best_ctas;
    return lbm_batch_set_tile_rows(b, best_rows);
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : "null batch"; }

void lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (lbm_ctx* c : b->ctx) lbm_destroy(c);
    delete b;
}

}  // extern "C"
