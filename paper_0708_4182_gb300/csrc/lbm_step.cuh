// lbm_step.cuh -- the fused D2Q9 Shan-Chen electrowetting time step (sm_103a).
//
// One launch = one time step of the update of Li, Li, Chen & Fang
// (arXiv:0708.4182): streaming (left side of Eq. 1, pull form with half-way
// bounce-back), moments (Eq. 2), pseudopotential psi, the forces of Eq. 5
// and Eq. 6, the electric force on the conductive wall layer (Eq. 9 and the
// critical-density paragraph), the body force, the velocity shift (Eq. 10)
// and BGK collision towards Eq. 3.
//
// State: post-collision populations f* in SoA planes fin[a][y][x] (FP32,
// row pitch `pitch` floats). Solid nodes hold the bit pattern kSolidBits in
// every plane; a pull that meets it knows the source node is solid, so the
// wall mask is never read on the hot path (0 extra bytes per node).
//
// Work decomposition (HBM-bound stencil, no tensor cores):
//  - a CTA of kThreads threads owns a strip of kThreads-2 columns plus one
//    halo column on each side, and marches up a segment of tile_rows rows;
//  - per row every thread pulls its node's 9 populations (coalesced along x),
//    forms rho and psi, and writes psi into a 4-row ring in shared memory;
//  - after one __syncthreads the interior threads compute the 8-neighbour
//    forces of the row below from the ring, collide, and store f*;
//  - the ring makes every DRAM element be read once per step except the 2
//    halo columns per strip and 2 halo rows per segment (L2 hits).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr uint32_t kSolidBits = 0xFFBADA55u;  // a NaN payload arithmetic never produces
constexpr int kThreads = 256;
constexpr int kInner = kThreads - 2;
constexpr int kPartialStride = 8;              // doubles per CTA in the partials array

struct Geom {
    int nx, ny;
    int pitch;  // floats per row
    int plane;  // ny * pitch
    int tile_rows;
};

struct Phys {
    float tau, inv_tau;
    float rho0, inv_rho0;
    float rho_c, f_elec;
    float bfx, bfy;
    float g_axis, g_diag;  // G_a of Eq. 4 on |e| = 1 and |e| = sqrt 2 links
    float w_axis, w_diag;  // W_a of Eq. 6
};

enum Mode { kStep = 0, kStepObs = 1, kObs = 2, kFields = 3 };

struct Pulled {
    float f[9];
    float rho, jx, jy;
    uint32_t sb;  // bit a set <=> the pull source x - e_a is solid
    bool solid;
};

__device__ __forceinline__ bool is_solid(float v) { return __float_as_uint(v) == kSolidBits; }

// Pull the 9 post-streaming populations of node (x, y) from the post-collision
// planes: f_a(x) = f*_a(x - e_a), or f*_opp(a)(x) when x - e_a is solid.
__device__ __forceinline__ void pull_node(const float* __restrict__ fin, const Geom& g, int x,
                                          int xm, int xp, int y, Pulled& n)
{
    const int ym = (y == 0) ? g.ny - 1 : y - 1;
    const int yp = (y == g.ny - 1) ? 0 : y + 1;
    const int P = g.plane;
    const int rc = y * g.pitch, rm = ym * g.pitch, rp = yp * g.pitch;
    const float v0 = __ldg(fin + rc + x);
    n.solid = is_solid(v0);
    if (n.solid) {
        n.rho = n.jx = n.jy = 0.f;
        n.sb = 0;
        return;
    }
    float v[9];
    v[0] = v0;
    v[1] = __ldg(fin + 1 * P + rc + xm);  // e1 = ( 1, 0): source (x-1, y)
    v[2] = __ldg(fin + 2 * P + rm + x);   // e2 = ( 0, 1): source (x, y-1)
    v[3] = __ldg(fin + 3 * P + rc + xp);  // e3 = (-1, 0): source (x+1, y)
    v[4] = __ldg(fin + 4 * P + rp + x);   // e4 = ( 0,-1): source (x, y+1)
    v[5] = __ldg(fin + 5 * P + rm + xm);  // e5 = ( 1, 1): source (x-1, y-1)
    v[6] = __ldg(fin + 6 * P + rm + xp);  // e6 = (-1, 1): source (x+1, y-1)
    v[7] = __ldg(fin + 7 * P + rp + xp);  // e7 = (-1,-1): source (x+1, y+1)
    v[8] = __ldg(fin + 8 * P + rp + xm);  // e8 = ( 1,-1): source (x-1, y+1)
    constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    uint32_t sb = 0;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        if (is_solid(v[a])) {
            sb |= 1u << a;
            v[a] = __ldg(fin + opp[a] * P + rc + x);  // half-way bounce-back
        }
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) n.f[a] = v[a];
    n.sb = sb;
    n.rho = ((v[0] + (v[1] + v[3])) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
    n.jx = (v[1] - v[3]) + (v[5] - v[7]) + (v[8] - v[6]);
    n.jy = (v[2] - v[4]) + (v[5] - v[7]) + (v[6] - v[8]);
}

__device__ __forceinline__ float pseudopotential(const Phys& p, const Pulled& n)
{
    // psi = rho0 (1 - exp(-rho/rho0)), via expm1 to keep small-rho accuracy
    return n.solid ? 0.f : -p.rho0 * expm1f(-n.rho * p.inv_rho0);
}

// Error-free accumulation s + c of FP32 terms (Knuth's TwoSum).
struct Acc {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float t = s + v;
        const float bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <int MODE>
__global__ void __launch_bounds__(kThreads)
    step_kernel(const float* __restrict__ fin, float* __restrict__ fout, Geom g, Phys p,
                double* __restrict__ partials, double* __restrict__ fields)
{
    __shared__ float psi_ring[4][kThreads];

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * kInner;
    const int nint = min(kInner, g.nx - x0);
    const bool active = t <= nint + 1;
    const bool interior = t >= 1 && t <= nint;
    int x = x0 - 1 + t;
    x = (x < 0) ? x + g.nx : (x >= g.nx ? x - g.nx : x);
    if (!active) x = 0;
    const int xm = (x == 0) ? g.nx - 1 : x - 1;
    const int xp = (x == g.nx - 1) ? 0 : x + 1;

    const int y0 = blockIdx.y * g.tile_rows;
    const int y1 = min(y0 + g.tile_rows, g.ny);
    auto wrap_y = [&](int y) { return y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y); };

    Pulled cur, nxt;
    if (active) {
        pull_node(fin, g, x, xm, xp, wrap_y(y0 - 1), nxt);
        psi_ring[(y0 + 3) & 3][t] = pseudopotential(p, nxt);
        pull_node(fin, g, x, xm, xp, y0, cur);
        psi_ring[y0 & 3][t] = pseudopotential(p, cur);
    }

    Acc a_mass, a_q, a_px, a_py;
    float umax2 = 0.f, rmin = __int_as_float(0x7f800000);  // +inf
    unsigned bad = 0;

    for (int r = y0; r < y1; ++r) {
        if (active) {
            pull_node(fin, g, x, xm, xp, wrap_y(r + 1), nxt);
            psi_ring[(r + 1) & 3][t] = pseudopotential(p, nxt);
        }
        __syncthreads();
        if (interior) {
            if (!cur.solid) {
                const float* pm = psi_ring[(r + 3) & 3];  // row r-1
                const float* pc = psi_ring[r & 3];
                const float* pp = psi_ring[(r + 1) & 3];  // row r+1
                const float psi = pc[t];
                // Eq. 5: sum_a G_a psi(x+e_a) e_a, axis and diagonal links
                const float sgx = p.g_axis * (pc[t + 1] - pc[t - 1]) +
                                  p.g_diag * ((pp[t + 1] - pp[t - 1]) + (pm[t + 1] - pm[t - 1]));
                const float sgy = p.g_axis * (pp[t] - pm[t]) +
                                  p.g_diag * ((pp[t + 1] + pp[t - 1]) - (pm[t + 1] + pm[t - 1]));
                // S(x + e_a) = solid flag of the pull source of the opposite direction
                const uint32_t sb = cur.sb;
                const float sE = (sb >> 3) & 1, sW = (sb >> 1) & 1;   // (x+1,y), (x-1,y)
                const float sN = (sb >> 4) & 1, sS = (sb >> 2) & 1;   // (x,y+1), (x,y-1)
                const float sNE = (sb >> 7) & 1, sNW = (sb >> 8) & 1; // (x+1,y+1), (x-1,y+1)
                const float sSW = (sb >> 5) & 1, sSE = (sb >> 6) & 1; // (x-1,y-1), (x+1,y-1)
                // Eq. 6: sum_a W_a S(x+e_a) e_a
                const float swx = p.w_axis * (sE - sW) + p.w_diag * ((sNE - sNW) + (sSE - sSW));
                const float swy = p.w_axis * (sN - sS) + p.w_diag * ((sNE + sNW) - (sSE + sSW));
                float Fx = -psi * (sgx + swx);
                float Fy = -psi * (sgy + swy);
                // electric force f n on the conductive single layer next to a wall
                if (cur.rho >= p.rho_c) {
                    Fx += p.f_elec * (sE - sW);
                    Fy += p.f_elec * (sN - sS);
                }
                // body force on every fluid node
                Fx += cur.rho * p.bfx;
                Fy += cur.rho * p.bfy;

                if constexpr (MODE == kStep || MODE == kStepObs) {
                    // Eq. 10 velocity shift, Eq. 3 equilibrium, Eq. 1 relaxation.
                    // FP32 care: u' by one correctly rounded division; the
                    // weights w_a rho all derive from one correctly rounded
                    // rho/9 by exact power-of-two scalings, so sum_a f_eq = rho
                    // has no systematic bias (1/9 in FP32 is 7.5e-9 too large,
                    // which would add mass every step); at tau = 1 f* = f_eq.
                    const float ux = __fdiv_rn(fmaf(p.tau, Fx, cur.jx), cur.rho);
                    const float uy = __fdiv_rn(fmaf(p.tau, Fy, cur.jy), cur.rho);
                    const float om = 1.f - 1.5f * fmaf(ux, ux, uy * uy);
                    const float r9 = __fdiv_rn(cur.rho, 9.f);
                    const float w0r = 4.f * r9, w1r = r9, w2r = 0.25f * r9;
                    const float d5 = ux + uy, d6 = uy - ux;
                    // f_eq_a = w_a rho (1 + 3 c + 4.5 c^2 - 1.5 u^2), c = e_a . u
                    auto poly = [om](float c) { return fmaf(c, fmaf(4.5f, c, 3.f), om); };
                    float feq[9];
                    feq[0] = w0r * om;
                    feq[1] = w1r * poly(ux);
                    feq[2] = w1r * poly(uy);
                    feq[3] = w1r * poly(-ux);
                    feq[4] = w1r * poly(-uy);
                    feq[5] = w2r * poly(d5);
                    feq[6] = w2r * poly(d6);
                    feq[7] = w2r * poly(-d5);
                    feq[8] = w2r * poly(-d6);
                    float* o = fout + r * g.pitch + x;
                    if (p.tau == 1.f) {
#pragma unroll
                        for (int a = 0; a < 9; ++a) o[a * g.plane] = feq[a];
                    } else {
#pragma unroll
                        for (int a = 0; a < 9; ++a) {
                            const float fa = cur.f[a];
                            o[a * g.plane] = fmaf(feq[a] - fa, p.inv_tau, fa);
                        }
                    }
                }
                if constexpr (MODE != kStep) {
                    // physical velocity u = (rho u + F/2)/rho
                    const float mx = fmaf(0.5f, Fx, cur.jx), my = fmaf(0.5f, Fy, cur.jy);
                    const float vx = __fdiv_rn(mx, cur.rho), vy = __fdiv_rn(my, cur.rho);
                    if constexpr (MODE == kFields) {
                        const size_t i = (size_t)r * g.nx + x, n = (size_t)g.nx * g.ny;
                        fields[i] = cur.rho;
                        fields[n + i] = vx;
                        fields[2 * n + i] = vy;
                    } else {
                        if (isfinite(cur.rho) && isfinite(vx) && isfinite(vy)) {
                            a_mass.add(cur.rho);
                            a_q.add(vx);
                            a_px.add(mx);
                            a_py.add(my);
                            umax2 = fmaxf(umax2, vx * vx + vy * vy);
                            rmin = fminf(rmin, cur.rho);
                        } else {
                            ++bad;
                        }
                    }
                }
            } else if constexpr (MODE == kFields) {
                const size_t i = (size_t)r * g.nx + x, n = (size_t)g.nx * g.ny;
                fields[i] = 0.0;
                fields[n + i] = 0.0;
                fields[2 * n + i] = 0.0;
            }
        }
        cur = nxt;
    }

    if constexpr (MODE == kStepObs || MODE == kObs) {
        // deterministic CTA reduction: warp shuffles, then warp 0 over warps
        __shared__ double red_d[4][kThreads / 32];
        __shared__ float red_f[2][kThreads / 32];
        __shared__ unsigned red_u[kThreads / 32];
        double d[4] = {a_mass.value(), a_q.value(), a_px.value(), a_py.value()};
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] += __shfl_down_sync(0xffffffffu, d[k], off);
            umax2 = fmaxf(umax2, __shfl_down_sync(0xffffffffu, umax2, off));
            rmin = fminf(rmin, __shfl_down_sync(0xffffffffu, rmin, off));
            bad += __shfl_down_sync(0xffffffffu, bad, off);
        }
        const int w = t >> 5, lane = t & 31;
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) red_d[k][w] = d[k];
            red_f[0][w] = umax2;
            red_f[1][w] = rmin;
            red_u[w] = bad;
        }
        __syncthreads();
        if (t == 0) {
            double s[4] = {0, 0, 0, 0};
            float um = 0.f, rm = __int_as_float(0x7f800000);
            unsigned b = 0;
            for (int k = 0; k < kThreads / 32; ++k) {
#pragma unroll
                for (int q = 0; q < 4; ++q) s[q] += red_d[q][k];
                um = fmaxf(um, red_f[0][k]);
                rm = fminf(rm, red_f[1][k]);
                b += red_u[k];
            }
            double* out = partials + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kPartialStride;
            out[0] = s[0];
            out[1] = s[1];
            out[2] = s[2];
            out[3] = s[3];
            out[4] = um;
            out[5] = rm;
            out[6] = b;
            out[7] = 0.0;
        }
    }
}

}  // namespace lbm
