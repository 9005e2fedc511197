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
// row pitch `pitch` floats, a multiple of 32). Solid nodes hold the bit
// pattern kSolidBits in every plane; a pull that meets it knows the source
// node is solid, so no wall mask is read on the hot path.
//
// Work decomposition (HBM-bound stencil, no tensor cores):
//  - a CTA owns a strip of kW columns and a segment of tile_rows rows;
//  - one producer warp streams every row the segment needs (all 9 planes,
//    columns x0-4 .. x0+kW+4) into a kStages-deep ring in shared memory:
//    one cp.async.bulk per plane row (completion counted on the stage's
//    "full" mbarrier); at the periodic seam and on ragged strips the
//    16-byte-aligned body goes in bulk and the few remaining columns by
//    4-byte cp.async that arrive on the same barrier, so the producer never
//    waits for a load;
//  - kW/32 consumer warps pull each node's 9 populations out of the ring
//    (bounce-back values come from the same stage, no dependent loads), form
//    rho and psi, write psi into a 4-row ring, meet at a named barrier, then
//    compute the 8-neighbour forces of the previous row, collide and store f*
//    with coalesced stores; each warp then frees its ring stage on the
//    stage's "empty" mbarrier;
//  - every mbarrier wait is bounded: on timeout the kernel sets a flag in
//    global memory, stops waiting and runs to completion, and the host
//    reports LBM_ETIMEOUT.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbm {

constexpr uint32_t kSolidBits = 0xFFBADA55u;  // a NaN payload arithmetic never produces
constexpr int kW = 256;                        // interior columns per CTA
constexpr int kConsumerWarps = kW / 32;
constexpr int kThreads = kW + 32;              // consumers + one producer warp
constexpr int kHalo = 4;                       // staged halo columns per side
constexpr int kRowLen = kW + 2 * kHalo;        // floats per staged plane row
constexpr int kStages = 6;                     // ring depth (rows)
constexpr int kPartialStride = 8;              // doubles per CTA in the partials array
constexpr uint32_t kWaitLimit = 1u << 22;      // try_wait rounds before giving up

constexpr size_t kStageBytes = size_t(9) * kRowLen * sizeof(float);
constexpr size_t kSmemBytes = kStages * kStageBytes + 4 * (kW + 2) * sizeof(float) +
                              2 * kStages * sizeof(uint64_t) + 128;

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

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on one phase of an mbarrier. Returns false (and raises the
// error flag) if the phase did not complete within kWaitLimit rounds.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err)
{
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicOr(err, 1);
    return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 4-byte asynchronous copy global -> shared (completion tracked per thread)
__device__ __forceinline__ void async_g2s_4(float* dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Arrive on `bar` once all of this thread's earlier cp.async copies have
// landed (the arrival is counted in the barrier's initial count).
__device__ __forceinline__ void async_arrive_noinc(uint64_t* bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Approximate reciprocal (hardware estimate, about 1 ulp).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Quotient n/d from an approximate reciprocal r ~ 1/d with one residual
// correction (Markstein, IBM J. Res. Dev. 34 (1990)): q0 = n r,
// e = n - q0 d computed exactly by FMA, q = q0 + e r. The result is within
// a hair of the correctly rounded quotient for the normal, positive d here.
__device__ __forceinline__ float div_corrected(float n, float d, float r)
{
    const float q0 = n * r;
    const float e = fmaf(-q0, d, n);
    return fmaf(e, r, q0);
}

__device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kW) : "memory");
}

// ------------------------------------------------------------------ node math

// Pull node (column c of the staged rows) from the three ring rows holding
// y-1 (sm), y (sc) and y+1 (sp): f_a(x) = f*_a(x - e_a), or f*_opp(a)(x)
// when x - e_a is solid.
__device__ __forceinline__ void pull_smem(const float* __restrict__ sm, const float* __restrict__ sc,
                                          const float* __restrict__ sp, int c, Pulled& n)
{
    const float v0 = sc[c];
    n.solid = is_solid(v0);
    if (n.solid) {
        n.rho = n.jx = n.jy = 0.f;
        n.sb = 0;
        return;
    }
    constexpr int R = kRowLen;
    float v[9];
    v[0] = v0;
    v[1] = sc[1 * R + c - 1];  // e1 = ( 1, 0): source (x-1, y)
    v[2] = sm[2 * R + c];      // e2 = ( 0, 1): source (x, y-1)
    v[3] = sc[3 * R + c + 1];  // e3 = (-1, 0): source (x+1, y)
    v[4] = sp[4 * R + c];      // e4 = ( 0,-1): source (x, y+1)
    v[5] = sm[5 * R + c - 1];  // e5 = ( 1, 1): source (x-1, y-1)
    v[6] = sm[6 * R + c + 1];  // e6 = (-1, 1): source (x+1, y-1)
    v[7] = sp[7 * R + c + 1];  // e7 = (-1,-1): source (x+1, y+1)
    v[8] = sp[8 * R + c - 1];  // e8 = ( 1,-1): source (x-1, y+1)
    constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    uint32_t sb = 0;
#pragma unroll
    for (int a = 1; a < 9; ++a) {
        if (is_solid(v[a])) {
            sb |= 1u << a;
            v[a] = sc[opp[a] * R + c];  // half-way bounce-back
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

struct ObsAcc {
    Acc mass, q, px, py;
    float umax2 = 0.f, rmin = __builtin_huge_valf();  // +inf
    unsigned bad = 0;
};

// Forces, velocity shift, collision and the mode's epilogue for one fluid node
// (x, r) whose pulled populations are `n`; psi rows r-1, r, r+1 are pm, pc, pp
// (indexed by ring column t = node column - x0 + 1).
template <int MODE>
__device__ __forceinline__ void collide_node(const Pulled& n, const float* pm, const float* pc,
                                             const float* pp, int t, const Phys& p, const Geom& g,
                                             float* __restrict__ fout, double* __restrict__ fields,
                                             int x, int r, ObsAcc& acc)
{
    const float psi = pc[t];
    // Eq. 5: sum_a G_a psi(x+e_a) e_a, axis and diagonal links
    const float sgx = p.g_axis * (pc[t + 1] - pc[t - 1]) +
                      p.g_diag * ((pp[t + 1] - pp[t - 1]) + (pm[t + 1] - pm[t - 1]));
    const float sgy = p.g_axis * (pp[t] - pm[t]) +
                      p.g_diag * ((pp[t + 1] + pp[t - 1]) - (pm[t + 1] + pm[t - 1]));
    float Fx, Fy;
    const uint32_t sb = n.sb;
    if (sb == 0) {
        // no solid neighbour: Eq. 6 and the electric force vanish
        Fx = -psi * sgx;
        Fy = -psi * sgy;
    } else {
        // S(x + e_a) = solid flag of the pull source of the opposite direction
        const float sE = (sb >> 3) & 1, sW = (sb >> 1) & 1;    // (x+1,y), (x-1,y)
        const float sN = (sb >> 4) & 1, sS = (sb >> 2) & 1;    // (x,y+1), (x,y-1)
        const float sNE = (sb >> 7) & 1, sNW = (sb >> 8) & 1;  // (x+1,y+1), (x-1,y+1)
        const float sSW = (sb >> 5) & 1, sSE = (sb >> 6) & 1;  // (x-1,y-1), (x+1,y-1)
        // Eq. 6: sum_a W_a S(x+e_a) e_a
        const float swx = p.w_axis * (sE - sW) + p.w_diag * ((sNE - sNW) + (sSE - sSW));
        const float swy = p.w_axis * (sN - sS) + p.w_diag * ((sNE + sNW) - (sSE + sSW));
        Fx = -psi * (sgx + swx);
        Fy = -psi * (sgy + swy);
        // electric force f n on the conductive single layer next to a wall
        if (n.rho >= p.rho_c) {
            Fx += p.f_elec * (sE - sW);
            Fy += p.f_elec * (sN - sS);
        }
    }
    // body force on every fluid node
    Fx += n.rho * p.bfx;
    Fy += n.rho * p.bfy;

    if constexpr (MODE == kStep || MODE == kStepObs) {
        // Eq. 10 velocity shift, Eq. 3 equilibrium, Eq. 1 relaxation.
        // FP32 care: u' by corrected quotients; the weights w_a rho all derive
        // from one corrected rho/9 by exact power-of-two scalings, so
        // sum_a f_eq = rho has no systematic bias (1/9 in FP32 is 7.5e-9 too
        // large, which would add mass every step); at tau = 1 f* = f_eq.
        const float rinv = rcp_approx(n.rho);
        const float ux = div_corrected(fmaf(p.tau, Fx, n.jx), n.rho, rinv);
        const float uy = div_corrected(fmaf(p.tau, Fy, n.jy), n.rho, rinv);
        const float om = 1.f - 1.5f * fmaf(ux, ux, uy * uy);
        const float r9 = div_corrected(n.rho, 9.f, 1.f / 9.f);
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
                const float fa = n.f[a];
                o[a * g.plane] = fmaf(feq[a] - fa, p.inv_tau, fa);
            }
        }
    }
    if constexpr (MODE != kStep) {
        // physical velocity u = (rho u + F/2)/rho
        const float mx = fmaf(0.5f, Fx, n.jx), my = fmaf(0.5f, Fy, n.jy);
        const float vx = __fdiv_rn(mx, n.rho), vy = __fdiv_rn(my, n.rho);
        if constexpr (MODE == kFields) {
            const size_t i = (size_t)r * g.nx + x, nn = (size_t)g.nx * g.ny;
            fields[i] = n.rho;
            fields[nn + i] = vx;
            fields[2 * nn + i] = vy;
        } else {
            if (isfinite(n.rho) && isfinite(vx) && isfinite(vy)) {
                acc.mass.add(n.rho);
                acc.q.add(vx);
                acc.px.add(mx);
                acc.py.add(my);
                acc.umax2 = fmaxf(acc.umax2, vx * vx + vy * vy);
                acc.rmin = fminf(acc.rmin, n.rho);
            } else {
                ++acc.bad;
            }
        }
    }
}

// ------------------------------------------------------------------ kernel

template <int MODE>
__global__ void __launch_bounds__(kThreads, 3)
    step_kernel(const float* __restrict__ fin, float* __restrict__ fout, Geom g, Phys p,
                double* __restrict__ partials, double* __restrict__ fields, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);                       // [kStages][9][kRowLen]
    float* psi_ring = ring + size_t(kStages) * 9 * kRowLen;                 // [4][kW + 2]
    uint64_t* full = reinterpret_cast<uint64_t*>(psi_ring + 4 * (kW + 2));  // [kStages]
    uint64_t* empty = full + kStages;                                       // [kStages]

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * kW;
    const int nint = min(kW, g.nx - x0);     // interior columns of this strip
    const int nbody = nint & ~3;             // columns moved by the bulk copies
    const int y0 = blockIdx.y * g.tile_rows;
    const int y1 = min(y0 + g.tile_rows, g.ny);
    const int nrows = (y1 - y0) + 4;         // staged rows y0-2 .. y1+1

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 32);               // 32 producer-lane arrivals + tx bytes
            mbar_init(&empty[s], kConsumerWarps);  // one arrival per consumer warp
        }
        fence_mbar_init();
    }
    __syncthreads();

    // staged rows reach two rows past the segment, which wraps more than
    // once around a domain of one row: reduce with a true modulo
    auto wrap_y = [&](int y) {
        y %= g.ny;
        return y < 0 ? y + g.ny : y;
    };
    auto wrap_x = [&](int x) {
        x %= g.nx;
        return x < 0 ? x + g.nx : x;
    };

    if (warp == kConsumerWarps) {
        // ---------------- producer warp: fill ring stages with rows y0-2 .. y1+1
        // Interior strips (halos inside [0, nx) and a 16-byte multiple wide)
        // take one bulk copy per plane row covering columns x0-4 .. x0+nint+4.
        // Edge and ragged strips copy the aligned body in bulk and fetch the
        // remaining <= 11 columns per plane with 4-byte cp.async; each lane's
        // column is fixed for the whole segment.
        const bool whole = (x0 >= kHalo) && (x0 + nint + kHalo <= g.nx) && ((nint & 3) == 0);
        const int b_col = whole ? -kHalo : 0;                   // first bulk column (rel. x0)
        const int b_len = whole ? nint + 2 * kHalo : nbody;     // bulk columns
        const uint32_t b_bytes = uint32_t(b_len) * sizeof(float);
        const int n_right = nint + kHalo - nbody;               // columns [x0+nbody, x0+nint+4)
        const int n_scalar = whole ? 0 : kHalo + n_right;       // <= 11
        int my_sc = 0, my_gx = 0;
        const bool has_scalar = lane < n_scalar;
        if (has_scalar) {
            const int col = (lane < kHalo) ? (lane - kHalo) : (nbody + (lane - kHalo));
            my_sc = kHalo + col;
            my_gx = wrap_x(x0 + col);
        }
        bool ok = true;
        for (int k = 0; k < nrows; ++k) {
            const int s = k % kStages;
            if (k >= kStages) ok = mbar_wait(&empty[s], ((k / kStages) - 1) & 1, err) && ok;
            const int row = wrap_y(y0 - 2 + k);
            float* st = ring + size_t(s) * 9 * kRowLen;
            const float* src = fin + size_t(row) * g.pitch;
            if (lane == 0 && b_len > 0) {
                mbar_expect_tx(&full[s], 9 * b_bytes);
#pragma unroll 1
                for (int a = 0; a < 9; ++a)
                    bulk_g2s(st + a * kRowLen + kHalo + b_col, src + size_t(a) * g.plane + x0 + b_col, b_bytes,
                             &full[s]);
            }
            if (has_scalar) {
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    async_g2s_4(st + a * kRowLen + my_sc, src + size_t(a) * g.plane + my_gx);
            }
            async_arrive_noinc(&full[s]);
        }
        // drain: every armed fill has been waited on by the consumers in the
        // normal path; wait (bounded) for the last phase of each stage anyway
        // so that no copy is in flight when the CTA exits
        for (int s = 0; s < kStages && s < nrows; ++s) {
            const int last_k = s + ((nrows - 1 - s) / kStages) * kStages;
            ok = mbar_wait(&full[s], (last_k / kStages) & 1, err) && ok;
        }
        (void)ok;
        return;
    }

    // ---------------- consumer warps
    const int t = tid;                  // column x0 + t
    const bool interior = t < nint;
    const int c = t + kHalo;            // staged column of this node
    const int x = x0 + t;
    float* psi_w = psi_ring;            // ring row stride kW + 2, column t + 1
    ObsAcc acc;
    Pulled cur, nxt;
    bool ok = true;
    // prologue: the two oldest staged rows (y0-2, y0-1) must be present
    ok = mbar_wait(&full[0], 0, err) && ok;
    if (nrows > 1) ok = mbar_wait(&full[1 % kStages], (1 / kStages) & 1, err) && ok;

    for (int k = 1; k <= nrows - 2; ++k) {
        // pull row r = y0 - 2 + k, which needs staged rows k-1, k, k+1
        const int r = y0 - 2 + k;
        const int kn = k + 1;
        ok = mbar_wait(&full[kn % kStages], (kn / kStages) & 1, err) && ok;
        const float* sm = ring + size_t((k - 1) % kStages) * 9 * kRowLen;
        const float* sc = ring + size_t(k % kStages) * 9 * kRowLen;
        const float* sp = ring + size_t(kn % kStages) * 9 * kRowLen;
        float* prow = psi_w + ((r + 4) & 3) * (kW + 2);
        if (interior) {
            pull_smem(sm, sc, sp, c, nxt);
            prow[t + 1] = pseudopotential(p, nxt);
            if (t == 0) {  // left halo column x0 - 1
                Pulled h;
                pull_smem(sm, sc, sp, c - 1, h);
                prow[0] = pseudopotential(p, h);
            }
            if (t == nint - 1) {  // right halo column x0 + nint
                Pulled h;
                pull_smem(sm, sc, sp, c + 1, h);
                prow[nint + 1] = pseudopotential(p, h);
            }
        }
        consumer_sync();
        // staged row k-1 is no longer needed by any consumer
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[(k - 1) % kStages]);
        if (k >= 3 && interior && !cur.solid) {
            // collide row r-1 with psi rows r-2, r-1, r
            const int rc = r - 1;
            const float* pm = psi_w + ((rc + 3) & 3) * (kW + 2);
            const float* pc = psi_w + ((rc + 4) & 3) * (kW + 2);
            const float* pp = psi_w + ((rc + 5) & 3) * (kW + 2);
            collide_node<MODE>(cur, pm, pc, pp, t + 1, p, g, fout, fields, x, rc, acc);
        } else if constexpr (MODE == kFields) {
            if (k >= 3 && interior) {
                const size_t i = (size_t)(r - 1) * g.nx + x, nn = (size_t)g.nx * g.ny;
                fields[i] = 0.0;
                fields[nn + i] = 0.0;
                fields[2 * nn + i] = 0.0;
            }
        }
        cur = nxt;
    }
    (void)ok;

    if constexpr (MODE == kStepObs || MODE == kObs) {
        // deterministic CTA reduction: warp shuffles, then one thread over warps
        __shared__ double red_d[4][kConsumerWarps];
        __shared__ float red_f[2][kConsumerWarps];
        __shared__ unsigned red_u[kConsumerWarps];
        double d[4] = {acc.mass.value(), acc.q.value(), acc.px.value(), acc.py.value()};
        float umax2 = acc.umax2, rmin = acc.rmin;
        unsigned bad = acc.bad;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] += __shfl_down_sync(0xffffffffu, d[q], off);
            umax2 = fmaxf(umax2, __shfl_down_sync(0xffffffffu, umax2, off));
            rmin = fminf(rmin, __shfl_down_sync(0xffffffffu, rmin, off));
            bad += __shfl_down_sync(0xffffffffu, bad, off);
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) red_d[q][warp] = d[q];
            red_f[0][warp] = umax2;
            red_f[1][warp] = rmin;
            red_u[warp] = bad;
        }
        consumer_sync();
        if (t == 0) {
            double s[4] = {0, 0, 0, 0};
            float um = 0.f, rm = __int_as_float(0x7f800000);
            unsigned b = 0;
            for (int w = 0; w < kConsumerWarps; ++w) {
#pragma unroll
                for (int q = 0; q < 4; ++q) s[q] += red_d[q][w];
                um = fmaxf(um, red_f[0][w]);
                rm = fminf(rm, red_f[1][w]);
                b += red_u[w];
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
