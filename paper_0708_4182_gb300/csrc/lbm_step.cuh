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
// Work decomposition (no tensor cores; the FP32 form is bound by DRAM, the
// 16-bit forms by instruction issue):
//  - a CTA owns a strip of columns and a segment of tile_rows rows;
//  - one producer warp streams every row the segment needs (all 9 planes of
//    a window a few columns wider than the strip) into a kStages-deep ring in
//    shared memory with cp.async.bulk copies whose completion is counted on
//    the stage's "full" mbarrier; pieces that cannot move in 16-byte units
//    (periodic seam, ragged strips of the FP32 forms) go by 4-byte cp.async
//    that arrive on the same barrier, so the producer never waits for a load;
//  - the consumer warps pull the 9 populations of one node per thread, or of
//    two neighbouring nodes per thread in the 32-bit forms' pair layout, out
//    of the ring (bounce-back values come from the same stage, no dependent loads),
//    form rho and psi, write psi into a 4-row ring, meet at a named barrier,
//    then compute the 8-neighbour forces of the previous row, collide and
//    store f* with coalesced stores; each warp then frees its ring stage on
//    the stage's "empty" mbarrier. The psi of the strip's two halo columns
//    comes from an extra pull by the threads at the strip's ends (32-bit
//    forms) or from two extra threads of overlapping strips (16-bit forms);
//    see run_tile;
//  - the pulled state of two consecutive rows lives in two register sets used
//    in turn, and a node whose 9 pulled values sum to a non-NaN value has no
//    solid neighbour and skips the per-direction bounce-back checks;
//  - every mbarrier wait is bounded: on timeout the kernel sets a flag in
//    global memory, stops waiting and runs to completion, and the host
//    reports LBM_ETIMEOUT.
//
// Storage forms (template parameter ST; the arithmetic is FP32 in all):
//  - kF32:     plane a holds f*_a (plain populations);
//  - kF32Dev:  plane 0 holds rho* = sum_a f*_a and planes 1..8 hold the
//              deviations d_a = f*_a - w_a rho* from the node's weighted rest
//              equilibrium, all FP32 (f*_0 = w_0 rho* - sum_a d_a). Small
//              per-step changes of a slow flow are representable in d_a,
//              where a plain FP32 f*_a of size ~w_a rho rounds them away;
//  - kF16Dev / kBF16Dev: as kF32Dev with d_a stored in 16 bits (FP16 or
//              BF16, rounded to nearest), the 8 of a node interleaved in 16
//              bytes after plane 0 (dev_index); 20 instead of 36 bytes per node.
// In the deviation forms the pull rebuilds f_a = w_a rho*(src) + d_a(src),
// and the kernel forms rho - rho*(x) and rho u from sums of small terms.
#pragma once

#include <cstdint>
#include <type_traits>
#include <utility>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

constexpr uint32_t kSolidBits = 0xFFBADA55u;  // a NaN payload arithmetic never produces
constexpr int kW = 256;                        // strip width of the 32-bit forms; consumer threads of the 16-bit forms
constexpr int kRowLen = kW + 8;                // staged columns per plane row (window + alignment)
constexpr int kPsiStride = kW + 4;             // floats per psi ring row
constexpr int kPartialStride = 8;              // doubles per CTA in the partials array
constexpr uint32_t kWaitLimit = 1u << 18;      // try_wait rounds before giving up (about 1 s on a GB300)

enum Storage { kF32 = 0, kF32Dev = 1, kF16Dev = 2, kBF16Dev = 3 };
__host__ __device__ constexpr bool is16(int st) { return st == kF16Dev || st == kBF16Dev; }

// Staging ring depth (rows) and resident CTAs per SM the launch bounds aim
// at. The one-node layout of the 32-bit forms (288 threads): 6 and 3. The
// 16-bit forms (288 threads): LBM_STAGES_16 / LBM_CTAS_16, 6 and 3. The pair
// layout of the 32-bit forms (160 threads, a pair of nodes per thread):
// LBM_STAGES_F32 / LBM_CTAS_F32 and LBM_STAGES_F32DEV / LBM_CTAS_F32DEV for
// the tau = 1 instances, whose register needs are lower; the tau != 1
// instances aim at 3. Shared memory and registers must allow that many CTAs.
// Measured at 16384x4096 (GLUPS, FP32 / FP32 deviations / batch FP32 / batch
// FP32 deviations): pairs at 6 stages x 3 CTAs 89.4 / 85.9 / 80.5 / 72.8;
// FP32 4 x 5 and deviations 5 x 4: 89.8 / 89.7 / 81.4 / 75.7 (the batch
// kernel keeps its domain parameters in shared memory, which keeps it from
// spilling at 4 CTAs). FP16 deviations at 4, 6 and 8 stages: 107.8 / 110.6
// / 104.4; at 2 or 4 CTAs per SM: 84.3 / 105.9.
#ifndef LBM_STAGES_F32
#define LBM_STAGES_F32 4
#endif
#ifndef LBM_CTAS_F32
#define LBM_CTAS_F32 5
#endif
#ifndef LBM_STAGES_F32DEV
#define LBM_STAGES_F32DEV 5
#endif
#ifndef LBM_CTAS_F32DEV
#define LBM_CTAS_F32DEV 4
#endif
#ifndef LBM_STAGES_16
#define LBM_STAGES_16 6
#endif
#ifndef LBM_CTAS_16
#define LBM_CTAS_16 3
#endif
// pair: the 32-bit forms' pair layout (ignored by the 16-bit forms)
__host__ __device__ constexpr int stages_of(int st, bool pair = true)
{
    return is16(st) ? LBM_STAGES_16 : !pair ? 6 : st == kF32 ? LBM_STAGES_F32 : LBM_STAGES_F32DEV;
}
__host__ __device__ constexpr int ctas_of(int st, bool t1 = true, bool pair = true)
{
    return is16(st) ? (t1 ? LBM_CTAS_16 : 3)
                    : !pair ? 3 : st == kF32 ? (t1 ? LBM_CTAS_F32 : 3) : (t1 ? LBM_CTAS_F32DEV : 3);
}
// the persistent batch kernel: as the single-domain step; its observing mode
// aims at 3 (it spills at 4)
__host__ __device__ constexpr int batch_ctas_of(int mode, int st, bool t1, bool pair = true)
{
    return mode == 0 ? ctas_of(st, t1, pair) : (ctas_of(st, t1, pair) > 3 ? 3 : ctas_of(st, t1, pair));
}
// the single-domain kernel of a mode: the observing modes keep their
// reduction state too and aim at one CTA less (no spills); the step with
// fused observables and tau != 1 (once per observation interval) at 2
__host__ __device__ constexpr int step_ctas_of(int mode, int st, bool t1, bool pair = true)
{
    return mode == 0 ? ctas_of(st, t1, pair)
           : !t1     ? 2
                     : (ctas_of(st, t1, pair) > 3 ? ctas_of(st, t1, pair) - 1 : ctas_of(st, t1, pair));
}

// T: type of the 8 values after plane 0 (populations or deviations); align:
// columns per 16 bytes of the narrowest plane (every staging copy starts and
// ends on such a boundary); overlap: the strip layout (see run_tile), 0 for
// the 32-bit forms, 1 for the 16-bit ones
template <int ST> struct StoreT;
template <> struct StoreT<kF32> { using T = float; static constexpr int align = 4, overlap = 0; };
template <> struct StoreT<kF32Dev> { using T = float; static constexpr int align = 4, overlap = 0; };
template <> struct StoreT<kF16Dev> { using T = __half; static constexpr int align = 8, overlap = 1; };
template <> struct StoreT<kBF16Dev> { using T = __nv_bfloat16; static constexpr int align = 8, overlap = 1; };

// Columns a CTA collides: kW, or kW - 2 where neighbouring strips overlap.
__host__ __device__ constexpr int strip_cols(int st) { return (st == kF16Dev || st == kBF16Dev) ? kW - 2 : kW; }

// Consumer threads per CTA: the pair layout of the 32-bit forms gives each
// thread a pair of neighbouring columns (packed two-lane FP32 arithmetic, see
// run_tile); the one-node layout and the 16-bit forms one column. One
// producer warp comes on top.
__host__ __device__ constexpr int consumers(int st, bool pair = true) { return (is16(st) || !pair) ? kW : kW / 2; }
__host__ __device__ constexpr int threads_of(int st, bool pair = true) { return consumers(st, pair) + 32; }

// Element index of deviation a (1..8) of the node at o = y * pitch + x among
// the deviation values that follow plane 0 (plane = ny * pitch): FP32
// deviations in 8 planes of `plane` elements; 16-bit deviations interleaved,
// the 8 of a node in 16 contiguous bytes (one vector store per node). The
// staged rows in shared memory use the same two layouts with R for plane.
template <typename T> __host__ __device__ __forceinline__ size_t dev_index(size_t o, int a, size_t plane)
{
    return sizeof(T) == 2 ? o * 8 + size_t(a - 1) : size_t(a - 1) * plane + o;
}

// staged row: plane 0 (FP32, kRowLen floats) then 8 x kRowLen deviations (type T)
template <int ST> __host__ __device__ constexpr size_t stage_bytes()
{
    return size_t(kRowLen) * (sizeof(float) + 8 * sizeof(typename StoreT<ST>::T));
}
template <int ST, bool PAIR = true> __host__ __device__ constexpr size_t smem_bytes()
{
    // ring stages, their two mbarriers each, the psi ring (one row per stage) and alignment slack
    return stages_of(ST, PAIR) * (stage_bytes<ST>() + 2 * sizeof(uint64_t) + kPsiStride * sizeof(float)) + 128;
}
// bytes of one node's state in global memory (plane 0 + the other 8 values)
template <int ST> __host__ __device__ constexpr int node_bytes() { return 4 + 8 * int(sizeof(typename StoreT<ST>::T)); }

// FP16 deviations are stored scaled by 2^12 (an exact scaling): |d| up to 16
// stays below the FP16 maximum 65504, and deviations down to 2^-26 stay in
// FP16's normal range. Unscaled, the deviations of slowly moving vapor
// (~1e-7) would be subnormal, with a few correct bits at most, and the flux
// of a body-force-driven channel would be off by percents.
constexpr float kF16Scale = 4096.f, kF16Unscale = 1.f / 4096.f;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v) * kF16Unscale; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v * kF16Scale); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

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
    float e_corner;        // electric force scale where two solid faces meet (1 or 1/sqrt 2)
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

// The NC consumer threads (once per staged row, and the observables reduction).
template <int NC> __device__ __forceinline__ void consumer_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NC) : "memory");
}

// ------------------------------------------------------------------ two-lane FP32
// In the pair layout a float2 holds one value of each of two neighbouring
// nodes (lane x: the left node A, lane y: the right node B); in the one-node
// functions it holds two values of the same node that go through the same
// operation (the x and y components of a vector, or the two halves of a sum).
// These map to Blackwell's paired FP32 instructions (add/mul/fma .rn on
// f32x2): each lane is rounded exactly as the scalar operation would be, and
// one instruction does both lanes' operation.
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as fma(b, -1, a): the product is exact, so this is the rounded difference
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ float lane_of(const float2& v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ void set_lane(float2& v, int k, float a)
{
    if (k == 0) v.x = a; else v.y = a;
}

// The compensated sum of Acc in both lanes at once (lane k accumulates the
// values of its lane, operation for operation as Acc::add).
struct Acc2 {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 v)
    {
        const float2 t = add2(s, v);
        const float2 bp = sub2(t, s);
        c = add2(c, add2(sub2(s, sub2(t, bp)), sub2(v, bp)));
        s = t;
    }
    __device__ __forceinline__ double value() const
    {
        return ((double)s.x + (double)c.x) + ((double)s.y + (double)c.y);
    }
};

// Observables state of the pair layout: lane k sums the nodes of lane k.
struct ObsAcc2 {
    Acc2 mass, q, px, py;
    float umax2 = 0.f, rmin = __builtin_huge_valf();  // +inf
    unsigned bad = 0;
    __device__ __forceinline__ double value(int k) const
    {
        return k == 0 ? mass.value() : k == 1 ? q.value() : k == 2 ? px.value() : py.value();
    }
};

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
    auto density = [&v]() { return ((v[0] + (v[1] + v[3])) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8])); };
    uint32_t sb = 0;
    float rho = density();
    // a solid source holds a NaN sentinel, so a sum that is not NaN has no
    // solid source; only a NaN sum (a wall nearby, or a state gone
    // non-finite) takes the per-direction checks
    if (isnan(rho)) {
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            if (is_solid(v[a])) {
                sb |= 1u << a;
                v[a] = sc[opp[a] * R + c];  // half-way bounce-back
            }
        }
        rho = density();
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) n.f[a] = v[a];
    n.sb = sb;
    n.rho = rho;
    n.jx = (v[1] - v[3]) + (v[5] - v[7]) + (v[8] - v[6]);
    n.jy = (v[2] - v[4]) + (v[5] - v[7]) + (v[6] - v[8]);
}

template <typename N>
__device__ __forceinline__ float pseudopotential(const Phys& p, const N& n)
{
    // psi = rho0 (1 - exp(-rho/rho0)), via expm1 to keep small-rho accuracy
    return n.solid ? 0.f : -p.rho0 * expm1f(-n.rho * p.inv_rho0);
}

// Error-free accumulation s + c of FP32 terms (Knuth's TwoSum).
// FP32 sum with the exact rounding error of every addition (TwoSum)
// collected in c: s + c carries about twice FP32's precision, so the sums of
// cancelling quantities (momentum) do not depend on how nodes are split
// among threads and tiles.
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
    // sum q (0 mass, 1 flux, 2 x momentum, 3 y momentum)
    __device__ __forceinline__ double value(int k) const
    {
        return k == 0 ? mass.value() : k == 1 ? q.value() : k == 2 ? px.value() : py.value();
    }
};

// Eq. 6 and the electric force of a node with solid pull sources (flags sb,
// nonzero), added to the negated Eq. 5 sums nsgx, nsgy: the node's force
// before the body force. Written with explicit roundings (no contraction
// left to the compiler) so that the one-node and the two-node kernels give
// the same bits.
__device__ __forceinline__ void wall_electric(uint32_t sb, float psi, float nsgx, float nsgy, float rho,
                                              const Phys& p, float& fx, float& fy)
{
    // S(x + e_a) = solid flag of the pull source of the opposite direction
    const float sE = (sb >> 3) & 1, sW = (sb >> 1) & 1;    // (x+1,y), (x-1,y)
    const float sN = (sb >> 4) & 1, sS = (sb >> 2) & 1;    // (x,y+1), (x,y-1)
    const float sNE = (sb >> 7) & 1, sNW = (sb >> 8) & 1;  // (x+1,y+1), (x-1,y+1)
    const float sSW = (sb >> 5) & 1, sSE = (sb >> 6) & 1;  // (x-1,y-1), (x+1,y-1)
    // Eq. 6: sum_a W_a S(x+e_a) e_a (the flag differences are exact)
    const float swx = fmaf(p.w_axis, sE - sW, __fmul_rn(p.w_diag, (sNE - sNW) + (sSE - sSW)));
    const float swy = fmaf(p.w_axis, sN - sS, __fmul_rn(p.w_diag, (sNE + sNW) - (sSE + sSW)));
    fx = __fmul_rn(psi, __fsub_rn(nsgx, swx));
    fy = __fmul_rn(psi, __fsub_rn(nsgy, swy));
    // electric force f n on the conductive single layer next to a wall
    if (rho >= p.rho_c) {
        const float ex = sE - sW, ey = sN - sS;
        const float fe = (ex != 0.f && ey != 0.f) ? __fmul_rn(p.f_elec, p.e_corner) : p.f_elec;
        fx = fmaf(fe, ex, fx);
        fy = fmaf(fe, ey, fy);
    }
}

// Total force on one fluid node: Eq. 5 from the psi rows pm, pc, pp (ring
// column t), Eq. 6 and the electric wall-layer force from the solid flags of
// the pull sources (n.sb), and the body force. N has fields rho and sb. The
// sign of Eq. 5 is carried by the constants (-G: round to nearest is
// symmetric, so this is exactly the negated sum); every operation is the
// two-node kernel's (node_force2) lane for lane. The x and y components go
// through the paired instructions together (lane x: the x component).
template <typename N>
__device__ __forceinline__ float2 node_force(const N& n, const float* pm, const float* pc, const float* pp,
                                             int t, const Phys& p)
{
    const float psi = pc[t];
    // (psi(x+1) - psi(x-1), psi(y+1) - psi(y-1)) on the node's row and column
    const float2 dc = sub2(make_float2(pc[t + 1], pp[t]), make_float2(pc[t - 1], pm[t]));
    // rows y+1 and y-1: right minus left, right plus left
    const float2 pr = make_float2(pp[t + 1], pm[t + 1]), pl = make_float2(pp[t - 1], pm[t - 1]);
    const float2 dd = sub2(pr, pl), ss = add2(pr, pl);
    // Eq. 5: -sum_a G_a psi(x+e_a) e_a, axis and diagonal links
    const float2 nsg = fma2(splat(-p.g_axis), dc,
                            mul2(splat(-p.g_diag), make_float2(__fadd_rn(dd.x, dd.y), __fsub_rn(ss.x, ss.y))));
    float2 F = mul2(splat(psi), nsg);
    if (n.sb != 0) wall_electric(n.sb, psi, nsg.x, nsg.y, n.rho, p, F.x, F.y);
    // body force on every fluid node
    return fma2(splat(n.rho), make_float2(p.bfx, p.bfy), F);
}

// Observables or fields epilogue of one fluid node (modes other than kStep).
// rinv is rcp_approx(rho); the quotients are corrected by one residual step.
template <int MODE>
__device__ __forceinline__ void node_observe(float rho, float rinv, float jx, float jy, float Fx, float Fy,
                                             const Geom& g, double* __restrict__ fields, int x, int r,
                                             ObsAcc& acc)
{
    // physical velocity u = (rho u + F/2)/rho
    const float mx = fmaf(0.5f, Fx, jx), my = fmaf(0.5f, Fy, jy);
    const float vx = div_corrected(mx, rho, rinv), vy = div_corrected(my, rho, rinv);
    if constexpr (MODE == kFields) {
        const size_t i = (size_t)r * g.nx + x, nn = (size_t)g.nx * g.ny;
        fields[i] = rho;
        fields[nn + i] = vx;
        fields[2 * nn + i] = vy;
    } else {
        // a NaN or infinity in any of the three makes the sum non-finite
        if (isfinite(rho + vx + vy)) {
            acc.mass.add(rho);
            acc.q.add(vx);
            acc.px.add(mx);
            acc.py.add(my);
            // explicit roundings: the same |u|^2 in every kernel instance
            acc.umax2 = fmaxf(acc.umax2, fmaf(vx, vx, __fmul_rn(vy, vy)));
            acc.rmin = fminf(acc.rmin, rho);
        } else {
            ++acc.bad;
        }
    }
}

// n / d by the corrected reciprocal r ~ 1/d (div_corrected) with nd = -d,
// written as the two-node kernel writes it (div2), operation for operation.
__device__ __forceinline__ float div1(float n, float nd, float r)
{
    const float q0 = __fmul_rn(n, r);
    const float e = fmaf(q0, nd, n);
    return fmaf(e, r, q0);
}

// The same in both lanes.
__device__ __forceinline__ float2 div2(float2 n, float2 nd, float2 r)
{
    const float2 q0 = mul2(n, r);
    const float2 e = fma2(q0, nd, n);
    return fma2(e, r, q0);
}

// Forces, velocity shift, collision and the mode's epilogue for one fluid node
// (x, r) in plain storage, whose pulled populations are `n`; psi rows r-1, r,
// r+1 are pm, pc, pp (indexed by the node's ring column t). Every operation is
// the two-node kernel's (collide_pair) lane for lane, so the one-node and
// two-node layouts store the same bits.
template <int MODE, bool T1>
__device__ __forceinline__ void collide_node(const Pulled& n, const float* pm, const float* pc,
                                             const float* pp, int t, const Phys& p, const Geom& g,
                                             float* __restrict__ fout, double* __restrict__ fields,
                                             int x, int r, ObsAcc& acc)
{
    const float2 F = node_force(n, pm, pc, pp, t, p);
    const float rinv = rcp_approx(n.rho);
    if constexpr (MODE == kStep || MODE == kStepObs) {
        // Eq. 10 velocity shift, Eq. 3 equilibrium, Eq. 1 relaxation.
        // FP32 care: u' by corrected quotients; the weights w_a rho all derive
        // from one corrected rho/9 by exact power-of-two scalings, so
        // sum_a f_eq = rho has no systematic bias (1/9 in FP32 is 7.5e-9 too
        // large, which would add mass every step); at tau = 1 f* = f_eq.
        // Lane pairs: (x, y) components, then the directions (1, 2), (3, 4),
        // (5, 6), (7, 8).
        const float2 u = div2(fma2(splat(p.tau), F, make_float2(n.jx, n.jy)), splat(-n.rho), splat(rinv));
        const float om = fmaf(-1.5f, fmaf(u.x, u.x, __fmul_rn(u.y, u.y)), 1.f);
        const float r9 = div1(n.rho, -9.f, 1.f / 9.f);
        const float w0r = __fmul_rn(4.f, r9), w2r = __fmul_rn(0.25f, r9);
        const float2 dg = make_float2(__fadd_rn(u.x, u.y), __fsub_rn(u.y, u.x));  // e5.u, e6.u
        // f_eq_a = w_a rho (1 + 3 c + 4.5 c^2 - 1.5 u^2) with c = +-(e_a . u):
        // (-c)(4.5(-c) + 3) = c (4.5 c - 3) exactly
        const float2 oms = splat(om);
        auto polyp = [oms](float2 c) { return fma2(c, fma2(splat(4.5f), c, splat(3.f)), oms); };
        auto polym = [oms](float2 c) { return fma2(c, fma2(splat(4.5f), c, splat(-3.f)), oms); };
        float fs[9];
        fs[0] = __fmul_rn(w0r, om);
        const float2 f12 = mul2(splat(r9), polyp(u)), f34 = mul2(splat(r9), polym(u));
        const float2 f56 = mul2(splat(w2r), polyp(dg)), f78 = mul2(splat(w2r), polym(dg));
        fs[1] = f12.x; fs[2] = f12.y; fs[3] = f34.x; fs[4] = f34.y;
        fs[5] = f56.x; fs[6] = f56.y; fs[7] = f78.x; fs[8] = f78.y;
        if (!T1 && p.tau != 1.f) {
#pragma unroll
            for (int a = 0; a < 9; ++a) fs[a] = fmaf(__fsub_rn(fs[a], n.f[a]), p.inv_tau, n.f[a]);
        }
        float* o = fout + r * g.pitch + x;
#pragma unroll
        for (int a = 0; a < 9; ++a) o[a * g.plane] = fs[a];
    }
    if constexpr (MODE != kStep) node_observe<MODE>(n.rho, rinv, n.jx, n.jy, F.x, F.y, g, fields, x, r, acc);
}

// ------------------------------------------------------------------ deviation storage

struct PulledDev {
    float rho, jx, jy;
    float g[9];   // f_a - w_a rho (only a = 1..8 are used)
    uint32_t sb;  // bit a set <=> the pull source x - e_a is solid
    bool solid;
};

// Stored deviations in raw units: FP16 planes hold d_a * kF16Scale, the
// other forms d_a itself. The deviation arithmetic below runs on raw values
// and applies the power-of-two factor kUnscale<T> once per sum; a
// power-of-two scaling commutes with FP32 rounding (no value here comes near
// FP32's range limits), so the results equal those of the unscaled sums bit
// for bit.
__device__ __forceinline__ float to_raw(float v) { return v; }
__device__ __forceinline__ float to_raw(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_raw(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_raw(float v);
template <> __device__ __forceinline__ float from_raw<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_raw<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_raw<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <typename T> struct RawScale { static constexpr float scale = 1.f, unscale = 1.f; };
template <> struct RawScale<__half> { static constexpr float scale = kF16Scale, unscale = kF16Unscale; };
// Two raw 16-bit values in one 32-bit word (lane x in the low half), to and
// from FP32 with one paired conversion each way.
template <typename T> __device__ __forceinline__ uint32_t pack_raw2(float2 v);
template <> __device__ __forceinline__ uint32_t pack_raw2<__half>(float2 v)
{
    const __half2 h = __floats2half2_rn(v.x, v.y);
    return *reinterpret_cast<const uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t pack_raw2<__nv_bfloat16>(float2 v)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    return *reinterpret_cast<const uint32_t*>(&h);
}
template <typename T> __device__ __forceinline__ float2 unpack_raw2(uint32_t w);
template <> __device__ __forceinline__ float2 unpack_raw2<__half>(uint32_t w)
{
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
}
template <> __device__ __forceinline__ float2 unpack_raw2<__nv_bfloat16>(uint32_t w)
{
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// Pull in deviation form: s0* are plane-0 rows (rho*) r-1, r, r+1; sd* the
// same rows' deviations (laid out by dev_index with plane R); c the node column.
// f_a(x) = w_a rho*(x - e_a) + d_a(x - e_a), or, if x - e_a is solid,
// f*_opp(a)(x) = w_a rho*(x) + d_opp(a)(x); f_0 = w_0 rho*(x) - sum_b d_b(x).
// n.g (tau != 1 only) is in raw units.
template <typename T, int R>
__device__ __forceinline__ void pull_dev(const float* __restrict__ s0m, const float* __restrict__ s0c,
                                         const float* __restrict__ s0p, const T* __restrict__ sdm,
                                         const T* __restrict__ sdc, const T* __restrict__ sdp, int c,
                                         bool need_g, PulledDev& n)
{
    constexpr float U = RawScale<T>::unscale, S = RawScale<T>::scale;
    const float r0 = s0c[c];
    n.solid = is_solid(r0);
    if (n.solid) {
        n.rho = n.jx = n.jy = 0.f;
        n.sb = 0;
        return;
    }
    auto dv = [](const T* sd, int col, int a) { return to_raw(sd[dev_index<T>(size_t(col), a, size_t(R))]); };
    // The 8 sources in four lane pairs (lane x an axis direction, lane y a
    // diagonal one): (1, 5), (3, 7), (2, 6), (4, 8), so that each sum below
    // runs its two halves in the two lanes.
    float2 rA = make_float2(s0c[c - 1], s0m[c - 1]);  // rho* at the sources of e1: (x-1, y), e5: (x-1, y-1)
    float2 rB = make_float2(s0c[c + 1], s0p[c + 1]);  // e3: (x+1, y), e7: (x+1, y+1)
    float2 rC = make_float2(s0m[c], s0m[c + 1]);      // e2: (x, y-1), e6: (x+1, y-1)
    float2 rD = make_float2(s0p[c], s0p[c - 1]);      // e4: (x, y+1), e8: (x-1, y+1)
    float2 dA = make_float2(dv(sdc, c - 1, 1), dv(sdm, c - 1, 5));
    float2 dB = make_float2(dv(sdc, c + 1, 3), dv(sdp, c + 1, 7));
    float2 dC = make_float2(dv(sdm, c, 2), dv(sdm, c + 1, 6));
    float2 dD = make_float2(dv(sdp, c, 4), dv(sdp, c - 1, 8));
    float own[9];
    if constexpr (sizeof(T) == 2) {
        // the node's own 8 deviations: one 16-byte load, paired conversions
        const uint4 qv = *reinterpret_cast<const uint4*>(sdc + size_t(c) * 8);
        const uint32_t w[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 v = unpack_raw2<T>(w[k]);
            own[2 * k + 1] = v.x;
            own[2 * k + 2] = v.y;
        }
    } else {
#pragma unroll
        for (int b = 1; b < 9; ++b) own[b] = dv(sdc, c, b);
    }
    const float2 r0s = splat(r0);
    float2 qa = sub2(rA, r0s), qb = sub2(rB, r0s), qc = sub2(rC, r0s), qd = sub2(rD, r0s);
    // (q1, q2) = sums of rho*_src - rho*(x) over the axis and the diagonal links
    float2 q = add2(add2(qa, qb), add2(qc, qd));
    uint32_t sb = 0;
    // a solid source holds a NaN sentinel in plane 0: only a NaN sum (a
    // wall nearby, or a state gone non-finite) takes the per-direction checks
    if (isnan(q.x + q.y)) {
        constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        float rs[9] = {0.f, rA.x, rC.x, rB.x, rD.x, rA.y, rC.y, rB.y, rD.y};
        float d[9] = {0.f, dA.x, dC.x, dB.x, dD.x, dA.y, dC.y, dB.y, dD.y};
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            if (is_solid(rs[a])) {  // half-way bounce-back: the node's own f*_opp(a)
                sb |= 1u << a;
                rs[a] = r0;
                d[a] = own[opp[a]];
            }
        }
        rA = make_float2(rs[1], rs[5]); rB = make_float2(rs[3], rs[7]);
        rC = make_float2(rs[2], rs[6]); rD = make_float2(rs[4], rs[8]);
        dA = make_float2(d[1], d[5]); dB = make_float2(d[3], d[7]);
        dC = make_float2(d[2], d[6]); dD = make_float2(d[4], d[8]);
        qa = sub2(rA, r0s); qb = sub2(rB, r0s); qc = sub2(rC, r0s); qd = sub2(rD, r0s);
        q = add2(add2(qa, qb), add2(qc, qd));
    }
    constexpr float w1 = 1.f / 9.f, w2 = 1.f / 36.f;
    // rho - rho*(x) = sum_a w_a (rho*_src - rho*(x)) + sum_a d_a(src) - sum_b d_b(x)
    const float2 ds = add2(add2(dA, dB), add2(dC, dD));
    const float2 dn = add2(add2(make_float2(own[1], own[5]), make_float2(own[3], own[7])),
                           add2(make_float2(own[2], own[6]), make_float2(own[4], own[8])));
    const float dsrc = ds.x + ds.y, down = dn.x + dn.y;
    const float drho = fmaf(w1, q.x, fmaf(w2, q.y, (dsrc - down) * U));
    n.rho = r0 + drho;
    // rho u: (jx, jy) in the two lanes; e_r = (rho*_1 - rho*_3, rho*_5 - rho*_7),
    // f_r = (rho*_2 - rho*_4, rho*_6 - rho*_8), the same for the deviations
    const float2 er = sub2(rA, rB), fr = sub2(rC, rD), ed = sub2(dA, dB), fd = sub2(dC, dD);
    float2 jd = make_float2((ed.x + ed.y) - fd.y, (fd.x + ed.y) + fd.y);
    if constexpr (U != 1.f) jd = mul2(jd, splat(U));
    const float2 j = fma2(splat(w1), make_float2(er.x, fr.x),
                          fma2(splat(w2), make_float2(er.y - fr.y, er.y + fr.y), jd));
    n.jx = j.x;
    n.jy = j.y;
    // g_a = f_a - w_a rho = w_a ((rho*_src - rho*(x)) - drho) + d_a(src), in
    // raw units; only the relaxation with tau != 1 reads it
    if (need_g) {
        const float2 wS = make_float2(w1 * S, w2 * S), dr = splat(drho);
        const float2 gA = fma2(wS, sub2(qa, dr), dA), gB = fma2(wS, sub2(qb, dr), dB);
        const float2 gC = fma2(wS, sub2(qc, dr), dC), gD = fma2(wS, sub2(qd, dr), dD);
        n.g[1] = gA.x; n.g[5] = gA.y; n.g[3] = gB.x; n.g[7] = gB.y;
        n.g[2] = gC.x; n.g[6] = gC.y; n.g[4] = gD.x; n.g[8] = gD.y;
    }
    n.g[0] = 0.f;
    n.sb = sb;
}

// Collision in deviation form: stores rho in plane 0 and the raw
// d*_a = f*_a - w_a rho after it (the equilibrium's deviation part
// w_a rho (3 c + 4.5 c^2 - 1.5 u^2) is formed without its leading 1). For
// FP32 deviations every operation is the two-node kernel's
// (collide_dev_pair) lane for lane.
template <int MODE, typename T, bool T1>
__device__ __forceinline__ void collide_dev(const PulledDev& n, const float* pm, const float* pc,
                                            const float* pp, int t, const Phys& p, const Geom& g,
                                            float* __restrict__ fout0, T* __restrict__ foutd,
                                            double* __restrict__ fields, int x, int r, ObsAcc& acc)
{
    const float2 F = node_force(n, pm, pc, pp, t, p);
    const float rinv = rcp_approx(n.rho);
    if constexpr (MODE == kStep || MODE == kStepObs) {
        // lane pairs as in collide_node; q[k] holds d*_(2k+1) and d*_(2k+2)
        const float2 u = div2(fma2(splat(p.tau), F, make_float2(n.jx, n.jy)), splat(-n.rho), splat(rinv));
        const float nusq = __fmul_rn(-1.5f, fmaf(u.x, u.x, __fmul_rn(u.y, u.y)));
        // power-of-two scaling to raw units: exact
        const float w1r = __fmul_rn(div1(n.rho, -9.f, 1.f / 9.f), RawScale<T>::scale);
        const float w2r = __fmul_rn(0.25f, w1r);
        const float2 dg = make_float2(__fadd_rn(u.x, u.y), __fsub_rn(u.y, u.x));  // e5.u, e6.u
        const float2 nus = splat(nusq);
        auto dpolyp = [nus](float2 c) { return fma2(c, fma2(splat(4.5f), c, splat(3.f)), nus); };
        auto dpolym = [nus](float2 c) { return fma2(c, fma2(splat(4.5f), c, splat(-3.f)), nus); };
        float2 q[4];
        q[0] = mul2(splat(w1r), dpolyp(u));
        q[1] = mul2(splat(w1r), dpolym(u));
        q[2] = mul2(splat(w2r), dpolyp(dg));
        q[3] = mul2(splat(w2r), dpolym(dg));
        if (!T1 && p.tau != 1.f) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float ga = n.g[2 * k + 1], gb = n.g[2 * k + 2];
                q[k] = make_float2(fmaf(__fsub_rn(q[k].x, ga), p.inv_tau, ga), fmaf(__fsub_rn(q[k].y, gb), p.inv_tau, gb));
            }
        }
        const int o = r * g.pitch + x;
        fout0[o] = n.rho;
        if constexpr (sizeof(T) == 2) {
            // the node's 8 deviations in one 16-byte store; each paired
            // conversion rounds both values to nearest, each as alone
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) w[k] = pack_raw2<T>(q[k]);
            *reinterpret_cast<uint4*>(foutd + size_t(o) * 8) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                foutd[(2 * k) * g.plane + o] = q[k].x;
                foutd[(2 * k + 1) * g.plane + o] = q[k].y;
            }
        }
    }
    if constexpr (MODE != kStep) node_observe<MODE>(n.rho, rinv, n.jx, n.jy, F.x, F.y, g, fields, x, r, acc);
}

// ------------------------------------------------------------------ node pairs (32-bit forms)
//
// A consumer thread of the 32-bit forms owns two neighbouring columns, A at
// staged column c (even) and B at c + 1, and carries their arithmetic in the
// two lanes of float2 values. Each node's arithmetic is the single-node
// arithmetic above, operation for operation; only the sources that lie on
// 8-byte boundaries come in one 64-bit shared-memory load (plane 0, 2 and 4
// and the node's own values), and both nodes store with one 64-bit store per
// plane.

struct Pulled2 {
    float2 f[9];
    float2 rho, jx, jy;
    uint32_t sb[2];  // per lane: bit a set <=> the pull source x - e_a is solid
    bool solid[2];   // per lane: solid node (B also when it lies past the pulled columns)
};

struct PulledDev2 {
    float2 rho, jx, jy;
    float2 g[9];     // f_a - w_a rho (a = 1..8, only with tau != 1)
    uint32_t sb[2];
    bool solid[2];
};

// Plain pull of the pair (c, c + 1) from the ring rows sm, sc, sp (see
// pull_smem); b_ok = false marks lane B as unused.
__device__ __forceinline__ void pull_pair(const float* __restrict__ sm, const float* __restrict__ sc,
                                          const float* __restrict__ sp, int c, bool b_ok, Pulled2& n)
{
    constexpr int R = kRowLen;
    const float2 v0 = ld2(sc + c);
    n.solid[0] = is_solid(v0.x);
    n.solid[1] = !b_ok || is_solid(v0.y);
    n.sb[0] = n.sb[1] = 0;
    if (n.solid[0] && n.solid[1]) {
        n.rho = n.jx = n.jy = splat(0.f);
        return;
    }
    float2 v[9];
    v[0] = v0;
    v[1] = make_float2(sc[1 * R + c - 1], sc[1 * R + c]);      // e1: source (x-1, y)
    v[2] = ld2(sm + 2 * R + c);                                 // e2: source (x, y-1)
    v[3] = make_float2(sc[3 * R + c + 1], sc[3 * R + c + 2]);  // e3: source (x+1, y)
    v[4] = ld2(sp + 4 * R + c);                                 // e4: source (x, y+1)
    v[5] = make_float2(sm[5 * R + c - 1], sm[5 * R + c]);      // e5: source (x-1, y-1)
    v[6] = make_float2(sm[6 * R + c + 1], sm[6 * R + c + 2]);  // e6: source (x+1, y-1)
    v[7] = make_float2(sp[7 * R + c + 1], sp[7 * R + c + 2]);  // e7: source (x+1, y+1)
    v[8] = make_float2(sp[8 * R + c - 1], sp[8 * R + c]);      // e8: source (x-1, y+1)
    auto density = [&v]() {
        return add2(add2(add2(v[0], add2(v[1], v[3])), add2(v[2], v[4])), add2(add2(v[5], v[7]), add2(v[6], v[8])));
    };
    float2 rho = density();
    const bool nan_a = !n.solid[0] && isnan(rho.x), nan_b = !n.solid[1] && isnan(rho.y);
    if (nan_a || nan_b) {
        constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            if (nan_a && is_solid(v[a].x)) {
                n.sb[0] |= 1u << a;
                v[a].x = sc[opp[a] * R + c];  // half-way bounce-back
            }
            if (nan_b && is_solid(v[a].y)) {
                n.sb[1] |= 1u << a;
                v[a].y = sc[opp[a] * R + c + 1];
            }
        }
        rho = density();
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) n.f[a] = v[a];
    n.rho = rho;
    n.jx = add2(add2(sub2(v[1], v[3]), sub2(v[5], v[7])), sub2(v[8], v[6]));
    n.jy = add2(add2(sub2(v[2], v[4]), sub2(v[5], v[7])), sub2(v[6], v[8]));
}

// Deviation-form pull of the pair (FP32 deviations; see pull_dev). The
// node's own deviations are one 64-bit load per plane; B's east source is
// A's own d_1 and A's west source is B's own d_3.
__device__ __forceinline__ void pull_dev_pair(const float* __restrict__ s0m, const float* __restrict__ s0c,
                                              const float* __restrict__ s0p, const float* __restrict__ sdm,
                                              const float* __restrict__ sdc, const float* __restrict__ sdp, int c,
                                              bool b_ok, bool need_g, PulledDev2& n)
{
    constexpr int R = kRowLen;
    const float2 r0 = ld2(s0c + c);
    n.solid[0] = is_solid(r0.x);
    n.solid[1] = !b_ok || is_solid(r0.y);
    n.sb[0] = n.sb[1] = 0;
    if (n.solid[0] && n.solid[1]) {
        n.rho = n.jx = n.jy = splat(0.f);
        return;
    }
    const float2 mM = ld2(s0m + c), pM = ld2(s0p + c);
    float2 rs[9], d[9], own[9];
    rs[1] = make_float2(s0c[c - 1], r0.x);
    rs[2] = mM;
    rs[3] = make_float2(r0.y, s0c[c + 2]);
    rs[4] = pM;
    rs[5] = make_float2(s0m[c - 1], mM.x);
    rs[6] = make_float2(mM.y, s0m[c + 2]);
    rs[7] = make_float2(pM.y, s0p[c + 2]);
    rs[8] = make_float2(s0p[c - 1], pM.x);
#pragma unroll
    for (int b = 1; b < 9; ++b) own[b] = ld2(sdc + (b - 1) * R + c);
    d[1] = make_float2(sdc[0 * R + c - 1], own[1].x);
    d[2] = ld2(sdm + 1 * R + c);
    d[3] = make_float2(own[3].y, sdc[2 * R + c + 2]);
    d[4] = ld2(sdp + 3 * R + c);
    d[5] = make_float2(sdm[4 * R + c - 1], sdm[4 * R + c]);
    d[6] = make_float2(sdm[5 * R + c + 1], sdm[5 * R + c + 2]);
    d[7] = make_float2(sdp[6 * R + c + 1], sdp[6 * R + c + 2]);
    d[8] = make_float2(sdp[7 * R + c - 1], sdp[7 * R + c]);
    auto qsum = [&rs, r0](float2& q1, float2& q2) {
        q1 = add2(add2(sub2(rs[1], r0), sub2(rs[3], r0)), add2(sub2(rs[2], r0), sub2(rs[4], r0)));
        q2 = add2(add2(sub2(rs[5], r0), sub2(rs[7], r0)), add2(sub2(rs[6], r0), sub2(rs[8], r0)));
    };
    float2 q1, q2;
    qsum(q1, q2);
    const bool nan_a = !n.solid[0] && isnan(q1.x + q2.x), nan_b = !n.solid[1] && isnan(q1.y + q2.y);
    if (nan_a || nan_b) {
        constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
        for (int a = 1; a < 9; ++a) {
            if (nan_a && is_solid(rs[a].x)) {  // half-way bounce-back: the node's own f*_opp(a)
                n.sb[0] |= 1u << a;
                rs[a].x = r0.x;
                d[a].x = own[opp[a]].x;
            }
            if (nan_b && is_solid(rs[a].y)) {
                n.sb[1] |= 1u << a;
                rs[a].y = r0.y;
                d[a].y = own[opp[a]].y;
            }
        }
        qsum(q1, q2);
    }
    const float2 w1 = splat(1.f / 9.f), w2 = splat(1.f / 36.f);
    const float2 dsrc = add2(add2(add2(d[1], d[3]), add2(d[2], d[4])), add2(add2(d[5], d[7]), add2(d[6], d[8])));
    const float2 down =
        add2(add2(add2(own[1], own[3]), add2(own[2], own[4])), add2(add2(own[5], own[7]), add2(own[6], own[8])));
    const float2 drho = fma2(w1, q1, fma2(w2, q2, sub2(dsrc, down)));
    n.rho = add2(r0, drho);
    n.jx = fma2(w1, sub2(rs[1], rs[3]),
                fma2(w2, add2(sub2(rs[5], rs[7]), sub2(rs[8], rs[6])),
                     add2(add2(sub2(d[1], d[3]), sub2(d[5], d[7])), sub2(d[8], d[6]))));
    n.jy = fma2(w1, sub2(rs[2], rs[4]),
                fma2(w2, add2(sub2(rs[5], rs[7]), sub2(rs[6], rs[8])),
                     add2(add2(sub2(d[2], d[4]), sub2(d[5], d[7])), sub2(d[6], d[8]))));
    if (need_g) {
#pragma unroll
        for (int a = 1; a < 9; ++a) n.g[a] = fma2(a <= 4 ? w1 : w2, sub2(sub2(rs[a], r0), drho), d[a]);
    }
    n.g[0] = splat(0.f);
}

// Total force on the pair (see node_force): psi ring rows pm, pc, pp with
// node A at ring column t (even) and B at t + 1.
__device__ __forceinline__ void node_force2(float2 rho, const uint32_t (&sb)[2], const float* pm, const float* pc,
                                            const float* pp, int t, const Phys& p, float2& Fx_out, float2& Fy_out)
{
    const float2 cM = ld2(pc + t), mM = ld2(pm + t), pM = ld2(pp + t);
    const float cL = pc[t - 1], cR = pc[t + 2], mL = pm[t - 1], mR = pm[t + 2], pL = pp[t - 1], pR = pp[t + 2];
    // lane A's left/right neighbours are (L, M.y), lane B's (M.x, R)
    const float2 dxc = make_float2(cM.y - cL, cR - cM.x);
    const float2 dxp = make_float2(pM.y - pL, pR - pM.x), dxm = make_float2(mM.y - mL, mR - mM.x);
    const float2 sxp = make_float2(pM.y + pL, pR + pM.x), sxm = make_float2(mM.y + mL, mR + mM.x);
    // Eq. 5: -sum_a G_a psi(x+e_a) e_a, the sign carried by the constants
    // (round to nearest is symmetric, so this is exactly the negated sum)
    const float2 nsgx = fma2(splat(-p.g_axis), dxc, mul2(splat(-p.g_diag), add2(dxp, dxm)));
    const float2 nsgy = fma2(splat(-p.g_axis), sub2(pM, mM), mul2(splat(-p.g_diag), sub2(sxp, sxm)));
    const float2 psi = cM;
    float2 Fx = mul2(psi, nsgx), Fy = mul2(psi, nsgy);
    if ((sb[0] | sb[1]) != 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (sb[k] == 0) continue;
            float fx, fy;
            wall_electric(sb[k], lane_of(psi, k), lane_of(nsgx, k), lane_of(nsgy, k), lane_of(rho, k), p, fx, fy);
            set_lane(Fx, k, fx);
            set_lane(Fy, k, fy);
        }
    }
    // body force on every fluid node
    Fx_out = fma2(rho, splat(p.bfx), Fx);
    Fy_out = fma2(rho, splat(p.bfy), Fy);
}

// Observables / fields epilogue of the lanes that are collided fluid nodes:
// node_observe lane for lane, the velocities and sums on the paired
// instructions (a lane that is not collided, or not finite, adds zero).
template <int MODE>
__device__ __forceinline__ void observe_pair(const float2& rho, const float2& rinv, const float2& jx,
                                             const float2& jy, const float2& Fx, const float2& Fy, const bool (&use)[2],
                                             const Geom& g, double* __restrict__ fields, int x, int r, ObsAcc2& acc)
{
    if constexpr (MODE == kFields) {
        ObsAcc unused;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (use[k])
                node_observe<MODE>(lane_of(rho, k), lane_of(rinv, k), lane_of(jx, k), lane_of(jy, k),
                                   lane_of(Fx, k), lane_of(Fy, k), g, fields, x + k, r, unused);
    } else {
        // physical velocity u = (rho u + F/2)/rho
        const float2 mx = fma2(splat(0.5f), Fx, jx), my = fma2(splat(0.5f), Fy, jy);
        const float2 nrho = make_float2(-rho.x, -rho.y);
        const float2 vx = div2(mx, nrho, rinv), vy = div2(my, nrho, rinv);
        const float2 u2 = fma2(vx, vx, mul2(vy, vy));
        bool ok[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            // a NaN or infinity in any of the three makes the sum non-finite
            ok[k] = use[k] && isfinite((lane_of(rho, k) + lane_of(vx, k)) + lane_of(vy, k));
            if (use[k] && !ok[k]) ++acc.bad;
            if (ok[k]) {
                acc.umax2 = fmaxf(acc.umax2, lane_of(u2, k));
                acc.rmin = fminf(acc.rmin, lane_of(rho, k));
            }
        }
        auto sel = [&ok](float2 v) { return make_float2(ok[0] ? v.x : 0.f, ok[1] ? v.y : 0.f); };
        acc.mass.add(sel(rho));
        acc.q.add(sel(vx));
        acc.px.add(sel(mx));
        acc.py.add(sel(my));
    }
}

// Shifted velocity (Eq. 10) of the pair from its force; rinv = 1/rho (approx).
__device__ __forceinline__ void shifted_velocity(const float2& rho, const float2& jx, const float2& jy,
                                                 const float2& Fx, const float2& Fy, const float2& rinv,
                                                 const Phys& p, float2& ux, float2& uy)
{
    const float2 nrho = make_float2(-rho.x, -rho.y);
    ux = div2(fma2(splat(p.tau), Fx, jx), nrho, rinv);
    uy = div2(fma2(splat(p.tau), Fy, jy), nrho, rinv);
}

// Forces, velocity shift, collision and store of a pair in plain storage
// (see collide_node); col[k]: lane k is a fluid node this CTA collides. Lane
// A is column x. Both lanes collided and fluid: one 64-bit store per plane.
template <int MODE, bool T1>
__device__ __forceinline__ void collide_pair(const Pulled2& n, const bool (&col)[2], const float* pm, const float* pc,
                                             const float* pp, int t, const Phys& p, const Geom& g,
                                             float* __restrict__ fout, double* __restrict__ fields, int x, int r,
                                             ObsAcc2& acc)
{
    float2 Fx, Fy;
    node_force2(n.rho, n.sb, pm, pc, pp, t, p, Fx, Fy);
    const float2 rinv = make_float2(rcp_approx(n.rho.x), rcp_approx(n.rho.y));
    if constexpr (MODE == kStep || MODE == kStepObs) {
        float2 ux, uy;
        shifted_velocity(n.rho, n.jx, n.jy, Fx, Fy, rinv, p, ux, uy);
        const float2 om = fma2(splat(-1.5f), fma2(ux, ux, mul2(uy, uy)), splat(1.f));
        const float2 r9 = div2(n.rho, splat(-9.f), splat(1.f / 9.f));
        const float2 w0r = mul2(splat(4.f), r9), w2r = mul2(splat(0.25f), r9);
        const float2 d5 = add2(ux, uy), d6 = sub2(uy, ux);
        // f_eq_a = w_a rho (1 + 3 c + 4.5 c^2 - 1.5 u^2) with c = +-(e_a . u):
        // (-c)(4.5(-c) + 3) = c (4.5 c - 3) exactly
        auto polyp = [om](float2 c) { return fma2(c, fma2(splat(4.5f), c, splat(3.f)), om); };
        auto polym = [om](float2 c) { return fma2(c, fma2(splat(4.5f), c, splat(-3.f)), om); };
        float2 fs[9];
        fs[0] = mul2(w0r, om);
        fs[1] = mul2(r9, polyp(ux));
        fs[2] = mul2(r9, polyp(uy));
        fs[3] = mul2(r9, polym(ux));
        fs[4] = mul2(r9, polym(uy));
        fs[5] = mul2(w2r, polyp(d5));
        fs[6] = mul2(w2r, polyp(d6));
        fs[7] = mul2(w2r, polym(d5));
        fs[8] = mul2(w2r, polym(d6));
        if (!T1 && p.tau != 1.f) {
#pragma unroll
            for (int a = 0; a < 9; ++a) fs[a] = fma2(sub2(fs[a], n.f[a]), splat(p.inv_tau), n.f[a]);
        }
        float* o = fout + r * g.pitch + x;
        if (col[0] && col[1]) {
#pragma unroll
            for (int a = 0; a < 9; ++a) *reinterpret_cast<float2*>(o + a * g.plane) = fs[a];
        } else {
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                if (col[0]) o[a * g.plane] = fs[a].x;
                if (col[1]) o[a * g.plane + 1] = fs[a].y;
            }
        }
    }
    if constexpr (MODE != kStep) observe_pair<MODE>(n.rho, rinv, n.jx, n.jy, Fx, Fy, col, g, fields, x, r, acc);
}

// The same in FP32 deviation storage (see collide_dev).
template <int MODE, bool T1>
__device__ __forceinline__ void collide_dev_pair(const PulledDev2& n, const bool (&col)[2], const float* pm,
                                                 const float* pc, const float* pp, int t, const Phys& p,
                                                 const Geom& g, float* __restrict__ fout0,
                                                 float* __restrict__ foutd, double* __restrict__ fields, int x,
                                                 int r, ObsAcc2& acc)
{
    float2 Fx, Fy;
    node_force2(n.rho, n.sb, pm, pc, pp, t, p, Fx, Fy);
    const float2 rinv = make_float2(rcp_approx(n.rho.x), rcp_approx(n.rho.y));
    if constexpr (MODE == kStep || MODE == kStepObs) {
        float2 ux, uy;
        shifted_velocity(n.rho, n.jx, n.jy, Fx, Fy, rinv, p, ux, uy);
        const float2 nusq = mul2(splat(-1.5f), fma2(ux, ux, mul2(uy, uy)));
        const float2 w1r = div2(n.rho, splat(-9.f), splat(1.f / 9.f));
        const float2 w2r = mul2(splat(0.25f), w1r);
        const float2 d5 = add2(ux, uy), d6 = sub2(uy, ux);
        auto dpolyp = [nusq](float2 c) { return fma2(c, fma2(splat(4.5f), c, splat(3.f)), nusq); };
        auto dpolym = [nusq](float2 c) { return fma2(c, fma2(splat(4.5f), c, splat(-3.f)), nusq); };
        float2 dq[9];
        dq[1] = mul2(w1r, dpolyp(ux));
        dq[2] = mul2(w1r, dpolyp(uy));
        dq[3] = mul2(w1r, dpolym(ux));
        dq[4] = mul2(w1r, dpolym(uy));
        dq[5] = mul2(w2r, dpolyp(d5));
        dq[6] = mul2(w2r, dpolyp(d6));
        dq[7] = mul2(w2r, dpolym(d5));
        dq[8] = mul2(w2r, dpolym(d6));
        if (!T1 && p.tau != 1.f) {
#pragma unroll
            for (int a = 1; a < 9; ++a) dq[a] = fma2(sub2(dq[a], n.g[a]), splat(p.inv_tau), n.g[a]);
        }
        const int o = r * g.pitch + x;
        if (col[0] && col[1]) {
            *reinterpret_cast<float2*>(fout0 + o) = n.rho;
#pragma unroll
            for (int a = 1; a < 9; ++a) *reinterpret_cast<float2*>(foutd + (a - 1) * g.plane + o) = dq[a];
        } else {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!col[k]) continue;
                fout0[o + k] = lane_of(n.rho, k);
#pragma unroll
                for (int a = 1; a < 9; ++a) foutd[(a - 1) * g.plane + o + k] = lane_of(dq[a], k);
            }
        }
    }
    if constexpr (MODE != kStep) observe_pair<MODE>(n.rho, rinv, n.jx, n.jy, Fx, Fy, col, g, fields, x, r, acc);
}

// ------------------------------------------------------------------ kernel

// f(std::integral_constant<int, J>) for J = 0, 1, ..., in order
template <typename F, int... J>
__device__ __forceinline__ void unroll_seq(std::integer_sequence<int, J...>, F&& f)
{
    (f(std::integral_constant<int, J>{}), ...);
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One CTA's work: a strip of columns of one domain and the segment of rows
// [by*tile_rows, (by+1)*tile_rows); per-CTA observables go to
// partials[slot]. smem_raw is the dynamic shared memory.
//
// Three layouts of the consumer threads (P = StoreT<ST>::overlap):
//  - P = 0, PAIR (32-bit forms, large domains, bound by DRAM): strips of kW
//    columns at x0 = bx*kW, kW/2 consumer threads, thread t owning the two
//    columns x0 + 2t and x0 + 2t + 1 (see the consumer section below);
//  - P = 0, one node per thread (32-bit forms, domains too small to fill the
//    GPU with pair CTAs, where twice the threads per CTA hide more latency):
//    thread t pulls and collides column x0 + t and writes its psi into ring
//    column t + 1; threads 0 and nint - 1 also pull the halo columns x0 - 1
//    and x0 + nint (ring columns 0 and nint + 1);
//  - P = 1 (16-bit forms, bound by instruction issue): strips of kW - 2
//    columns at x0 = bx*(kW-2). Thread t pulls column x0 - 1 + t into ring
//    column t, so the halo columns come from threads 0 and nint + 1 like
//    every other column and all consumer warps do the same work; threads
//    1 .. nint collide. Neighbouring strips overlap by two pulled columns.
// Warp stores cover whole 128-byte lines in the 32-bit layouts. In all three
// the producer warp only stages rows, running ahead of the consumers. The
// two 32-bit layouts store the same bits.
template <int MODE, int ST, bool T1, bool PAIR>
__device__ __forceinline__ void run_tile(const float* __restrict__ fin, float* __restrict__ fout, const Geom& g,
                                         const Phys& p, double* __restrict__ partials,
                                         double* __restrict__ fields, int* __restrict__ err, int bx, int by,
                                         int slot, unsigned char* smem_raw)
{
    using T = typename StoreT<ST>::T;
    constexpr int kStages = stages_of(ST, PAIR);
    constexpr int A = StoreT<ST>::align;
    constexpr int P = StoreT<ST>::overlap;
    constexpr bool PR = P == 0 && PAIR;  // the pair layout
    constexpr int R = kRowLen;
    constexpr size_t SB = stage_bytes<ST>();
    // ring stage s: plane 0 (FP32, R) then the deviations in the layout of
    // dev_index with plane = R (8 planes of R for FP32, 8 per node for 16 bits)
    float* psi_ring = reinterpret_cast<float*>(smem_raw + kStages * SB);            // [kStages][kPsiStride]
    uint64_t* full = reinterpret_cast<uint64_t*>(psi_ring + kStages * kPsiStride);  // [kStages]
    uint64_t* empty = full + kStages;                                         // [kStages]
    auto stage_ptr = [&](int s) { return smem_raw + size_t(s) * SB; };

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int x0 = bx * strip_cols(ST);
    const int nint = min(strip_cols(ST), g.nx - x0);  // columns collided: x0 .. x0 + nint - 1
    const int y0 = by * g.tile_rows;
    const int y1 = min(y0 + g.tile_rows, g.ny);
    const int nrows = (y1 - y0) + 4;                  // staged rows y0-2 .. y1+1
    // Staged window: global columns ws .. ws + L - 1 (periodic in x), with ws
    // the multiple of A at or below x0 - P - 1 and L a multiple of A, so that
    // the pulls of columns x0 - P .. x0 - P + kW - 1 (which read one column
    // more on each side) find their sources; node column x sits at staged
    // column x - ws, so thread t's node at t + 1 + o with o = x0 - P - 1 - ws.
    // P = 0: x0 is a multiple of kW, so o = A - 1 for every strip (a
    // compile-time offset). P = 1: x0 - 2 >= -2 is even and o <= A - 2.
    // L = kW + 2 + o rounded up to A <= kRowLen.
    const int o = P == 0 ? A - 1 : (x0 >= 2 ? (x0 - 2) % A : A - 2);
    const int ws = x0 - P - 1 - o;
    const int L = ((kW + 2 + o) + A - 1) / A * A;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 32);               // 32 producer-lane arrivals + tx bytes
            mbar_init(&empty[s], consumers(ST, PAIR) / 32);  // one arrival per consumer warp
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

    using PT = std::conditional_t<ST == kF32, Pulled, PulledDev>;
    constexpr int NC = consumers(ST, PAIR);
    constexpr int NCW = NC / 32;
    // the state of what a consumer thread pulls per row: a pair of nodes or one
    using PT2 = std::conditional_t<PR, std::conditional_t<ST == kF32, Pulled2, PulledDev2>, PT>;
    // pull the node in staged column col of the row held by stage bc, whose
    // neighbour rows are in stages bm (row - 1) and bp (row + 1)
    auto pull = [&](const unsigned char* bm, const unsigned char* bc, const unsigned char* bp, int col, PT& n) {
        const float* s0m = reinterpret_cast<const float*>(bm);
        const float* s0c = reinterpret_cast<const float*>(bc);
        const float* s0p = reinterpret_cast<const float*>(bp);
        if constexpr (ST == kF32) {
            pull_smem(s0m, s0c, s0p, col, n);
        } else {
            const T* sdm = reinterpret_cast<const T*>(bm + R * sizeof(float));
            const T* sdc = reinterpret_cast<const T*>(bc + R * sizeof(float));
            const T* sdp = reinterpret_cast<const T*>(bp + R * sizeof(float));
            pull_dev<T, R>(s0m, s0c, s0p, sdm, sdc, sdp, col, !T1 && p.tau != 1.f, n);
        }
    };
    float* psi_w = psi_ring;

    if (warp == NCW) {
        // ---------------- producer warp: fill ring stages with rows y0-2 .. y1+1
        bool ok = true;
        // Staged row k goes to stage k % kStages.
        if constexpr (P == 0) {
            // 32-bit planes, strips at multiples of kW. Interior strips (the
            // window x0-4 .. x0+nint+4 inside [0, nx) and a 16-byte multiple
            // wide) take one bulk copy per plane row; edge and ragged strips
            // copy the aligned body in bulk and fetch the remaining <= 11
            // columns per plane with 4-byte cp.async (each lane's column is
            // fixed for the whole segment). The producer runs ahead on its
            // own, refilling each stage as soon as the consumers free it.
            constexpr int H = A;                                 // staged columns left of x0 (o = H - 1)
            const int nbody = nint & ~3;                         // columns moved by the bulk copies
            const bool whole = (x0 >= H) && (x0 + nint + H <= g.nx) && ((nint & 3) == 0);
            const int b_col = whole ? -H : 0;                    // first bulk column (rel. x0)
            const int b_len = whole ? nint + 2 * H : nbody;      // bulk columns
            const uint32_t b_bytes = uint32_t(b_len) * sizeof(float);
            const int n_right = nint + H - nbody;                // columns [x0+nbody, x0+nint+4)
            const int n_scalar = whole ? 0 : H + n_right;        // <= 11
            int my_sc = 0, my_gx = 0;
            const bool has_scalar = lane < n_scalar;
            if (has_scalar) {
                const int col = (lane < H) ? (lane - H) : (nbody + (lane - H));
                my_sc = H + col;
                my_gx = wrap_x(x0 + col);
            }
            auto fill = [&](int k) {
                const int s = k % kStages;
                const int row = wrap_y(y0 - 2 + k);
                float* st = reinterpret_cast<float*>(stage_ptr(s));
                const float* src = fin + size_t(row) * g.pitch;
                if (lane == 0 && b_len > 0) {
                    mbar_expect_tx(&full[s], 9 * b_bytes);
#pragma unroll 1
                    for (int a = 0; a < 9; ++a)
                        bulk_g2s(st + a * R + H + b_col, src + size_t(a) * g.plane + x0 + b_col, b_bytes,
                                 &full[s]);
                }
                if (has_scalar) {
#pragma unroll
                    for (int a = 0; a < 9; ++a) async_g2s_4(st + a * R + my_sc, src + size_t(a) * g.plane + my_gx);
                }
                async_arrive_noinc(&full[s]);
            };
            for (int k = 0; k < nrows; ++k) {
                if (k >= kStages) ok = mbar_wait(&empty[k % kStages], ((k / kStages) - 1) & 1, err) && ok;
                fill(k);
            }
        } else {
            // 16-bit deviations (nx % 8 == 0): the window splits at the
            // periodic seam into pieces that start and end on 16-byte
            // boundaries, the same for every row; lane l moves pieces l,
            // l + 32, ... with two cp.async.bulk copies each (plane 0 and the
            // node-interleaved deviations). The producer runs ahead on its
            // own, as above.
            const uint32_t tx = uint32_t(L) * uint32_t(sizeof(float) + 8 * sizeof(T));
            const T* dbase = reinterpret_cast<const T*>(fin + g.plane);
            // piece q covers window positions [max(ws, (m0+q) nx), min(ws+L, (m0+q+1) nx))
            const int m0 = ws >= 0 ? ws / g.nx : -((-ws + g.nx - 1) / g.nx);
            const int npieces = (ws + L - 1 - m0 * g.nx) / g.nx + 1;
            auto piece = [&](int q, int& j, int& gx, int& len) {
                const int base = (m0 + q) * g.nx;
                const int start = max(ws, base), end = min(ws + L, base + g.nx);
                j = start - ws;
                gx = start - base;
                len = end - start;
            };
            int pj = 0, pgx = 0, plen = 0;  // this lane's first piece
            if (lane < npieces) piece(lane, pj, pgx, plen);
            // plane 0 and the node-interleaved deviations (16 bytes a node)
            auto copy_piece = [&](float* s0, int row, int j, int gx, int len, uint64_t* bar) {
                T* sd = reinterpret_cast<T*>(s0 + R);
                const float* g0 = fin + size_t(row) * g.pitch;
                const T* gd = dbase + size_t(row) * g.pitch * 8;
                bulk_g2s(s0 + j, g0 + gx, uint32_t(len) * 4u, bar);
                bulk_g2s(sd + size_t(j) * 8, gd + size_t(gx) * 8, uint32_t(len) * 16u, bar);
            };
            auto fill = [&](int k) {
                const int s = k % kStages;
                int row = y0 - 2 + k;
                if (row < 0 || row >= g.ny) row = wrap_y(row);
                float* s0 = reinterpret_cast<float*>(stage_ptr(s));
                if (lane == 0) mbar_expect_tx(&full[s], tx);
                __syncwarp();
                if (lane < npieces) copy_piece(s0, row, pj, pgx, plen, &full[s]);
                for (int q = lane + 32; q < npieces; q += 32) {  // windows wider than 31 domain widths
                    int j, gx, len;
                    piece(q, j, gx, len);
                    copy_piece(s0, row, j, gx, len, &full[s]);
                }
                async_arrive_noinc(&full[s]);
            };
            for (int k = 0; k < nrows; ++k) {
                if (k >= kStages) ok = mbar_wait(&empty[k % kStages], ((k / kStages) - 1) & 1, err) && ok;
                fill(k);
            }
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
    // P = 1: thread t pulls node column x0 - 1 + t (staged column t + 1 + o,
    // psi ring column t) and collides it if it lies inside the strip.
    // P = 0, one node: thread t pulls column x0 + t (staged column t + 1 + o,
    // ring column t + 1) and collides it if it lies inside the strip.
    // P = 0, pairs: thread t owns the pair of columns x0 + 2t (lane A) and
    // x0 + 2t + 1 (lane B): staged columns c, c + 1 with c = 2t + 1 + o
    // (even, as o = 3), psi ring columns 2t + 2 and 2t + 3. The pulled
    // columns are x0 .. x0 + nint, the last one being the right halo; the left
    // halo x0 - 1 (ring column 1) is one extra pull by thread 0, and a full
    // strip's right halo x0 + kW (ring column kW + 2) one by the last thread.
    const int t = tid;
    const int np = nint + 1;                                       // pairs: pulled columns
    const bool active = PR ? 2 * t < np : P == 0 ? t < nint : t < nint + 2;  // pulls something
    const bool b_ok = 2 * t + 1 < np;                               // pairs: lane B pulled
    const bool col_a = PR ? 2 * t < nint : P == 0 ? t < nint : (t >= 1 && t <= nint);
    const bool col_b = 2 * t + 1 < nint;                            // pairs: lane B collided
    const bool halo_r = PR && t == NC - 1 && np > 2 * NC;
    const int c = PR ? 2 * t + 1 + o : t + 1 + o;                  // staged column (of lane A)
    const int x = PR ? x0 + 2 * t : x0 - P + t;
    const int tr = PR ? 2 * t + 2 : t + 1 - P;                     // psi ring column (of lane A)
    std::conditional_t<PR, ObsAcc2, ObsAcc> acc;
    bool ok = true;
    // prologue: the two oldest staged rows (y0-2, y0-1) must be present
    // (a segment stages at least 5 rows)
    ok = mbar_wait(&full[0], 0, err) && ok;
    ok = mbar_wait(&full[1], 0, err) && ok;

    auto psi_of = [&](bool solid, float rho) { return solid ? 0.f : -p.rho0 * expm1f(-rho * p.inv_rho0); };
    // all-zero fields of the collided solid lanes (kFields)
    auto zero_fields = [&](int xs, int rs) {
        const size_t i = (size_t)rs * g.nx + xs, nn = (size_t)g.nx * g.ny;
        fields[i] = 0.0;
        fields[nn + i] = 0.0;
        fields[2 * nn + i] = 0.0;
    };

    // Row k: pull row r = y0 - 2 + k (staged rows k-1, k, k+1, in stages
    // s_m, s_c, s_p; row k+1 filled in phase ph_p) into `into`, then collide
    // row r - 1, pulled at row k - 1 into `prev`. Staged row k sits in stage
    // k % kStages and its psi in the psi ring row of the same index.
    auto body = [&](int k, PT2& into, const PT2& prev, int s_m, int s_c, int s_p, uint32_t ph_p) {
        const int r = y0 - 2 + k;
        const unsigned char* b_m = stage_ptr(s_m);
        const unsigned char* b_c = stage_ptr(s_c);
        const unsigned char* b_p = stage_ptr(s_p);
        ok = mbar_wait(&full[s_p], ph_p, err) && ok;
        float* prow = psi_w + s_c * kPsiStride;
        if (active) {
            if constexpr (PR) {
                const float* s0m = reinterpret_cast<const float*>(b_m);
                const float* s0c = reinterpret_cast<const float*>(b_c);
                const float* s0p = reinterpret_cast<const float*>(b_p);
                if constexpr (ST == kF32)
                    pull_pair(s0m, s0c, s0p, c, b_ok, into);
                else
                    pull_dev_pair(s0m, s0c, s0p, s0m + R, s0c + R, s0p + R, c, b_ok, !T1 && p.tau != 1.f, into);
                *reinterpret_cast<float2*>(prow + tr) =
                    make_float2(psi_of(into.solid[0], into.rho.x), psi_of(into.solid[1], into.rho.y));
                if (t == 0) {  // left halo column x0 - 1
                    PT h;
                    pull(b_m, b_c, b_p, c - 1, h);
                    prow[1] = pseudopotential(p, h);
                }
                if (halo_r) {  // right halo column x0 + kW
                    PT h;
                    pull(b_m, b_c, b_p, c + 2, h);
                    prow[tr + 2] = pseudopotential(p, h);
                }
            } else {
                pull(b_m, b_c, b_p, c, into);
                prow[tr] = pseudopotential(p, into);
                if constexpr (P == 0) {
                    if (t == 0) {  // left halo column x0 - 1
                        PT h;
                        pull(b_m, b_c, b_p, c - 1, h);
                        prow[tr - 1] = pseudopotential(p, h);
                    }
                    if (t == nint - 1) {  // right halo column x0 + nint
                        PT h;
                        pull(b_m, b_c, b_p, c + 1, h);
                        prow[tr + 1] = pseudopotential(p, h);
                    }
                }
            }
        }
        consumer_sync<NC>();
        // staged row k-1 is no longer needed by any consumer
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s_m]);
        if (k >= 3) {
            // collide row r-1 with psi rows r-2, r-1, r
            const int rc = r - 1;
            const float* pm = psi_w + (s_m == 0 ? kStages - 1 : s_m - 1) * kPsiStride;
            const float* pc = psi_w + s_m * kPsiStride;
            const float* pp = psi_w + s_c * kPsiStride;
            if constexpr (PR) {
                const bool col[2] = {col_a && !prev.solid[0], col_b && !prev.solid[1]};
                if (col[0] || col[1]) {
                    if constexpr (ST == kF32)
                        collide_pair<MODE, T1>(prev, col, pm, pc, pp, tr, p, g, fout, fields, x, rc, acc);
                    else
                        collide_dev_pair<MODE, T1>(prev, col, pm, pc, pp, tr, p, g, fout, fout + g.plane, fields, x,
                                               rc, acc);
                }
                if constexpr (MODE == kFields) {
                    if (col_a && prev.solid[0]) zero_fields(x, rc);
                    if (col_b && prev.solid[1]) zero_fields(x + 1, rc);
                }
            } else {
                if (col_a && !prev.solid) {
                    if constexpr (ST == kF32)
                        collide_node<MODE, T1>(prev, pm, pc, pp, tr, p, g, fout, fields, x, rc, acc);
                    else
                        collide_dev<MODE, T, T1>(prev, pm, pc, pp, tr, p, g, fout,
                                                 reinterpret_cast<T*>(fout + g.plane), fields, x, rc, acc);
                } else if constexpr (MODE == kFields) {
                    if (col_a) zero_fields(x, rc);
                }
            }
        }
    };

    // two pulled-state register sets used in turn, so that no copy is made
    PT2 n0, n1;
    if constexpr (PR) {
        n0.solid[0] = n0.solid[1] = n1.solid[0] = n1.solid[1] = true;
    } else {
        n0.solid = n1.solid = true;
    }
    const int kmax = nrows - 2;
    if constexpr (is16(ST) && MODE == kStep) {
    // The plain step of the 16-bit forms (bound by instruction issue) unrolls the row loop by
    // U rows, a multiple of the ring depth and even: every stage index,
    // mbarrier address, psi ring row and register set is a compile-time
    // constant; the fill phase of row k+1 is that of the iteration
    // (U = kStages) or a constant (U = 2 kStages). Measured at 16384x4096:
    // 110.7 / 112.0 GLUPS (FP16 / BF16) against 102.9 / 104.5 rolled. The
    // 32-bit forms keep the rolled loop: unrolled, the pair kernels lost
    // 2-3% (FP32, 4 rows) and 60% (FP32 deviations, 10 rows of code).
    constexpr int U = (kStages % 2 == 0) ? kStages : 2 * kStages;
    uint32_t it = 0;
    for (int k0 = 1; k0 <= kmax; k0 += U) {
        unroll_seq(std::make_integer_sequence<int, U>{}, [&](auto jc) {
            constexpr int J = decltype(jc)::value;
            constexpr int sm = J % kStages, sc = (J + 1) % kStages, sp = (J + 2) % kStages;
            const uint32_t ph = (U == kStages ? it : 0u) ^ uint32_t(((J + 2) / kStages) & 1);
            if (k0 + J <= kmax) {
                if constexpr (J % 2 == 0)
                    body(k0 + J, n0, n1, sm, sc, sp, ph);
                else
                    body(k0 + J, n1, n0, sm, sc, sp, ph);
            }
        });
        it ^= 1u;
    }
    } else {
        int s_m = 0, s_c = 1, s_p = 2;
        uint32_t ph_p = 0;
        auto advance = [&]() {
            s_m = s_c;
            s_c = s_p;
            s_p = (s_p == kStages - 1) ? 0 : s_p + 1;
            ph_p ^= (s_p == 0) ? 1u : 0u;
        };
        for (int k = 1; k <= kmax; k += 2) {
            body(k, n0, n1, s_m, s_c, s_p, ph_p);
            advance();
            if (k + 1 <= kmax) {
                body(k + 1, n1, n0, s_m, s_c, s_p, ph_p);
                advance();
            }
        }
    }
    (void)ok;

    if constexpr (MODE == kStepObs || MODE == kObs) {
        // deterministic CTA reduction: warp shuffles, then one thread over warps
        __shared__ double red_d[4][NCW];
        __shared__ float red_f[2][NCW];
        __shared__ unsigned red_u[NCW];
        double d[4] = {acc.value(0), acc.value(1), acc.value(2), acc.value(3)};
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
        consumer_sync<NC>();
        if (t == 0) {
            double s[4] = {0, 0, 0, 0};
            float um = 0.f, rm = __int_as_float(0x7f800000);
            unsigned b = 0;
            for (int w = 0; w < NCW; ++w) {
#pragma unroll
                for (int q = 0; q < 4; ++q) s[q] += red_d[q][w];
                um = fmaxf(um, red_f[0][w]);
                rm = fminf(rm, red_f[1][w]);
                b += red_u[w];
            }
            double* out = partials + (size_t)slot * kPartialStride;
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

// T1: tau = 1 (the relaxation sets f* = f_eq, so no pulled population is
// kept for it); the modes that only observe use T1 = true.
template <int MODE, int ST = kF32, bool T1 = true, bool PAIR = true>
__global__ void __launch_bounds__(threads_of(ST, PAIR), step_ctas_of(MODE, ST, T1, PAIR))
    step_kernel(const float* __restrict__ fin, float* __restrict__ fout, Geom g, Phys p,
                double* __restrict__ partials, double* __restrict__ fields, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    run_tile<MODE, ST, T1, PAIR>(fin, fout, g, p, partials, fields, err, blockIdx.x, blockIdx.y,
                                 blockIdx.y * gridDim.x + blockIdx.x, smem_raw);
}

// One domain of a batch: geometry, model parameters, its two population
// buffers and its per-CTA partials.
struct DomainDev {
    Geom g;
    Phys p;
    float* buf[2];
    double* partials;
};

// Persistent batched step: every CTA walks the tile list (domain, strip,
// segment, partial slot) with stride gridDim.x, so domains of any size share
// one launch; buffers alternate with `parity`. Between tiles the CTA
// invalidates and re-arms its mbarriers.
template <int MODE, int ST = kF32, bool T1 = true, bool PAIR = true>
__global__ void __launch_bounds__(threads_of(ST, PAIR), batch_ctas_of(MODE, ST, T1, PAIR))
    batch_step_kernel(const DomainDev* __restrict__ doms, const int4* __restrict__ tiles, int ntiles,
                      int parity, int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // the tile's domain parameters live in shared memory, read where used, so
    // that they hold no registers across the tile (the single-domain kernel
    // reads them from its parameter space)
    __shared__ Geom g;
    __shared__ Phys p;
    for (int i = blockIdx.x; i < ntiles; i += gridDim.x) {
        const int4 tl = tiles[i];
        const DomainDev& d = doms[tl.x];
        if (threadIdx.x == 0) {
            g = d.g;
            p = d.p;
        }
        __syncthreads();
        run_tile<MODE, ST, T1, PAIR>(d.buf[parity], d.buf[parity ^ 1], g, p, d.partials, nullptr, err, tl.y, tl.z,
                                     tl.w, smem_raw);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t* bars = reinterpret_cast<uint64_t*>(
                smem_raw + stages_of(ST, PAIR) * (stage_bytes<ST>() + kPsiStride * sizeof(float)));
            for (int s = 0; s < 2 * stages_of(ST, PAIR); ++s) mbar_inval(&bars[s]);
        }
        __syncthreads();
    }
}

}  // namespace lbm
