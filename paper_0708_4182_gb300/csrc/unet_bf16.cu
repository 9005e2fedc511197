// unet_bf16.cu -- hand-written kernels of the warm-start U-Net (sm_103a).
//
// The surrogate maps a channel's wall mask, electric-force level and fill
// fraction to its steady density and velocity, which then initialise the
// lattice Boltzmann run (the warm start). Activations are BF16, channels-last
// (NHWC); every sum accumulates in FP32; the optimizer keeps FP32 master
// weights and moments.
//
// The 3x3 convolutions run on the 5th-generation tensor cores: tcgen05.mma
// (kind::f16, BF16 operands from shared memory, FP32 accumulator in tensor
// memory) issued by one thread per CTA, operands staged by cp.async into the
// canonical no-swizzle layout (8-row x 16-byte core matrices), completion
// tracked by tcgen05.commit on mbarriers, the accumulator read back with
// tcgen05.ld for the epilogue. Forward and input-gradient convolutions are an
// implicit GEMM with M = 128 output pixels (one row of 128, or 4 rows x 32
// columns for narrower images), N = a tile of output channels, K = 16 input
// channels of one of the 9 taps per MMA (both operands K-major: channels are
// contiguous per pixel). The weight gradient is a GEMM per tap with M = 128
// output channels, N = a tile of input channels and K = 16 pixels per MMA
// (both operands MN-major), the 3 taps of a row sharing a CTA's staged operands.
//
// A tensor "view" is (pointer to its first channel, channels per pixel of
// the underlying buffer), so a layer reads or writes a channel range of a
// larger buffer (the decoder's concatenations); nothing is copied. Padding of
// the 3x3 convolutions: circular in x (the channels are periodic along the
// flow), zero in y (walls).
#include "unet_bf16.h"

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace unet {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kT = 256;                      // threads of the SIMT kernels
constexpr int kTcThreads = 128;              // threads of the tensor-core kernels (4 warps = 128 TMEM lanes)
constexpr uint32_t kWaitLimit = 1u << 18;    // try_wait rounds before giving up (about 1 s on a GB300)
constexpr int kTileRows = 4, kTileCols = 32; // output pixels of one conv CTA (M = 128)
constexpr int kSmemPerSm = 233472;           // shared memory of one SM (bytes)

__device__ __forceinline__ float ld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ int wrapx(int x, int w) { return x < 0 ? x + w : (x >= w ? x - w : x); }

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait on one phase of an mbarrier. On timeout raise *err and set
// alive = false: the thread waits no more (each later call returns at once),
// so a kernel that lost a phase ends after one time limit per thread rather
// than one per wait, and nothing hangs.
__device__ __forceinline__ void mbar_wait_alive(uint64_t* bar, uint32_t parity, int* err, bool& alive)
{
    if (!alive) return;
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return;
    }
    atomicOr(err, 1);
    alive = false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16-byte global -> shared copy; src_bytes = 0 fills zeros (src is not read)
__device__ __forceinline__ void cp_async16_ca(void* dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async16_cg(void* dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// shared-memory matrix descriptor, no swizzle: core matrix (8 rows x 16 B)
// (i, j) at start + i * sbo + j * lbo, j along K, i along M (or N)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
// M = 128, N = n; a_mn / b_mn select MN-major operands
__host__ __device__ constexpr uint32_t idesc_bf16(int n, bool a_mn, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn ? 1u << 15 : 0u) | (b_mn ? 1u << 16 : 0u) |
           (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 consecutive FP32 columns: thread t of the warp gets lane t
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// TMEM columns to allocate for accumulators spanning n FP32 columns (a power
// of two >= 32, at most the 512 of an SM; n > 512 cannot be allocated)
__host__ __device__ constexpr uint32_t tmem_cols(int n)
{
    return n <= 32 ? 32u : (n <= 64 ? 64u : (n <= 128 ? 128u : (n <= 256 ? 256u : 512u)));
}

// Dynamic shared memory that lets at most 512 / cols CTAs share an SM, so
// their tensor-memory allocations (cols columns each) always fit in the 512.
__host__ constexpr int smem_for_tmem(int cols, int needed)
{
    const int ctas = 512 / cols;
    const int cap = kSmemPerSm / (ctas + 1) + 1024;
    return needed > cap ? needed : cap;
}

// output-channel tile of a convolution with n output channels
__host__ __device__ constexpr int conv_ntile(int n) { return n % 128 == 0 ? 128 : (n % 64 == 0 ? 64 : 32); }

// ------------------------------------------------------------------ tensor-core 3x3 convolution
// y[b, p, co] = act(bias[co] + sum_{tap, k} B[co][k](tap) x[b, p + off(tap), k])
// x: NHWC view (channels per pixel ct_in, K = 16 kc channels used), y: NHWC
// view (ct_out per pixel), wt: packed weights (conv_pack_kernel), one CTA =
// 128 pixels (4 rows x 32 columns) x NT channels of one image.
//
// K runs over (chunk group, tap): a ring slot holds CK chunks of 16 input
// channels of one tap (A: 128 pixels x 16 channels per chunk, K-major; B:
// NT x 16 weights per chunk) and gets CK MMAs. Warp roles as in the weight
// gradient (wgrad_tc_kernel): warps 1-3 stage the slots with cp.async and
// arrive on the slot's "full" mbarrier kConvLag steps later (after their own
// copies landed and were fenced for the async proxy); one thread issues the
// MMAs and commits them to the slot's "empty" mbarrier; no CTA-wide barrier
// runs inside the K loop.
constexpr int kConvStages = 4;   // operand ring depth
constexpr int kConvLag = 2;      // K-steps between a producer's copies and its "full" arrival
constexpr int kConvProducers = kTcThreads - 32;
template <int NT, int CK> __host__ __device__ constexpr int conv_smem_needed()
{
    return kConvStages * CK * (128 * 16 * 2 + NT * 16 * 2) + 2 * kConvStages * 8 + 16;
}

template <int NT, int CK>
__global__ void __launch_bounds__(kTcThreads) conv3x3_tc_kernel(const bf16* __restrict__ x, int ct_in, int kc,
                                                                const bf16* __restrict__ wt,
                                                                const float* __restrict__ bias,
                                                                bf16* __restrict__ y, int ct_out, int H, int W,
                                                                int relu, int* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    static_assert(NT <= int(tmem_cols(NT)), "the accumulator must fit the allocation");
    static_assert(kConvLag < kConvStages, "a producer arrives on a slot before it needs it again");
    constexpr int kAChunk = 128 * 16 * 2;  // 128 pixels x 16 channels
    constexpr int kBChunk = NT * 16 * 2;   // NT channels x 16 channels
    constexpr int kABytes = CK * kAChunk, kBBytes = CK * kBChunk;
    unsigned char* sa = smem;
    unsigned char* sb = smem + kConvStages * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sb + kConvStages * kBBytes);
    uint64_t* empty = full + kConvStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(empty + kConvStages);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / kTileCols;
    const int ty0 = (blockIdx.x / tiles_x) * kTileRows, tx0 = (blockIdx.x % tiles_x) * kTileCols;
    const int nb = blockIdx.y, b = blockIdx.z;
    const int KT = (kc / CK) * 9;
    const bf16* wblk = wt + size_t(nb) * kc * 9 * NT * 16;

    if (tid == 0) {
        for (int s = 0; s < kConvStages; ++s) {
            mbar_init(&full[s], kConvProducers);
            mbar_init(&empty[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, tmem_cols(NT));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool alive = true;

    if (warp == 0) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(NT, false, false);
#pragma unroll 1
            for (int it = 0; it < KT; ++it) {
                const int s = it % kConvStages;
                mbar_wait_alive(&full[s], uint32_t(it / kConvStages) & 1u, err, alive);
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < CK; ++j) {
                    const uint64_t da = smem_desc(smem_u32(sa + s * kABytes + j * kAChunk), 128, 256);
                    const uint64_t db = smem_desc(smem_u32(sb + s * kBBytes + j * kBChunk), 128, 256);
                    mma_bf16(tmem, da, db, idesc, (it > 0 || j > 0) ? 1u : 0u);
                }
                mma_commit(&empty[s]);
            }
        }
        __syncwarp();
    } else {
        const int pt = tid - 32;
#pragma unroll 1
        for (int it = 0; it < KT; ++it) {
            const int s = it % kConvStages;
            if (it >= kConvStages) mbar_wait_alive(&empty[s], uint32_t((it / kConvStages) - 1) & 1u, err, alive);
            const int t = it % 9, cg = it / 9;
            const int dy = t / 3 - 1, dx = t % 3 - 1;
            unsigned char* da = sa + s * kABytes;
            unsigned char* db = sb + s * kBBytes;
            // A: CK chunks x 256 pieces of 16 B (pixel q / 2, channel half q % 2)
            for (int q = pt; q < CK * 256; q += kConvProducers) {
                const int j = q >> 8, p = (q & 255) >> 1, h = q & 1;
                const int yy = ty0 + (p >> 5) + dy, xx = wrapx(tx0 + (p & 31) + dx, W);
                const bool ok = yy >= 0 && yy < H;
                const bf16* src = ok ? x + (size_t(b * H + yy) * W + xx) * ct_in + (cg * CK + j) * 16 + h * 8 : x;
                cp_async16_ca(da + j * kAChunk + (p >> 3) * 256 + h * 128 + (p & 7) * 16, src, ok ? 16u : 0u);
            }
            // B: CK chunks x NT * 2 pieces of the packed (chunk, tap) blocks
            for (int q = pt; q < CK * NT * 2; q += kConvProducers) {
                const int j = q / (NT * 2), r = q % (NT * 2);
                const bf16* wsrc = wblk + size_t((cg * CK + j) * 9 + t) * NT * 16;
                cp_async16_cg(db + j * kBChunk + r * 16, wsrc + r * 8, 16u);
            }
            cp_async_commit();
            if (it >= kConvLag) {
                cp_async_wait<kConvLag>();
                fence_proxy_async();
                mbar_arrive(&full[(it - kConvLag) % kConvStages]);
            }
        }
        cp_async_wait<0>();
        fence_proxy_async();
        for (int it = KT > kConvLag ? KT - kConvLag : 0; it < KT; ++it) mbar_arrive(&full[it % kConvStages]);
    }
    mbar_wait_alive(&empty[(KT - 1) % kConvStages], uint32_t((KT - 1) / kConvStages) & 1u, err, alive);
    tc_fence_after();

    // epilogue: lane = pixel, 16 columns at a time
    const int p = warp * 32 + lane;
    const int yy = ty0 + (p >> 5), xx = tx0 + (p & 31);
    bf16* out = y + (size_t(b * H + yy) * W + xx) * ct_out + nb * NT;
#pragma unroll 1
    for (int n0 = 0; n0 < NT; n0 += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + n0, v);
        __align__(16) bf16 o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float a = v[j] + (bias ? bias[nb * NT + n0 + j] : 0.f);
            if (relu) a = fmaxf(a, 0.f);
            o[j] = __float2bfloat16_rn(a);
        }
        uint4* dst = reinterpret_cast<uint4*>(out + n0);
        dst[0] = reinterpret_cast<const uint4*>(o)[0];
        dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols(NT));
}

// The same convolution for images at least 128 pixels wide: one CTA = 128
// consecutive pixels of one image row. Per 16-channel chunk the CTA stages a
// halo of 3 rows x 130 pixels once, pixels at a uniform 16-byte pitch (two
// planes of 8 channels, LBO = the plane distance, SBO = 8 pixels), and the 9
// taps are 9 MMAs whose A descriptors start at that halo shifted by dx pixels
// (16 bytes each) and dy rows: the input crosses shared memory once per chunk
// instead of once per tap. Three ring slots of one chunk each, with the warp
// roles of conv3x3_tc_kernel: the next chunks load while this one's MMAs run.
constexpr int kRowPix = 128, kHaloPix = kRowPix + 2;
constexpr int kHaloPlane = kHaloPix * 16;      // bytes of one 8-channel plane of one halo row
constexpr int kHaloBytes = 3 * 2 * kHaloPlane; // 3 rows x 2 planes
constexpr int kRowStages = 3;                  // ring slots (one chunk each)
constexpr int kRowLag = 1;                     // chunks between a producer's copies and its "full" arrival

template <int NT>
__global__ void __launch_bounds__(kTcThreads) conv3x3_tc_row_kernel(const bf16* __restrict__ x, int ct_in, int kc,
                                                                    const bf16* __restrict__ wt,
                                                                    const float* __restrict__ bias,
                                                                    bf16* __restrict__ y, int ct_out, int H, int W,
                                                                    int relu, int* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    static_assert(NT <= int(tmem_cols(NT)), "the accumulator must fit the allocation");
    static_assert(kRowLag < kRowStages, "a producer arrives on a slot before it needs it again");
    constexpr int kBBytes = 9 * NT * 16 * 2;  // the 9 taps' weights of one chunk
    unsigned char* sa = smem;
    unsigned char* sb = smem + kRowStages * kHaloBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sb + kRowStages * kBBytes);
    uint64_t* empty = full + kRowStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(empty + kRowStages);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = W / kRowPix;
    const int y0 = blockIdx.x / tiles_x, x0 = (blockIdx.x % tiles_x) * kRowPix;
    const int nb = blockIdx.y, b = blockIdx.z;
    const bf16* wblk = wt + size_t(nb) * kc * 9 * NT * 16;

    if (tid == 0) {
        for (int s = 0; s < kRowStages; ++s) {
            mbar_init(&full[s], kConvProducers);
            mbar_init(&empty[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, tmem_cols(NT));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool alive = true;

    if (warp == 0) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(NT, false, false);
#pragma unroll 1
            for (int c = 0; c < kc; ++c) {
                const int s = c % kRowStages;
                mbar_wait_alive(&full[s], uint32_t(c / kRowStages) & 1u, err, alive);
                tc_fence_after();
                const uint32_t a0 = smem_u32(sa + s * kHaloBytes);
                const uint32_t b0 = smem_u32(sb + s * kBBytes);
#pragma unroll
                for (int t = 0; t < 9; ++t) {
                    const int dy = t / 3, dx = t % 3;  // halo row and pixel shift of this tap
                    const uint64_t da = smem_desc(a0 + dy * 2 * kHaloPlane + dx * 16, kHaloPlane, 128);
                    const uint64_t db = smem_desc(b0 + t * NT * 32, 128, 256);
                    mma_bf16(tmem, da, db, idesc, (c > 0 || t > 0) ? 1u : 0u);
                }
                mma_commit(&empty[s]);
            }
        }
        __syncwarp();
    } else {
        const int pt = tid - 32;
#pragma unroll 1
        for (int c = 0; c < kc; ++c) {
            const int s = c % kRowStages;
            if (c >= kRowStages) mbar_wait_alive(&empty[s], uint32_t((c / kRowStages) - 1) & 1u, err, alive);
            unsigned char* da = sa + s * kHaloBytes;
            // 3 rows x 130 pixels x 2 planes of 16 bytes
            for (int q = pt; q < 3 * kHaloPix * 2; q += kConvProducers) {
                const int h = q & 1, pix = (q >> 1) % kHaloPix, r = (q >> 1) / kHaloPix;
                const int yy = y0 + r - 1, xx = wrapx(x0 + pix - 1, W);
                const bool ok = yy >= 0 && yy < H;
                const bf16* src = ok ? x + (size_t(b * H + yy) * W + xx) * ct_in + c * 16 + h * 8 : x;
                cp_async16_ca(da + (r * 2 + h) * kHaloPlane + pix * 16, src, ok ? 16u : 0u);
            }
            const bf16* wsrc = wblk + size_t(c) * 9 * NT * 16;
            unsigned char* db = sb + s * kBBytes;
            for (int q = pt; q < 9 * NT * 2; q += kConvProducers) cp_async16_cg(db + q * 16, wsrc + q * 8, 16u);
            cp_async_commit();
            if (c >= kRowLag) {
                cp_async_wait<kRowLag>();
                fence_proxy_async();
                mbar_arrive(&full[(c - kRowLag) % kRowStages]);
            }
        }
        cp_async_wait<0>();
        fence_proxy_async();
        for (int c = kc > kRowLag ? kc - kRowLag : 0; c < kc; ++c) mbar_arrive(&full[c % kRowStages]);
    }
    mbar_wait_alive(&empty[(kc - 1) % kRowStages], uint32_t((kc - 1) / kRowStages) & 1u, err, alive);
    tc_fence_after();

    const int p = warp * 32 + lane;
    bf16* out = y + (size_t(b * H + y0) * W + x0 + p) * ct_out + nb * NT;
#pragma unroll 1
    for (int n0 = 0; n0 < NT; n0 += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + n0, v);
        __align__(16) bf16 o[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            float a = v[j] + (bias ? bias[nb * NT + n0 + j] : 0.f);
            if (relu) a = fmaxf(a, 0.f);
            o[j] = __float2bfloat16_rn(a);
        }
        uint4* dst = reinterpret_cast<uint4*>(out + n0);
        dst[0] = reinterpret_cast<const uint4*>(o)[0];
        dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tmem_cols(NT));
}

// Packed B operand of the tensor-core convolution. Forward (transpose = 0):
// row n = output channel, column k = input channel, B[n][k](tap) =
// w[n][k][tap]. Input gradient (transpose = 1): row n = input channel of the
// forward layer, column k = its output channel, B[n][k](tap) = w[k][n][8 - tap]
// (the transposed, flipped kernel). w: FP32 master weights [co][ci][9]. Out:
// blocks [n tile][k chunk of 16][tap] of NT x 16 BF16 in core-matrix order
// (row group i at 256 B, k half j at 128 B, row r at 16 B); k beyond the real
// channels is 0.
__device__ __forceinline__ void pack_one(const float* __restrict__ w, int co, int ci, int transpose, int nt, int kc,
                                         long long i, bf16* __restrict__ out)
{
    const int kreal = transpose ? co : ci;
    const int k = int(i % (kc * 16));
    const long long r1 = i / (kc * 16);
    const int t = int(r1 % 9);
    const int n = int(r1 / 9);
    float v = 0.f;
    if (k < kreal) v = transpose ? w[(size_t(k) * ci + n) * 9 + (8 - t)] : w[(size_t(n) * ci + k) * 9 + t];
    const int nbk = n / nt, nn = n % nt, c = k / 16, kk = k % 16;
    const size_t blk = (size_t(nbk) * kc + c) * 9 + t;
    const size_t off = blk * nt * 16 + ((nn >> 3) * 2 + (kk >> 3)) * 64 + (nn & 7) * 8 + (kk & 7);
    out[off] = __float2bfloat16_rn(v);
}

__global__ void conv_pack_kernel(const float* __restrict__ w, int co, int ci, int transpose, int nt, int kc,
                                 bf16* __restrict__ out)
{
    const int nrows = transpose ? ci : co;
    const long long total = (long long)nrows * kc * 16 * 9;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        pack_one(w, co, ci, transpose, nt, kc, i, out);
}

// Several packings in one launch: job blockIdx.y is the record
// jobs[5 y .. 5 y + 4] = (address of w, co, ci, transpose, address of out).
__global__ void conv_pack_many_kernel(const long long* __restrict__ jobs)
{
    const long long* j = jobs + 5 * blockIdx.y;
    const float* w = reinterpret_cast<const float*>(j[0]);
    const int co = int(j[1]), ci = int(j[2]), transpose = int(j[3]);
    bf16* out = reinterpret_cast<bf16*>(j[4]);
    const int nrows = transpose ? ci : co, kreal = transpose ? co : ci;
    const int kc = (kreal + 15) / 16, nt = conv_ntile(nrows);
    const long long total = (long long)nrows * kc * 16 * 9;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        pack_one(w, co, ci, transpose, nt, kc, i, out);
}

// ------------------------------------------------------------------ tensor-core weight gradient
// dw[co][ci][tap] += sum over pixels p of dy[p][co] x[p + off(tap)][ci]: per
// tap a GEMM with M = 128 output channels, N = NT input channels and K = the
// pixels. One CTA takes one tap row (dy = -1, 0, 1 of the 3x3 stencil) and a
// range of npix pixels. Per K-step of P pixels of one image row (P = 16, 32
// or 64, dividing the row), dy (A, 128 output channels x P pixels, MN-major:
// 8 channels of a pixel in 16 bytes, pixels at a 16-byte pitch, so LBO = 8
// pixels and SBO = P pixels) is staged once, and x as a halo row of P + 2
// pixels x NT channels (B, MN-major likewise: SBO = P + 2 pixels). Each
// 16-pixel piece j of the step gives three MMAs, one per tap (dx = -1, 0, 1)
// of the row: A starts 16 j pixels in, B 16 j + dx pixels in, into three
// accumulators of NT columns (3 NT <= 512 tensor-memory columns). With SW
// (layers with more input than output channels) the operands swap roles:
// the x halo row is A (M = 128 input channels) and dy is B (N = NT output
// channels), so that the wider side fills the MMA's 128 rows; the shared
// layouts and descriptors are the same, and the accumulators hold dw
// transposed (lane = input channel).
//
// Warp roles: warps 1-3 stage the operands with 16-byte cp.async into a ring
// of kWgStages slots; each producer thread waits for its own copies of a slot
// two steps later, fences them for the tensor core's (async) proxy and
// arrives on the slot's "full" mbarrier (96 arrivals). One thread of warp 0
// waits on "full", issues the MMAs and commits them to the slot's "empty"
// mbarrier, which the producers wait on before refilling the slot. No
// CTA-wide barrier runs inside the K loop. The epilogue adds the three
// accumulators into dw (FP32 atomics; the grid splits the pixels).
constexpr int kWgStages = 4;   // operand ring depth of the weight gradient
constexpr int kWgLag = 2;      // K-steps between a producer's copies and its "full" arrival
constexpr int kWgThreads = 256;                 // 8 warps: one issues the MMAs, seven stage operands
constexpr int kWgProducers = kWgThreads - 32;
template <int P> __host__ __device__ constexpr int wgrad_halo_pix() { return P + 2; }
// dy and x channels per CTA
template <int NT, bool SW> __host__ __device__ constexpr int wgrad_co_tile() { return SW ? NT : 128; }
template <int NT, bool SW> __host__ __device__ constexpr int wgrad_ci_tile() { return SW ? 128 : NT; }
template <int NT, int P, bool SW> __host__ __device__ constexpr int wgrad_smem_needed()
{
    return kWgStages * (wgrad_co_tile<NT, SW>() * P * 2 + (wgrad_ci_tile<NT, SW>() / 8) * wgrad_halo_pix<P>() * 16) +
           2 * kWgStages * 8 + 16;
}

template <int NT, int P, bool SW>
__global__ void __launch_bounds__(kWgThreads) wgrad_tc_kernel(const bf16* __restrict__ x, int ct_x, int ci,
                                                              const bf16* __restrict__ dy, int ct_dy, int co,
                                                              float* __restrict__ dw, int H, int W, int npix,
                                                              int* __restrict__ err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    static_assert(3 * NT <= 512, "three accumulators must fit the tensor memory");
    static_assert(P == 16 || P == 32 || P == 64, "K-step of 16, 32 or 64 pixels");
    static_assert(kWgLag < kWgStages, "a producer arrives on a slot before it needs it again");
    constexpr int COT = wgrad_co_tile<NT, SW>(), CIT = wgrad_ci_tile<NT, SW>();
    constexpr int HP = wgrad_halo_pix<P>();                // halo row pixels
    constexpr int kABytes = COT * P * 2;                   // dy: COT output channels x P pixels
    constexpr int kBBytes = (CIT / 8) * HP * 16;           // x: one halo row of CIT input channels
    constexpr uint32_t kCols = tmem_cols(3 * NT);
    unsigned char* sa = smem;
    unsigned char* sb = smem + kWgStages * kABytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sb + kWgStages * kBBytes);
    uint64_t* empty = full + kWgStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(empty + kWgStages);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int co0 = blockIdx.x * COT, ci0 = blockIdx.y * CIT;
    const int trow = blockIdx.z % 3;                       // taps 3 trow .. 3 trow + 2 (row offset trow - 1)
    const int co_here = co - co0 < COT ? co - co0 : COT;
    const int ci_here = ci - ci0 < CIT ? ci - ci0 : CIT;
    const int KT = npix / P;

    // rows of A beyond co_here and channel groups of B beyond ci_here are never loaded: zero them once
    for (int i = tid; i < kWgStages * (kABytes + kBBytes) / 16; i += kWgThreads)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            mbar_init(&full[s], kWgProducers);
            mbar_init(&empty[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, kCols);
    fence_proxy_async();  // the zeroed slots, before the tensor core reads them
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool alive = true;

    if (warp == 0) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(NT, true, true);
#pragma unroll 1
            for (int k = 0; k < KT; ++k) {
                const int s = k % kWgStages;
                mbar_wait_alive(&full[s], uint32_t(k / kWgStages) & 1u, err, alive);
                tc_fence_after();
                const uint32_t a0 = smem_u32(sa + s * kABytes);
                const uint32_t b0 = smem_u32(sb + s * kBBytes);
#pragma unroll
                for (int j = 0; j < P / 16; ++j) {
                    const uint64_t dd = smem_desc(a0 + j * 256, 128, P * 16);  // dy piece j
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const uint64_t dh = smem_desc(b0 + (16 * j + dx) * 16, 128, HP * 16);  // x, shifted dx
                        if constexpr (SW)
                            mma_bf16(tmem + dx * NT, dh, dd, idesc, (k > 0 || j > 0) ? 1u : 0u);
                        else
                            mma_bf16(tmem + dx * NT, dd, dh, idesc, (k > 0 || j > 0) ? 1u : 0u);
                    }
                }
                mma_commit(&empty[s]);
            }
        }
        __syncwarp();
    } else {
        const int pt = tid - 32;                           // producer thread 0 .. 95
        const int ga = (co_here + 7) / 8, gb = (ci_here + 7) / 8;
        // position of K-step k: image bimg, row yy, first column x0 (each step
        // lies inside one image row), advanced incrementally
        const long long p_begin = (long long)(blockIdx.z / 3) * npix;
        int bimg = int(p_begin / ((long long)H * W));
        const int rem = int(p_begin - (long long)bimg * H * W);
        int yy = rem / W, x0 = rem % W;
#pragma unroll 1
        for (int k = 0; k < KT; ++k) {
            const int s = k % kWgStages;
            if (k >= kWgStages) mbar_wait_alive(&empty[s], uint32_t((k / kWgStages) - 1) & 1u, err, alive);
            unsigned char* da = sa + s * kABytes;
            unsigned char* db = sb + s * kBBytes;
            const bf16* arow = dy + (size_t(bimg * H + yy) * W + x0) * ct_dy + co0;
            for (int q = pt; q < P * ga; q += kWgProducers) {
                const int kk = q % P, g = q / P;
                cp_async16_cg(da + g * (P * 16) + kk * 16, arow + size_t(kk) * ct_dy + g * 8, 16u);
            }
            const int ys = yy + trow - 1;
            const bool ok = ys >= 0 && ys < H;
            const bf16* brow = x + size_t(bimg * H + (ok ? ys : 0)) * W * ct_x + ci0;
            for (int q = pt; q < HP * gb; q += kWgProducers) {
                const int pix = q % HP, g = q / HP;
                const int xs = wrapx(x0 + pix - 1, W);
                cp_async16_ca(db + g * (HP * 16) + pix * 16, ok ? brow + size_t(xs) * ct_x + g * 8 : x, ok ? 16u : 0u);
            }
            cp_async_commit();
            if (k >= kWgLag) {
                cp_async_wait<kWgLag>();
                fence_proxy_async();
                mbar_arrive(&full[(k - kWgLag) % kWgStages]);
            }
            x0 += P;
            if (x0 == W) {
                x0 = 0;
                if (++yy == H) {
                    yy = 0;
                    ++bimg;
                }
            }
        }
        cp_async_wait<0>();
        fence_proxy_async();
        for (int k = KT > kWgLag ? KT - kWgLag : 0; k < KT; ++k) mbar_arrive(&full[k % kWgStages]);
    }
    // every warp: the last commit completes when all MMAs have
    mbar_wait_alive(&empty[(KT - 1) % kWgStages], uint32_t((KT - 1) / kWgStages) & 1u, err, alive);
    tc_fence_after();

    // warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its quadrant) and
    // the accumulator columns of every (w / 4)-th 16-column block
    const int quad = warp & 3, half = warp >> 2;
    const int m = quad * 32 + lane;  // accumulator row: output channel co0 + m (input channel ci0 + m with SW)
    const int m_here = SW ? ci_here : co_here, n_here = SW ? co_here : ci_here;
#pragma unroll 1
    for (int dx = 0; dx < 3; ++dx) {
        const int tap = trow * 3 + dx;
#pragma unroll 1
        for (int n0 = 16 * half; n0 < NT; n0 += 16 * (kWgThreads / 128)) {
            float v[16];
            tmem_ld16(tmem + (uint32_t(quad * 32) << 16) + dx * NT + n0, v);
            if (m < m_here) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (n0 + j >= n_here) continue;
                    const size_t o = SW ? (size_t(co0 + n0 + j) * ci + ci0 + m) : (size_t(co0 + m) * ci + ci0 + n0 + j);
                    atomicAdd(&dw[o * 9 + tap], v[j]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ------------------------------------------------------------------ SIMT kernels (NHWC)
// db[c] += sum over pixels of dy[p, c]; block = channels, grid over pixel ranges
__global__ void bias_grad_kernel(const bf16* __restrict__ dy, int ct, int C, long long npix, int per_block,
                                 float* __restrict__ db)
{
    const int c = threadIdx.x;
    if (c >= C) return;
    const long long p0 = (long long)blockIdx.x * per_block;
    const long long p1 = p0 + per_block < npix ? p0 + per_block : npix;
    float s = 0.f;
    for (long long p = p0; p < p1; ++p) s += ld(dy + p * ct + c);
    atomicAdd(&db[c], s);
}

// 8 BF16 values (16 bytes) <-> FP32
__device__ __forceinline__ void unpack8(const uint4& q, float (&v)[8])
{
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[2 * k] = __uint_as_float(w[k] << 16);
        v[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
}
__device__ __forceinline__ uint4 pack8(const float (&v)[8])
{
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
        w[k] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// 1x1 head: y[b, o, p] = bias[o] + sum_i w[o][i] x[b, p, i] (x NHWC view, y FP32 NCHW)
__global__ void head_fwd_kernel(const bf16* __restrict__ x, int ct, int Ci, const bf16* __restrict__ w,
                                const float* __restrict__ bias, float* __restrict__ y, int Co, int HW, int B)
{
    // the Co x Ci weights (at most 8 x 64) once per block, read as broadcasts
    __shared__ float ws[8 * 64];
    for (int k = threadIdx.x; k < Co * Ci; k += blockDim.x) ws[k] = ld(w + k);
    __syncthreads();
    const long long n = (long long)B * HW;
    const bool vec = (Ci % 8 == 0) && (ct % 8 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int b = int(i / HW), p = int(i % HW);
        const bf16* xp = x + i * ct;
        float s[8];
        for (int o = 0; o < Co; ++o) s[o] = bias[o];
        if (vec) {
            // the pixel's channels 8 at a time (16-byte loads), each used by every output
            for (int c0 = 0; c0 < Ci; c0 += 8) {
                float xv[8];
                unpack8(*reinterpret_cast<const uint4*>(xp + c0), xv);
                for (int o = 0; o < Co; ++o) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) s[o] = fmaf(ws[o * Ci + c0 + k], xv[k], s[o]);
                }
            }
        } else {
            for (int c = 0; c < Ci; ++c) {
                const float xv = ld(xp + c);
                for (int o = 0; o < Co; ++o) s[o] = fmaf(ws[o * Ci + c], xv, s[o]);
            }
        }
        for (int o = 0; o < Co; ++o) y[((long long)b * Co + o) * HW + p] = s[o];
    }
}

// head backward: dx[b, p, i] = sum_o w[o][i] dy[b, o, p] (NHWC BF16 out);
// dw[o][i] += sum dy x, db[o] += sum dy (FP32). Block: Ci channels x
// (256 / Ci) pixel lanes; each thread keeps its CO partial sums of dw and db
// in registers, reduced per block in shared memory.
template <int CO>
__global__ void head_bwd_kernel(const bf16* __restrict__ x, int ct, int Ci, const bf16* __restrict__ w,
                                const float* __restrict__ dy, int HW, int B, bf16* __restrict__ dx, int ct_dx,
                                float* __restrict__ dw, float* __restrict__ db)
{
    __shared__ float red[kT][CO];
    const int lanes = kT / Ci;
    const int c = threadIdx.x % Ci, lane = threadIdx.x / Ci;
    float wc[CO], sw[CO], sb[CO];
#pragma unroll
    for (int o = 0; o < CO; ++o) {
        wc[o] = ld(w + o * Ci + c);
        sw[o] = sb[o] = 0.f;
    }
    const long long n = (long long)B * HW;
    if (lane < lanes) {
        for (long long i = (long long)blockIdx.x * lanes + lane; i < n; i += (long long)gridDim.x * lanes) {
            const int b = int(i / HW), p = int(i % HW);
            const float xv = ld(x + i * ct + c);
            float s = 0.f;
#pragma unroll
            for (int o = 0; o < CO; ++o) {
                const float g = dy[((long long)b * CO + o) * HW + p];
                s = fmaf(wc[o], g, s);
                sw[o] = fmaf(g, xv, sw[o]);
                sb[o] += g;
            }
            dx[i * ct_dx + c] = __float2bfloat16_rn(s);
        }
    }
#pragma unroll
    for (int o = 0; o < CO; ++o) red[threadIdx.x][o] = lane < lanes ? sw[o] : 0.f;
    __syncthreads();
    if (lane == 0) {
        for (int o = 0; o < CO; ++o) {
            float t = red[c][o];
            for (int k = 1; k < lanes; ++k) t += red[k * Ci + c][o];
            atomicAdd(&dw[o * Ci + c], t);
        }
    }
    __syncthreads();
    // db: every channel's thread saw the same dy values, so channel 0's lanes suffice
#pragma unroll
    for (int o = 0; o < CO; ++o) red[threadIdx.x][o] = (c == 0 && lane < lanes) ? sb[o] : 0.f;
    __syncthreads();
    if (threadIdx.x < CO) {
        float t = 0.f;
        for (int k = 0; k < lanes; ++k) t += red[k * Ci][threadIdx.x];
        atomicAdd(&db[threadIdx.x], t);
    }
}

// 2x2 average pooling of an (H, W) NHWC view and its adjoint
// 2x2 average pooling of an (H, W) NHWC view and its adjoint. One thread per
// coarse pixel and 8 channels (16-byte accesses): C, ctx, cty multiples of 8,
// views 16-byte aligned (checked by the host entries).
__global__ void pool2_fwd_kernel(const bf16* __restrict__ x, int ctx, bf16* __restrict__ y, int cty, int C, int H,
                                 int W, int B)
{
    const int h = H / 2, w = W / 2, C8 = C / 8;
    const int n = B * h * w * C8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = (i % C8) * 8, pix = i / C8;
        const int xx = pix % w, r = pix / w;  // r = b * h + yy
        const bf16* s = x + (size_t(2 * r) * W + 2 * xx) * ctx + c;
        float a[8], b2[8], c2[8], d[8];
        unpack8(*reinterpret_cast<const uint4*>(s), a);
        unpack8(*reinterpret_cast<const uint4*>(s + ctx), b2);
        unpack8(*reinterpret_cast<const uint4*>(s + size_t(W) * ctx), c2);
        unpack8(*reinterpret_cast<const uint4*>(s + size_t(W + 1) * ctx), d);
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = 0.25f * ((a[k] + b2[k]) + (c2[k] + d[k]));
        *reinterpret_cast<uint4*>(y + size_t(pix) * cty + c) = pack8(o);
    }
}

__global__ void pool2_bwd_kernel(const bf16* __restrict__ dy, int cty, bf16* __restrict__ dx, int ctx, int C, int H,
                                 int W, int B, int accumulate)
{
    const int h = H / 2, w = W / 2, C8 = C / 8;
    const int n = B * h * w * C8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = (i % C8) * 8, pix = i / C8;
        const int xx = pix % w, r = pix / w;
        float g[8];
        unpack8(*reinterpret_cast<const uint4*>(dy + size_t(pix) * cty + c), g);
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] *= 0.25f;
        bf16* o = dx + (size_t(2 * r) * W + 2 * xx) * ctx + c;
        const size_t offs[4] = {0, size_t(ctx), size_t(W) * ctx, size_t(W + 1) * ctx};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4* dst = reinterpret_cast<uint4*>(o + offs[q]);
            float v[8];
            if (accumulate) {
                unpack8(*dst, v);
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] += g[k];
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = g[k];
            }
            *dst = pack8(v);
        }
    }
}

// nearest 2x upsampling of an (h, w) NHWC view and its adjoint (sum over the
// 4 copies); the forward copies 8 channels (16 bytes) per thread, so C, ctx,
// cty must be multiples of 8 and the views 16-byte aligned
__global__ void up2_fwd_kernel(const bf16* __restrict__ x, int ctx, bf16* __restrict__ y, int cty, int C, int h,
                               int w, int B)
{
    const int H = 2 * h, W = 2 * w, C8 = C / 8;
    const long long n = (long long)B * H * W * C8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % C8) * 8;
        const long long pix = i / C8;
        const int xx = int(pix % W), yy = int((pix / W) % H), b = int(pix / ((long long)W * H));
        *reinterpret_cast<uint4*>(y + (size_t(b * H + yy) * W + xx) * cty + c) =
            *reinterpret_cast<const uint4*>(x + (size_t(b * h + yy / 2) * w + xx / 2) * ctx + c);
    }
}

__global__ void up2_bwd_kernel(const bf16* __restrict__ dy, int cty, bf16* __restrict__ dx, int ctx, int C, int h,
                               int w, int B)
{
    const int W = 2 * w, C8 = C / 8;
    const int n = B * h * w * C8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = (i % C8) * 8, pix = i / C8;
        const int xx = pix % w, r = pix / w;
        const bf16* s = dy + (size_t(2 * r) * W + 2 * xx) * cty + c;
        float a[8], b2[8], c2[8], d[8];
        unpack8(*reinterpret_cast<const uint4*>(s), a);
        unpack8(*reinterpret_cast<const uint4*>(s + cty), b2);
        unpack8(*reinterpret_cast<const uint4*>(s + size_t(W) * cty), c2);
        unpack8(*reinterpret_cast<const uint4*>(s + size_t(W + 1) * cty), d);
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = (a[k] + b2[k]) + (c2[k] + d[k]);
        *reinterpret_cast<uint4*>(dx + size_t(pix) * ctx + c) = pack8(o);
    }
}

// dy <- dy * (y > 0): gradient through a ReLU whose output is y (NHWC views,
// C <= 256 channels, C, cty, ctd multiples of 8, 16-byte aligned); with db !=
// NULL also db[c] += sum over pixels of the masked dy (the bias gradient of the
// layer that produced y). A thread handles 8 channels of a pixel with 16-byte
// loads and keeps 8 partial sums; the block sums them per channel in shared
// memory, one atomic per channel.
__global__ void relu_bwd_kernel(const bf16* __restrict__ y, int cty, bf16* __restrict__ dy, int ctd, int C,
                                long long npix, float* __restrict__ db)
{
    __shared__ float red[kT][8];
    const int G = C / 8, lanes = kT / G;
    const int grp = threadIdx.x % G, lane = threadIdx.x / G;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // each pixel's 8 gradients: zero where y <= 0, else kept and summed
    auto step = [&](const uint4& yv, uint4& gv) {
        const bf16* ye = reinterpret_cast<const bf16*>(&yv);
        bf16* ge = reinterpret_cast<bf16*>(&gv);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (__bfloat162float(ye[j]) > 0.f)
                s[j] += __bfloat162float(ge[j]);
            else
                ge[j] = __float2bfloat16_rn(0.f);
        }
    };
    if (lane < lanes) {
        // four pixels per round, their loads issued together
        const long long stride = (long long)gridDim.x * lanes;
        long long p = (long long)blockIdx.x * lanes + lane;
        for (; p + 3 * stride < npix; p += 4 * stride) {
            uint4 yv[4], gv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                yv[u] = *reinterpret_cast<const uint4*>(y + (p + u * stride) * cty + grp * 8);
                gv[u] = *reinterpret_cast<const uint4*>(dy + (p + u * stride) * ctd + grp * 8);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                step(yv[u], gv[u]);
                *reinterpret_cast<uint4*>(dy + (p + u * stride) * ctd + grp * 8) = gv[u];
            }
        }
        for (; p < npix; p += stride) {
            const uint4 yv = *reinterpret_cast<const uint4*>(y + p * cty + grp * 8);
            uint4 gv = *reinterpret_cast<const uint4*>(dy + p * ctd + grp * 8);
            step(yv, gv);
            *reinterpret_cast<uint4*>(dy + p * ctd + grp * 8) = gv;
        }
    }
    if (!db) return;
    if (lane >= lanes) {
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] = 0.f;
    }
    // bias gradient: the partial sums of group grp over the block's pixels
    const int tid = threadIdx.x;
    if ((G & (G - 1)) == 0) {
        // G divides 32: threads tid ^ m (m = G, 2G, .., 16) hold the same
        // group, so shuffles sum a warp's lanes; then one value per warp and
        // group goes through shared memory
        for (int m = G; m < 32; m <<= 1) {
#pragma unroll
            for (int j = 0; j < 8; ++j) s[j] += __shfl_xor_sync(0xffffffffu, s[j], m);
        }
        const int wl = tid & 31, wp = tid >> 5;
        if (wl < G) {
#pragma unroll
            for (int j = 0; j < 8; ++j) red[wp * G + wl][j] = s[j];
        }
        __syncthreads();
        if (tid < C) {
            const int g = tid / 8, j = tid % 8;
            float t = 0.f;
            for (int w = 0; w < kT / 32; ++w) t += red[w * G + g][j];
            atomicAdd(&db[g * 8 + j], t);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) red[tid][j] = s[j];
        __syncthreads();
        if (tid < C) {
            const int g = tid / 8, j = tid % 8;
            float t = 0.f;
            for (int k = 0; k < lanes; ++k) t += red[k * G + g][j];
            atomicAdd(&db[g * 8 + j], t);
        }
    }
}

// FP32 NCHW planes -> BF16 NHWC with ct channels per pixel (channels >= c are 0)
__global__ void input_nhwc_kernel(const float* __restrict__ x, int C, int HW, int B, bf16* __restrict__ y, int ct)
{
    const long long n = (long long)B * HW * ct;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = int(i % ct);
        const long long pix = i / ct;
        const int b = int(pix / HW), p = int(pix % HW);
        y[i] = __float2bfloat16_rn(c < C ? x[((long long)b * C + c) * HW + p] : 0.f);
    }
}

// weighted mean squared error over n = B*C*HW values, weight per channel:
// loss = sum_i wc (p - t)^2 / n; grad = 2 wc (p - t) / n (FP32, NCHW)
__global__ void mse_kernel(const float* __restrict__ p, const float* __restrict__ t, const float* __restrict__ wc,
                           int C, int HW, long long n, float* __restrict__ grad, double* __restrict__ loss)
{
    __shared__ double red[kT];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
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

// Adam on FP32 master weights; writes the BF16 compute copy if wb != NULL
// hyper (may be NULL): lr, c1 = 1 - b1^t, c2 = 1 - b2^t read from device
// memory instead of the arguments (a replayable graph of training steps)
__global__ void adam_kernel(float* __restrict__ wm, bf16* __restrict__ wb, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, float wd, const float* __restrict__ hyper)
{
    if (hyper) {
        lr = hyper[0];
        c1 = hyper[1];
        c2 = hyper[2];
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
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

// One training step's Adam scalars on the device. state: [0] t, [1] b1^t,
// [2] b2^t (running products, multiplied in FP32 as the host entry does),
// then the step's [3] lr = lr_sched[t - 1] (the last entry beyond the end),
// [4] 1 - b1^t, [5] 1 - b2^t.
__global__ void adam_hyper_kernel(float* __restrict__ state, const float* __restrict__ lr_sched, int n, float b1,
                                  float b2)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int t = int(state[0]) + 1;
    const float p1 = state[1] * b1, p2 = state[2] * b2;
    state[0] = float(t);
    state[1] = p1;
    state[2] = p2;
    state[3] = lr_sched[t - 1 < n ? t - 1 : n - 1];
    state[4] = 1.f - p1;
    state[5] = 1.f - p2;
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, bf16* __restrict__ y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// Warm-start fields from the network output y [n][3][hw] (normalised): on
// fluid nodes (mask 0) rho = clamp(y0 rho_std + rho_mean, lo, hi), u = y1,2
// u_scale; 0 on solids. out [n][3][hw] FP64; sums[b] += sum of rho over image b.
__global__ void warm_decode_kernel(const float* __restrict__ y, int hw, int n, const uint8_t* __restrict__ mask,
                                   float rho_mean, float rho_std, float u_scale, double lo, double hi,
                                   double* __restrict__ out, double* __restrict__ sums)
{
    __shared__ double red[kT];
    const int b = blockIdx.y;
    double s = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < hw; p += gridDim.x * blockDim.x) {
        const bool fluid = mask[(size_t)b * hw + p] == 0;
        const float* yb = y + (size_t)b * 3 * hw;
        double r = double(yb[p]) * rho_std + rho_mean;
        r = fluid ? fmin(fmax(r, lo), hi) : 0.0;
        double* ob = out + (size_t)b * 3 * hw;
        ob[p] = r;
        ob[hw + p] = fluid ? double(yb[hw + p]) * u_scale : 0.0;
        ob[2 * hw + p] = fluid ? double(yb[2 * hw + p]) * u_scale : 0.0;
        s += r;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&sums[b], red[0]);
}

// rho of image b scaled by mass[b] / sums[b]
__global__ void warm_scale_kernel(int hw, const double* __restrict__ mass, const double* __restrict__ sums,
                                  double* __restrict__ out)
{
    const int b = blockIdx.y;
    const double k = sums[b] > 0.0 ? mass[b] / sums[b] : 1.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < hw; p += gridDim.x * blockDim.x)
        out[(size_t)b * 3 * hw + p] *= k;
}

int blocks_for(long long n) { return int(n / kT + 1 < 4096 ? n / kT + 1 : 4096); }

int status(cudaError_t e) { return e == cudaSuccess ? 0 : int(e); }

__device__ int g_err = 0;  // set by a tensor-core kernel whose mbarrier wait timed out

int* err_ptr()
{
    static int* p = nullptr;
    if (!p) cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_err);
    return p;
}

template <int NT>
int launch_conv_row(const void* x, int ct_in, int kc, const void* wt, const float* bias, void* y, int ct_out,
                    int cout, int n, int h, int wd, int relu, cudaStream_t st)
{
    constexpr int needed = kRowStages * (kHaloBytes + 9 * NT * 32) + 2 * kRowStages * 8 + 16;
    const int smem = smem_for_tmem(int(tmem_cols(NT)), needed);
    auto k = conv3x3_tc_row_kernel<NT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return int(e);
    dim3 grid(h * (wd / kRowPix), cout / NT, n);
    k<<<grid, kTcThreads, smem, st>>>((const bf16*)x, ct_in, kc, (const bf16*)wt, bias, (bf16*)y, ct_out, h, wd, relu,
                                      err_ptr());
    return status(cudaGetLastError());
}

template <int NT, int CK>
int launch_conv_tile(const void* x, int ct_in, int kc, const void* wt, const float* bias, void* y, int ct_out,
                     int cout, int n, int h, int wd, int relu, cudaStream_t st)
{
    const int smem = smem_for_tmem(int(tmem_cols(NT)), conv_smem_needed<NT, CK>());
    auto k = conv3x3_tc_kernel<NT, CK>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return int(e);
    dim3 grid((h / kTileRows) * (wd / kTileCols), cout / NT, n);
    k<<<grid, kTcThreads, smem, st>>>((const bf16*)x, ct_in, kc, (const bf16*)wt, bias, (bf16*)y, ct_out, h, wd, relu,
                                      err_ptr());
    return status(cudaGetLastError());
}

template <int NT>
int launch_conv(const void* x, int ct_in, int kc, const void* wt, const float* bias, void* y, int ct_out, int cout,
                int n, int h, int wd, int relu, cudaStream_t st)
{
    if (wd % kRowPix == 0) return launch_conv_row<NT>(x, ct_in, kc, wt, bias, y, ct_out, cout, n, h, wd, relu, st);
    // chunks of 16 channels per ring slot: 4, 2 or 1, dividing kc
    if (kc % 4 == 0) return launch_conv_tile<NT, 4>(x, ct_in, kc, wt, bias, y, ct_out, cout, n, h, wd, relu, st);
    if (kc % 2 == 0) return launch_conv_tile<NT, 2>(x, ct_in, kc, wt, bias, y, ct_out, cout, n, h, wd, relu, st);
    return launch_conv_tile<NT, 1>(x, ct_in, kc, wt, bias, y, ct_out, cout, n, h, wd, relu, st);
}

template <int NT, int P, bool SW>
int launch_wgrad_p(const void* x, int ct_x, int ci, const void* dy, int ct_dy, int co, float* dw, int h, int wd,
                   int npix, long long total, cudaStream_t st)
{
    const int smem = smem_for_tmem(int(tmem_cols(3 * NT)), wgrad_smem_needed<NT, P, SW>());
    auto k = wgrad_tc_kernel<NT, P, SW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return int(e);
    constexpr int COT = wgrad_co_tile<NT, SW>(), CIT = wgrad_ci_tile<NT, SW>();
    dim3 grid((co + COT - 1) / COT, (ci + CIT - 1) / CIT, int(3 * (total / npix)));
    k<<<grid, kWgThreads, smem, st>>>((const bf16*)x, ct_x, ci, (const bf16*)dy, ct_dy, co, dw, h, wd, npix,
                                      err_ptr());
    return status(cudaGetLastError());
}

// CTAs of the weight gradient that fit on one SM (shared and tensor memory)
template <int NT, int P, bool SW> int wgrad_ctas_per_sm()
{
    const int smem = smem_for_tmem(int(tmem_cols(3 * NT)), wgrad_smem_needed<NT, P, SW>());
    const int by_smem = kSmemPerSm / (smem + 1024), by_tmem = 512 / int(tmem_cols(3 * NT));
    return by_smem < by_tmem ? (by_smem > 0 ? by_smem : 1) : by_tmem;
}

template <int NT, int P, bool SW>
int launch_wgrad_np(const void* x, int ct_x, int ci, const void* dy, int ct_dy, int co, float* dw, int n, int h,
                    int wd, cudaStream_t st)
{
    // pixels per CTA: a power of two dividing the total, at most 4096 (long
    // K loops: the tensor time of one layer is a few microseconds, and each
    // split adds its co x ci x 3 partial sums into dw with atomics), halved
    // while the grid fills less than half of the CTA slots, down to 8 K-steps
    const long long total = (long long)n * h * wd;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const long long slots = (long long)(sms > 0 ? sms : 148) * wgrad_ctas_per_sm<NT, P, SW>();
    constexpr int COT = wgrad_co_tile<NT, SW>(), CIT = wgrad_ci_tile<NT, SW>();
    const long long tiles = 3LL * ((co + COT - 1) / COT) * ((ci + CIT - 1) / CIT);
    int npix = 4096;
    while (npix > P && total % npix) npix >>= 1;
    while (npix > 8 * P && tiles * (total / npix) < slots / 2 && total % (npix / 2) == 0) npix >>= 1;
    return launch_wgrad_p<NT, P, SW>(x, ct_x, ci, dy, ct_dy, co, dw, h, wd, npix, total, st);
}

template <int NT, bool SW>
int launch_wgrad(const void* x, int ct_x, int ci, const void* dy, int ct_dy, int co, float* dw, int n, int h,
                 int wd, cudaStream_t st)
{
    // K-step: the widest of 64, 32, 16 pixels that divides the row (every
    // step stays inside one image row)
    if (wd % 64 == 0) return launch_wgrad_np<NT, 64, SW>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
    if (wd % 32 == 0) return launch_wgrad_np<NT, 32, SW>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
    return launch_wgrad_np<NT, 16, SW>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
}

}  // namespace
}  // namespace unet

using namespace unet;

extern "C" {

int unet_conv_ntile(int channels) { return conv_ntile(channels); }

size_t unet_conv_pack_elems(int co, int ci, int transpose)
{
    const int nrows = transpose ? ci : co, kreal = transpose ? co : ci;
    const int kc = (kreal + 15) / 16;
    return size_t(nrows) * kc * 16 * 9;
}

int unet_conv_pack(const float* w, int co, int ci, int transpose, void* out, void* stream)
{
    const int nrows = transpose ? ci : co, kreal = transpose ? co : ci;
    if (nrows % 32) return -1;
    const int kc = (kreal + 15) / 16;
    const long long total = (long long)nrows * kc * 16 * 9;
    conv_pack_kernel<<<blocks_for(total), kT, 0, (cudaStream_t)stream>>>(w, co, ci, transpose, conv_ntile(nrows), kc,
                                                                        (bf16*)out);
    return status(cudaGetLastError());
}

int unet_conv_pack_many(const long long* jobs, int njobs, long max_elems, void* stream)
{
    if (!jobs || njobs < 1 || njobs > 65535 || max_elems < 1) return -1;
    conv_pack_many_kernel<<<dim3(blocks_for(max_elems), njobs), kT, 0, (cudaStream_t)stream>>>(jobs);
    return status(cudaGetLastError());
}

int unet_conv3x3(const void* x, int ct_in, int cin, const void* wt, const float* bias, void* y, int ct_out, int cout,
                 int n, int h, int wd, int relu, void* stream)
{
    // K runs over kc chunks of 16 channels: cin a multiple of 16, or cin < 16
    // in a view whose first 16 channels are readable (channels >= cin zero)
    const int kc = (cin + 15) / 16;
    if (wd % kTileCols || h % kTileRows || cout % 32 || ct_in % 8 || ct_out % 8 || cin < 1 ||
        (cin % 16 && cin > 16) || kc * 16 > ct_in ||
        (reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(wt)) & 15)
        return -1;
    cudaStream_t st = (cudaStream_t)stream;
    switch (conv_ntile(cout)) {
    case 128: return launch_conv<128>(x, ct_in, kc, wt, bias, y, ct_out, cout, n, h, wd, relu, st);
    case 64: return launch_conv<64>(x, ct_in, kc, wt, bias, y, ct_out, cout, n, h, wd, relu, st);
    default: return launch_conv<32>(x, ct_in, kc, wt, bias, y, ct_out, cout, n, h, wd, relu, st);
    }
}

int unet_conv3x3_bwd_weight(const void* x, int ct_x, int ci, const void* dy, int ct_dy, int co, float* dw, float* db,
                            int n, int h, int wd, void* stream)
{
    if (wd % 16 || co % 8 || ct_x % 8 || ct_dy % 8 ||
        (reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(dy)) & 15)
        return -1;
    cudaStream_t st = (cudaStream_t)stream;
    // The MMA's 128 rows take the wider of the two channel counts: output
    // channels (tiles of 128; input channels in N tiles of 128, 64, 32 or 16,
    // at most ci rounded up to 16), or with more input than output channels
    // (at most 128 of them) input channels (tiles of 128; output channels in
    // one N tile of 32, 64 or 128).
    int rc;
    if (ci > co && co <= 128) {
        if (co <= 32)
            rc = launch_wgrad<32, true>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
        else if (co <= 64)
            rc = launch_wgrad<64, true>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
        else
            rc = launch_wgrad<128, true>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
    } else if (ci > 64)
        rc = launch_wgrad<128, false>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
    else if (ci > 32)
        rc = launch_wgrad<64, false>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
    else if (ci > 16)
        rc = launch_wgrad<32, false>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
    else
        rc = launch_wgrad<16, false>(x, ct_x, ci, dy, ct_dy, co, dw, n, h, wd, st);
    if (rc || !db) return rc;
    const long long npix = (long long)n * h * wd;
    const int per = 1024;
    bias_grad_kernel<<<int((npix + per - 1) / per), co <= kT ? co : kT, 0, st>>>((const bf16*)dy, ct_dy, co, npix, per,
                                                                                db);
    return status(cudaGetLastError());
}

int unet_tc_error(void* stream, int reset)
{
    int h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, err_ptr(), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return -int(e);
    if (reset && h) {
        const int z = 0;
        cudaMemcpyAsync(err_ptr(), &z, sizeof(int), cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
    }
    return h;
}

int unet_head_fwd(const void* x, int ct, int ci, const void* w, const float* bias, float* y, int co, int n, int hw,
                  void* stream)
{
    if (co < 1 || co > 8 || ci < 1 || ci > 64) return -1;
    head_fwd_kernel<<<blocks_for((long long)n * hw), kT, 0, (cudaStream_t)stream>>>((const bf16*)x, ct, ci,
                                                                                   (const bf16*)w, bias, y, co, hw, n);
    return status(cudaGetLastError());
}

int unet_head_bwd(const void* x, int ct, int ci, const void* w, const float* dy, int co, int n, int hw, void* dx,
                  int ct_dx, float* dw, float* db, void* stream)
{
    if (co != 3 || ci < 1 || ci > kT) return -1;
    // at most 8 blocks per SM: each block adds its partial sums into the same
    // 3 (ci + 1) addresses of dw and db
    long long blocks = (long long)n * hw * ci / (kT * 4) + 1;
    if (blocks > 1184) blocks = 1184;
    head_bwd_kernel<3><<<int(blocks), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, ct, ci, (const bf16*)w, dy, hw, n, (bf16*)dx, ct_dx, dw, db);
    return status(cudaGetLastError());
}

// the vector pooling/upsampling kernels: 8-channel groups, 16-byte aligned
// views, 32-bit element counts
static bool vec8_ok(const void* a, int cta, const void* b, int ctb, int c, long long elems)
{
    return c % 8 == 0 && cta % 8 == 0 && ctb % 8 == 0 && elems / 8 < (1LL << 31) &&
           ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

int unet_pool2_fwd(const void* x, int ctx, void* y, int cty, int c, int n, int h, int wd, void* stream)
{
    if (!vec8_ok(x, ctx, y, cty, c, (long long)n * c * h * wd) || h % 2 || wd % 2) return -1;
    pool2_fwd_kernel<<<blocks_for((long long)n * c / 8 * h * wd / 4), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, ctx, (bf16*)y, cty, c, h, wd, n);
    return status(cudaGetLastError());
}

int unet_pool2_bwd(const void* dy, int cty, void* dx, int ctx, int c, int n, int h, int wd, int accumulate,
                   void* stream)
{
    if (!vec8_ok(dy, cty, dx, ctx, c, (long long)n * c * h * wd) || h % 2 || wd % 2) return -1;
    pool2_bwd_kernel<<<blocks_for((long long)n * c / 8 * h * wd / 4), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)dy, cty, (bf16*)dx, ctx, c, h, wd, n, accumulate);
    return status(cudaGetLastError());
}

int unet_up2_fwd(const void* x, int ctx, void* y, int cty, int c, int n, int h, int wd, void* stream)
{
    if (c % 8 || ctx % 8 || cty % 8 || (reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15)
        return -1;
    up2_fwd_kernel<<<blocks_for((long long)n * c / 8 * h * wd * 4), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)x, ctx, (bf16*)y, cty, c, h, wd, n);
    return status(cudaGetLastError());
}

int unet_up2_bwd(const void* dy, int cty, void* dx, int ctx, int c, int n, int h, int wd, void* stream)
{
    if (!vec8_ok(dy, cty, dx, ctx, c, (long long)n * c * h * wd * 4)) return -1;
    up2_bwd_kernel<<<blocks_for((long long)n * c / 8 * h * wd), kT, 0, (cudaStream_t)stream>>>(
        (const bf16*)dy, cty, (bf16*)dx, ctx, c, h, wd, n);
    return status(cudaGetLastError());
}

int unet_relu_bwd(const void* y, int cty, void* dy, int ctd, int c, long npix, float* db, void* stream)
{
    if (c < 8 || c > kT || c % 8 || cty % 8 || ctd % 8 ||
        (reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(dy)) & 15)
        return -1;
    long long blocks = (long long)npix * (c / 8) / (kT * 4) + 1;  // about 4 pixels per thread: one round
    if (blocks > 1184) blocks = 1184;                                 // 8 per SM
    relu_bwd_kernel<<<int(blocks), kT, 0, (cudaStream_t)stream>>>((const bf16*)y, cty, (bf16*)dy, ctd, c, npix, db);
    return status(cudaGetLastError());
}

int unet_input_nhwc(const float* x, int c, int hw, int n, void* y, int ct, void* stream)
{
    input_nhwc_kernel<<<blocks_for((long long)n * hw * ct), kT, 0, (cudaStream_t)stream>>>(x, c, hw, n, (bf16*)y, ct);
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
                                                                    weight_decay, nullptr);
    return status(cudaGetLastError());
}

int unet_adam_dev(float* w_master, void* w_bf16, const float* grad, float* m, float* v, long count,
                  const float* hyper, float beta1, float beta2, float eps, float weight_decay, void* stream)
{
    if (!hyper) return -1;
    adam_kernel<<<blocks_for(count), kT, 0, (cudaStream_t)stream>>>(w_master, (bf16*)w_bf16, grad, m, v, count, 0.f,
                                                                    beta1, beta2, eps, 1.f, 1.f, weight_decay, hyper);
    return status(cudaGetLastError());
}

int unet_adam_hyper(float* state, const float* lr_schedule, int n, float beta1, float beta2, void* stream)
{
    if (!state || !lr_schedule || n < 1) return -1;
    adam_hyper_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(state, lr_schedule, n, beta1, beta2);
    return status(cudaGetLastError());
}

int unet_warm_fields(const float* y, int n, int hw, const uint8_t* mask, const double* mass, float rho_mean,
                     float rho_std, float u_scale, double lo, double hi, double* out, double* sums, void* stream)
{
    if (n < 1 || n > 65535 || hw < 1) return -1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(sums, 0, size_t(n) * sizeof(double), st);
    if (e != cudaSuccess) return int(e);
    const int bx = (hw + kT - 1) / kT < 64 ? (hw + kT - 1) / kT : 64;
    warm_decode_kernel<<<dim3(bx, n), kT, 0, st>>>(y, hw, n, mask, rho_mean, rho_std, u_scale, lo, hi, out, sums);
    warm_scale_kernel<<<dim3(bx, n), kT, 0, st>>>(hw, mass, sums, out);
    return status(cudaGetLastError());
}

int unet_f32_to_bf16(const float* x, void* y, long count, void* stream)
{
    f32_to_bf16_kernel<<<blocks_for(count), kT, 0, (cudaStream_t)stream>>>(x, (bf16*)y, count);
    return status(cudaGetLastError());
}

}  // extern "C"
