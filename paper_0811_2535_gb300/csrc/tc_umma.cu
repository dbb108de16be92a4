// Reduced-precision path on the 5th-generation tensor cores (tcgen05).
//
// A radix-16 stage multiplies every 16-point vector by the DFT-16 matrix.
// With real and imaginary parts interleaved on both sides this is, for the
// 256 vectors of a 4096-point block, one real GEMM
//     D[v][2k + c'] = sum_{m, c} A[v][2m + c] * W[2k + c'][2m + c]
// (M = 256 vectors as two M = 128 tiles, N = 32 outputs, K = 32 inputs).
// A (the data, split into FP16 or BF16 parts) lives in tensor memory: row v
// is TMEM lane v % 128 of tile v / 128, two 16-bit K entries per 32-bit
// column, written by its own thread with tcgen05.st.  W (split the same way)
// lives in shared memory in the K-major canonical layout without swizzle
// (core matrices of 8 rows x 16 bytes, 128 bytes apart along K, 512 bytes
// apart along N).  The FP32 accumulators D live in tensor memory too.  One
// thread issues the products and commits them to an mbarrier; thread v then
// reads row v of D (tcgen05.ld), applies the FP32 twiddle and writes its 16
// outputs to their rows of the next stage through a padded FP32 exchange
// buffer (the Stockham reordering of the index digits), reads back its own
// new row, splits it and stores it to tensor memory.
//
// Compensation: FP16 hi + lo with the three products of order up to 2^-11,
// each row scaled by the power of two that puts its largest |re|, |im| in
// [2^10, 2^11) (exact, undone on the same row of D); BF16 hi + mid + lo with
// the six products of order up to 2^-16 and no scaling.
//
// Index digits, N = 4096: j = j0 + 16 j1 + 256 j2, k = k0 + 16 k1 + 256 k2.
//   stage 0: row u = j0 + 16 j1, points j2, twiddle w_4096^(u k0)
//   stage 1: row j0 + 16 k0, points j1, twiddle w_256^(j0 k1)
//   stage 2: row k0 + 16 k1, points j0, output X[row + 256 k2]
// N = 256, sixteen transforms rho per block of 4096 points: j = j0 + 16 j1.
//   stage 0: row j0 + 16 rho, points j1, twiddle w_256^(j0 k0)
//   stage 1: row k0 + 16 rho, points j0, output X_rho[k0 + 16 k1]
// These maps make the global loads and stores coalesced and the exchange
// (row stride 17 complex64) free of bank conflicts.
#include "fft_core.cuh"
#include "internal.h"
#include "tc_common.cuh"
#include "tmem.cuh"

namespace moa {

namespace {

__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor for tcgen05.mma: start address, leading
// byte offset (between core matrices adjacent along K), stride byte offset
// (between 8-row groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B format FP16 (0) or BF16 (1) in bits 7-9 and 10-12, both K-major, N / 8 in
// bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc(bool bf16, int M, int N)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Arrive on `bar` once every tcgen05.mma issued so far by this thread is complete.
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
                 : "memory");
}

// D[tmem] (+)= A * B^T with A in tensor memory (M rows = lanes, two 16-bit
// K entries per 32-bit column) and B in shared memory.
__device__ __forceinline__ void umma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mbar_init1(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; false when the phase did not complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t polls = 0; polls < (1u << 24); ++polls)
        if (mbar_try(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <bool BF16> struct TcLayout {
    static constexpr int PARTS = tc::Split2<BF16>::PARTS;
    static constexpr int RS = 17;                          // exchange row stride (complex64 entries)
    static constexpr uint32_t EX_BYTES = 256 * RS * 8;     // [256][17] complex64
    static constexpr uint32_t W_PLANE = 2048;              // 32 rows x 32 16-bit entries
    static constexpr uint32_t W_OFF = EX_BYTES;
    static constexpr uint32_t TW_OFF = W_OFF + PARTS * W_PLANE;     // stage twiddle table (4096 + 256 complex64)
    static constexpr uint32_t TW_BYTES = (4096 + 256) * 8;
    static constexpr uint32_t MISC_OFF = TW_OFF + TW_BYTES;           // mbarrier, TMEM slot, abort flag
    // at most two blocks per SM (their TMEM columns must fit the SM's 512)
    static constexpr uint32_t BYTES = 84 * 1024;
    static_assert(MISC_OFF + 64 <= BYTES, "shared memory layout");
    // TMEM columns: D of tile t at 32 t; A part p of tile t at 64 + 16 (2 p + t)
    static constexpr uint32_t A_COL = 64;
    static constexpr uint32_t COLS = BF16 ? 256 : 128;
};

// One block of 4096 points (one 4096-point transform, or sixteen 256-point
// transforms) per iteration; persistent over blocks.  256 threads: thread t
// owns row t of A and D at every stage (tile t / 128, TMEM lane t % 128).
template <bool BF16, int LOGN>
__global__ void __launch_bounds__(256, 2)
    tc_umma_kernel(const float2 *in, float2 *out, int64_t rows, const float2 *__restrict__ tw, int flags, int *status)
{
    using L = TcLayout<BF16>;
    using SP = tc::Split<BF16>;
    using S2 = tc::Split2<BF16>;
    constexpr int PARTS = L::PARTS;
    constexpr int S = LOGN / 4;
    constexpr int RPG = 4096 >> LOGN;   // transforms per block of 4096 points
    constexpr int RS = L::RS;
    constexpr uint32_t IDESC = umma_idesc(BF16, 128, 32);
    static_assert(LOGN == 12 || LOGN == 8, "N = 4096 or 256");
    extern __shared__ __align__(1024) uint8_t smem[];
    float2 *ex = reinterpret_cast<float2 *>(smem);
    uint8_t *sW = smem + L::W_OFF;
    float2 *stw = reinterpret_cast<float2 *>(smem + L::TW_OFF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::MISC_OFF);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + L::MISC_OFF + 8);
    int *abort_flag = reinterpret_cast<int *>(smem + L::MISC_OFF + 12);

    const int tid = threadIdx.x, warp = tid >> 5, tile = tid >> 7;
    const int64_t groups = (rows + RPG - 1) / RPG;

    // W split into parts, K-major: entry (o, kk) at (o/8)*512 + (kk/8)*128 + (o%8)*16 + (kk%8)*2
    for (int e = tid; e < 1024; e += 256) {
        const int o = e >> 5, kk = e & 31;
        uint16_t p[3];
        SP::run(tc::w_interleaved(o, kk), p);
        const uint32_t off = (o >> 3) * 512 + (kk >> 3) * 128 + (o & 7) * 16 + (kk & 7) * 2;
#pragma unroll
        for (int q = 0; q < PARTS; ++q)
            *reinterpret_cast<uint16_t *>(sW + q * L::W_PLANE + off) = p[q];
    }
    // the stage twiddles, read every stage by every thread, kept on chip
    constexpr int TW_N = LOGN == 12 ? 4096 + 256 : 256;
    for (int e = tid; e < TW_N; e += 256)
        stw[e] = tw[e];
    if (warp == 0)
        tmem_alloc(tslot, L::COLS);
    if (tid == 0) {
        mbar_init1(bar);
        *abort_flag = 0;
    }
    fence_async_smem();
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;   // this warp's quarter of the lanes
    const uint32_t d_row = tmem + lanes + 32 * tile;

    const float cin = (flags & FLAG_CONJ_IN) ? -1.f : 1.f;
    const float cout = (flags & FLAG_CONJ_OUT) ? -1.f : 1.f;

    // stage-0 points of this thread's row for block g (zeros past the last transform)
    auto load_block = [&](int64_t g, float2 (&x)[16]) {
        if constexpr (LOGN == 12) {
            const float2 *src = in + g * 4096 + tid;   // row u = tid, points x[u + 256 m]
#pragma unroll
            for (int m = 0; m < 16; ++m)
                x[m] = __ldcs(src + 256 * m);
        } else {
            const int rho = tid >> 4, j0 = tid & 15;   // row j0 + 16 rho, points x_rho[j0 + 16 m]
            const bool valid = g * 16 + rho < rows;
            const float2 *src = in + (g * 16 + rho) * 256 + j0;
#pragma unroll
            for (int m = 0; m < 16; ++m)
                x[m] = valid ? __ldcs(src + 16 * m) : make_float2(0.f, 0.f);
        }
    };

    // row `tid` of A from 16 points: FP16 scaled by a power of two putting the
    // row's largest |re|, |im| in [2^10, 2^11); parts into TMEM.  Returns the
    // factor that undoes the scaling on row `tid` of D.
    auto store_a = [&](float2 (&v)[16]) -> float {
        float scale = 1.f;
        if constexpr (!BF16) {
            float mx = 0.f;
#pragma unroll
            for (int m = 0; m < 16; ++m)
                mx = fmaxf(mx, fmaxf(fabsf(v[m].x), fabsf(v[m].y)));
            scale = mx > 0.f ? ldexpf(1.f, 10 - ilogbf(mx)) : 1.f;
#pragma unroll
            for (int m = 0; m < 16; ++m)
                v[m] = make_float2(v[m].x * scale, v[m].y * scale);
        }
#pragma unroll
        for (int p = 0; p < PARTS; ++p) {
            uint32_t w[16];
#pragma unroll
            for (int m = 0; m < 16; ++m)
                w[m] = S2::take(v[m]);
            tmem_st16(tmem + lanes + L::A_COL + 16 * (2 * p + tile), w);
        }
        tmem_st_wait();
        return 1.f / scale;   // a power of two: exact
    };

    // all products of one stage into D, then a bounded wait for them
    uint32_t phase = 0;
    auto mma_stage = [&]() -> bool {
        tmem_fence_before();
        __syncthreads();
        if (tid == 0) {
            tmem_fence_after();
            const uint32_t b0 = s_u32(sW);
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                uint32_t acc = 0;
#pragma unroll
                for (int ord = PARTS - 1; ord >= 0; --ord)
#pragma unroll
                    for (int pa = 0; pa <= ord; ++pa) {
                        const int pb = ord - pa;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            umma_f16_ts(tmem + 32 * t, tmem + L::A_COL + 16 * (2 * pa + t) + 8 * h,
                                        umma_desc(b0 + pb * L::W_PLANE + h * 256, 128, 512), IDESC, acc);
                            acc = 1;
                        }
                    }
            }
            umma_commit(bar);
            if (!mbar_wait_bounded(bar, phase)) {
                atomicExch(status, 6);   // MOA_ERR_TIMEOUT
                *abort_flag = 1;
            }
        }
        phase ^= 1u;
        __syncthreads();
        tmem_fence_after();
        return *abort_flag == 0;
    };

    float2 x[16];
    int64_t g = blockIdx.x;
    if (g < groups)
        load_block(g, x);
    bool ok = true;
    for (; g < groups && ok; g += gridDim.x) {
#pragma unroll
        for (int m = 0; m < 16; ++m)
            x[m].y *= cin;
        float unscale = store_a(x);
        if (g + gridDim.x < groups)
            load_block(g + gridDim.x, x);   // next block's inputs, in flight during the stages

#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!mma_stage()) {
                ok = false;
                break;
            }
            uint32_t d[32];
            tmem_ld32(d_row, d);
            float2 y[16];
#pragma unroll
            for (int k = 0; k < 16; ++k)
                y[k] = make_float2(__uint_as_float(d[2 * k]) * unscale, __uint_as_float(d[2 * k + 1]) * unscale);

            if (s < S - 1) {
                // twiddle, then output k to row rbase + 16 k (LOGN 12) or rbase + k
                // (LOGN 8), point mp, of the next stage through the exchange buffer
                int rbase, rstep, mp;
                if constexpr (LOGN == 12) {
                    if (s == 0) {   // row u = j0 + 16 j1 -> row j0 + 16 k0, point j1
#pragma unroll
                        for (int k = 1; k < 16; ++k)
                            y[k] = cmul(y[k], stw[k * 256 + tid]);
                        rbase = tid & 15;
                        mp = tid >> 4;
                    } else {        // row j0 + 16 k0 -> row k0 + 16 k1, point j0
#pragma unroll
                        for (int k = 1; k < 16; ++k)
                            y[k] = cmul(y[k], stw[4096 + k * 16 + (tid & 15)]);
                        rbase = tid >> 4;
                        mp = tid & 15;
                    }
                    rstep = 16;
                } else {            // row j0 + 16 rho -> row k0 + 16 rho, point j0
#pragma unroll
                    for (int k = 1; k < 16; ++k)
                        y[k] = cmul(y[k], stw[k * 16 + (tid & 15)]);
                    rbase = 16 * (tid >> 4);
                    rstep = 1;
                    mp = tid & 15;
                }
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    ex[(rbase + rstep * k) * RS + mp] = y[k];
                __syncthreads();
#pragma unroll
                for (int m = 0; m < 16; ++m)
                    y[m] = ex[tid * RS + m];
                unscale = store_a(y);
            } else if constexpr (LOGN == 12) {
                // row k0 + 16 k1 = tid: X[tid + 256 k2], coalesced across the warp
                float2 *dst = out + g * 4096 + tid;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    __stcs(dst + 256 * k, make_float2(y[k].x, y[k].y * cout));
            } else {
                // row k0 + 16 rho = tid: X_rho[k0 + 16 k1]
                const int rho = tid >> 4, k0 = tid & 15;
                if (g * 16 + rho < rows) {
                    float2 *dst = out + (g * 16 + rho) * 256 + k0;
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        __stcs(dst + 16 * k, make_float2(y[k].x, y[k].y * cout));
                }
            }
        }
    }

    tmem_fence_before();
    __syncthreads();
    if (!ok && tid == 0)
        mbar_wait_bounded(bar, phase ^ 1u);   // products still in flight after a timeout
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after();
        tmem_dealloc(tmem, L::COLS);
    }
}

template <bool BF16, int LOGN>
cudaError_t launch_umma_typed(const PassDesc &d, const float2 *in, float2 *out, const float2 *tw, int flags,
                              cudaStream_t stream, int *status)
{
    using L = TcLayout<BF16>;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_umma_kernel<BF16, LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)L::BYTES);
    if (e != cudaSuccess)
        return e;
    const int64_t groups = LOGN == 12 ? d.O : (d.O + 15) / 16;
    const int64_t grid = groups < (int64_t)sms * 2 ? groups : (int64_t)sms * 2;
    tc_umma_kernel<BF16, LOGN><<<(unsigned)grid, 256, L::BYTES, stream>>>(in, out, d.O, tw, flags, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_umma_pass(const PassDesc &d, bool bf16, const float2 *in, float2 *out, const float2 *tw, int flags,
                             cudaStream_t stream, int *status)
{
    if (d.logN == 12)
        return bf16 ? launch_umma_typed<true, 12>(d, in, out, tw, flags, stream, status)
                    : launch_umma_typed<false, 12>(d, in, out, tw, flags, stream, status);
    if (d.logN == 8)
        return bf16 ? launch_umma_typed<true, 8>(d, in, out, tw, flags, stream, status)
                    : launch_umma_typed<false, 8>(d, in, out, tw, flags, stream, status);
    return cudaErrorInvalidValue;
}

}  // namespace moa
