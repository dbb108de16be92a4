// Pipelined strided passes for N = 1024..4096 with four transforms per tile.
//
// These are the two halves of the dimension-lifted transform that touch
// memory with a stride: the column pass (paper's block phase, Fig. 4.8-4.9:
// r-point transforms down the columns of the r x c array, then the twiddle
// w_n^(j2*k1)) and the transposed row pass (cyclic phase: c-point
// transforms along rows, stored at X[k1 + r*k2]).  Four transforms per tile
// make every row segment a whole 32-byte sector; with N = 4096 that tile is
// 128 KiB, so only one tile fits an SM (registers hold the tile being
// computed, shared memory its exchange buffer).  To keep HBM busy anyway
// each block is persistent and refills its shared memory asynchronously:
//
//   H (landing buffer): TMA brings the first part of tile i+1 while tile i
//     computes: for columns, as many 256-row boxes (256 rows x 32 bytes) as
//     fit beside E, 11 of 16 at N = 4096, in one cp.async.bulk.tensor copy
//     whose box spans those 256-row blocks; for rows, the first half of each
//     row (cp.async.bulk);
//   E (exchange buffer, (N + N/16) x 4 complex64): the single-round register
//     exchanges of tile i's radix-16 stages; as soon as the last exchange has
//     been read, TMA lands the rest of tile i+1 in it, overlapping the last
//     stage, the epilogue and the stores of tile i.
//
// Completion is tracked on two mbarriers.  One elected thread waits on them
// with an iteration limit; on timeout it records MOA_ERR_TIMEOUT in the
// status word and the whole block returns.
#include <cuda.h>

#include <cstdlib>

#include "fft_core.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace moa {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z,
                                            int w)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Asynchronous stores from shared memory (TMA, bulk-group completion).
__device__ __forceinline__ void bulk_store(void *gdst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
                 "r"(y), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *src, int x, int y, int z, int w)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(src))
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the staged data has been read out of shared memory (it may be reused)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// the stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Upper bound on mbarrier polls before a wait is declared failed (each
// try_wait may suspend the thread for a while; a normal tile load completes
// within a few thousand polls).
constexpr uint32_t kMaxPolls = 1u << 26;

__device__ __forceinline__ float2 two_level_tw(const float2 *__restrict__ lo, const float2 *__restrict__ hi, int h,
                                               int64_t e)
{
    return cmul(__ldg(&lo[e & ((int64_t(1) << h) - 1)]), __ldg(&hi[e >> h]));
}

struct PipeSmem {
    // entries (float2) of the exchange buffer E, which also lands the second
    // half of the next tile, and of the first-half landing buffer H
    template <int LOGN> __host__ __device__ static constexpr int E_entries() { return ((1 << LOGN) + (1 << LOGN) / 16) * 4; }
    template <int LOGN> __host__ __device__ static constexpr int row_pitch() { return (1 << LOGN) / 2 + 4; }
    template <int LOGN> __host__ __device__ static constexpr int H_entries() { return 4 * row_pitch<LOGN>(); }
    template <int LOGN> __host__ __device__ static constexpr size_t bytes()
    {
        return (size_t)(E_entries<LOGN>() + H_entries<LOGN>() + 64) * 8 + 64;
    }
    // column kernel: per-tile twiddle tables behind H (three tables of
    // [16][4] entries: the four-step factors of the tile's columns)
    static constexpr int kTwEntries = 192;
    // column kernel: rows of the next tile that land early (while the tile
    // computes) in a buffer of their own; the rest lands in the exchange
    // buffer after its last use.  As many whole 256-row boxes as fit next to
    // the exchange buffer and the tables, at most all but one.
    template <int LOGN> __host__ __device__ static constexpr int early_rows()
    {
        return ((((232448 - E_entries<LOGN>() * 8 - kTwEntries * 8 - 64) / 32) / 256) * 256) < (1 << LOGN) - 256
                   ? (((232448 - E_entries<LOGN>() * 8 - kTwEntries * 8 - 64) / 32) / 256) * 256
                   : (1 << LOGN) - 256;
    }
};

__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase by one thread; on timeout the status word
// gets MOA_ERR_TIMEOUT and *abort_flag is set.  With FLAG_SHORT_WAIT (fault
// injection for tests) the wait is a single test, which gives up on a load
// still in flight.
__device__ __forceinline__ void bounded_wait(uint64_t *bar, uint32_t parity, int *status, int *abort_flag, int flags)
{
    if (flags & FLAG_SHORT_WAIT) {
        if (!mbar_test_wait(bar, parity)) {
            atomicExch(status, 6);   // MOA_ERR_TIMEOUT
            *abort_flag = 1;
        }
        return;
    }
    uint32_t polls = 0;
    while (!mbar_try_wait(bar, parity)) {
        if (++polls >= kMaxPolls) {
            atomicExch(status, 6);   // MOA_ERR_TIMEOUT
            *abort_flag = 1;
            return;
        }
    }
}

// After a wait gave up: wait (bounded) for the tile's loads still in flight,
// so that no copy lands in shared memory the block has given up.
__device__ __forceinline__ void drain_in_flight(uint64_t *bar, uint32_t parity)
{
    for (int b = 0; b < 2; ++b)
        for (uint32_t polls = 0; polls < kMaxPolls && !mbar_try_wait(&bar[b], parity); ++polls) {
        }
}

// Rows [0, HR) (h = 0) or [HR, N) (h = 1) of a column tile's four columns:
// one TMA copy of HR / 256 (or (N - HR) / 256) boxes of 256 rows x 32 bytes,
// through the tensor map of that depth (tmapH for h = 0, tmapE for h = 1).
template <int LOGN, int BLK>
__device__ __forceinline__ void issue_tile_part(const CUtensorMap *tmapH, const CUtensorMap *tmapE, int logTpo,
                                                int tile, int h, float2 *dst, uint64_t *b)
{
    constexpr int N = 1 << LOGN;
    constexpr int HR = PipeSmem::early_rows<LOGN>();
    const int o = tile >> logTpo;
    const int c0 = (tile & ((1 << logTpo) - 1)) << 2;
    const int r0 = h ? HR : 0, nb = (h ? N - HR : HR) / 256;
    const CUtensorMap *map = h ? tmapE : tmapH;
    mbar_arrive_expect_tx(b, nb * 256 * 4 * (uint32_t)sizeof(float2));
    if constexpr (BLK == 3)
        tma_load_3d(dst, map, b, 2 * (c0 & 255), o * 256, 16 * (c0 >> 8) + (r0 >> 8));
    else if constexpr (BLK == 2)
        tma_load_4d(dst, map, b, 0, c0 >> 2, 0, (o * N + r0) >> 8);
    else
        tma_load_3d(dst, map, b, 2 * c0, 0, (o * N + r0) >> 8);
}

// The three radix stages of N = 1024, 2048, 4096 (radix 4/8/16, 16, 16) with
// single-round exchanges through E; `after_last_read` runs once E is no
// longer needed (used to start refilling it).
template <int LOGN, bool TW0 = true, typename F>
__device__ __forceinline__ void three_stages(float2 (&v)[16], float2 *E, int tau, int f, const float2 *__restrict__ tw,
                                             F after_last_read)
{
    static_assert(Sched<LOGN>::S == 3, "three-stage schedule expected");
    stage_compute<LOGN, 0, TW0>(v, tau, tw);
    stage_write<LOGN, 0, 2>(v, E, tau, f);
    __syncthreads();
    stage_read<LOGN, 1, 2>(v, E, tau, f);
    __syncthreads();
    stage_compute<LOGN, 1>(v, tau, tw);
    stage_write<LOGN, 1, 2>(v, E, tau, f);
    __syncthreads();
    stage_read<LOGN, 2, 2>(v, E, tau, f);
    __syncthreads();
    after_last_read();
    stage_compute<LOGN, 2>(v, tau, tw);
}

// Column pass: view [O][N][C], tile = 4 consecutive columns of one o.
//
// BLK selects the blocked workspace of the lifted transform, in which the
// r x c intermediate is stored as 4 x 4 blocks of 128 bytes: element
// (k1, j2) at ((j2/4)*(r/4) + k1/4)*16 + (j2%4)*4 + k1%4.  A tile of four
// columns then writes whole blocks (256 contiguous bytes per warp) and the
// tile of four rows of the second pass reads whole blocks.
//   BLK = 0: rows of the tile from a 2-D tensor map, output in the [O][N][C]
//            view (32-byte row segments);
//   BLK = 1: lifted pass 1 (N = r, C = c): 2-D tensor map in, blocked out;
//   BLK = 2: lifted pass 2 (N = c, C = r): the blocked workspace through a
//            3-D tensor map {32 floats, r/4, O*c/4}, output in the [O][N][C]
//            view, i.e. X[k1 + r*k2].
//   BLK = 3: second pass of the two-pass 3-D transform of 256 x 256 x 256
//            arrays (N = 4096, C = 256; the tile index within a transform is
//            64*k1b + g): the 16 rows 16*k1b + j1a of every plane j0 and
//            columns 4g..4g+3 land as element e = j0 + 256*j1a through a 3-D
//            tensor map {512 floats, O*256 planes, 256 rows}.  The stage-0
//            DFT (over j1a) takes no twiddle, so the tile computes the 2-D DFT
//            over (j1a, j0); output k = k1a + 16*k0 goes to
//            X[k0][k1b + 16*k1a][column].
//
// Staged stores (N = 4096, `staged` != 0): once the last exchange has been
// read, the exchange buffer E has room for the late rows of the next tile
// (its first 40 KiB) and for twelve of the tile's sixteen output slices
// (slice k = outputs tau + 256k of the four columns, 8 KiB each).  The
// threads write those slices to E and one thread hands them to TMA stores
// (BLK = 1: one bulk copy of the tile's first 96 KiB of blocked output;
// BLK = 0, 2: a 2-D tensor map over the output rows, one 256-row box per
// slice; BLK = 3: a 4-D tensor map {columns, k1b, k1a, planes}, one box of
// 16 x 16 rows per slice); the other four slices go out as plain stores.
// The TMA engine then drains the outputs while the next tile lands and
// computes; the slices must have left E before the next tile's first
// exchange, which one thread waits for at the tile start.
template <int LOGN, bool TW4, int BLK>
__global__ void __launch_bounds__(1 << (LOGN - 2), 1)
    pipe_col_kernel(const __grid_constant__ CUtensorMap tmapH, const __grid_constant__ CUtensorMap tmapE,
                    const __grid_constant__ CUtensorMap omap, float2 *out,
                    int C, int logTpo, int ntiles, const float2 *__restrict__ tw, const float2 *__restrict__ tw_lo,
                    const float2 *__restrict__ tw_hi, int tw_h, int flags, int staged, int *status)
{
    using Sc = Sched<LOGN>;
    constexpr int N = Sc::N, T = Sc::T;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2 *E = reinterpret_cast<float2 *>(smem_raw);
    float2 *H = E + PipeSmem::E_entries<LOGN>();
    constexpr int HR = PipeSmem::early_rows<LOGN>();   // rows landing in H; rows HR..N-1 land in E
    float2 *tk = H + 4 * HR;                           // [16][4] four-step twiddle factors
    uint64_t *bar = reinterpret_cast<uint64_t *>(tk + PipeSmem::kTwEntries);   // [0]: H, [1]: the rest in E
    int *abort_flag = reinterpret_cast<int *>(bar + 2);

    const int tid = threadIdx.x;
    const int f = tid & 3, tau = tid >> 2;
    const unsigned tpo_mask = (1u << logTpo) - 1;

    auto issue_half = [&](int tile, int h, float2 *dst, uint64_t *b) {
        issue_tile_part<LOGN, BLK>(&tmapH, &tmapE, logTpo, tile, h, dst, b);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    __syncthreads();
    int tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) {
        pdl_wait_prior();   // the input may be the previous kernel's output
        issue_half(tile, 0, H, &bar[0]);
        issue_half(tile, 1, E, &bar[1]);
    }
    uint32_t parity = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        const int o = tile >> logTpo;
        const int col = ((tile & tpo_mask) << 2) + f;
        const int next = tile + (int)gridDim.x;
        if (next >= ntiles)
            pdl_launch_dependents();   // the block's last tile: let the next kernel launch
        if (tid == 0) {
            bounded_wait(&bar[0], parity, status, abort_flag, flags);
            bounded_wait(&bar[1], parity, status, abort_flag, flags);
            if (*abort_flag)
                drain_in_flight(bar, parity);
        }
        __syncthreads();
        if (*abort_flag) {
            if (LOGN == 12 && staged && tid == 0)
                bulk_wait_all();   // no staged store may still read E
            return;
        }
        parity ^= 1u;

        // element tau + T*q lands in register (q % NB0)*R0 + q / NB0 (stage-0 order);
        // rows below HR (q < HR / T) are in H, the others in E
        constexpr int R0 = 1 << Sc::rlog(0), NB0 = 16 / R0;
        static_assert(HR % T == 0, "early rows must be whole row blocks");
        float2 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float2 *src = q * T < HR ? H + (tau + T * q) * 4 : E + (tau + T * q - HR) * 4;
            v[(q % NB0) * R0 + q / NB0] = src[f];
        }
        if (LOGN == 12 && staged && tid == 0)
            bulk_wait_read();   // the previous tile's staged outputs have left E
        __syncthreads();   // H and E have been read
        if (tid == 0 && next < ntiles) {
            fence_proxy_async();
            issue_half(next, 0, H, &bar[0]);
        }
        if (flags & FLAG_CONJ_IN) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
                v[r].y = -v[r].y;
        }
        if constexpr (TW4) {
            if (tau < 16)
                tk[tau * 4 + f] = two_level_tw(tw_lo, tw_hi, tw_h, (int64_t)col * (T * tau));
        }

        three_stages<LOGN, BLK != 3>(v, E, tau, f, tw, [&] {
            if (tid == 0 && next < ntiles) {
                fence_proxy_async();
                issue_half(next, 1, E, &bar[1]);
            }
        });

        if constexpr (TW4) {
            const float2 A = two_level_tw(tw_lo, tw_hi, tw_h, (int64_t)col * tau);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                v[k] = cmul(v[k], cmul(A, tk[k * 4 + f]));
        }
        if (flags & FLAG_CONJ_OUT) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
                v[k].y = -v[k].y;
        }
        // outputs k >= k0 of the thread with plain stores
        auto store_plain = [&](int k0) {
            if constexpr (BLK == 3) {
                // output k = k1a + 16*k0 with tau + T*k = k: k1a = tau % 16, k0 = tau/16 + 16*k
                static_assert(N == 4096 && T == 256, "the 3-D second pass is a 16 x 256 tile");
                float2 *dst = out + ((int64_t)o << 24) + (int64_t)(tau >> 4) * 65536 +
                              ((col >> 8) + 16 * (tau & 15)) * 256 + (col & 255);
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k >= k0)
                        dst[(int64_t)k << 20] = v[k];
            } else if constexpr (BLK == 1) {
                // element (tau + T*k, col) of the tile: block ((col/4)*(N/4) + (tau + T*k)/4),
                // slot f*4 + tau%4 (T is a multiple of 4)
                float2 *dst = out + (int64_t)o * N * C + (int64_t)((col >> 2) * (N >> 2)) * 16 + f * 4 +
                              (tau >> 2) * 16 + (tau & 3);
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k >= k0)
                        dst[k * 4 * T] = v[k];
            } else {
                float2 *dst = out + (int64_t)o * N * C + col + (int64_t)tau * C;
                const int64_t step = (int64_t)T * C;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k >= k0)
                        dst[k * step] = v[k];
            }
        };
        if (LOGN == 12 && staged) {
            // slices 0..KS-1 to E behind the late rows of the next tile, the rest plain
            constexpr int LATE = N - HR;
            constexpr int KS = (PipeSmem::E_entries<LOGN>() - 4 * LATE) / (4 * T);
            static_assert(KS >= 1 && KS < 16 && (4 * LATE * 8) % 1024 == 0, "staging slices");
            float2 *stg = E + 4 * LATE;
            const int sidx = BLK == 1 ? (tau >> 2) * 16 + f * 4 + (tau & 3) : tau * 4 + f;
#pragma unroll
            for (int k = 0; k < KS; ++k)
                stg[k * 4 * T + sidx] = v[k];
            store_plain(KS);
            __syncthreads();   // the staged slices are complete
            if (tid == 0) {
                fence_proxy_async();   // written through the generic proxy, read by TMA
                const int c0 = (tile & tpo_mask) << 2;
                if constexpr (BLK == 1) {
                    bulk_store(out + (int64_t)o * N * C + (int64_t)(c0 >> 2) * (N >> 2) * 16, stg,
                               (uint32_t)(KS * 4 * T * sizeof(float2)));
                } else {
#pragma unroll 1
                    for (int k = 0; k < KS; ++k) {
                        if constexpr (BLK == 3)
                            tma_store_4d(&omap, stg + k * 4 * T, 2 * (c0 & 255), c0 >> 8, 0, o * 256 + 16 * k);
                        else
                            tma_store_2d(&omap, stg + k * 4 * T, 2 * c0, o * N + T * k);
                    }
                }
                bulk_commit();
            }
        } else {
            store_plain(0);
        }
    }
    if (LOGN == 12 && staged && tid == 0)
        bulk_wait_all();   // the staged stores are complete before the block exits
}

// ---------------------------------------------------------------------------
// Two columns per thread (N = 4096).  The four columns of a tile are four
// independent transforms with the same butterflies and the same stage
// twiddles, so a thread can carry two of them: 512 threads, thread (tau, g)
// holds columns 2g and 2g+1 in v and u.  The shared-memory layouts stay those
// of the four-column kernel (element e of column f at byte 32*pad16(e) + 8f),
// in which the two columns of a thread are 16 contiguous bytes: every
// landing and exchange access, and the staging of row outputs, moves a float4
// (half the shared-memory instructions; the blocked staging of lifted pass 1
// is two 8-byte stores, the two columns being 32 bytes apart in a 4 x 4
// block); the stage twiddle rows are loaded and their products formed once
// for both columns.  The arithmetic of each column is that of the
// four-column kernel, operation for operation.  Lifted pass 1 (BLK = 1) also
// differs in its four-step twiddle tables and its landing order (see the
// kernel).

// Stage s of the three radix-16 stages on the two transforms of a thread;
// TWID = false leaves out the stage twiddles (as stage_compute does).
template <int s, bool TWID = true>
__device__ __forceinline__ void stage_compute2(float2 (&v)[16], float2 (&u)[16], int tau,
                                               const float2 *__restrict__ tw)
{
    using Sc = Sched<12>;
    dft16(v);
    dft16(u);
    if constexpr (TWID && s != Sc::S - 1) {
        // twiddle w_M^(uu*k) on output k: rows k = 1, 2, 3, 4, 8, 12 of the
        // stage table, the others as products (the rows and products of
        // apply_twiddles<16>)
        constexpr int M1 = Sc::M1(s);
        const float2 *t = tw + Sc::tw_offset(s);
        const int uu = tau & (M1 - 1);
        const float2 w1 = __ldg(&t[uu]), w2 = __ldg(&t[M1 + uu]), w3 = __ldg(&t[2 * M1 + uu]);
        v[1] = cmul(v[1], w1);
        u[1] = cmul(u[1], w1);
        v[2] = cmul(v[2], w2);
        u[2] = cmul(u[2], w2);
        v[3] = cmul(v[3], w3);
        u[3] = cmul(u[3], w3);
#pragma unroll
        for (int j = 1; j < 4; ++j) {
            const float2 wj = __ldg(&t[(j + 2) * M1 + uu]);   // k = 4, 8, 12
            const float2 a = cmul(wj, w1), b = cmul(wj, w2), c = cmul(wj, w3);
            v[4 * j] = cmul(v[4 * j], wj);
            u[4 * j] = cmul(u[4 * j], wj);
            v[4 * j + 1] = cmul(v[4 * j + 1], a);
            u[4 * j + 1] = cmul(u[4 * j + 1], a);
            v[4 * j + 2] = cmul(v[4 * j + 2], b);
            u[4 * j + 2] = cmul(u[4 * j + 2], b);
            v[4 * j + 3] = cmul(v[4 * j + 3], c);
            u[4 * j + 3] = cmul(u[4 * j + 3], c);
        }
    }
}

// Stage s outputs e = tau + 256k of both columns to the exchange buffer.
template <int s>
__device__ __forceinline__ void stage_write2(const float2 (&v)[16], const float2 (&u)[16], float4 *sm, int tau, int g)
{
    using Sc = Sched<12>;
    constexpr int KM1 = Sc::K(s) * Sc::M1(s);   // 256
    float4 *p = sm + (pad16(tau) << 1) + g;
#pragma unroll
    for (int k = 0; k < 16; ++k)
        p[pad16(KM1 * k) << 1] = make_float4(v[k].x, v[k].y, u[k].x, u[k].y);
}

// Stage s inputs e = w + M1*m of both columns from the exchange buffer.
template <int s>
__device__ __forceinline__ void stage_read2(float2 (&v)[16], float2 (&u)[16], const float4 *sm, int tau, int g)
{
    using Sc = Sched<12>;
    constexpr int M1 = Sc::M1(s), M = M1 * 16;
    const int w = (tau / M1) * M + (tau & (M1 - 1));
    const float4 *p = sm + (pad16(w) << 1) + g;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const float4 a = p[pad16(M1 * m) << 1];
        v[m] = make_float2(a.x, a.y);
        u[m] = make_float2(a.z, a.w);
    }
}

// BLK as in pipe_col_kernel; N = 4096, 512 threads.  The output must be
// 16-byte aligned (the plain stores write both columns as one float4).
template <bool TW4, int BLK>
__global__ void __launch_bounds__(512, 1)
    pipe_col2_kernel(const __grid_constant__ CUtensorMap tmapH, const __grid_constant__ CUtensorMap tmapE,
                     const __grid_constant__ CUtensorMap omap, float2 *out, int C, int logTpo, int ntiles,
                     const float2 *__restrict__ tw, const float2 *__restrict__ tw_lo,
                     const float2 *__restrict__ tw_hi, int tw_h, int flags, int staged, int *status)
{
    constexpr int N = 4096, T = 256;
    // landing order: the split order for lifted pass 1 (see the tile start)
    constexpr bool kSplitLanding = BLK == 1;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2 *E = reinterpret_cast<float2 *>(smem_raw);
    float2 *H = E + PipeSmem::E_entries<12>();
    constexpr int HR = PipeSmem::early_rows<12>();   // rows landing in H; rows HR..N-1 land in E
    // four-step twiddle tables of the tile, [16][4] each (entry i*4 + f for
    // column c0 + f): tl[i] = w^(col*i), th[i] = w^(col*16i), tk[i] = w^(col*256i),
    // so that w^(col*(tau + 256k)) = tl[tau % 16] * th[tau / 16] * tk[k]
    float2 *twt = H + 4 * HR;
    uint64_t *bar = reinterpret_cast<uint64_t *>(twt + PipeSmem::kTwEntries);
    int *abort_flag = reinterpret_cast<int *>(bar + 2);
    float4 *E4 = reinterpret_cast<float4 *>(E);
    const float4 *H4 = reinterpret_cast<const float4 *>(H);

    const int tid = threadIdx.x;
    const int g = tid & 1, tau = tid >> 1;
    const unsigned tpo_mask = (1u << logTpo) - 1;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    __syncthreads();
    int tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) {
        pdl_wait_prior();   // the input may be the previous kernel's output
        issue_tile_part<12, BLK>(&tmapH, &tmapE, logTpo, tile, 0, H, &bar[0]);
        issue_tile_part<12, BLK>(&tmapH, &tmapE, logTpo, tile, 1, E, &bar[1]);
    }
    uint32_t parity = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        const int o = tile >> logTpo;
        const int c0 = (tile & tpo_mask) << 2;
        const int col = c0 + 2 * g;   // the thread's first column; the second is col + 1
        const int next = tile + (int)gridDim.x;
        if (next >= ntiles)
            pdl_launch_dependents();   // the block's last tile: let the next kernel launch
        // the tile's twiddle table entries (threads below 192, one each, from
        // the two-level table), loaded before the tile wait so that their
        // latency is spent behind it
        float2 el, eh;
        if constexpr (TW4) {
            if (tid < PipeSmem::kTwEntries) {
                const int j = tid >> 6, i = (tid >> 2) & 15;
                const int64_t e = (int64_t)(c0 + (tid & 3)) * (i << (4 * j));
                el = __ldg(&tw_lo[e & ((int64_t(1) << tw_h) - 1)]);
                eh = __ldg(&tw_hi[e >> tw_h]);
            }
        }
        // element tau + T*q of both columns (rows below HR in H, the others in E)
        float2 v[16], u[16];
        if constexpr (kSplitLanding) {
            // Lifted pass 1 drains its staged outputs as three 32 KiB stores,
            // which may still be reading E when the next tile has landed.  The
            // early rows are read as soon as they are in; the late rows (in E)
            // after their own wait, while the next tile's early rows are already
            // on their way into H; the wait for the staged stores comes just
            // before the first exchange writes E.  (Measured: pass 1 61.3 ->
            // 58.8 us; for the row-output passes, whose twelve 8 KiB stores have
            // left E by then, the extra barrier costs 0.7-2.6 us.)
            if (tid == 0) {
                bounded_wait(&bar[0], parity, status, abort_flag, flags);
                if (*abort_flag)
                    drain_in_flight(bar, parity);
            }
            __syncthreads();
            if (*abort_flag) {
                if (staged && tid == 0)
                    bulk_wait_all();   // no staged store may still read E
                return;
            }
#pragma unroll
            for (int q = 0; q * T < HR; ++q) {
                const float4 a = H4[(tau + T * q) * 2 + g];
                v[q] = make_float2(a.x, a.y);
                u[q] = make_float2(a.z, a.w);
            }
            if (tid == 0) {
                bounded_wait(&bar[1], parity, status, abort_flag, flags);
                if (*abort_flag)
                    drain_in_flight(bar, parity);
            }
            __syncthreads();   // H has been read; the late rows have landed
            if (*abort_flag) {
                if (staged && tid == 0)
                    bulk_wait_all();
                return;
            }
            if (tid == 0 && next < ntiles) {
                fence_proxy_async();
                issue_tile_part<12, BLK>(&tmapH, &tmapE, logTpo, next, 0, H, &bar[0]);
            }
#pragma unroll
            for (int q = HR / T; q < 16; ++q) {
                const float4 a = E4[(tau + T * q - HR) * 2 + g];
                v[q] = make_float2(a.x, a.y);
                u[q] = make_float2(a.z, a.w);
            }
        } else {
            if (tid == 0) {
                bounded_wait(&bar[0], parity, status, abort_flag, flags);
                bounded_wait(&bar[1], parity, status, abort_flag, flags);
                if (*abort_flag)
                    drain_in_flight(bar, parity);
            }
            __syncthreads();
            if (*abort_flag) {
                if (staged && tid == 0)
                    bulk_wait_all();   // no staged store may still read E
                return;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float4 a = q * T < HR ? H4[(tau + T * q) * 2 + g] : E4[(tau + T * q - HR) * 2 + g];
                v[q] = make_float2(a.x, a.y);
                u[q] = make_float2(a.z, a.w);
            }
            if (staged && tid == 0)
                bulk_wait_read();   // the previous tile's staged outputs have left E
            __syncthreads();   // H and E have been read
            if (tid == 0 && next < ntiles) {
                fence_proxy_async();
                issue_tile_part<12, BLK>(&tmapH, &tmapE, logTpo, next, 0, H, &bar[0]);
            }
        }
        parity ^= 1u;
        if (flags & FLAG_CONJ_IN) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                v[r].y = -v[r].y;
                u[r].y = -u[r].y;
            }
        }
        if constexpr (TW4) {
            if (tid < PipeSmem::kTwEntries)
                twt[tid] = cmul(el, eh);
        }

        stage_compute2<0, BLK != 3>(v, u, tau, tw);
        if constexpr (kSplitLanding) {
            // the previous tile's staged outputs must have left E, and every
            // thread have read its late rows from E, before the first
            // exchange writes it
            if (staged && tid == 0)
                bulk_wait_read();
            __syncthreads();
        }
        stage_write2<0>(v, u, E4, tau, g);
        __syncthreads();
        stage_read2<1>(v, u, E4, tau, g);
        __syncthreads();
        stage_compute2<1>(v, u, tau, tw);
        stage_write2<1>(v, u, E4, tau, g);
        __syncthreads();
        stage_read2<2>(v, u, E4, tau, g);
        __syncthreads();
        if (tid == 0 && next < ntiles) {
            fence_proxy_async();
            issue_tile_part<12, BLK>(&tmapH, &tmapE, logTpo, next, 1, E, &bar[1]);
        }
        stage_compute2<2>(v, u, tau, tw);

        if constexpr (TW4) {
            // w^(col * (tau + T*k)) = A * tk[k][col], A = tl[tau % 16][col] * th[tau / 16][col]
            const float4 *t4 = reinterpret_cast<const float4 *>(twt);
            const float4 l = t4[(tau & 15) * 2 + g], h = t4[32 + (tau >> 4) * 2 + g];
            const float2 A0 = cmul(make_float2(l.x, l.y), make_float2(h.x, h.y));
            const float2 A1 = cmul(make_float2(l.z, l.w), make_float2(h.z, h.w));
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float4 t = t4[64 + k * 2 + g];
                v[k] = cmul(v[k], cmul(A0, make_float2(t.x, t.y)));
                u[k] = cmul(u[k], cmul(A1, make_float2(t.z, t.w)));
            }
        }
        if (flags & FLAG_CONJ_OUT) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                v[k].y = -v[k].y;
                u[k].y = -u[k].y;
            }
        }
        // outputs k >= k0 of the thread with plain stores
        auto store_plain = [&](int k0) {
            if constexpr (BLK == 3) {
                // output k = k1a + 16*k0 with tau + T*k = k: k1a = tau % 16, k0 = tau/16 + 16*k
                float4 *dst = reinterpret_cast<float4 *>(out + ((int64_t)o << 24) + (int64_t)(tau >> 4) * 65536 +
                                                         ((col >> 8) + 16 * (tau & 15)) * 256 + (col & 255));
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k >= k0)
                        dst[(int64_t)k << 19] = make_float4(v[k].x, v[k].y, u[k].x, u[k].y);
            } else if constexpr (BLK == 1) {
                // element (tau + T*k, col) of the tile: block ((col/4)*(N/4) + (tau + T*k)/4),
                // slot (col%4)*4 + tau%4; the second column is 4 slots on
                float2 *dst = out + (int64_t)o * N * C + (int64_t)((col >> 2) * (N >> 2)) * 16 + (col & 3) * 4 +
                              (tau >> 2) * 16 + (tau & 3);
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k >= k0) {
                        dst[k * 4 * T] = v[k];
                        dst[k * 4 * T + 4] = u[k];
                    }
            } else {
                float4 *dst = reinterpret_cast<float4 *>(out + (int64_t)o * N * C + col + (int64_t)tau * C);
                const int64_t step = (int64_t)T * C / 2;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k >= k0)
                        dst[k * step] = make_float4(v[k].x, v[k].y, u[k].x, u[k].y);
            }
        };
        if (staged) {
            // slices 0..KS-1 to E behind the late rows of the next tile, the rest plain
            constexpr int LATE = N - HR;
            constexpr int KS = (PipeSmem::E_entries<12>() - 4 * LATE) / (4 * T);
            static_assert(KS >= 1 && KS < 16 && (4 * LATE * 8) % 1024 == 0, "staging slices");
            float2 *stg = E + 4 * LATE;
            if constexpr (BLK == 1) {
                // slot (col%4)*4 + tau%4 of block (tau/4 + 64k), stored with the
                // 128-byte swizzle of the output tensor map (16-byte chunk j of
                // block b at chunk j ^ (b % 8)), so that the blocks of a warp's
                // four tau groups fall on different banks; b % 8 = (tau/4) % 8
                // The 8-byte stores are served per half-warp (two blocks): lanes
                // of odd blocks store their second column first, so that the
                // two blocks of a half-warp fill disjoint chunks in each store.
                char *sb = reinterpret_cast<char *>(stg) + (tau >> 2) * 128 + (tau & 1) * 8;
                const int sw = (tau >> 2) & 7, ch = 4 * g + ((tau >> 1) & 1);   // chunk of the first column
                const bool odd = ((tau >> 2) & 1) != 0;
                float2 *p0 = reinterpret_cast<float2 *>(sb + (((odd ? ch + 2 : ch)) ^ sw) * 16);
                float2 *p1 = reinterpret_cast<float2 *>(sb + (((odd ? ch : ch + 2)) ^ sw) * 16);
#pragma unroll
                for (int k = 0; k < KS; ++k) {
                    p0[k * 4 * T] = odd ? u[k] : v[k];
                    p1[k * 4 * T] = odd ? v[k] : u[k];
                }
            } else {
                float4 *sp = reinterpret_cast<float4 *>(stg) + tau * 2 + g;
#pragma unroll
                for (int k = 0; k < KS; ++k)
                    sp[k * 2 * T] = make_float4(v[k].x, v[k].y, u[k].x, u[k].y);
            }
            store_plain(KS);
            __syncthreads();   // the staged slices are complete
            if (tid == 0) {
                fence_proxy_async();   // written through the generic proxy, read by TMA
                if constexpr (BLK == 1) {
                    // three boxes of 256 blocks (32 KiB) of the map over the blocked output
                    static_assert(KS * 64 == 3 * 256, "three boxes of 256 blocks");
                    const int b0 = o * (N / 16) * C + (c0 >> 2) * (N >> 2);
#pragma unroll 1
                    for (int j = 0; j < 3; ++j)
                        tma_store_2d(&omap, stg + j * 256 * 16, 0, b0 + 256 * j);
                } else {
                    // three boxes of four slices (32 KiB) each
                    static_assert(KS == 12, "twelve staged slices");
#pragma unroll 1
                    for (int j = 0; j < 3; ++j) {
                        if constexpr (BLK == 3)
                            tma_store_4d(&omap, stg + j * 16 * T, 2 * (c0 & 255), c0 >> 8, 0, o * 256 + 64 * j);
                        else
                            tma_store_3d(&omap, stg + j * 16 * T, 2 * c0, 0, o * (N / 256) + 4 * j);
                    }
                }
                bulk_commit();
            }
        } else {
            store_plain(0);
        }
    }
    if (staged && tid == 0)
        bulk_wait_all();   // the staged stores are complete before the block exits
}

// Transposed row pass: rows o = 4*tile + f of the [O][N] view; output
// element k of row o goes to (o / Rt)*(N*Rt) + (o % Rt) + Rt*k.
template <int LOGN>
__global__ void __launch_bounds__(1 << (LOGN - 2), 1)
    pipe_rowT_kernel(const float2 *in, float2 *out, int64_t O, int64_t Rt, int ntiles,
                     const float2 *__restrict__ tw, int flags, int *status)
{
    using Sc = Sched<LOGN>;
    constexpr int N = Sc::N, T = Sc::T, NH = N / 2;
    constexpr int PITCH = PipeSmem::row_pitch<LOGN>();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    float2 *E = reinterpret_cast<float2 *>(smem_raw);
    float2 *H = E + PipeSmem::E_entries<LOGN>();
    uint64_t *bar = reinterpret_cast<uint64_t *>(H + PipeSmem::H_entries<LOGN>() + 64);
    int *abort_flag = reinterpret_cast<int *>(bar + 2);

    const int tid = threadIdx.x;
    const int f = tid & 3, tau = tid >> 2;

    auto issue_half = [&](int tile, int h, float2 *dst, uint64_t *b) {
        const int64_t o0 = (int64_t)tile * 4;
        const int rows = (int)((O - o0) < 4 ? (O - o0) : 4);
        mbar_arrive_expect_tx(b, rows * NH * (uint32_t)sizeof(float2));
        for (int r = 0; r < rows; ++r)
            bulk_load(dst + r * PITCH, in + (o0 + r) * N + h * NH, NH * (uint32_t)sizeof(float2), b);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        *abort_flag = 0;
    }
    __syncthreads();
    int tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) {
        pdl_wait_prior();   // the input may be the previous kernel's output
        issue_half(tile, 0, H, &bar[0]);
        issue_half(tile, 1, E, &bar[1]);
    }
    uint32_t parity = 0;
    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t o = (int64_t)tile * 4 + f;
        const bool active = o < O;
        const int next = tile + (int)gridDim.x;
        if (next >= ntiles)
            pdl_launch_dependents();   // the block's last tile: let the next kernel launch
        if (tid == 0) {
            bounded_wait(&bar[0], parity, status, abort_flag, flags);
            bounded_wait(&bar[1], parity, status, abort_flag, flags);
            if (*abort_flag)
                drain_in_flight(bar, parity);
        }
        __syncthreads();
        if (*abort_flag)
            return;
        parity ^= 1u;

        constexpr int R0 = 1 << Sc::rlog(0), NB0 = 16 / R0;
        float2 v[16];
        if (active) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float2 *src = q < 8 ? H : E;
                v[(q % NB0) * R0 + q / NB0] = src[f * PITCH + tau + T * (q & 7)];
            }
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)
                v[q] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (tid == 0 && next < ntiles) {
            fence_proxy_async();
            issue_half(next, 0, H, &bar[0]);
        }
        if (flags & FLAG_CONJ_IN) {
#pragma unroll
            for (int r = 0; r < 16; ++r)
                v[r].y = -v[r].y;
        }

        three_stages<LOGN>(v, E, tau, f, tw, [&] {
            if (tid == 0 && next < ntiles) {
                fence_proxy_async();
                issue_half(next, 1, E, &bar[1]);
            }
        });

        if (flags & FLAG_CONJ_OUT) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
                v[k].y = -v[k].y;
        }
        if (active) {
            const int64_t ob = o / Rt, orow = o - ob * Rt;
            float2 *dst = out + ob * (N * Rt) + orow + (int64_t)tau * Rt;
            const int64_t step = (int64_t)T * Rt;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                dst[k * step] = v[k];
        }
    }
}

// ---------------------------------------------------------------------------
// Host side: tensor-map encoding through the driver entry point (no libcuda
// link), launch configuration, dispatch.

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// E, H (the early rows of the next tile), the twiddle table tk [16][4], two
// mbarriers and a flag
template <int LOGN> size_t col_smem()
{
    return (size_t)(PipeSmem::E_entries<LOGN>() + 4 * PipeSmem::early_rows<LOGN>() + PipeSmem::kTwEntries) * 8 + 64;
}
template <int LOGN> size_t rowT_smem() { return PipeSmem::bytes<LOGN>(); }

// SM count of each device (set by prepare_pipe_kernels for the current
// device; the persistent grids are sized from the device they launch on).
constexpr int kMaxDev = 64;
int g_num_sms[kMaxDev] = {0};

int num_sms_current()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
        return 1;
    int n = __atomic_load_n(&g_num_sms[dev], __ATOMIC_RELAXED);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return 1;
        __atomic_store_n(&g_num_sms[dev], n, __ATOMIC_RELAXED);
    }
    return n;
}

// Staged stores of the N = 4096 column passes (MOA_STAGED=0 turns them off).
bool staged_enabled()
{
    static const bool on = [] {
        const char *s = std::getenv("MOA_STAGED");
        return !(s && *s && std::atoi(s) == 0);
    }();
    return on;
}

// Two columns per thread at N = 4096 (MOA_COL2=0: the four-column kernel).
bool col2_enabled()
{
    static const bool on = [] {
        const char *s = std::getenv("MOA_COL2");
        return !(s && *s && std::atoi(s) == 0);
    }();
    return on;
}

// Output tensor map of the staged stores over the [O][N][C] view: {2C floats,
// O*N rows}, boxes of 4 columns x 256 rows.  False when the output cannot be
// a TMA target (not 16-byte aligned).
bool encode_out_rows(CUtensorMap *map, float2 *out, int64_t O, int64_t C, int logN)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || (reinterpret_cast<uintptr_t>(out) & 15) != 0)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * C), (cuuint64_t)(O << logN)};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * C * sizeof(float))};
    const cuuint32_t box[2] = {8, 256};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output tensor map of the two-column kernel's staged row stores over the
// [O][N][C] view: {2C floats, 256 rows, O*N/256 row blocks}, boxes of 4
// columns x 256 rows x 4 row blocks (four slices, 32 KiB).  False when the
// output cannot be a TMA target (not 16-byte aligned).
bool encode_out_rows4(CUtensorMap *map, float2 *out, int64_t O, int64_t C, int logN)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || (reinterpret_cast<uintptr_t>(out) & 15) != 0)
        return false;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * C), 256, (cuuint64_t)((O << logN) >> 8)};
    const cuuint64_t strides[2] = {(cuuint64_t)(2 * C * sizeof(float)), (cuuint64_t)(256 * 2 * C * sizeof(float))};
    const cuuint32_t box[3] = {8, 256, 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output tensor map of the two-column kernel's staged blocked stores: the
// blocked workspace as {32 floats (one 4 x 4 block), blocks}, boxes of 256
// blocks, 128-byte swizzle.  False when it cannot be encoded.
bool encode_out_blocked(CUtensorMap *map, float2 *out, int64_t nblocks)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || (reinterpret_cast<uintptr_t>(out) & 15) != 0)
        return false;
    const cuuint64_t dims[2] = {32, (cuuint64_t)nblocks};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {32, 256};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Column pass over the [O][N][C] view (BLK 0 or 1) or the second pass of the
// lifted transform over the blocked workspace (BLK 2; O = B, C = r).
template <int LOGN>
cudaError_t launch_col(const PassDesc &d, int64_t O, int64_t C, int blk, const float2 *in, float2 *out,
                       const TwiddleSet &tw, int flags, cudaStream_t stream, int *status)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return cudaErrorNotSupported;
    // the tile's first HR rows (early landing) and the rest, each one TMA copy
    // of whole 256-row boxes: depth HR/256 and (N - HR)/256 along a dimension
    // of 256-row blocks
    constexpr int HR = PipeSmem::early_rows<LOGN>();
    const cuuint32_t depth[2] = {(cuuint32_t)(HR / 256), (cuuint32_t)(((1 << LOGN) - HR) / 256)};
    CUtensorMap maps[2];
    CUresult r = CUDA_SUCCESS;
    for (int h = 0; h < 2 && r == CUDA_SUCCESS; ++h) {
        if (blk == 2) {
            // {floats of one 4 x 4 block, blocks along k1, 64 blocks along j2, 256-row blocks of every o}
            const cuuint64_t dims[4] = {32, (cuuint64_t)(C >> 2), 64, (cuuint64_t)((O << LOGN) >> 8)};
            const cuuint64_t strides[3] = {128, (cuuint64_t)((C >> 2) * 128), (cuuint64_t)(64 * (C >> 2) * 128)};
            const cuuint32_t box[4] = {32, 1, 64, depth[h]};
            const cuuint32_t estr[4] = {1, 1, 1, 1};
            r = enc(&maps[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2 *>(in), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        } else {
            // {floats of a row, rows of a 256-row block, 256-row blocks of every o}
            const cuuint64_t dims[3] = {(cuuint64_t)(2 * C), 256, (cuuint64_t)((O << LOGN) >> 8)};
            const cuuint64_t strides[2] = {(cuuint64_t)(2 * C * sizeof(float)), (cuuint64_t)(256 * 2 * C * sizeof(float))};
            const cuuint32_t box[3] = {8, 256, depth[h]};
            const cuuint32_t estr[3] = {1, 1, 1};
            r = enc(&maps[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(in), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        }
    }
    const CUtensorMap &map = maps[0];
    if (r != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    int logTpo = 0;
    while ((int64_t(1) << logTpo) < (C >> 2))
        ++logTpo;
    const int ntiles = (int)(O << logTpo);
    const int nsm = num_sms_current();
    const int grid = ntiles < nsm ? ntiles : nsm;
    const size_t smem = col_smem<LOGN>();
    const int Ci = (int)C;
    // staged stores: blocked output by bulk copy (16-byte aligned output),
    // row output through a tensor map
    CUtensorMap omap = map;
    int staged = 0;
    if (LOGN == 12 && staged_enabled())
        staged = blk == 1 ? (reinterpret_cast<uintptr_t>(out) & 15) == 0 : encode_out_rows(&omap, out, O, C, LOGN);
    if (LOGN == 12 && col2_enabled() && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        if (staged)
            staged = blk == 1 ? encode_out_blocked(&omap, out, (O << LOGN) * C / 16)
                              : encode_out_rows4(&omap, out, O, C, LOGN);
        auto kern2 = blk == 2 ? pipe_col2_kernel<false, 2>
                              : (d.tw4 && blk == 1 ? pipe_col2_kernel<true, 1>
                                                   : (d.tw4 ? pipe_col2_kernel<true, 0> : pipe_col2_kernel<false, 0>));
        return launch_maybe_dependent(kern2, grid, 512, smem, stream, flags & FLAG_PDL, maps[0], maps[1], omap, out,
                                      Ci, logTpo, ntiles, tw.stage[LOGN], tw.lo, tw.hi, tw.h, flags,
                                      staged, status);
    }
    auto kern = blk == 2 ? pipe_col_kernel<LOGN, false, 2>
                         : (d.tw4 && blk == 1 ? pipe_col_kernel<LOGN, true, 1>
                                              : (d.tw4 ? pipe_col_kernel<LOGN, true, 0> : pipe_col_kernel<LOGN, false, 0>));
    return launch_maybe_dependent(kern, grid, 1 << (LOGN - 2), smem, stream, flags & FLAG_PDL, maps[0], maps[1], omap,
                                  out, Ci, logTpo, ntiles, tw.stage[LOGN], tw.lo, tw.hi, tw.h, flags, staged, status);
}

// Second pass of the two-pass 3-D transform of O arrays of 256^3 (BLK = 3).
cudaError_t launch_plane2(int64_t O, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                          cudaStream_t stream, int *status)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc)
        return cudaErrorNotSupported;
    // {floats of one row, planes of all O arrays, rows of a plane}; the early
    // and the late part of a tile as one copy each (boxes of 11 and 5 rows)
    constexpr int HR = PipeSmem::early_rows<12>();
    CUtensorMap maps[2];
    for (int h = 0; h < 2; ++h) {
        const cuuint64_t dims[3] = {512, (cuuint64_t)(O * 256), 256};
        const cuuint64_t strides[2] = {(cuuint64_t)65536 * sizeof(float2), (cuuint64_t)256 * sizeof(float2)};
        const cuuint32_t box[3] = {8, 256, (cuuint32_t)(h ? (4096 - HR) / 256 : HR / 256)};
        const cuuint32_t estr[3] = {1, 1, 1};
        if (enc(&maps[h], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(in), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    const CUtensorMap &map = maps[0];
    const int ntiles = (int)(O << 10);   // 16 row groups x 64 column groups per array
    const int nsm = num_sms_current();
    const int grid = ntiles < nsm ? ntiles : nsm;
    // staged stores: the output X[k0][k1b + 16 k1a][col] of every array as
    // {512 floats, k1b (16), k1a (16, 16 rows apart), O*256 planes}
    CUtensorMap omap = map;
    int staged = 0;
    if (staged_enabled() && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        const cuuint64_t odims[4] = {512, 16, 16, (cuuint64_t)(O * 256)};
        const cuuint64_t ostrides[3] = {256 * sizeof(float2), 16 * 256 * sizeof(float2),
                                        65536 * sizeof(float2)};
        const bool two = col2_enabled();   // (the two-column kernel stores four slices per box)
        const cuuint32_t obox[4] = {8, 1, 16, two ? 64u : 16u};
        const cuuint32_t oestr[4] = {1, 1, 1, 1};
        staged = enc(&omap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, out, odims, ostrides, obox, oestr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (col2_enabled() && (reinterpret_cast<uintptr_t>(out) & 15) == 0)
        return launch_maybe_dependent(pipe_col2_kernel<false, 3>, grid, 512, col_smem<12>(), stream,
                                      flags & FLAG_PDL, maps[0], maps[1], omap, out, 256, 10, ntiles, tw.stage[12],
                                      tw.lo, tw.hi, tw.h, flags, staged, status);
    return launch_maybe_dependent(pipe_col_kernel<12, false, 3>, grid, 1024, col_smem<12>(), stream, flags & FLAG_PDL,
                                  maps[0], maps[1], omap, out, 256, 10, ntiles, tw.stage[12], tw.lo, tw.hi, tw.h,
                                  flags, staged, status);
}

template <int LOGN>
cudaError_t launch_rowT(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                        cudaStream_t stream, int *status)
{
    const int ntiles = (int)((d.O + 3) / 4);
    const int nsm = num_sms_current();
    const int grid = ntiles < nsm ? ntiles : nsm;
    return launch_maybe_dependent(pipe_rowT_kernel<LOGN>, grid, 1 << (LOGN - 2), rowT_smem<LOGN>(), stream,
                                  flags & FLAG_PDL, in, out, d.O, d.Rt, ntiles, tw.stage[LOGN], flags, status);
}

template <int LOGN>
cudaError_t set_pipe_attrs()
{
    cudaError_t e;
    const int cs = (int)col_smem<LOGN>();
    if ((e = cudaFuncSetAttribute(pipe_col_kernel<LOGN, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(pipe_col_kernel<LOGN, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(pipe_col_kernel<LOGN, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(pipe_col_kernel<LOGN, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)))
        return e;
    return cudaFuncSetAttribute(pipe_rowT_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rowT_smem<LOGN>());
}

}  // namespace

bool pipe_supported() { return encode_fn() != nullptr; }

bool pipe_col2_active() { return col2_enabled(); }

bool encode_c64_map(CUtensorMap *map, const void *base, int rank, const uint64_t *dims, const uint64_t *strides,
                    const uint32_t *box)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || rank < 1 || rank > 5)
        return false;
    cuuint64_t d[5], st[4];
    cuuint32_t b[5], es[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank)
            st[i] = strides[i];
    }
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, const_cast<void *>(base), d, st, b, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t prepare_pipe_kernels()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    int nsm = 0;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if (dev < kMaxDev)
        __atomic_store_n(&g_num_sms[dev], nsm, __ATOMIC_RELAXED);
    if ((e = set_pipe_attrs<10>()) || (e = set_pipe_attrs<11>()) || (e = set_pipe_attrs<12>()))
        return e;
    const int cs = (int)col_smem<12>();
    if ((e = cudaFuncSetAttribute(pipe_col_kernel<12, false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(pipe_col2_kernel<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(pipe_col2_kernel<false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(pipe_col2_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(pipe_col2_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)) ||
        (e = cudaFuncSetAttribute(pipe_col2_kernel<false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs)))
        return e;
    return cudaSuccess;
}

cudaError_t launch_pipe_plane2(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                               cudaStream_t stream, int *status)
{
    return launch_plane2(d.O, in, out, tw, flags, stream, status);
}

cudaError_t launch_pipe_pass(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                             cudaStream_t stream, int *status)
{
    if (d.kind == PASS_COL || d.blk == 2) {
        // blocked second pass: O = B transforms of the r x c array, C = r columns
        const int64_t O = d.kind == PASS_COL ? d.O : d.O / d.Rt;
        const int64_t C = d.kind == PASS_COL ? d.C : d.Rt;
        switch (d.logN) {
        case 10: return launch_col<10>(d, O, C, d.blk, in, out, tw, flags, stream, status);
        case 11: return launch_col<11>(d, O, C, d.blk, in, out, tw, flags, stream, status);
        case 12: return launch_col<12>(d, O, C, d.blk, in, out, tw, flags, stream, status);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (d.logN) {
    case 10: return launch_rowT<10>(d, in, out, tw, flags, stream, status);
    case 11: return launch_rowT<11>(d, in, out, tw, flags, stream, status);
    case 12: return launch_rowT<12>(d, in, out, tw, flags, stream, status);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace moa
