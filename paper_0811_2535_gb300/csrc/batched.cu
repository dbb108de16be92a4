// Batched transforms of uneven power-of-two lengths in one persistent launch.
//
// Many independent problems share one launch the way the paper's plans
// share processors among the columns of one problem (Sec. 4.3): the host
// turns the list of lengths into a work queue of tasks, longest first, and
// persistent blocks take tasks in queue order with an atomic ticket.
//
//   small task  one to 4096/n transforms of the same length n <= 4096, all
//               in one 256-thread block (n/16 threads per transform), in
//               shared memory and registers: one HBM read, one HBM write.
//   large transform  n = r*c in [2^13, 2^16], split into n/4096 column
//               tiles (r-point transforms on 4096/r columns, twiddle
//               w_n^(j2*k1), result to a workspace) and n/4096 row tiles
//               (c-point transforms on 4096/c rows, stored at X[k1 + r*k2]).
//               A row tile waits for a per-transform counter of finished
//               column tiles (bounded wait; MOA_ERR_TIMEOUT on expiry).  The
//               queue puts every row tile after all column tiles of its
//               transform, about one wave of blocks later, so that the
//               workspace is read back while it is still in L2; column tiles
//               never wait, so every wait ends.
//
// A launch is one memset (ticket and counters) plus one kernel, both on
// the caller's stream, so an exec can be captured in a CUDA graph.
#include "batched.h"
#include "fft_core.cuh"

namespace moa {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;   // resident blocks per SM (64 registers, 32 bytes of spill; faster than 3 at 80)

__device__ __forceinline__ float2 two_level_b(const float2 *__restrict__ lo, const float2 *__restrict__ hi, int h,
                                              int64_t e)
{
    return cmul(__ldg(&lo[e & ((int64_t(1) << h) - 1)]), __ldg(&hi[e >> h]));
}

template <int LOGN>
__device__ __forceinline__ void small_task(const BatchTask &t, const int64_t *__restrict__ offs,
                                           const float2 *in, float2 *out, const BatchTables &tb, float2 *sm,
                                           int flags)
{
    using Sc = Sched<LOGN>;
    constexpr int T = Sc::T;
    const int tid = threadIdx.x;
    const int f = tid / T, tau = tid % T;   // lanes run along a transform: contiguous loads and stores
    const bool active = f < t.count;
    const int64_t base = active ? offs[t.first + f] : 0;
    constexpr int R0 = 1 << Sc::rlog(0), NB0 = Sc::P / R0;
    float2 v[16];
    if (active) {
        const float2 *src = in + base + tau;
#pragma unroll
        for (int q = 0; q < Sc::P; ++q)
            v[(q % NB0) * R0 + q / NB0] = src[q * T];
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            v[q] = make_float2(0.f, 0.f);
    }
    if (flags & FLAG_CONJ_IN) {
#pragma unroll
        for (int r = 0; r < Sc::P; ++r)
            v[r].y = -v[r].y;
    }
    fft_tile<LOGN, -1>(v, sm, tau, f, tb.stage[LOGN]);
    if (flags & FLAG_CONJ_OUT) {
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            v[k].y = -v[k].y;
    }
    if (active) {
        float2 *dst = out + base + tau;
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            dst[k * T] = v[k];
    }
}

// One column tile of a large transform: r = 2^LOGR points per column,
// 4096/r columns starting at column 4096/r * tile, c columns in all.
template <int LOGR>
__device__ __forceinline__ void large_col_tile(const float2 *x, float2 *b, int c, int logn, int tile,
                                            const BatchTables &tb, float2 *sm, int flags)
{
    using Sc = Sched<LOGR>;
    constexpr int T = Sc::T;
    constexpr int LOGF = 12 - LOGR;   // 4096/r columns per tile, adjacent lanes
    constexpr int F = 1 << LOGF;
    const int tid = threadIdx.x;
    const int f = tid & (F - 1), tau = tid >> LOGF;
    const float2 *lo = tb.lo[logn], *hi = tb.hi[logn];
    const int h = tb.h[logn];
    constexpr int R0 = 1 << Sc::rlog(0), NB0 = Sc::P / R0;
    const int col = tile * F + f;
    float2 v[16];
    const float2 *src = x + col + (int64_t)tau * c;
#pragma unroll
    for (int q = 0; q < Sc::P; ++q)
        v[(q % NB0) * R0 + q / NB0] = src[(int64_t)q * T * c];
    if (flags & FLAG_CONJ_IN) {
#pragma unroll
        for (int r = 0; r < Sc::P; ++r)
            v[r].y = -v[r].y;
    }
    fft_tile<LOGR, LOGF>(v, sm, tau, f, tb.stage[LOGR]);
    float2 *dst = b + col + (int64_t)tau * c;
    // twiddle w_n^(col*k1), k1 = tau + T*k, from the two-level table
#pragma unroll 4
    for (int k = 0; k < Sc::P; ++k)
        dst[(int64_t)k * T * c] = cmul(v[k], two_level_b(lo, hi, h, (int64_t)col * (tau + T * k)));
}

// The workspace lines a row tile has read are not needed again (each is read
// by exactly one row tile): drop them from L2 without a write-back, so that
// the column-pass results never travel to DRAM.  Only whole 128-byte lines
// inside the region [p, p + n) are dropped (a transform's offset in the batch
// is only 16-byte aligned).  The caller has consumed every load of the
// region in every thread before the call (a block barrier after their use).
__device__ __forceinline__ void discard_read_lines(const float2 *p, int64_t n)
{
    uint64_t a;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(a) : "l"(p));
    const uint64_t first = (a + 127) & ~uint64_t(127), last = (a + (uint64_t)n * sizeof(float2)) & ~uint64_t(127);
    for (uint64_t l = first + (uint64_t)threadIdx.x * 128; l < last; l += (uint64_t)blockDim.x * 128)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(l) : "memory");
}

// One row tile of a large transform: c = 2^LOGC points per row, 4096/c
// rows starting at row 4096/c * tile, transposed store into X (r rows).  The
// rows are read with c/16 consecutive threads per row (whole runs of one row
// per warp) and stage 0 runs in that order; the first exchange (row-major,
// odd row pitch: conflict-free for both orders) hands the data to the
// row-interleaved order in which the other stages run and the transposed
// stores cover whole segments of consecutive rows.
template <int LOGC>
__device__ __forceinline__ void large_row_tile(const float2 *b, float2 *X, int r, int tile, const BatchTables &tb,
                                            float2 *sm, int flags)
{
    using Sc = Sched<LOGC>;
    constexpr int N = Sc::N, T = Sc::T;
    constexpr int LOGT = LOGC - 4;
    constexpr int LOGF = 12 - LOGC;   // 4096/c rows per tile
    constexpr int F = 1 << LOGF;
    const int tid = threadIdx.x;
    constexpr int R0 = 1 << Sc::rlog(0), NB0 = Sc::P / R0;
    const int fb = tid & (F - 1), tau_b = tid >> LOGF;
    constexpr int LR = F >= 16 ? -2 : (F == 8 ? -3 : -4);   // row pitch padding for F rows
    float2 v[16];
    if constexpr (Sc::S == 1) {
        // one stage: one thread per row, no exchange
        const float2 *src = b + (int64_t)(tile * F + fb) * N;
#pragma unroll
        for (int q = 0; q < Sc::P; ++q)
            v[q] = src[q];
        stage_compute<LOGC, 0>(v, 0, tb.stage[LOGC]);
        __syncthreads();   // every load of the tile has been used
        discard_read_lines(b + (int64_t)tile * F * N, (int64_t)F * N);
    } else {
        const int tau_a = tid & (T - 1), fa = tid >> LOGT;
        const float2 *src = b + (int64_t)(tile * F + fa) * N + tau_a;
#pragma unroll
        for (int q = 0; q < Sc::P; ++q)
            v[(q % NB0) * R0 + q / NB0] = src[q * T];
        stage_compute<LOGC, 0>(v, tau_a, tb.stage[LOGC]);
        stage_write<LOGC, 0, LR>(v, sm, tau_a, fa);
        __syncthreads();   // also: every load of the tile has been used
        discard_read_lines(b + (int64_t)tile * F * N, (int64_t)F * N);
        stage_read<LOGC, 1, LR>(v, sm, tau_b, fb);
        __syncthreads();
        stage_compute<LOGC, 1>(v, tau_b, tb.stage[LOGC]);
        run_stages<LOGC, 2, LR>(v, sm, tau_b, fb, tb.stage[LOGC]);
    }
    if (flags & FLAG_CONJ_OUT) {
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            v[k].y = -v[k].y;
    }
    const int k1 = tile * F + fb;
    float2 *dst = X + k1 + (int64_t)tau_b * r;
#pragma unroll
    for (int k = 0; k < Sc::P; ++k)
        dst[(int64_t)k * T * r] = v[k];
}

__device__ __forceinline__ void run_small(const BatchTask &t, const int64_t *offs, const float2 *in, float2 *out,
                          const BatchTables &tb, float2 *sm, int flags)
{
    switch (t.logn) {
    case 1: small_task<1>(t, offs, in, out, tb, sm, flags); break;
    case 2: small_task<2>(t, offs, in, out, tb, sm, flags); break;
    case 3: small_task<3>(t, offs, in, out, tb, sm, flags); break;
    case 4: small_task<4>(t, offs, in, out, tb, sm, flags); break;
    case 5: small_task<5>(t, offs, in, out, tb, sm, flags); break;
    case 6: small_task<6>(t, offs, in, out, tb, sm, flags); break;
    case 7: small_task<7>(t, offs, in, out, tb, sm, flags); break;
    case 8: small_task<8>(t, offs, in, out, tb, sm, flags); break;
    case 9: small_task<9>(t, offs, in, out, tb, sm, flags); break;
    case 10: small_task<10>(t, offs, in, out, tb, sm, flags); break;
    case 11: small_task<11>(t, offs, in, out, tb, sm, flags); break;
    case 12: small_task<12>(t, offs, in, out, tb, sm, flags); break;
    default: break;
    }
}


__device__ __forceinline__ int load_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void run_large(const BatchTask &t, const int64_t *offs, const float2 *in, float2 *out, float2 *ws,
                          int *counters, const BatchTables &tb, float2 *sm, int flags, int *status, int *s_flag,
                          int max_polls, int wait_extra)
{
    const int64_t base = offs[t.first];
    const int c = 1 << (t.logn - t.logr), r = 1 << t.logr;
    float2 *b = ws + base;
    if (t.kind == 1) {
        const float2 *x = in + base;
        switch (t.logr) {
        case 4: large_col_tile<4>(x, b, c, t.logn, t.tile, tb, sm, flags); break;
        case 5: large_col_tile<5>(x, b, c, t.logn, t.tile, tb, sm, flags); break;
        case 6: large_col_tile<6>(x, b, c, t.logn, t.tile, tb, sm, flags); break;
        case 7: large_col_tile<7>(x, b, c, t.logn, t.tile, tb, sm, flags); break;
        case 8: large_col_tile<8>(x, b, c, t.logn, t.tile, tb, sm, flags); break;
        case 9: large_col_tile<9>(x, b, c, t.logn, t.tile, tb, sm, flags); break;
        case 10: large_col_tile<10>(x, b, c, t.logn, t.tile, tb, sm, flags); break;
        default: break;
        }
        __syncthreads();   // all of the tile's workspace stores are issued
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&counters[t.first], 1);
        }
        return;
    }
    // row tile: wait until every column tile of this transform is done
    if (threadIdx.x == 0) {
        const int need = (1 << (t.logn - 12)) + wait_extra;
        int polls = 0, ok = 1;
        while (load_acquire(&counters[t.first]) < need) {
            if (++polls >= max_polls) {
                atomicExch(status, 6);   // MOA_ERR_TIMEOUT
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        *s_flag = ok;
    }
    __syncthreads();
    const bool ok = *s_flag != 0;
    if (ok) {
        switch (t.logn - t.logr) {
        case 4: large_row_tile<4>(b, out + base, r, t.tile, tb, sm, flags); break;
        case 5: large_row_tile<5>(b, out + base, r, t.tile, tb, sm, flags); break;
        case 6: large_row_tile<6>(b, out + base, r, t.tile, tb, sm, flags); break;
        case 7: large_row_tile<7>(b, out + base, r, t.tile, tb, sm, flags); break;
        case 8: large_row_tile<8>(b, out + base, r, t.tile, tb, sm, flags); break;
        case 9: large_row_tile<9>(b, out + base, r, t.tile, tb, sm, flags); break;
        case 10: large_row_tile<10>(b, out + base, r, t.tile, tb, sm, flags); break;
        default: break;
        }
    }
}

__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    batched_kernel(const BatchTask *__restrict__ tasks, int ntasks, int *ticket, const int64_t *__restrict__ offs,
                   const float2 *in, float2 *out, float2 *ws, const BatchTables *__restrict__ tbp, int flags,
                   int *status, int max_polls, int wait_extra)
{
    const BatchTables &tb = *tbp;
    __shared__ float2 sm[4480];   // exchange buffer: 4096 points + padding (up to 128 rows of N + N/16 + 1)
    __shared__ int s_task, s_flag;
    int *counters = ticket + 1;
    for (;;) {
        if (threadIdx.x == 0)
            s_task = atomicAdd(ticket, 1);
        __syncthreads();
        const int ti = s_task;
        __syncthreads();   // everyone has read s_task before it is overwritten
        if (ti >= ntasks)
            break;
        const BatchTask t = tasks[ti];
        if (t.kind == 0)
            run_small(t, offs, in, out, tb, sm, flags);
        else
            run_large(t, offs, in, out, ws, counters, tb, sm, flags, status, &s_flag, max_polls, wait_extra);
        __syncthreads();   // the exchange buffer is reused by the next task
    }
}

}  // namespace

int batched_blocks_per_sm() { return kBlocksPerSM; }

cudaError_t launch_batched(const BatchLaunch &b, const float2 *in, float2 *out, int flags, cudaStream_t stream,
                           int *status)
{
    cudaError_t e = cudaMemsetAsync(b.ticket, 0, sizeof(int) * (size_t)(1 + b.ncounters), stream);
    if (e != cudaSuccess)
        return e;
    batched_kernel<<<b.grid, kThreads, 0, stream>>>(b.tasks, b.ntasks, b.ticket, b.offs, in, out, b.ws, b.tables,
                                                    flags, status, b.max_polls, b.wait_extra);
    return cudaGetLastError();
}

}  // namespace moa
