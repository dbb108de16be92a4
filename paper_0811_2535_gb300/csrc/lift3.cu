// Second and third passes of a three-level lifted 1-D transform, fused in
// one persistent launch.
//
// The transform of n = r * c points is lifted as r x c (first pass: r-point
// transforms down the c columns with the twiddle w_n^(j2 k1), col_pass_kernel)
// and every row k1 of the r x c intermediate is itself a c-point transform,
// lifted again as cA x cB (the paper's dimension lifting applied to the
// rows, Sec. 4.4):
//   middle pass: cA-point transforms down the cB columns of each row, times
//                w_c^(j3 k2), in place in the workspace;
//   last pass:   cB-point transforms along the rows of each row's cA x cB
//                array, stored at X[k1 + r (k2 + cA k3)].
// A last-pass tile takes 4096/cB consecutive rows k1 at one k2, so its
// stores are whole 128-byte segments (cB = 256) of X.  Those rows form a
// unit; the middle-pass tiles of one unit rewrite 4096/cB * cA * cB * 8 bytes
// (8 MiB for cB = 256), which the last-pass tiles of the same unit read back
// shortly after, from L2.  DRAM sees the workspace read once and X written
// once: the two passes cost the traffic of one.
//
// The middle pass writes its output to a ring of four units (not back to
// the workspace): rewriting a slot that is still in L2 sends nothing to
// DRAM, so DRAM sees the workspace read once and X written once.
//
// Scheduling: the queue holds the middle-pass tiles of unit u followed (two
// units later) by the last-pass tiles of unit u; persistent blocks take
// tasks in order with an atomic ticket, fetched one task ahead, and decode
// them arithmetically.  Each task's 32 KiB tile is brought into shared
// memory by TMA while the block computes the task before it.  Dependencies:
// a last-pass tile's load is issued once all middle tiles of its unit are
// counted; a middle tile's stores wait until the last pass has read the
// ring slot's previous unit.  A block counts its finished middle tile at
// the top of its next task and only then waits for anything (a load that
// was not ready during the previous task is started there, waiting); so no
// block waits while holding an uncounted tile, every wait is for tiles
// taken earlier by running blocks, and every wait ends.  The waits are
// bounded nonetheless (MOA_ERR_TIMEOUT on expiry).
#include "fft_core.cuh"
#include "internal.h"

namespace moa {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 3;
constexpr int kMaxPolls = 1 << 22;
constexpr uint32_t kTileBytes = 4096 * 8;

__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float2 tw2(const float2 *__restrict__ lo, const float2 *__restrict__ hi, int h, int64_t e)
{
    return cmul(__ldg(&lo[e & ((int64_t(1) << h) - 1)]), __ldg(&hi[e >> h]));
}

__device__ __forceinline__ int load_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait by one thread until *p >= need; false (and MOA_ERR_TIMEOUT in
// the status word) when the limit is reached.
__device__ __forceinline__ bool wait_count(const int *p, int need, int *status)
{
    for (int polls = 0; load_acquire(p) < need; ++polls) {
        if (polls >= kMaxPolls) {
            atomicExch(status, 6);   // MOA_ERR_TIMEOUT
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ void mbar_init1(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (int polls = 0; polls < (1 << 24); ++polls) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(s_u32(bar)), "r"(parity)
            : "memory");
        if (ok)
            return true;
    }
    return false;
}

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(s_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(s_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(s_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(s_u32(bar))
        : "memory");
}

// Task `ti` of the queue: LAG units of middle tiles, then for each further
// unit its middle tiles followed by the last tiles of the unit LAG before,
// then the last tiles of the final LAG units.  kind 1 = middle, 2 = last.
__device__ __forceinline__ void decode(int ti, const Lift3Launch &l, int &kind, int &unit, int &idx)
{
    const int per = l.middle_per_unit, lag = l.lag, U = l.nunits;
    const int head = lag * per;
    if (ti < head) {
        kind = 1;
        unit = ti / per;
        idx = ti % per;
        return;
    }
    const int t = ti - head, mid = (U - lag) * 2 * per;
    if (t < mid) {
        const int p = t / (2 * per), w = t % (2 * per);
        kind = w < per ? 1 : 2;
        unit = w < per ? p + lag : p;
        idx = w < per ? w : w - per;
        return;
    }
    kind = 2;
    unit = (U - lag) + (t - mid) / per;
    idx = (t - mid) % per;
}

// Thread 0: start the TMA load of task ti's tile into `land`.  Middle tile:
// rows R*cA .. R*cA + cA-1, columns jb*F .. jb*F + F-1 of the workspace.
// Last tile: its unit's F_B rows at k2 from the ring slot, which may be read
// only once all middle tiles of the unit are counted: with `may_wait` the
// thread waits for that (bounded); without it the load is not started and
// false is returned.
__device__ __forceinline__ bool start_load(int ti, const Lift3Launch &l, float2 *land, uint64_t *bar,
                                           const int *mid_done, int *status, bool may_wait)
{
    int kind, unit, idx;
    decode(ti, l, kind, unit, idx);
    const int rows_per_unit = 1 << (12 - l.logb);
    if (kind == 1) {
        const int fa = 12 - l.loga;
        const int blocks = 1 << (l.logb - fa);
        const int R = unit * rows_per_unit + idx / blocks;
        mbar_expect(bar, kTileBytes);
        tma_2d(land, l.map_mid, bar, (idx % blocks) << fa, R << l.loga);
        return true;
    }
    if (may_wait)
        wait_count(&mid_done[unit], l.middle_per_unit, status);
    else if (load_acquire(&mid_done[unit]) < l.middle_per_unit)
        return false;
    asm volatile("fence.proxy.async.global;" ::: "memory");   // generic writes of the ring, then TMA reads
    mbar_expect(bar, kTileBytes);
    tma_3d(land, l.map_last, bar, 0, idx, (unit % l.ring_units) * rows_per_unit);
    return true;
}


// What a tile needs to start the next task's load once its landing buffer
// has been read (thread 0 only; `issued` records whether it did).
struct Next {
    int ti, ntasks;
    float2 *land;
    uint64_t *bar;
    const int *mid_done;
    int *status;
    bool *issued;
};

// Middle pass: columns jb*F .. jb*F + F-1 of row R's cA x cB array (landed
// as [cA rows][F]), cA-point transforms, twiddle w_c^(j3 k2), written to the
// same place in the row's slot of the ring.  The twiddle of output k2 =
// tau + T k is A * B_k with A = w_c^(j3 tau) per thread and B_k = w_c^(j3 T k)
// per column (a table in shared memory).  Thread 0 checks, before the
// exchange barrier, that the last pass has read the slot's previous unit.
template <int LOGA>
__device__ __forceinline__ void middle_tile(const float2 *land, float2 *slot_row, int jb, int logb,
                                            const Lift3Launch &l, const float2 *__restrict__ stage, float2 *sm,
                                            float2 *tk, const int *prev, int *s_ok, int *status, const Next nx)
{
    using Sc = Sched<LOGA>;
    static_assert(Sc::S == 2, "two-stage transforms only");
    constexpr int T = Sc::T;
    constexpr int LOGF = 12 - LOGA;
    constexpr int F = 1 << LOGF;
    const int tid = threadIdx.x;
    const int f = tid & (F - 1), tau = tid >> LOGF;
    const int cB = 1 << logb;
    constexpr int R0 = 1 << Sc::rlog(0), NB0 = Sc::P / R0;
    const int col = jb * F + f;
    float2 v[16];
#pragma unroll
    for (int q = 0; q < Sc::P; ++q)
        v[(q % NB0) * R0 + q / NB0] = land[(tau + q * T) * F + f];
#pragma unroll
    for (int k = tau; k < 16; k += T)
        tk[k * F + f] = tw2(l.lo, l.hi, l.h, (int64_t)col * (T * k));
    const float2 A = tw2(l.lo, l.hi, l.h, (int64_t)col * tau);
    stage_compute<LOGA, 0>(v, tau, stage);
    stage_write<LOGA, 0, LOGF>(v, sm, tau, f);
    if (tid == 0)
        *s_ok = prev ? wait_count(prev, l.middle_per_unit, status) : 1;
    __syncthreads();
    if (tid == 0 && nx.ti < nx.ntasks)   // the landing buffer has been read: next task's load, if ready
        *nx.issued = start_load(nx.ti, l, nx.land, nx.bar, nx.mid_done, nx.status, false);
    stage_read<LOGA, 1, LOGF>(v, sm, tau, f);
    stage_compute<LOGA, 1>(v, tau, stage);
    if (*s_ok) {
        float2 *y = slot_row + col + (int64_t)tau * cB;
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            y[(int64_t)k * T * cB] = cmul(v[k], cmul(A, tk[k * F + f]));
    }
}

// Last pass: the unit's F rows (consecutive k1) at k2 (landed as [F][cB]),
// cB-point transforms, stored at X[o n + k1 + r (k2 + cA k3)].  Stage 0 runs
// with N/16 consecutive threads per row; the one exchange hands the data to
// the row-interleaved order (consecutive threads on consecutive rows) in
// which stage 1 runs and the stores cover whole 128-byte segments of X.
template <int LOGB>
__device__ __forceinline__ void last_tile(const float2 *land, float2 *X, int64_t unit, int k2, int loga,
                                          const Lift3Launch &l, const float2 *__restrict__ stage, float2 *sm, int flags,
                                          int *read_done, const Next nx)
{
    using Sc = Sched<LOGB>;
    static_assert(Sc::S == 2, "two-stage transforms only");
    constexpr int N = Sc::N, T = Sc::T;
    constexpr int LOGT = LOGB - 4;
    constexpr int LOGF = 12 - LOGB;
    constexpr int F = 1 << LOGF;
    const int tid = threadIdx.x;
    constexpr int R0 = 1 << Sc::rlog(0), NB0 = Sc::P / R0;
    const int logc = loga + LOGB;
    const int tau_a = tid & (T - 1), fa = tid >> LOGT;
    float2 v[16];
#pragma unroll
    for (int q = 0; q < Sc::P; ++q)
        v[(q % NB0) * R0 + q / NB0] = land[fa * N + tau_a + q * T];
    stage_compute<LOGB, 0>(v, tau_a, stage);
    stage_write<LOGB, 0, -2>(v, sm, tau_a, fa);
    __syncthreads();
    if (tid == 0) {
        atomicAdd(read_done, 1);   // this tile's part of the ring slot has been consumed
        if (nx.ti < nx.ntasks)     // the landing buffer has been read: next task's load, if ready
            *nx.issued = start_load(nx.ti, l, nx.land, nx.bar, nx.mid_done, nx.status, false);
    }
    const int fb = tid & (F - 1), tau_b = tid >> LOGF;
    stage_read<LOGB, 1, -2>(v, sm, tau_b, fb);
    stage_compute<LOGB, 1>(v, tau_b, stage);
    if (flags & FLAG_CONJ_OUT) {
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            v[k].y = -v[k].y;
    }
    const int64_t R = unit * F + fb;
    const int64_t o = R >> l.logr, k1 = R & ((int64_t(1) << l.logr) - 1);
    const int64_t rcA = int64_t(1) << (l.logr + loga);   // X stride of k3
    float2 *dst = X + (o << (l.logr + logc)) + k1 + ((int64_t)k2 << l.logr) + tau_b * rcA;
#pragma unroll
    for (int k = 0; k < Sc::P; ++k)
        dst[(int64_t)k * T * rcA] = v[k];
}

__global__ void __launch_bounds__(kThreads, kBlocksPerSM)
    lift3_kernel(const Lift3Launch l, float2 *out, const float2 *__restrict__ stage_a,
                 const float2 *__restrict__ stage_b, int flags, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    float2 *land = reinterpret_cast<float2 *>(smem);   // the current task's tile (TMA)
    float2 *sm = land + 4096;                           // exchange buffer
    float2 *tk = sm + l.ex_entries;                     // middle pass: w_c^(j3 T k) per column
    uint64_t *bar = reinterpret_cast<uint64_t *>(tk + (16 << (12 - l.loga)));
    int *s_ticket = reinterpret_cast<int *>(bar + 1);   // [2]
    int *s_ok = s_ticket + 2;
    int *s_mid_ok = s_ticket + 3;
    int *s_issued = s_ticket + 4;
    int *mid_done = l.ticket + 1;                 // middle tiles finished, per unit
    int *read_done = mid_done + l.nunits;         // last tiles that have read their data, per unit
    const int tid = threadIdx.x;
    const int ntasks = 2 * l.nunits * l.middle_per_unit;
    const int rows_per_unit = 1 << (12 - l.logb);
    const int64_t unit_elems = (int64_t)rows_per_unit << (l.loga + l.logb);

    if (tid == 0) {
        mbar_init1(bar);
        s_ticket[0] = atomicAdd(l.ticket, 1);
    }
    __syncthreads();
    uint32_t phase = 0;
    int pending = -1;      // (every thread) unit of this block's previous task if it was a middle tile
    bool issued = false;   // thread 0: the next task's load has been started
    bool ok = true;
    int next_ti = ntasks;  // thread 0: the next task's ticket
    for (int it = 0;; ++it) {
        const int ti = s_ticket[it & 1];
        if (ti >= ntasks)
            break;
        // s_issued: whether this task's load was started during the previous task
        // (written at the end of that task, read here, rewritten only at the end of this one)
        const bool loaded = it > 0 && *s_issued != 0;
        if (tid == 0) {
            next_ti = atomicAdd(l.ticket, 1);   // the next task; its value is first needed mid-task
            if (!loaded) {
                // this load may have to wait for other tiles: count this block's own tile first
                if (pending >= 0) {
                    __threadfence();   // its stores were issued before the last barrier
                    atomicAdd(&mid_done[pending], 1);
                }
                start_load(ti, l, land, bar, mid_done, status, true);
            }
            *s_ok = mbar_wait_bounded(bar, phase) ? 1 : 0;
            if (!*s_ok)
                atomicExch(status, 6);   // MOA_ERR_TIMEOUT
        } else if (tid == 32 && loaded && pending >= 0) {
            // count the previous middle tile off thread 0's path
            __threadfence();
            atomicAdd(&mid_done[pending], 1);
        }
        __syncthreads();
        phase ^= 1u;
        if (!*s_ok) {
            ok = false;
            pending = -1;   // counted above, before any wait
            break;
        }
        int kind, unit, idx;
        decode(ti, l, kind, unit, idx);
        issued = false;
        const Next nx{tid == 0 ? next_ti : ntasks, ntasks, land, bar, mid_done, status, &issued};
        float2 *slot = l.ring + (int64_t)(unit % l.ring_units) * unit_elems;
        if (kind == 1) {
            const int blocks = 1 << (l.logb - (12 - l.loga));
            const int row = idx / blocks, jb = idx % blocks;
            float2 *slot_row = slot + ((int64_t)row << (l.loga + l.logb));
            const int *prev = unit >= l.ring_units ? &read_done[unit - l.ring_units] : nullptr;
            switch (l.loga) {
            case 6: middle_tile<6>(land, slot_row, jb, l.logb, l, stage_a, sm, tk, prev, s_mid_ok, status, nx); break;
            case 7: middle_tile<7>(land, slot_row, jb, l.logb, l, stage_a, sm, tk, prev, s_mid_ok, status, nx); break;
            case 8: middle_tile<8>(land, slot_row, jb, l.logb, l, stage_a, sm, tk, prev, s_mid_ok, status, nx); break;
            default: break;
            }
            pending = unit;
        } else {
            switch (l.logb) {
            case 6: last_tile<6>(land, out, unit, idx, l.loga, l, stage_b, sm, flags, &read_done[unit], nx); break;
            case 7: last_tile<7>(land, out, unit, idx, l.loga, l, stage_b, sm, flags, &read_done[unit], nx); break;
            case 8: last_tile<8>(land, out, unit, idx, l.loga, l, stage_b, sm, flags, &read_done[unit], nx); break;
            default: break;
            }
            pending = -1;
        }
        if (tid == 0) {
            s_ticket[(it + 1) & 1] = next_ti;
            *s_issued = issued ? 1 : 0;
        }
        __syncthreads();   // exchange buffer and twiddle table reuse; next ticket and s_issued visible
    }
    if (tid == 0) {
        if (pending >= 0) {
            __threadfence();
            atomicAdd(&mid_done[pending], 1);
        }
        if (!ok)
            mbar_wait_bounded(bar, phase ^ 1u);   // a copy still in flight after a timeout
    }
}

}  // namespace

int lift3_blocks_per_sm() { return kBlocksPerSM; }

cudaError_t launch_lift3(const Lift3Launch &l, float2 *out, const float2 *stage_a, const float2 *stage_b, int flags,
                         cudaStream_t stream, int *status)
{
    cudaError_t e = cudaFuncSetAttribute(lift3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)l.smem_bytes);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(l.ticket, 0, sizeof(int) * (size_t)(1 + 2 * l.nunits), stream);
    if (e != cudaSuccess)
        return e;
    lift3_kernel<<<l.grid, kThreads, l.smem_bytes, stream>>>(l, out, stage_a, stage_b, flags, status);
    return cudaGetLastError();
}

}  // namespace moa
