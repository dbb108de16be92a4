// Pass kernels: the column pass (strided axis, paper's block phase with the
// four-step twiddle in its epilogue) and the row pass (contiguous axis,
// paper's cyclic phase with the transposed store).  See internal.h for the
// views each pass works on.
//
// Tiles: F transforms of length N per thread block (F*N <= 2^14 complex64,
// 128 KiB), one thread per 16 points.  Loads and stores go straight between
// HBM and registers: in the column pass the F lanes that share a row read
// or write F*8 contiguous bytes (F >= 4 gives whole 32-byte sectors); in the
// row pass the F lanes that share a column index write the F outputs of the
// four-step transpose X[k1 + r*k2] next to each other.

#include "fft_core.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace moa {

namespace {

__device__ __forceinline__ float2 two_level(const float2 *__restrict__ lo, const float2 *__restrict__ hi,
                                            int h, int64_t e)
{
    return cmul(__ldg(&lo[e & ((int64_t(1) << h) - 1)]), __ldg(&hi[e >> h]));
}

template <int LOGN, bool TW4, int V = 0>
__global__ void __launch_bounds__(1024) col_pass_kernel(const float2 *in, float2 *out, int C, int logF,
                                                        int logTpo, const float2 *__restrict__ tw,
                                                        const float2 *__restrict__ tw_lo,
                                                        const float2 *__restrict__ tw_hi, int tw_h, int flags,
                                                        int Rt, int log_cdiv)
{
    using Sc = Sched<LOGN, V>;
    extern __shared__ float2 smem[];
    const int F = 1 << logF;
    const int tid = threadIdx.x;
    const int f = tid & (F - 1);
    const int tau = tid >> logF;
    const unsigned tile = blockIdx.x;
    const unsigned o = tile >> logTpo;
    const int col = (int)((tile & ((1u << logTpo) - 1)) << logF) + f;
    // N*Rt*C < 2^31 (checked at plan time), so in-column offsets fit in 32 bits
    const int64_t base = (int64_t)o * ((int64_t)Sc::N * C) + col + (int64_t)tau * C;
    const int step = Sc::T * C;
    // output: row k of o at row (o % Rt) + Rt*k of the [O/Rt][N*Rt][C] view
    const unsigned ob = o / (unsigned)Rt, orow = o - ob * (unsigned)Rt;
    const int64_t obase = (int64_t)ob * ((int64_t)Sc::N * Rt * C) + (int64_t)orow * C + col + (int64_t)tau * Rt * C;
    const int ostep = Sc::T * Rt * C;
    const int64_t tcol = col >> log_cdiv;   // the twiddle's column index

    pdl_wait_prior();   // `in` may be the previous kernel's output, `out` its input
    float2 v[16];
    {
        constexpr int R0 = 1 << Sc::rlog(0);
        constexpr int NB0 = Sc::P / R0;
        const float2 *src = in + base;
        // element tau + T*q lands in register (q % NB0)*R0 + q / NB0
#pragma unroll
        for (int q = 0; q < Sc::P; ++q)
            v[(q % NB0) * R0 + q / NB0] = src[q * step];
    }
    if (flags & FLAG_CONJ_IN) {
#pragma unroll
        for (int r = 0; r < Sc::P; ++r)
            v[r].y = -v[r].y;
    }

    constexpr int LAY = max_logF_interleaved(LOGN);
    constexpr int kExchange = Sc::S > 1 ? ((Sc::N + Sc::N / 16) << LAY) : 0;
    float2 *tk = smem + kExchange;
    (void)tk;
    if constexpr (TW4) {
        // w_M^(tcol*row), row = orow + Rt*(tau + T*k), as A * Tk[k]:
        // A = w_M^(tcol*(orow + Rt*tau)) per thread, Tk[k] = w_M^(tcol*Rt*T*k)
        // shared by the lanes of one column.
        for (int k = tau; k < Sc::P; k += Sc::T)
            tk[(k << LAY) + f] = two_level(tw_lo, tw_hi, tw_h, tcol * ((int64_t)Rt * Sc::T * k));
    }

    fft_tile<LOGN, LAY, V>(v, smem, tau, f, tw);

    if constexpr (TW4) {
        const float2 A = two_level(tw_lo, tw_hi, tw_h, tcol * (orow + (int64_t)Rt * tau));
        if constexpr (Sc::S == 1)
            __syncthreads();
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            v[k] = cmul(v[k], cmul(A, tk[(k << LAY) + f]));
    }
    if (flags & FLAG_CONJ_OUT) {
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            v[k].y = -v[k].y;
    }
    float2 *dst = out + obase;
#pragma unroll
    for (int k = 0; k < Sc::P; ++k)
        dst[k * ostep] = v[k];
    pdl_launch_dependents();   // after the stores: the next kernel launches as the last blocks finish
}

template <int LOGN, bool TRANS, int V = 0>
__global__ void __launch_bounds__(1024) row_pass_kernel(const float2 *in, float2 *out, int64_t O, int64_t Rt,
                                                        int logF, const float2 *__restrict__ tw, int flags)
{
    using Sc = Sched<LOGN, V>;
    extern __shared__ float2 smem[];
    const int F = 1 << logF;
    const int tid = threadIdx.x;
    // Natural-order store: consecutive lanes take consecutive points of one
    // row, so loads and stores are contiguous along the row.  Transposed
    // store: consecutive lanes take the F rows first, so the F outputs
    // X[k1 + r*k2], k1 = o0..o0+F-1, land side by side.
    constexpr int LAY = TRANS ? max_logF_interleaved(LOGN) : -1;
    const int f = TRANS ? (tid & (F - 1)) : (tid / Sc::T);
    const int tau = TRANS ? (tid >> logF) : (tid & (Sc::T - 1));
    const int64_t o = ((int64_t)blockIdx.x << logF) + f;
    const bool active = o < O;
    pdl_wait_prior();   // `in` may be the previous kernel's output, `out` its input
    float2 v[16];
    if (active) {
        constexpr int R0 = 1 << Sc::rlog(0);
        constexpr int NB0 = Sc::P / R0;
        const float2 *src = in + o * Sc::N + tau;
#pragma unroll
        for (int q = 0; q < Sc::P; ++q)
            v[(q % NB0) * R0 + q / NB0] = src[q * Sc::T];
    } else {
#pragma unroll
        for (int r = 0; r < Sc::P; ++r)
            v[r] = make_float2(0.f, 0.f);
    }
    if (flags & FLAG_CONJ_IN) {
#pragma unroll
        for (int r = 0; r < Sc::P; ++r)
            v[r].y = -v[r].y;
    }

    fft_tile<LOGN, LAY, V>(v, smem, tau, f, tw);

    if (flags & FLAG_CONJ_OUT) {
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            v[k].y = -v[k].y;
    }
    if (active) {
        const int64_t ob = o / Rt, orow = o - ob * Rt;
        float2 *dst = out + ob * (Sc::N * Rt) + orow + (int64_t)tau * Rt;
        const int64_t step = (int64_t)Sc::T * Rt;
#pragma unroll
        for (int k = 0; k < Sc::P; ++k)
            dst[k * step] = v[k];
    }
    pdl_launch_dependents();
}

// Row pass (natural order) for N = 128, 256, 512 with the butterflies that
// cross lanes done by warp shuffles: no shared-memory exchange between the
// radix stages and no block barrier.  N = 16 * T, element j = lam + T*q of a
// transform in lane lam (< T) of its group of T lanes, register q:
//   1. a radix-16 DFT over q in registers (outputs k1), then the twiddle
//      w_N^(lam*k1) (the first step of the lifting n = 16 x T, Sec. 4.2);
//   2. the T-point DFTs over lam as log2 T radix-2 stages across lanes
//      (decimation in frequency, Sec. 3.5-3.6's butterfly on lane pairs
//      lam, lam ^ h): each lane sends its value with shfl.xor, the lower lane
//      keeps the sum, the upper one the difference times w_2h^(lam mod h);
//      the lane then holds k2 = bitrev(lam), i.e. X[k1 + 16*bitrev(lam)];
//   3. the warp's outputs (32/T transforms, 512 complex64 contiguous in
//      memory) pass through a warp-private staging area (row = lane, 17
//      entries a row: conflict-free both ways) behind __syncwarp, so every
//      store instruction writes 256 contiguous bytes.
// Each block holds T << logF threads, a multiple of 32 up to 256 (the plan
// uses this kernel only then), so every shuffle has its whole warp.  `tw` holds rows
// k = 1, 2, 3, 4, 8, 12 of w_N^(u*k), u < T, then w_T^u, u < T.
template <int LOGN>
__global__ void __launch_bounds__(256) row_warp_kernel(const float2 *in, float2 *out, int64_t O, int logF,
                                                       const float2 *__restrict__ tw, int flags)
{
    constexpr int N = 1 << LOGN, T = N / 16, LT = LOGN - 4;
    static_assert(T >= 8 && T <= 32, "N = 128, 256, 512");
    extern __shared__ float2 smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lam = lane & (T - 1), g = lane >> LT;
    const int64_t o0 = ((int64_t)blockIdx.x << logF) + (int64_t)warp * (32 / T);   // the warp's first row
    const int64_t o = o0 + g;
    pdl_wait_prior();   // `in` may be the previous kernel's output, `out` its input
    float2 v[16];
    if (o < O) {
        const float2 *src = in + o * N + lam;
#pragma unroll
        for (int q = 0; q < 16; ++q)
            v[q] = src[q * T];
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            v[q] = make_float2(0.f, 0.f);
    }
    if (flags & FLAG_CONJ_IN) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            v[q].y = -v[q].y;
    }
    dft16(v);
    apply_twiddles<16>(v, tw, lam, T);
    const float2 *wT = tw + 6 * T;   // w_T^u
#pragma unroll
    for (int h = T / 2; h >= 1; h >>= 1) {
        const bool upper = (lam & h) != 0;
        const float sg = upper ? -1.f : 1.f;
        // w_2h^(lam mod h) = w_T^((lam mod h) * T / 2h) on the upper lane, 1 on the lower
        const float2 w = upper ? __ldg(&wT[(lam & (h - 1)) * (T / (2 * h))]) : make_float2(1.f, 0.f);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float px = __shfl_xor_sync(0xffffffffu, v[k].x, h);
            const float py = __shfl_xor_sync(0xffffffffu, v[k].y, h);
            // lower: mine + partner; upper: partner - mine
            v[k] = cmul(make_float2(fmaf(sg, v[k].x, px), fmaf(sg, v[k].y, py)), w);
        }
    }
    if (flags & FLAG_CONJ_OUT) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
            v[k].y = -v[k].y;
    }
    float2 *stg = smem + warp * (32 * 17);
#pragma unroll
    for (int k = 0; k < 16; ++k)
        stg[lane * 17 + k] = v[k];
    __syncwarp();
    float2 *dst = out + o0 * N;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int p = lane + 32 * m;            // position in the warp's 32 x 16 outputs
        const int fl = p >> LOGN, k = p & (N - 1);
        const int row = fl * T + (int)(__brev((unsigned)(k >> 4)) >> (32 - LT));
        if (o0 + fl < O)
            dst[p] = stg[row * 17 + (k & 15)];
    }
    pdl_launch_dependents();
}

// First pass of the two-pass 3-D transform of 256 x 256 x 256 arrays.  Axis
// 1 is lifted as j1 = j1a + 16*j1b (Sec. 4.2 applied to that axis).  Tile
// (array o, plane j0, j1a): the 16 rows j1a + 16*j1b of the plane.  Their
// 256-point transforms along axis 2 (16 threads per row), then, per column
// k2 (one thread each), the 16-point DFT over j1b and the twiddle
// w_256^(j1a*k1b); the result for k1b goes to row j1a + 16*k1b of the
// workspace.  The second pass (the DFT over j1a and the axis-0 transform)
// runs in pipe_col_kernel<12, false, 3>.
__global__ void __launch_bounds__(256, 5) plane3d_p1_kernel(const float2 *in, float2 *ws, int ntiles,
                                                         const float2 *__restrict__ tw8,
                                                         const float2 *__restrict__ w256, int flags)
{
    using Sc = Sched<8>;
    static_assert(Sc::T == 16 && Sc::P == 16, "256-point rows, 16 threads per row");
    __shared__ float2 sm[16 * (256 + 16)];   // the row exchange, then the 16 x 256 block
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    if (tile >= ntiles)
        return;
    const int j1a = tile & 15;
    const int64_t plane = tile >> 4;   // o*256 + j0
    const float2 *base = in + plane * 65536 + j1a * 256;

    pdl_wait_prior();   // `in` may be the previous kernel's output, `ws` its input
    const int f = tid >> 4, tau = tid & 15;   // row j1a + 16*f, 16 threads per row
    float2 v[16];
    const float2 *src = base + f * 4096 + tau;
#pragma unroll
    for (int q = 0; q < 16; ++q)   // radix 16 first: element tau + 16*q in register q
        v[q] = src[q * 16];
    if (flags & FLAG_CONJ_IN) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            v[q].y = -v[q].y;
    }
    fft_tile<8, -1>(v, sm, tau, f, tw8);   // v[k]: point tau + 16*k of row f's transform
    // fft_tile's last exchange read is behind a block barrier: sm is free
#pragma unroll
    for (int k = 0; k < 16; ++k)
        sm[f * 256 + tau + 16 * k] = v[k];
    __syncthreads();
    const int c = tid;   // column k2
    float2 u[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
        u[j] = sm[j * 256 + c];
    dft16(u);
#pragma unroll
    for (int k = 1; k < 16; ++k)
        u[k] = cmul(u[k], __ldg(&w256[(j1a * k) & 255]));
    float2 *dst = ws + plane * 65536 + j1a * 256 + c;
#pragma unroll
    for (int k = 0; k < 16; ++k)
        dst[k * 4096] = u[k];
    pdl_launch_dependents();   // after the stores
}

template <int LOGN, int V>
cudaError_t launch_typed_v(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                           cudaStream_t stream)
{
    const int threads = pass_threads(d);
    const size_t smem = pass_smem_bytes(d);
    const float2 *stage = V == 0 ? tw.stage[LOGN] : tw.vstage[V][LOGN];
    if (d.kind == PASS_COL) {
        int logTpo = 0;
        while ((int64_t(1) << logTpo) < (d.C >> d.logF))
            ++logTpo;
        const int64_t grid = d.O << logTpo;
        int log_cdiv = 0;
        while ((1 << log_cdiv) < d.cdiv)
            ++log_cdiv;
        const bool xt = d.twlog > 0;   // a further table (a lifted axis) instead of the main one
        return launch_maybe_dependent(d.tw4 ? col_pass_kernel<LOGN, true, V> : col_pass_kernel<LOGN, false, V>,
                                      (unsigned)grid, threads, smem, stream, flags & FLAG_PDL, in, out, (int)d.C,
                                      d.logF, logTpo, stage, xt ? tw.xlo[d.twlog] : tw.lo,
                                      xt ? tw.xhi[d.twlog] : tw.hi, xt ? tw.xh[d.twlog] : tw.h, flags,
                                      (int)(d.Rt > 1 ? d.Rt : 1), log_cdiv);
    }
    const int64_t grid = (d.O + (int64_t(1) << d.logF) - 1) >> d.logF;
    return launch_maybe_dependent(d.Rt > 1 ? row_pass_kernel<LOGN, true, V> : row_pass_kernel<LOGN, false, V>,
                                  (unsigned)grid, threads, smem, stream, flags & FLAG_PDL, in, out, d.O, d.Rt,
                                  d.logF, stage, flags);
}

template <int LOGN>
cudaError_t launch_typed(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                         cudaStream_t stream)
{
    if constexpr (LOGN >= 7 && LOGN <= 9) {
        if (d.sched == 3) {
            if (d.kind != PASS_ROW || d.Rt > 1 || pass_threads(d) % 32 != 0 || pass_threads(d) > 256 ||
                !tw.vstage[3][LOGN])
                return cudaErrorInvalidValue;
            const int64_t grid = (d.O + (int64_t(1) << d.logF) - 1) >> d.logF;
            return launch_maybe_dependent(row_warp_kernel<LOGN>, (unsigned)grid, pass_threads(d),
                                          pass_smem_bytes(d), stream, flags & FLAG_PDL, in, out, d.O, d.logF,
                                          tw.vstage[3][LOGN], flags);
        }
    }
    if constexpr (sched_variant_ok(LOGN, 1)) {
        if (d.sched == 1)
            return launch_typed_v<LOGN, 1>(d, in, out, tw, flags, stream);
    }
    if constexpr (sched_variant_ok(LOGN, 2)) {
        if (d.sched == 2)
            return launch_typed_v<LOGN, 2>(d, in, out, tw, flags, stream);
    }
    if (d.sched != 0)
        return cudaErrorInvalidValue;
    return launch_typed_v<LOGN, 0>(d, in, out, tw, flags, stream);
}

template <int LOGN, int V>
cudaError_t set_attrs_v()
{
    const int max_smem = 227 * 1024;
    cudaError_t e = cudaFuncSetAttribute(col_pass_kernel<LOGN, true, V>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(col_pass_kernel<LOGN, false, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             max_smem);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(row_pass_kernel<LOGN, true, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             max_smem);
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(row_pass_kernel<LOGN, false, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem);
}

template <int LOGN>
cudaError_t set_attrs()
{
    cudaError_t e = set_attrs_v<LOGN, 0>();
    if constexpr (sched_variant_ok(LOGN, 1))
        if (e == cudaSuccess)
            e = set_attrs_v<LOGN, 1>();
    if constexpr (sched_variant_ok(LOGN, 2))
        if (e == cudaSuccess)
            e = set_attrs_v<LOGN, 2>();
    return e;
}

}  // namespace

cudaError_t launch_plane1(const PassDesc &d, const float2 *in, float2 *ws, const TwiddleSet &tw, const float2 *w256,
                          int flags, cudaStream_t stream)
{
    const int ntiles = (int)(d.O * 256 * 16);   // arrays x planes x j1a
    return launch_maybe_dependent(plane3d_p1_kernel, (unsigned)ntiles, 256, 0, stream, flags & FLAG_PDL, in, ws,
                                  ntiles, tw.stage[8], w256, flags);
}

int pass_threads(const PassDesc &d)
{
    const int N = 1 << d.logN;
    const int T = N < 16 ? 1 : N / 16;
    return T << d.logF;
}

size_t pass_smem_bytes(const PassDesc &d)
{
    if (d.sched == 3)   // row_warp_kernel: 17 entries per lane of staged outputs
        return (size_t)pass_threads(d) * 17 * sizeof(float2);
    const int N = 1 << d.logN;
    const int P = N < 16 ? N : 16;
    const size_t F = size_t(1) << d.logF;
    const size_t FP = size_t(1) << max_logF_interleaved(d.logN);
    const bool interleaved = d.kind == PASS_COL || d.Rt > 1;
    size_t entries = 0;
    if (d.logN > 4)
        entries += (size_t)(N + N / 16) * (interleaved ? FP : F);
    if (d.kind == PASS_COL && d.tw4)
        entries += (size_t)P * FP;
    return entries * sizeof(float2);
}

cudaError_t prepare_kernels()
{
    cudaError_t e = cudaSuccess;

    if ((e = set_attrs<1>()) || (e = set_attrs<2>()) || (e = set_attrs<3>()) || (e = set_attrs<4>()) ||
        (e = set_attrs<5>()) || (e = set_attrs<6>()) || (e = set_attrs<7>()) || (e = set_attrs<8>()) ||
        (e = set_attrs<9>()) || (e = set_attrs<10>()) || (e = set_attrs<11>()) || (e = set_attrs<12>()))
        return e;
    return cudaSuccess;
}

cudaError_t launch_pass(const PassDesc &d, const float2 *in, float2 *out, const TwiddleSet &tw, int flags,
                        cudaStream_t stream, int *status)
{
    if (d.pipe && (reinterpret_cast<uintptr_t>(in) & 15) == 0)
        return launch_pipe_pass(d, in, out, tw, flags, stream, status);
    switch (d.logN) {
    case 1: return launch_typed<1>(d, in, out, tw, flags, stream);
    case 2: return launch_typed<2>(d, in, out, tw, flags, stream);
    case 3: return launch_typed<3>(d, in, out, tw, flags, stream);
    case 4: return launch_typed<4>(d, in, out, tw, flags, stream);
    case 5: return launch_typed<5>(d, in, out, tw, flags, stream);
    case 6: return launch_typed<6>(d, in, out, tw, flags, stream);
    case 7: return launch_typed<7>(d, in, out, tw, flags, stream);
    case 8: return launch_typed<8>(d, in, out, tw, flags, stream);
    case 9: return launch_typed<9>(d, in, out, tw, flags, stream);
    case 10: return launch_typed<10>(d, in, out, tw, flags, stream);
    case 11: return launch_typed<11>(d, in, out, tw, flags, stream);
    case 12: return launch_typed<12>(d, in, out, tw, flags, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace moa
