// Twiddle generator.  The weights w_M^e = exp(-2 pi i e / M) (Sec. 3.1: the
// diagonal of Omega in B_L holds consecutive powers of w_L; Fig. 3.8 computes
// them directly per stage, not by recurrence) are evaluated once per plan in
// FP64 with sincospi on the device and rounded once to FP32.  The kernels
// only read these tables.
#include "fft_core.cuh"
#include "internal.h"

namespace moa {

namespace {

struct StageGen {
    int M, M1, offset;
};

__global__ void stage_table_kernel(float2 *dst, int total, StageGen s0, StageGen s1, StageGen s2, int nst)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total)
        return;
    StageGen g = s0;
    if (nst > 1 && idx >= s1.offset)
        g = s1;
    if (nst > 2 && idx >= s2.offset)
        g = s2;
    const int local = idx - g.offset;
    const int j = local / g.M1, u = local % g.M1;
    const int e = (int)(((int64_t)u * tw_row_k(j)) % g.M);
    double s, c;
    sincospi(2.0 * (double)e / (double)g.M, &s, &c);
    dst[idx] = make_float2((float)c, (float)(-s));
}

__global__ void power_table_kernel(float2 *dst, int64_t count, int64_t step, int64_t modulus)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= count)
        return;
    const int64_t e = (idx * step) % modulus;
    double s, c;
    sincospi(2.0 * (double)e / (double)modulus, &s, &c);
    dst[idx] = make_float2((float)c, (float)(-s));
}

__global__ void full_stage_kernel(float2 *dst, int64_t M, int64_t M1)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 16 * M1)
        return;
    const int64_t k = idx / M1, u = idx % M1;
    const int64_t e = (u * k) % M;
    double s, c;
    sincospi(2.0 * (double)e / (double)M, &s, &c);
    dst[idx] = make_float2((float)c, (float)(-s));
}

template <int LOGN, int V>
int entries_typed()
{
    if constexpr (V == 3)
        return 7 * ((1 << LOGN) / 16);
    else
        return Sched<LOGN, V>::tw_entries();
}

template <int LOGN, int V>
cudaError_t gen_typed(float2 *dst, cudaStream_t stream)
{
    StageGen g[3] = {{1, 1, 0}, {1, 1, 0}, {1, 1, 0}};
    int nst = 0, total = 0;
    if constexpr (V == 3) {
        // rows of w_N^(u*k), u < T, then one row of w_T^u
        constexpr int N = 1 << LOGN, T = N / 16;
        g[0] = StageGen{N, T, 0};
        g[1] = StageGen{T, T, 6 * T};
        nst = 2;
        total = 7 * T;
    } else {
        using Sc = Sched<LOGN, V>;
        total = Sc::tw_entries();
        nst = Sc::S - 1;
        for (int s = 0; s < nst; ++s)
            g[s] = StageGen{Sc::M1(s) << Sc::rlog(s), Sc::M1(s), Sc::tw_offset(s)};
    }
    if (total == 0)
        return cudaSuccess;
    stage_table_kernel<<<(total + 255) / 256, 256, 0, stream>>>(dst, total, g[0], g[1], g[2], nst);
    return cudaGetLastError();
}

constexpr bool exists(int logN, int V) { return V == 3 ? (logN >= 7 && logN <= 9) : sched_variant_ok(logN, V); }

template <int LOGN>
int entries_any(int V)
{
    switch (V) {
    case 0: return entries_typed<LOGN, 0>();
    case 1: if constexpr (exists(LOGN, 1)) return entries_typed<LOGN, 1>(); else return -1;
    case 2: if constexpr (exists(LOGN, 2)) return entries_typed<LOGN, 2>(); else return -1;
    case 3: if constexpr (exists(LOGN, 3)) return entries_typed<LOGN, 3>(); else return -1;
    default: return -1;
    }
}

template <int LOGN>
cudaError_t gen_any(float2 *dst, int V, cudaStream_t stream)
{
    switch (V) {
    case 0: return gen_typed<LOGN, 0>(dst, stream);
    case 1: if constexpr (exists(LOGN, 1)) return gen_typed<LOGN, 1>(dst, stream); else return cudaErrorInvalidValue;
    case 2: if constexpr (exists(LOGN, 2)) return gen_typed<LOGN, 2>(dst, stream); else return cudaErrorInvalidValue;
    case 3: if constexpr (exists(LOGN, 3)) return gen_typed<LOGN, 3>(dst, stream); else return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool sched_exists(int logN, int V) { return V >= 0 && V <= 3 && exists(logN, V); }

int stage_table_entries(int logN, int V)
{
    switch (logN) {
    case 1: return entries_any<1>(V);
    case 2: return entries_any<2>(V);
    case 3: return entries_any<3>(V);
    case 4: return entries_any<4>(V);
    case 5: return entries_any<5>(V);
    case 6: return entries_any<6>(V);
    case 7: return entries_any<7>(V);
    case 8: return entries_any<8>(V);
    case 9: return entries_any<9>(V);
    case 10: return entries_any<10>(V);
    case 11: return entries_any<11>(V);
    case 12: return entries_any<12>(V);
    default: return -1;
    }
}

cudaError_t generate_stage_table(float2 *dst, int logN, cudaStream_t stream, int V)
{
    switch (logN) {
    case 1: return gen_any<1>(dst, V, stream);
    case 2: return gen_any<2>(dst, V, stream);
    case 3: return gen_any<3>(dst, V, stream);
    case 4: return gen_any<4>(dst, V, stream);
    case 5: return gen_any<5>(dst, V, stream);
    case 6: return gen_any<6>(dst, V, stream);
    case 7: return gen_any<7>(dst, V, stream);
    case 8: return gen_any<8>(dst, V, stream);
    case 9: return gen_any<9>(dst, V, stream);
    case 10: return gen_any<10>(dst, V, stream);
    case 11: return gen_any<11>(dst, V, stream);
    case 12: return gen_any<12>(dst, V, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t generate_full_stage(float2 *dst, int64_t M, int64_t M1, cudaStream_t stream)
{
    full_stage_kernel<<<(unsigned)((16 * M1 + 255) / 256), 256, 0, stream>>>(dst, M, M1);
    return cudaGetLastError();
}

cudaError_t generate_two_level(float2 *lo, float2 *hi, int logn, int h, cudaStream_t stream)
{
    const int64_t n = int64_t(1) << logn;
    const int64_t nlo = int64_t(1) << h, nhi = n >> h;
    power_table_kernel<<<(unsigned)((nlo + 255) / 256), 256, 0, stream>>>(lo, nlo, 1, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    power_table_kernel<<<(unsigned)((nhi + 255) / 256), 256, 0, stream>>>(hi, nhi, nlo, n);
    return cudaGetLastError();
}

}  // namespace moa
