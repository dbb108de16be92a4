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

template <int LOGN>
int entries_typed() { return Sched<LOGN>::tw_entries(); }

template <int LOGN>
cudaError_t gen_typed(float2 *dst, cudaStream_t stream)
{
    using Sc = Sched<LOGN>;
    const int total = Sc::tw_entries();
    if (total == 0)
        return cudaSuccess;
    StageGen g[3] = {{1, 1, 0}, {1, 1, 0}, {1, 1, 0}};
    const int nst = Sc::S - 1;
    for (int s = 0; s < nst; ++s)
        g[s] = StageGen{Sc::M1(s) << Sc::rlog(s), Sc::M1(s), Sc::tw_offset(s)};
    stage_table_kernel<<<(total + 255) / 256, 256, 0, stream>>>(dst, total, g[0], g[1], g[2], nst);
    return cudaGetLastError();
}

}  // namespace

int stage_table_entries(int logN)
{
    switch (logN) {
    case 1: return entries_typed<1>();
    case 2: return entries_typed<2>();
    case 3: return entries_typed<3>();
    case 4: return entries_typed<4>();
    case 5: return entries_typed<5>();
    case 6: return entries_typed<6>();
    case 7: return entries_typed<7>();
    case 8: return entries_typed<8>();
    case 9: return entries_typed<9>();
    case 10: return entries_typed<10>();
    case 11: return entries_typed<11>();
    case 12: return entries_typed<12>();
    default: return -1;
    }
}

cudaError_t generate_stage_table(float2 *dst, int logN, cudaStream_t stream)
{
    switch (logN) {
    case 1: return gen_typed<1>(dst, stream);
    case 2: return gen_typed<2>(dst, stream);
    case 3: return gen_typed<3>(dst, stream);
    case 4: return gen_typed<4>(dst, stream);
    case 5: return gen_typed<5>(dst, stream);
    case 6: return gen_typed<6>(dst, stream);
    case 7: return gen_typed<7>(dst, stream);
    case 8: return gen_typed<8>(dst, stream);
    case 9: return gen_typed<9>(dst, stream);
    case 10: return gen_typed<10>(dst, stream);
    case 11: return gen_typed<11>(dst, stream);
    case 12: return gen_typed<12>(dst, stream);
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
