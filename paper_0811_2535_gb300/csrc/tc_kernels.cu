// Reduced-precision path: the radix-16 DFT blocks on tensor cores.
//
// A radix-16 stage multiplies every 16-point vector by the 16 x 16 complex
// DFT matrix.  Written on real and imaginary parts that is one real GEMM
//     [Re y; Im y] = W [Re x; Im x],   W = [[C, S], [-S, C]],
//     C[k][m] = cos(2 pi k m / 16), S[k][m] = sin(2 pi k m / 16)
// (exponent sign -1; the opposite sign conjugates input and output), with
// eight vectors per mma.sync.m16n8k16 (FP32 accumulate).  FP16 and BF16
// carry too few mantissa bits for the 1e-5 target, so both operands are
// split and the products recombined in FP32:
//   FP16: x = x_hi + x_lo, W = W_hi + W_lo;  W x ~ Wh xh + Wh xl + Wl xh
//   BF16: three parts (hi, mid, lo) each;    the six products of order
//         up to 2^-16 of the leading term.
// FP16 has a small range, so each stage's inputs are scaled by a power of
// two chosen from the tile's largest magnitude (exact, undone after the
// product).  Twiddles between stages and all data movement stay FP32.
//
// One block transforms one row of N = 256 or 4096 points at a time
// (persistent over rows): coalesced load to shared memory, three (or two)
// stages whose fragments are read from and written back to shared memory
// at their Stockham positions, coalesced store.
#include "fft_core.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace moa {

namespace {

template <bool BF16> struct TC;

template <> struct TC<false> {
    static constexpr int PARTS = 2;
    __device__ static void split(float v, uint16_t (&p)[3]) { tc::Split<false>::run(v, p); }
    __device__ static void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
    {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

template <> struct TC<true> {
    static constexpr int PARTS = 3;
    __device__ static void split(float v, uint16_t (&p)[3]) { tc::Split<true>::run(v, p); }
    __device__ static void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
    {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

using tc::pack;

// W[row][col] of the 32 x 32 real DFT-16 matrix (sign -1)
__device__ __forceinline__ float wval(int row, int col)
{
    const int k = row & 15, m = col & 15, j = (k * m) & 15;
    const float c = tc::cos16(j), s = tc::sin16(j);
    if (row < 16)
        return col < 16 ? c : s;     // Re y_k = sum C x_re + S x_im
    return col < 16 ? -s : c;        // Im y_k = sum -S x_re + C x_im
}

// Padded shared-memory slot of element e of the row (one pad per 16).
__device__ __forceinline__ int tslot(int e) { return e + (e >> 4); }

// Largest |re|, |im| over the block's values (every thread passes its own).
__device__ __forceinline__ float block_absmax(float v, float *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        red[warp] = v;
    __syncthreads();
    float m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        m = fmaxf(m, red[w]);
    __syncthreads();
    return m;
}

template <bool BF16, int LOGN>
__global__ void __launch_bounds__(256, 2) tc_row_kernel(const float2 *in, float2 *out, int64_t rows,
                                                        const float2 *__restrict__ tw, int flags)
{
    using P = TC<BF16>;
    constexpr int N = 1 << LOGN;
    constexpr int S = LOGN / 4;          // radix-16 stages
    constexpr int NV = N / 16;           // 16-point vectors per stage
    constexpr int NB = NV / 8;           // blocks of eight vectors (one mma N dimension)
    constexpr int WARPS = 8;
    constexpr int NBW = (NB + WARPS - 1) / WARPS;   // vector blocks per warp
    static_assert(NB % WARPS == 0 || NB < WARPS, "vector blocks must spread evenly over warps");
    __shared__ float2 sm[N + N / 16];
    __shared__ float red[WARPS];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;

    // A fragments of W, split into parts: a[part][mb][kb][4]
    uint32_t a[P::PARTS][2][2][4];
#pragma unroll
    for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                // register r holds (row, col), (row, col+1) with row = gid + 8*(r&1), col = 2*tig + 8*(r>>1)
                const int row = 16 * mb + gid + 8 * (r & 1), col = 16 * kb + 2 * tig + 8 * (r >> 1);
                uint16_t p0[3], p1[3];
                P::split(wval(row, col), p0);
                P::split(wval(row, col + 1), p1);
#pragma unroll
                for (int q = 0; q < P::PARTS; ++q)
                    a[q][mb][kb][r] = pack(p0[q], p1[q]);
            }

    const float cin = (flags & FLAG_CONJ_IN) ? -1.f : 1.f;
    const float cout = (flags & FLAG_CONJ_OUT) ? -1.f : 1.f;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const float2 *src = in + row * N;
        for (int e = tid; e < N; e += 256) {
            float2 v = src[e];
            v.y *= cin;
            sm[tslot(e)] = v;
        }
        __syncthreads();

        int K = 1;   // product of the radices of the stages done
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int M = N / K, M1 = M / 16;
            // power-of-two scale keeping the FP16 parts in range (BF16: none)
            float scale = 1.f, unscale = 1.f;
            if constexpr (!BF16) {
                float m = 0.f;
                for (int e = tid; e < N; e += 256) {
                    const float2 v = sm[tslot(e)];
                    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
                }
                m = block_absmax(m, red);
                if (m > 0.f) {
                    const int ex = ilogbf(m);           // m in [2^ex, 2^(ex+1))
                    scale = ldexpf(1.f, 10 - ex);       // largest part below 2^11
                    unscale = ldexpf(1.f, ex - 10);
                }
            }
            float d[NBW][2][4];
#pragma unroll
            for (int j = 0; j < NBW; ++j) {
                const int nb = warp + WARPS * j;
                if (nb >= NB)
                    continue;
                // this lane's inputs: points m = 2*tig + {0, 1, 8, 9} of vector b = 8*nb + gid
                const int b = 8 * nb + gid;
                const int kappa = b / M1, u = b % M1;
                const int base = kappa * M + u;
                uint16_t re[4][3], im[4][3];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int mm = 2 * tig + (i & 1) + 8 * (i >> 1);
                    const float2 v = sm[tslot(base + M1 * mm)];
                    P::split(v.x * scale, re[i]);
                    P::split(v.y * scale, im[i]);
                }
#pragma unroll
                for (int mb = 0; mb < 2; ++mb)
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        d[j][mb][r] = 0.f;
                // products, smallest first: for parts (p, q) with p + q < PARTS
#pragma unroll
                for (int ord = P::PARTS - 1; ord >= 0; --ord)
#pragma unroll
                    for (int pa = 0; pa <= ord; ++pa) {
                        const int pb = ord - pa;
                        const uint32_t bre0 = pack(re[0][pb], re[1][pb]), bre1 = pack(re[2][pb], re[3][pb]);
                        const uint32_t bim0 = pack(im[0][pb], im[1][pb]), bim1 = pack(im[2][pb], im[3][pb]);
#pragma unroll
                        for (int mb = 0; mb < 2; ++mb) {
                            P::mma(d[j][mb], a[pa][mb][0], bre0, bre1);
                            P::mma(d[j][mb], a[pa][mb][1], bim0, bim1);
                        }
                    }
            }
            __syncthreads();   // every stage input has been read
#pragma unroll
            for (int j = 0; j < NBW; ++j) {
                const int nb = warp + WARPS * j;
                if (nb >= NB)
                    continue;
                // d[j][0][r]: Re y_k, d[j][1][r]: Im y_k, k = gid + 8*(r>>1), vector 8*nb + 2*tig + (r&1)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int k = gid + 8 * (r >> 1);
                    const int b = 8 * nb + 2 * tig + (r & 1);
                    const int kappa = b / M1, u = b % M1;
                    float2 y = make_float2(d[j][0][r] * unscale, d[j][1][r] * unscale);
                    if (s != S - 1)
                        y = cmul(y, __ldg(&tw[(s == 0 ? 0 : 16 * (N / 16)) + k * M1 + u]));
                    sm[tslot((kappa + K * k) * M1 + u)] = y;
                }
            }
            __syncthreads();
            K *= 16;
        }
        float2 *dst = out + row * N;
        for (int e = tid; e < N; e += 256) {
            float2 v = sm[tslot(e)];
            v.y *= cout;
            dst[e] = v;
        }
        __syncthreads();
    }
}

template <bool BF16, int LOGN>
cudaError_t launch_tc_typed(const PassDesc &d, const float2 *in, float2 *out, const float2 *tw, int flags,
                            cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int64_t grid = d.O < (int64_t)sms * 2 ? d.O : (int64_t)sms * 2;
    tc_row_kernel<BF16, LOGN><<<(unsigned)grid, 256, 0, stream>>>(in, out, d.O, tw, flags);
    return cudaGetLastError();
}

}  // namespace

int tc_table_entries(int logN) { return logN == 12 ? 16 * 256 + 16 * 16 : (logN == 8 ? 16 * 16 : -1); }

cudaError_t launch_tc_pass(const PassDesc &d, bool bf16, const float2 *in, float2 *out, const float2 *tw, int flags,
                           cudaStream_t stream)
{
    if (d.logN == 12)
        return bf16 ? launch_tc_typed<true, 12>(d, in, out, tw, flags, stream)
                    : launch_tc_typed<false, 12>(d, in, out, tw, flags, stream);
    if (d.logN == 8)
        return bf16 ? launch_tc_typed<true, 8>(d, in, out, tw, flags, stream)
                    : launch_tc_typed<false, 8>(d, in, out, tw, flags, stream);
    return cudaErrorInvalidValue;
}

}  // namespace moa
