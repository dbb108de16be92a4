// Pieces shared by the two tensor-core kernels (tc_kernels.cu: mma.sync;
// tc_umma.cu: tcgen05): the DFT-16 matrix entries and the splitting of an
// FP32 value into FP16 or BF16 parts whose sum approximates it.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace moa {
namespace tc {

// cos(2 pi j / 16) and sin(2 pi j / 16) for any integer j, from the three
// constants cos(pi/8), sqrt(2)/2, sin(pi/8) by the symmetries of the cosine.
__device__ __forceinline__ float cos16(int j)
{
    j &= 15;
    if (j > 8)
        j = 16 - j;   // cos(2 pi (16 - j) / 16) = cos(2 pi j / 16), now 0..8
    const int a = j <= 4 ? j : 8 - j;   // cos(pi - x) = -cos(x)
    const float c = a == 0 ? 1.f : a == 1 ? MOA_C8 : a == 2 ? MOA_R2 : a == 3 ? MOA_S8 : 0.f;
    return j <= 4 ? c : -c;
}
__device__ __forceinline__ float sin16(int j) { return cos16(j + 12); }   // sin x = cos(x - pi/2)

// Entry (row, col) of the real 32 x 32 form of the DFT-16 matrix (sign -1)
// with real and imaginary parts interleaved on both sides: row 2k + c' is
// Re y_k (c' = 0) or Im y_k (c' = 1), column 2m + c multiplies Re x_m (c = 0)
// or Im x_m (c = 1).  Re y = sum C x_re + S x_im, Im y = sum -S x_re + C x_im.
__device__ __forceinline__ float w_interleaved(int row, int col)
{
    const int j = ((row >> 1) * (col >> 1)) & 15;
    const float c = cos16(j), s = sin16(j);
    if ((row & 1) == 0)
        return (col & 1) == 0 ? c : s;
    return (col & 1) == 0 ? -s : c;
}

template <bool BF16> struct Split;

// FP16: v ~ hi + lo (22 significand bits)
template <> struct Split<false> {
    static constexpr int PARTS = 2;
    __device__ static void run(float v, uint16_t (&p)[3])
    {
        const __half h = __float2half_rn(v);
        const __half l = __float2half_rn(v - __half2float(h));
        p[0] = __half_as_ushort(h);
        p[1] = __half_as_ushort(l);
        p[2] = 0;
    }
};

// BF16: v ~ hi + mid + lo (24 significand bits)
template <> struct Split<true> {
    static constexpr int PARTS = 3;
    __device__ static void run(float v, uint16_t (&p)[3])
    {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
        p[0] = __bfloat16_as_ushort(h);
        p[1] = __bfloat16_as_ushort(m);
        p[2] = __bfloat16_as_ushort(l);
    }
};

__device__ __forceinline__ uint32_t pack(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// The same splitting on a complex value, one part at a time: take() returns
// the next part as a packed (re | im) pair of 16-bit values (re in the low
// half) and leaves the FP32 residual in v.
template <bool BF16> struct Split2;

template <> struct Split2<false> {
    static constexpr int PARTS = 2;
    __device__ static uint32_t take(float2 &v)
    {
        const __half2 h = __float22half2_rn(v);
        const float2 b = __half22float2(h);
        v.x -= b.x;
        v.y -= b.y;
        return *reinterpret_cast<const uint32_t *>(&h);
    }
};

template <> struct Split2<true> {
    static constexpr int PARTS = 3;
    __device__ static uint32_t take(float2 &v)
    {
        const __nv_bfloat162 h = __float22bfloat162_rn(v);
        const float2 b = __bfloat1622float2(h);
        v.x -= b.x;
        v.y -= b.y;
        return *reinterpret_cast<const uint32_t *>(&h);
    }
};

}  // namespace tc
}  // namespace moa
