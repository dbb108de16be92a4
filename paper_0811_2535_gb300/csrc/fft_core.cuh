// In-register radix-2^k FFT core for lengths N = 2^L <= 4096 (sm_103a).
//
// The radix-2 butterfly loop of the paper (Fig. 2.1, Sec. 3.5-3.6) is
// regrouped so that up to four consecutive radix-2 stages run in registers:
// each thread holds P = 16 points (fewer when N < 16), computes a radix-R
// DFT (R in {2, 4, 8, 16}) on them, multiplies by the stage twiddles and
// exchanges through shared memory.  That is the paper's dimension lifting
// applied recursively inside one tile: N = R_1 * R_2 * ..., with the first
// radix over the slowest index (the "block phase" for a column of length
// N/R_1, Sec. 4.2) and each exchange playing the role of the block-to-cyclic
// redistribution (Sec. 4.6, Fig. 4.9).  The stages form a self-sorting
// (Stockham) sequence, so input and output are in natural order and no bit
// reversal (the first step of Fig. 2.1) is ever materialised.
//
// Stage s (K = R_1..R_{s-1} product, M = N/K, M1 = M/R_s):
//   butterfly b = kappa*M1 + u, kappa < K, u < M1,
//   reads  e = kappa*M + u + M1*m            (m < R_s)
//   y[k] = sum_m x_m w_{R_s}^{m k} * w_M^{u k}
//   writes e = (kappa + K*k)*M1 + u          (k < R_s)
// Thread tau (< T = N/P) owns butterflies b = tau + T*i, i < P/R_s.
//
// All arithmetic is FP32, exponent sign -1 (w_N = exp(-2 pi i/N)); the
// opposite sign is obtained by conjugating input and output.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace moa {

// Complex addition and subtraction as one packed FP32 instruction (sm_100 and
// later; each lane rounded to nearest like a scalar add): half the
// instructions of the radix-2/4/8/16 butterflies.  Being opaque to the
// compiler, a packed add is never contracted with a preceding multiply into
// an FMA, which the scalar form allowed; results differ from the scalar form
// in the last bits only where that happened.
__device__ __forceinline__ unsigned long long f2_bits(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long r)
{
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(r);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiplication by -i (the w_4 of the forward transform)
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// ---------------------------------------------------------------------------
// Small DFTs, exponent sign -1, natural order in and out, in place.
// Constants: cos/sin of pi/8 and sqrt(2)/2.
#define MOA_C8 0.92387953251128675613f
#define MOA_S8 0.38268343236508977173f
#define MOA_R2 0.70710678118654752440f

__device__ __forceinline__ void dft2(float2 &a, float2 &b)
{
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3)
{
    float2 s02 = cadd(x0, x2), d02 = csub(x0, x2);
    float2 s13 = cadd(x1, x3), d13 = mul_mi(csub(x1, x3));
    x0 = cadd(s02, s13);
    x2 = csub(s02, s13);
    x1 = cadd(d02, d13);
    x3 = csub(d02, d13);
}

// w_8^j, j = 1, 3 (forward): (sqrt2/2)(1 - i), (sqrt2/2)(-1 - i)
__device__ __forceinline__ float2 mul_w8_1(float2 a) { return make_float2(MOA_R2 * (a.x + a.y), MOA_R2 * (a.y - a.x)); }
__device__ __forceinline__ float2 mul_w8_3(float2 a) { return make_float2(MOA_R2 * (a.y - a.x), -MOA_R2 * (a.x + a.y)); }

// DFT-8 as 2 x 4: index m = 4*m1 + m2; k = k1 + 2*k2.
__device__ __forceinline__ void dft8(float2 *v)
{
    dft2(v[0], v[4]);
    dft2(v[1], v[5]);
    dft2(v[2], v[6]);
    dft2(v[3], v[7]);
    // twiddle w_8^(m2*k1) on the k1 = 1 half
    v[5] = mul_w8_1(v[5]);
    v[6] = mul_mi(v[6]);
    v[7] = mul_w8_3(v[7]);
    dft4(v[0], v[1], v[2], v[3]);   // k1 = 0: outputs k = 0, 2, 4, 6
    dft4(v[4], v[5], v[6], v[7]);   // k1 = 1: outputs k = 1, 3, 5, 7
    float2 t1 = v[1], t2 = v[2], t3 = v[3], t4 = v[4], t5 = v[5], t6 = v[6];
    v[1] = t4;
    v[2] = t1;
    v[3] = t5;
    v[4] = t2;
    v[5] = t6;
    v[6] = t3;
}

// DFT-16 as 4 x 4: index m = 4*m1 + m2; k = k1 + 4*k2.
__device__ __forceinline__ void dft16(float2 *v)
{
    dft4(v[0], v[4], v[8], v[12]);
    dft4(v[1], v[5], v[9], v[13]);
    dft4(v[2], v[6], v[10], v[14]);
    dft4(v[3], v[7], v[11], v[15]);
    // t[k1][m2] sits at v[4*k1 + m2]; twiddle w_16^(m2*k1)
    v[5] = cmul(v[5], make_float2(MOA_C8, -MOA_S8));    // w^1
    v[6] = mul_w8_1(v[6]);                              // w^2
    v[7] = cmul(v[7], make_float2(MOA_S8, -MOA_C8));    // w^3
    v[9] = mul_w8_1(v[9]);                              // w^2
    v[10] = mul_mi(v[10]);                              // w^4
    v[11] = mul_w8_3(v[11]);                            // w^6
    v[13] = cmul(v[13], make_float2(MOA_S8, -MOA_C8));  // w^3
    v[14] = mul_w8_3(v[14]);                            // w^6
    v[15] = cmul(v[15], make_float2(-MOA_C8, MOA_S8));  // w^9
    dft4(v[0], v[1], v[2], v[3]);
    dft4(v[4], v[5], v[6], v[7]);
    dft4(v[8], v[9], v[10], v[11]);
    dft4(v[12], v[13], v[14], v[15]);
    // y[k1 + 4*k2] = v[4*k1 + k2]: a 4x4 transpose of the register block
    float2 t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

template <int R> __device__ __forceinline__ void dft(float2 *v);
template <> __device__ __forceinline__ void dft<2>(float2 *v) { dft2(v[0], v[1]); }
template <> __device__ __forceinline__ void dft<4>(float2 *v) { dft4(v[0], v[1], v[2], v[3]); }
template <> __device__ __forceinline__ void dft<8>(float2 *v) { dft8(v); }
template <> __device__ __forceinline__ void dft<16>(float2 *v) { dft16(v); }

// ---------------------------------------------------------------------------
// Radix schedules for N = 2^L (any factorisation is a valid breakpoint,
// Sec. 4.8; the autotuner picks one by timing).  V selects the schedule:
//   V = 0: one stage of radix N when L <= 4, otherwise stages of radix 16
//          preceded by one stage of radix 2^(L mod 4) when L is not a
//          multiple of 4 (the small radix first, so the last stage reads
//          contiguous groups of 16 from shared memory);
//   V = 1: the same radices with the small one last;
//   V = 2: stages of radix 8, preceded by one of radix 2^(L mod 3) when L is
//          not a multiple of 3.
// Every thread holds P = 16 points in every schedule (two butterflies per
// stage of radix 8, eight of radix 2).
template <int LOGN, int V = 0> struct Sched {
    static_assert(V >= 0 && V <= 2, "radix schedules 0, 1, 2");
    static constexpr int N = 1 << LOGN;
    static constexpr int P = N < 16 ? N : 16;          // points per thread
    static constexpr int T = N / P;                    // threads per transform
    static constexpr int S = V == 2 ? (LOGN <= 3 ? 1 : (LOGN + 2) / 3) : (LOGN <= 4 ? 1 : (LOGN + 3) / 4);
    __host__ __device__ static constexpr int rlog(int s)
    {
        if (V == 2)
            return LOGN <= 3 ? LOGN : ((s == 0 && (LOGN % 3) != 0) ? (LOGN % 3) : 3);
        if (V == 1)
            return LOGN <= 4 ? LOGN : ((s == S - 1 && (LOGN % 4) != 0) ? (LOGN % 4) : 4);
        return LOGN <= 4 ? LOGN : ((s == 0 && (LOGN % 4) != 0) ? (LOGN % 4) : 4);
    }
    __host__ __device__ static constexpr int K(int s)  // product of earlier radices
    {
        int k = 1;
        for (int i = 0; i < s; ++i)
            k <<= rlog(i);
        return k;
    }
    __host__ __device__ static constexpr int M1(int s) { return N / K(s) >> rlog(s); }
    // offset (in entries) of stage s's twiddle block: 6 rows of M1(s) entries
    __host__ __device__ static constexpr int tw_offset(int s)
    {
        int o = 0;
        for (int i = 0; i < s; ++i)
            o += 6 * M1(i);
        return o;
    }
    __host__ __device__ static constexpr int tw_entries() { return tw_offset(S - 1); }
    // The exchanges address element e = w + off as a per-thread base plus a
    // compile-time offset (Layout below), which needs every stage but the
    // last to write at offsets N/R * k that are multiples of 16.  (The reads
    // always qualify: their base mod 16 plus their offset mod 16 stays below
    // 16 for power-of-two radices.)
    __host__ __device__ static constexpr bool valid()
    {
        if (P != 16 && S > 1)
            return false;
        for (int s = 0; s + 1 < S; ++s)
            if (((N >> rlog(s)) & 15) != 0)
                return false;
        return true;
    }
};

// Whether schedule V exists for 2^logN points and differs from schedule 0
// (V = 1 only when L is not a multiple of 4, L >= 9; V = 2 for L >= 7).
__host__ __device__ constexpr bool sched_variant_ok(int logN, int V)
{
    return V == 0 ? (logN >= 1 && logN <= 12)
                  : V == 1 ? (logN >= 9 && logN <= 11) : V == 2 ? (logN >= 7 && logN <= 12) : false;
}

// exponent multipliers of the six stored twiddle rows
__host__ __device__ constexpr int tw_row_k(int j) { return j < 4 ? j + 1 : (j == 4 ? 8 : 12); }

// Shared-memory layouts of the exchange buffer.  Element e of transform f
// is stored at padded index pe = e + e/16 (one slot of padding per 16
// elements, which keeps the stride-16 reads of a radix-16 stage free of
// bank conflicts) in one of two arrangements:
//   LAY >= 0  interleaved: slot (pe << LAY) + f, f < 2^LAY  (lanes vary f first)
//   LAY <  0  row-major:   slot f * (N + N/16) + pe        (lanes vary e first)
// Every index used below has the form e = w + off with a per-thread w and a
// compile-time off, and either off is a multiple of 16 or w is; then
// pe(w + off) = pe(w) + off + off/16 exactly, so every access is a per-thread
// base plus an immediate offset.
__host__ __device__ __forceinline__ constexpr int pad16(int e) { return e + (e >> 4); }

template <int N, int LAY>
struct Layout {
    __device__ __forceinline__ static int base(int pw, int f)
    {
        if constexpr (LAY >= 0)
            return (pw << LAY) + f;
        else if constexpr (LAY <= -2)
            // row pitch N + N/16 + 2^(-2-LAY): with 16, 8 or 4 rows per half-warp
            // (LAY = -2, -3, -4) both row-wise and row-interleaved lanes are conflict-free
            return f * (N + N / 16 + (1 << (-2 - LAY))) + pw;
        else
            return f * (N + N / 16) + pw;
    }
    __host__ __device__ static constexpr int off(int o)
    {
        return LAY >= 0 ? (pad16(o) << (LAY >= 0 ? LAY : 0)) : pad16(o);
    }
};

// Multiply butterfly outputs v[1..R-1] by w_M^(u*k) from the stage table
// (rows k = 1,2,3,4,8,12 of M1 entries each; others formed as products).
template <int R>
__device__ __forceinline__ void apply_twiddles(float2 *v, const float2 *__restrict__ t, int u, int M1)
{
    float2 w1 = __ldg(&t[u]);
    if constexpr (R == 2) {
        v[1] = cmul(v[1], w1);
    } else {
        float2 w2 = __ldg(&t[M1 + u]);
        float2 w3 = __ldg(&t[2 * M1 + u]);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        if constexpr (R >= 8) {
            float2 w4 = __ldg(&t[3 * M1 + u]);
            v[4] = cmul(v[4], w4);
            v[5] = cmul(v[5], cmul(w4, w1));
            v[6] = cmul(v[6], cmul(w4, w2));
            v[7] = cmul(v[7], cmul(w4, w3));
            if constexpr (R == 16) {
                float2 w8 = __ldg(&t[4 * M1 + u]);
                float2 w12 = __ldg(&t[5 * M1 + u]);
                v[8] = cmul(v[8], w8);
                v[9] = cmul(v[9], cmul(w8, w1));
                v[10] = cmul(v[10], cmul(w8, w2));
                v[11] = cmul(v[11], cmul(w8, w3));
                v[12] = cmul(v[12], w12);
                v[13] = cmul(v[13], cmul(w12, w1));
                v[14] = cmul(v[14], cmul(w12, w2));
                v[15] = cmul(v[15], cmul(w12, w3));
            }
        }
    }
}

// Element index (within the transform) held in register r before stage 0.
template <int LOGN, int V = 0>
__device__ __forceinline__ int load_index(int r, int tau)
{
    using Sc = Sched<LOGN, V>;
    constexpr int R = 1 << Sc::rlog(0);
    constexpr int NB = Sc::P / R;
    return tau + Sc::T * ((r / R) + NB * (r % R));
}

// Radix-R DFTs and twiddles of stage s on the registers of one thread.
// TWID = false leaves out the twiddles (a 2-D DFT whose slowest axis is the
// stage-0 digit: the stage-0 DFT is then a transform of its own).
template <int LOGN, int s, bool TWID = true, int V = 0>
__device__ __forceinline__ void stage_compute(float2 (&v)[16], int tau, const float2 *__restrict__ tw)
{
    using Sc = Sched<LOGN, V>;
    constexpr int R = 1 << Sc::rlog(s);
    constexpr int NB = Sc::P / R;
    constexpr int M1 = Sc::M1(s);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        dft<R>(&v[i * R]);
        if constexpr (TWID && s != Sc::S - 1) {
            const int b = tau + Sc::T * i;
            apply_twiddles<R>(&v[i * R], tw + Sc::tw_offset(s), b & (M1 - 1), M1);
        }
    }
}

// Scatter stage s outputs to their Stockham positions in shared memory.
template <int LOGN, int s, int LAY, int V = 0>
__device__ __forceinline__ void stage_write(const float2 (&v)[16], float2 *sm, int tau, int f)
{
    using Sc = Sched<LOGN, V>;
    using Ly = Layout<Sc::N, LAY>;
    constexpr int R = 1 << Sc::rlog(s);
    constexpr int NB = Sc::P / R;
    constexpr int M1 = Sc::M1(s);
    constexpr int KM1 = Sc::K(s) * M1;   // = N / R, a multiple of 16
    static_assert(KM1 % 16 == 0, "stage write offsets must be multiples of 16");
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = tau + Sc::T * i;
        // e = (kappa + K*k)*M1 + u = b + (N/R)*k
        float2 *p = sm + Ly::base(pad16(b), f);
#pragma unroll
        for (int k = 0; k < R; ++k)
            p[Ly::off(KM1 * k)] = v[i * R + k];
    }
}

// Gather stage s inputs from shared memory.
template <int LOGN, int s, int LAY, int V = 0>
__device__ __forceinline__ void stage_read(float2 (&v)[16], const float2 *sm, int tau, int f)
{
    using Sc = Sched<LOGN, V>;
    using Ly = Layout<Sc::N, LAY>;
    constexpr int R = 1 << Sc::rlog(s);
    constexpr int NB = Sc::P / R;
    constexpr int M1 = Sc::M1(s);
    constexpr int M = M1 * R;
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        const int b = tau + Sc::T * i;
        const int w = (b / M1) * M + (b & (M1 - 1));      // kappa*M + u
        const float2 *p = sm + Ly::base(pad16(w), f);
#pragma unroll
        for (int m = 0; m < R; ++m)
            v[i * R + m] = p[Ly::off(M1 * m)];
    }
}

// Stages 1..S-1 (stage 0 has been computed by the caller).  Every thread of
// the block must call this (it contains block barriers).  On return the
// thread holds the last stage's outputs: butterfly b = tau + T*i, output k
// (element X[b + (N/R)*k] for the last radix R) in v[i*R + k].
template <int LOGN, int s, int LAY, int V = 0>
__device__ __forceinline__ void run_stages(float2 (&v)[16], float2 *sm, int tau, int f,
                                           const float2 *__restrict__ tw)
{
    if constexpr (s < Sched<LOGN, V>::S) {
        stage_write<LOGN, s - 1, LAY, V>(v, sm, tau, f);
        __syncthreads();
        stage_read<LOGN, s, LAY, V>(v, sm, tau, f);
        __syncthreads();
        stage_compute<LOGN, s, true, V>(v, tau, tw);
        run_stages<LOGN, s + 1, LAY, V>(v, sm, tau, f, tw);
    }
}

// The whole transform of the registers v (loaded in the order of
// load_index).  On return the thread holds X[tau + T*q] in v[q], q < P, in
// every schedule: when the last radix R is below P, the thread's P/R last
// butterflies b = tau + T*i give X[tau + T*(i + (P/R)*k)] as output k, and the
// registers are renamed into that order (a compile-time permutation).
template <int LOGN, int LAY, int V = 0>
__device__ __forceinline__ void fft_tile(float2 (&v)[16], float2 *sm, int tau, int f, const float2 *__restrict__ tw)
{
    using Sc = Sched<LOGN, V>;
    static_assert(Sc::valid(), "radix schedule not usable for this length");
    stage_compute<LOGN, 0, true, V>(v, tau, tw);
    run_stages<LOGN, 1, LAY, V>(v, sm, tau, f, tw);
    constexpr int RL = 1 << Sc::rlog(Sc::S - 1);
    constexpr int NBL = Sc::P / RL;
    if constexpr (NBL > 1) {
        float2 t[16];
#pragma unroll
        for (int r = 0; r < Sc::P; ++r)
            t[r] = v[r];
#pragma unroll
        for (int i = 0; i < NBL; ++i)
#pragma unroll
            for (int k = 0; k < RL; ++k)
                v[i + NBL * k] = t[i * RL + k];
    }
}

// Largest number of transforms per tile of the interleaved layout for
// length 2^LOGN (tiles of 2^12 points, at least 4 transforms so column
// accesses cover whole 32-byte sectors); the exchange buffer is sized for it.
__host__ __device__ constexpr int max_logF_interleaved(int logN) { return logN >= 10 ? 2 : 12 - logN; }

}  // namespace moa
