/*
 * The paper's shared-memory all-processor templates on the host cores.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this directory: the tests and
 * the CPU baseline leg of the benchmark call it.  It shares no code with the
 * CUDA path.  It is the CPU comparison point for the GPU path: the paper's
 * own parallel method, in FP64, on every host core.
 *
 *   tmpl_fft_partitioned  Sec. 6.3, Fig. 6.4: the combined plan of Fig. 4.9
 *                         with both p loops made parallel.  Thread p copies
 *                         its consecutive block of psize = n/m elements into
 *                         private memory, runs stages q < breakpoint there and
 *                         copies it back (Fig. 6.5, block <-> centralized);
 *                         after the first parallel loop ends, thread p copies
 *                         the stride-m subset x(p), x(p+m), ... into private
 *                         memory, runs stages q >= breakpoint with only its
 *                         weights w_L^(m*row' + p) (Sec. 4.4-4.5) and copies it
 *                         back.  The copy through the shared array between the
 *                         loops is the block-to-cyclic redistribution.
 *   tmpl_fft_nd           Appendix B, Eq. B.6 with the lines of each axis as
 *                         the parallel loop (Sec. 6.1 style: the lines are
 *                         disjoint, so each is one thread's work), each line a
 *                         sequential radix-2 transform (Fig. 2.1).
 *
 * The arithmetic of each butterfly, the weights and the order of the stages
 * are those of the sequential plans, so the results equal them bit for bit:
 * only which core runs which p changes.  Built with OpenMP where the compiler
 * has it; without it the parallel loops run on one thread and
 * tmpl_max_threads() returns 1.  Return codes: 0, -1 bad argument, -2 no
 * memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559

int tmpl_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int pow2_ge2(int64_t n)
{
    return n >= 2 && (n & (n - 1)) == 0;
}

static int ilog2(int64_t n)
{
    int t = 0;
    while (((int64_t)1 << t) < n)
        ++t;
    return t;
}

/* w = exp(s * 2*pi*i * num/den), den a power of two (num/den exact). */
static void root(int64_t num, int64_t den, int s, double *re, double *im)
{
    double a = TWO_PI * ((double)num / (double)den);
    *re = cos(a);
    *im = (double)s * sin(a);
}

static int64_t bitrev(int64_t j, int t)
{
    int64_t k = 0;
    for (int b = 0; b < t; ++b)
        if (j & ((int64_t)1 << b))
            k |= (int64_t)1 << (t - 1 - b);
    return k;
}

/* The butterflies of one stage over `len` consecutive complex entries of v,
 * in columns of `col` entries whose two halves are `half` apart, the half
 * rows taking the weights w[0 .. half-1]:
 *   c = w * v_hi, v_lo' = d + c, v_hi' = d - c with d = v_lo. */
static void stage(double *v, int64_t len, int64_t col, int64_t half, const double *w)
{
    for (int64_t c0 = 0; c0 < len; c0 += col) {
        for (int64_t r = 0; r < half; ++r) {
            double *lo = &v[2 * (c0 + r)];
            double *hi = &v[2 * (c0 + r + half)];
            double wr = w[2 * r], wi = w[2 * r + 1];
            double cr = wr * hi[0] - wi * hi[1];
            double ci = wr * hi[1] + wi * hi[0];
            double dr = lo[0], di = lo[1];
            lo[0] = dr + cr;
            lo[1] = di + ci;
            hi[0] = dr - cr;
            hi[1] = di - ci;
        }
    }
}

/* Sequential Fig. 2.1 on one private vector: bit reversal, then q = 1..t
 * with the Fig. 3.8 weights w_L^row. */
static void radix2_private(double *v, int64_t len, int sign, double *w)
{
    const int t = ilog2(len);
    for (int64_t j = 0; j < len; ++j) {
        int64_t k = bitrev(j, t);
        if (j < k) {
            double r = v[2 * j], i = v[2 * j + 1];
            v[2 * j] = v[2 * k];
            v[2 * j + 1] = v[2 * k + 1];
            v[2 * k] = r;
            v[2 * k + 1] = i;
        }
    }
    for (int q = 1; q <= t; ++q) {
        const int64_t L = (int64_t)1 << q;
        for (int64_t r = 0; r < L / 2; ++r)
            root(r, L, sign, &w[2 * r], &w[2 * r + 1]);
        stage(v, len, L, L / 2, w);
    }
}

/* Fig. 6.4 on m "processors" (a power of two, m <= psize = n/m) with the
 * stages split at `breakpoint`, log2(m) + 1 <= breakpoint <= log2(psize) + 1
 * (Sec. 4.8).  In place; x is n interleaved complex doubles. */
int tmpl_fft_partitioned(double *x, int64_t n, int64_t m, int breakpoint, int sign)
{
    if (!pow2_ge2(n) || m < 1 || (m & (m - 1)) != 0 || (sign != 1 && sign != -1))
        return -1;
    const int t = ilog2(n);
    const int64_t psize = n / m;
    if (m > psize || breakpoint < ilog2(m) + 1 || breakpoint > ilog2(psize) + 1)
        return -1;
    int failed = 0;

    /* Fig. 2.1 begins with P_n x.  Each pair (j, bitrev(j)) is swapped by the
     * iteration with the smaller index only, so the iterations are disjoint. */
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        int64_t k = bitrev(j, t);
        if (j < k) {
            double r = x[2 * j], i = x[2 * j + 1];
            x[2 * j] = x[2 * k];
            x[2 * j + 1] = x[2 * k + 1];
            x[2 * k] = r;
            x[2 * k + 1] = i;
        }
    }

    /* first parallel do: block partitioned, stages 1 .. breakpoint-1 */
#pragma omp parallel for schedule(static) reduction(| : failed)
    for (int64_t p = 0; p < m; ++p) {
        double *xblock = (double *)malloc(sizeof(double) * 2 * (size_t)psize);
        double *weight = (double *)malloc(sizeof(double) * (size_t)psize);
        if (xblock && weight) {
            memcpy(xblock, x + 2 * psize * p, sizeof(double) * 2 * (size_t)psize);
            for (int q = 1; q <= breakpoint - 1; ++q) {
                const int64_t L = (int64_t)1 << q;
                for (int64_t r = 0; r < L / 2; ++r)
                    root(r, L, sign, &weight[2 * r], &weight[2 * r + 1]);
                stage(xblock, psize, L, L / 2, weight);
            }
            memcpy(x + 2 * psize * p, xblock, sizeof(double) * 2 * (size_t)psize);
        } else {
            failed = 1;
        }
        free(xblock);
        free(weight);
    }
    if (failed)
        return -2;

    /* second parallel do: cyclic partitioned, stages breakpoint .. t.  In the
     * private copy xcyclic(i) = x(m*i + p) a length-L column takes L/m
     * consecutive entries and its butterflies pair entries L/(2m) apart. */
#pragma omp parallel for schedule(static) reduction(| : failed)
    for (int64_t p = 0; p < m; ++p) {
        double *xcyclic = (double *)malloc(sizeof(double) * 2 * (size_t)psize);
        double *weight = (double *)malloc(sizeof(double) * (size_t)psize);
        if (xcyclic && weight) {
            for (int64_t i = 0; i < psize; ++i) {
                xcyclic[2 * i] = x[2 * (m * i + p)];
                xcyclic[2 * i + 1] = x[2 * (m * i + p) + 1];
            }
            for (int q = breakpoint; q <= t; ++q) {
                const int64_t L = (int64_t)1 << q, half = L / (2 * m);
                for (int64_t r = 0; r < half; ++r)
                    root(m * r + p, L, sign, &weight[2 * r], &weight[2 * r + 1]);
                stage(xcyclic, psize, L / m, half, weight);
            }
            for (int64_t i = 0; i < psize; ++i) {
                x[2 * (m * i + p)] = xcyclic[2 * i];
                x[2 * (m * i + p) + 1] = xcyclic[2 * i + 1];
            }
        } else {
            failed = 1;
        }
        free(xcyclic);
        free(weight);
    }
    return failed ? -2 : 0;
}

/* Eq. B.6 in parallel: `batch` row-major arrays of shape[0..dims-1], each
 * axis (last first) transformed line by line, the lines of one axis spread
 * over the threads.  The end of each axis's loop is a barrier. */
int tmpl_fft_nd(double *x, const int64_t *shape, int dims, int64_t batch, int sign)
{
    if (dims < 1 || dims > 8 || batch < 1 || (sign != 1 && sign != -1))
        return -1;
    int64_t total = 1, maxlen = 1;
    for (int a = 0; a < dims; ++a) {
        if (!pow2_ge2(shape[a]))
            return -1;
        total *= shape[a];
        if (shape[a] > maxlen)
            maxlen = shape[a];
    }
    int failed = 0;
#pragma omp parallel reduction(| : failed)
    {
        double *line = (double *)malloc(sizeof(double) * 2 * (size_t)maxlen);
        double *weight = (double *)malloc(sizeof(double) * (size_t)maxlen);
        if (!line || !weight)
            failed = 1;
        for (int64_t b = 0; b < batch; ++b) {
            double *arr = x + 2 * total * b;
            for (int a = dims - 1; a >= 0; --a) {
                int64_t stride = 1;
                for (int k = a + 1; k < dims; ++k)
                    stride *= shape[k];
                const int64_t len = shape[a], lines = total / len;
#pragma omp for schedule(static)
                for (int64_t li = 0; li < lines; ++li) {
                    if (!line || !weight)
                        continue;
                    double *base = arr + 2 * ((li / stride) * len * stride + li % stride);
                    for (int64_t j = 0; j < len; ++j) {
                        line[2 * j] = base[2 * j * stride];
                        line[2 * j + 1] = base[2 * j * stride + 1];
                    }
                    radix2_private(line, len, sign, weight);
                    for (int64_t j = 0; j < len; ++j) {
                        base[2 * j * stride] = line[2 * j];
                        base[2 * j * stride + 1] = line[2 * j + 1];
                    }
                }
            }
        }
        free(line);
        free(weight);
    }
    return failed ? -2 : 0;
}
