/*
 * FP64 CPU oracle for the MoA reshape-transpose radix-2 FFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may call this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Data layout: complex values are interleaved (re, im) doubles.  Multi-D
 * arrays are row-major (MoA gamma ordering, Appendix A, Definition A.1),
 * batch outermost.  Transforms are unnormalised.  The exponent sign s is a
 * parameter: X[k] = sum_j x[j] * exp(s * 2*pi*i * j*k / n).  The paper's
 * weight formula EXP((2*pi*i*row)/L) (Fig. 3.8) is the s = +1 case.
 *
 * Functions and the passages they follow:
 *   oracle_dft_naive        the DFT definition itself (the "Output: the FFT
 *                           of x" of Fig. 2.1), O(n^2), exact angle reduction
 *   oracle_fft_radix2       Fig. 2.1 (bit reversal P_n, then the q loop of
 *                           B_L products) scalarised as in Sec. 3.5-3.6
 *                           (in-place butterfly c = w*x_hi, x_lo' = d + c,
 *                           x_hi' = d - c), weights computed directly per
 *                           stage as in Fig. 3.8
 *   oracle_fft_partitioned  Sec. 4.2-4.7, Fig. 4.9: q loop split at
 *                           `breakpoint`, block phase on private copies of
 *                           consecutive psize-element blocks, cyclic phase
 *                           on private copies of the stride-m subsets with
 *                           only the needed weights (Sec. 4.4-4.5)
 *   oracle_fft_four_step    the dimension-lifting restatement: x viewed as
 *                           an r x c array, r-point column DFTs, twiddle
 *                           exp(s*2*pi*i*j2*k1/n), c-point row DFTs,
 *                           transposed output index k1 + r*k2
 *   oracle_fft_nd           Appendix B, Eq. B.6 (Omega): a d-dimensional
 *                           DFT as the 1-D transform applied along each axis
 *   oracle_gamma            Appendix A, Definition A.1: row-major offset
 *
 * Every function returns 0 on success and a negative value on a bad
 * argument (n not a power of two >= 2, or a split outside the range the
 * paper allows).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559

static int is_pow2_at_least_2(int64_t n)
{
    return n >= 2 && (n & (n - 1)) == 0;
}

static int log2_exact(int64_t n)
{
    int t = 0;
    while (((int64_t)1 << t) < n)
        ++t;
    return t;
}

/* exp(s * 2*pi*i * num / den) with 0 <= num < den; num/den is exact for the
 * power-of-two denominators used here, so the only rounding is in the
 * multiplication by 2*pi and in cos/sin. */
static void unit_root(int64_t num, int64_t den, int s, double *re, double *im)
{
    double a = TWO_PI * ((double)num / (double)den);
    *re = cos(a);
    *im = (double)s * sin(a);
}

/* ---------------------------------------------------------------------- */
/* Definition A.1: gamma(s, p) = x_{d-1}, x_0 = p_0, x_j = x_{j-1}*s_j + p_j */
int64_t oracle_gamma(const int64_t *shape, const int64_t *index, int d)
{
    if (d <= 0)
        return 0;
    int64_t x = index[0];
    for (int j = 1; j < d; ++j)
        x = x * shape[j] + index[j];
    return x;
}

/* ---------------------------------------------------------------------- */
/* The DFT by its definition: y[k] = sum_j x[j] w^(j*k), with the exponent
 * reduced exactly (j*k mod n) before the trigonometric evaluation. */
int oracle_dft_naive(const double *x, double *y, int64_t n, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1))
        return -1;
    for (int64_t k = 0; k < n; ++k) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            int64_t e = (int64_t)(((unsigned __int128)j * (unsigned __int128)k) % (unsigned __int128)n);
            double wr, wi;
            unit_root(e, n, sign, &wr, &wi);
            double xr = x[2 * j], xi = x[2 * j + 1];
            sr += xr * wr - xi * wi;
            si += xr * wi + xi * wr;
        }
        y[2 * k] = sr;
        y[2 * k + 1] = si;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Fig. 2.1 begins with x <- P_n x, the bit-reversal permutation.  Element j
 * moves to position bitrev_t(j); the permutation is an involution, so each
 * pair is swapped once. */
static void bit_reverse_permute(double *x, int64_t n, int t)
{
    for (int64_t j = 0; j < n; ++j) {
        int64_t k = 0;
        for (int b = 0; b < t; ++b)
            if (j & ((int64_t)1 << b))
                k |= (int64_t)1 << (t - 1 - b);
        if (j < k) {
            double r = x[2 * j], i = x[2 * j + 1];
            x[2 * j] = x[2 * k];
            x[2 * j + 1] = x[2 * k + 1];
            x[2 * k] = r;
            x[2 * k + 1] = i;
        }
    }
}

/* One stage q of the butterfly loop over the whole vector: x_{L x r} <-
 * B_L x_{L x r} with L = 2^q, the L x r matrix stored column-wise in x so
 * that element (row, col) is x(L*col + row) (Sec. 3.3).  B_L = [I, W; I, -W]
 * with W = diag(w_L^0 .. w_L^{L/2-1}) (Fig. 2.1); the product is done with
 * the optimised in-place basic block of Sec. 3.5-3.6. */
static void butterfly_stage(double *x, int64_t n, int q, int sign, double *weight)
{
    const int64_t L = (int64_t)1 << q, half = L / 2;
    for (int64_t row = 0; row < half; ++row)               /* Fig. 3.8 weights */
        unit_root(row, L, sign, &weight[2 * row], &weight[2 * row + 1]);
    for (int64_t col0 = 0; col0 < n; col0 += L) {           /* each column */
        for (int64_t row = 0; row < half; ++row) {
            double *lo = &x[2 * (col0 + row)];
            double *hi = &x[2 * (col0 + row + half)];
            double wr = weight[2 * row], wi = weight[2 * row + 1];
            double cr = wr * hi[0] - wi * hi[1];            /* c = weight*x_hi */
            double ci = wr * hi[1] + wi * hi[0];
            double dr = lo[0], di = lo[1];                  /* d = x_lo */
            lo[0] = dr + cr;
            lo[1] = di + ci;
            hi[0] = dr - cr;
            hi[1] = di - ci;
        }
    }
}

/* Fig. 2.1 as scalarised in Sec. 3: bit reversal, then q = 1..t. In place. */
int oracle_fft_radix2(double *x, int64_t n, int sign)
{
    if (!is_pow2_at_least_2(n) || (sign != 1 && sign != -1))
        return -1;
    const int t = log2_exact(n);
    double *weight = (double *)malloc(sizeof(double) * (size_t)n);
    if (!weight)
        return -2;
    bit_reverse_permute(x, n, t);
    for (int q = 1; q <= t; ++q)
        butterfly_stage(x, n, q, sign, weight);
    free(weight);
    return 0;
}

/* Batched form: `batch` consecutive transforms of length n. */
int oracle_fft_radix2_batch(double *x, int64_t n, int64_t batch, int sign)
{
    for (int64_t b = 0; b < batch; ++b) {
        int rc = oracle_fft_radix2(x + 2 * n * b, n, sign);
        if (rc)
            return rc;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Sec. 4, Fig. 4.9: the combined plan using partitioned data.
 *
 * m "processors" (a power of two), psize = n/m elements each.  After the
 * bit reversal that begins Fig. 2.1, stages q < breakpoint run in the block
 * phase: processor p copies the psize consecutive elements starting at
 * p*psize into a private vector xblock, runs those stages on it (each column
 * of length L = 2^q <= psize lies inside the block) and copies it back.
 * Stages q >= breakpoint run in the cyclic phase: processor p copies the
 * elements whose position is congruent to p mod m into a private vector
 * xcyclic (xcyclic(i) = x(m*i + p)), where each length-L column of x
 * occupies L/m consecutive entries, and uses only its weights
 * weightcyclic(row') = w_L^(m*row' + p) (Sec. 4.4-4.5).  The allowed range
 * is log2(m) + 1 <= breakpoint <= log2(psize) + 1 (Sec. 4.8); that range
 * needs m <= psize.  The p loops run one after another here: their data
 * sets are disjoint (Sec. 4.3), so the order does not matter. */
int oracle_fft_partitioned(double *x, int64_t n, int64_t m, int breakpoint, int sign)
{
    if (!is_pow2_at_least_2(n) || m < 1 || (m & (m - 1)) != 0 || (sign != 1 && sign != -1))
        return -1;
    const int t = log2_exact(n);
    const int64_t psize = n / m;
    if (m > psize)
        return -1;
    const int lo_bp = log2_exact(m) + 1, hi_bp = log2_exact(psize) + 1;
    if (breakpoint < lo_bp || breakpoint > hi_bp)
        return -1;

    double *priv = (double *)malloc(sizeof(double) * 2 * (size_t)psize);
    double *weight = (double *)malloc(sizeof(double) * (size_t)n);
    if (!priv || !weight) {
        free(priv);
        free(weight);
        return -2;
    }
    bit_reverse_permute(x, n, t);

    /* block phase */
    for (int64_t p = 0; p < m; ++p) {
        memcpy(priv, x + 2 * p * psize, sizeof(double) * 2 * (size_t)psize);
        for (int q = 1; q <= breakpoint - 1; ++q)
            butterfly_stage(priv, psize, q, sign, weight);
        memcpy(x + 2 * p * psize, priv, sizeof(double) * 2 * (size_t)psize);
    }

    /* cyclic phase */
    for (int64_t p = 0; p < m; ++p) {
        for (int64_t i = 0; i < psize; ++i) {
            priv[2 * i] = x[2 * (m * i + p)];
            priv[2 * i + 1] = x[2 * (m * i + p) + 1];
        }
        for (int q = breakpoint; q <= t; ++q) {
            const int64_t L = (int64_t)1 << q;
            const int64_t col_len = L / m, half = L / (2 * m);
            for (int64_t rp = 0; rp < half; ++rp)
                unit_root(m * rp + p, L, sign, &weight[2 * rp], &weight[2 * rp + 1]);
            for (int64_t col0 = 0; col0 < psize; col0 += col_len) {
                for (int64_t rp = 0; rp < half; ++rp) {
                    double *lo = &priv[2 * (col0 + rp)];
                    double *hi = &priv[2 * (col0 + rp + half)];
                    double wr = weight[2 * rp], wi = weight[2 * rp + 1];
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
        for (int64_t i = 0; i < psize; ++i) {
            x[2 * (m * i + p)] = priv[2 * i];
            x[2 * (m * i + p) + 1] = priv[2 * i + 1];
        }
    }
    free(priv);
    free(weight);
    return 0;
}

/* In-place length-len transform of a vector (len 1 is the identity). */
static int line_fft(double *v, int64_t len, int sign)
{
    if (len == 1)
        return 0;
    return oracle_fft_radix2(v, len, sign);
}

/* ---------------------------------------------------------------------- */
/* Dimension lifting (Sec. 1, "reshape-transpose"): n = r*c.
 *   A[j1][j2] = x[c*j1 + j2]                          (reshape, no movement)
 *   B[k1][j2] = sum_j1 A[j1][j2] w_r^(j1*k1)          (r-point column DFTs)
 *   B'[k1][j2] = B[k1][j2] * w_n^(j2*k1 mod n)        (twiddle)
 *   E[k1][k2] = sum_j2 B'[k1][j2] w_c^(j2*k2)         (c-point row DFTs)
 *   y[k1 + r*k2] = E[k1][k2]                          (transpose)
 * Each 1-D piece is oracle_fft_radix2. */
int oracle_fft_four_step(const double *x, double *y, int64_t r, int64_t c, int sign)
{
    if (r < 1 || c < 1 || (r & (r - 1)) || (c & (c - 1)) || r * c < 2 || (sign != 1 && sign != -1))
        return -1;
    const int64_t n = r * c;
    double *B = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    double *line = (double *)malloc(sizeof(double) * 2 * (size_t)(r > c ? r : c));
    if (!B || !line) {
        free(B);
        free(line);
        return -2;
    }
    for (int64_t j2 = 0; j2 < c; ++j2) {
        for (int64_t j1 = 0; j1 < r; ++j1) {
            line[2 * j1] = x[2 * (c * j1 + j2)];
            line[2 * j1 + 1] = x[2 * (c * j1 + j2) + 1];
        }
        line_fft(line, r, sign);
        for (int64_t k1 = 0; k1 < r; ++k1) {
            double wr, wi;
            unit_root((j2 * k1) % n, n, sign, &wr, &wi);
            double br = line[2 * k1], bi = line[2 * k1 + 1];
            B[2 * (c * k1 + j2)] = br * wr - bi * wi;
            B[2 * (c * k1 + j2) + 1] = br * wi + bi * wr;
        }
    }
    for (int64_t k1 = 0; k1 < r; ++k1) {
        memcpy(line, B + 2 * c * k1, sizeof(double) * 2 * (size_t)c);
        line_fft(line, c, sign);
        for (int64_t k2 = 0; k2 < c; ++k2) {
            y[2 * (k1 + r * k2)] = line[2 * k2];
            y[2 * (k1 + r * k2) + 1] = line[2 * k2 + 1];
        }
    }
    free(B);
    free(line);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Appendix B, Eq. B.6: Omega applies an operation along a chosen axis.  The
 * d-dimensional DFT of a row-major array of shape n[0..d-1] is the 1-D DFT
 * applied along every axis in turn (the axis order does not matter).  Each
 * of the `batch` arrays is transformed independently, in place. */
int oracle_fft_nd(double *x, const int64_t *shape, int dims, int64_t batch, int sign)
{
    if (dims < 1 || dims > 8 || batch < 1 || (sign != 1 && sign != -1))
        return -1;
    int64_t total = 1, maxlen = 1;
    for (int a = 0; a < dims; ++a) {
        if (!is_pow2_at_least_2(shape[a]))
            return -1;
        total *= shape[a];
        if (shape[a] > maxlen)
            maxlen = shape[a];
    }
    double *line = (double *)malloc(sizeof(double) * 2 * (size_t)maxlen);
    if (!line)
        return -2;
    for (int64_t b = 0; b < batch; ++b) {
        double *arr = x + 2 * total * b;
        for (int a = dims - 1; a >= 0; --a) {
            int64_t stride = 1;
            for (int k = a + 1; k < dims; ++k)
                stride *= shape[k];
            const int64_t len = shape[a], outer = total / (len * stride);
            for (int64_t o = 0; o < outer; ++o) {
                for (int64_t i = 0; i < stride; ++i) {
                    double *base = arr + 2 * (o * len * stride + i);
                    for (int64_t j = 0; j < len; ++j) {
                        line[2 * j] = base[2 * j * stride];
                        line[2 * j + 1] = base[2 * j * stride + 1];
                    }
                    oracle_fft_radix2(line, len, sign);
                    for (int64_t j = 0; j < len; ++j) {
                        base[2 * j * stride] = line[2 * j];
                        base[2 * j * stride + 1] = line[2 * j + 1];
                    }
                }
            }
        }
    }
    free(line);
    return 0;
}
