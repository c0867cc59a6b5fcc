/*
 * CPU oracle for the sparse embedding (CountSketch) of Clarkson & Woodruff,
 * "Low Rank Approximation and Regression in Input Sparsity Time".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the GPU library is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * never does.  It shares no code with the GPU path.
 *
 * What it computes (paper Section 2, definition of the sparse embedding matrix):
 *   S = Phi D with Phi in {0,1}^{t x n}, Phi[h(i), i] = 1, and D = diag(sigma),
 *   sigma(i) in {+1, -1}.  Hence (SA)[j, :] = sum over rows i with h(i) = j of
 *   sigma(i) * A[i, :], and the same for Sb (Theorem "lin reg" sketches A and b
 *   with the same S).  Sums are taken in float64, rows in ascending order.
 *
 * The random map: the paper takes h uniform on [t] and D with independent
 * signs.  This build fixes a seeded 4-wise independent family instead:
 *   p = 2^61 - 1;  coefficients from the SplitMix64 stream (Steele, Lea and
 *   Flood, 2014) started at `seed`: each draw z gives c = z & (2^61 - 1),
 *   drawing again when c == 2^61 - 1; draws 0..3 are the bucket polynomial
 *   (c0..c3), draws 4..7 the sign polynomial.
 *   g(x) = c3 x^3 + c2 x^2 + c1 x + c0 (mod p), x = the 0-based row index.
 *   h(i) = g_bucket(i) mod m;  sigma(i) = +1 if g_sign(i) is even, else -1.
 * Arithmetic here is the textbook one: 128-bit products reduced with `%`.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <omp.h>

#define ORC_P ((uint64_t)0x1FFFFFFFFFFFFFFFull) /* 2^61 - 1 */

typedef struct {
    uint64_t cb[4]; /* bucket polynomial c0..c3 */
    uint64_t cs[4]; /* sign polynomial c0..c3 */
} orc_poly;

static uint64_t orc_splitmix_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ull;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void orc_coefficients(uint64_t seed, orc_poly *P)
{
    uint64_t state = seed;
    uint64_t c[8];
    int k;
    for (k = 0; k < 8; ++k) {
        uint64_t v;
        do {
            v = orc_splitmix_next(&state) & ORC_P;
        } while (v == ORC_P);
        c[k] = v;
    }
    for (k = 0; k < 4; ++k) {
        P->cb[k] = c[k];
        P->cs[k] = c[4 + k];
    }
}

/* g(x) = ((c3 x + c2) x + c1) x + c0 mod p, with exact 128-bit intermediates. */
static uint64_t orc_poly_eval(const uint64_t c[4], uint64_t x)
{
    unsigned __int128 acc = c[3];
    unsigned __int128 xx = x % ORC_P;
    acc = (acc * xx + c[2]) % ORC_P;
    acc = (acc * xx + c[1]) % ORC_P;
    acc = (acc * xx + c[0]) % ORC_P;
    return (uint64_t)acc;
}

static void orc_bucket_sign(const orc_poly *P, uint64_t i, uint64_t m, int64_t *bucket, int *sign)
{
    *bucket = (int64_t)(orc_poly_eval(P->cb, i) % m);
    *sign = (orc_poly_eval(P->cs, i) % 2 == 0) ? 1 : -1;
}

/* ---- exported entry points (host arrays only) -------------------------- */

void orc_coeffs(uint64_t seed, uint64_t out[8])
{
    orc_poly P;
    int k;
    orc_coefficients(seed, &P);
    for (k = 0; k < 4; ++k) {
        out[k] = P.cb[k];
        out[4 + k] = P.cs[k];
    }
}

/* Raw polynomial values g_bucket(i), g_sign(i) for i = i0 .. i0+count-1. */
void orc_poly_values(uint64_t seed, int64_t i0, int64_t count, uint64_t *gb, uint64_t *gs)
{
    orc_poly P;
    int64_t k;
    orc_coefficients(seed, &P);
    for (k = 0; k < count; ++k) {
        gb[k] = orc_poly_eval(P.cb, (uint64_t)(i0 + k));
        gs[k] = orc_poly_eval(P.cs, (uint64_t)(i0 + k));
    }
}

/* h(i) and sigma(i) for i = i0 .. i0+count-1. */
void orc_hash(uint64_t seed, int64_t m, int64_t i0, int64_t count, int32_t *bucket, int8_t *sign)
{
    orc_poly P;
    int64_t k;
    orc_coefficients(seed, &P);
    for (k = 0; k < count; ++k) {
        int64_t h;
        int s;
        orc_bucket_sign(&P, (uint64_t)(i0 + k), (uint64_t)m, &h, &s);
        bucket[k] = (int32_t)h;
        sign[k] = (int8_t)s;
    }
}

/*
 * SA (m x d, row-major, float64) and Sb (m, float64; skipped when b == NULL)
 * for CSR A with n rows.  Global row index of local row i is i0 + i (a row
 * shard hashes with its global indices).  Outputs are overwritten.
 */
void orc_sketch_csr(int64_t n, int64_t d, const int32_t *row_ptr, const int32_t *col,
                    const float *val, const float *b, int64_t m, uint64_t seed, int64_t i0,
                    double *SA, double *Sb)
{
    orc_poly P;
    int64_t i, k;
    orc_coefficients(seed, &P);
    memset(SA, 0, sizeof(double) * (size_t)m * (size_t)d);
    if (Sb) memset(Sb, 0, sizeof(double) * (size_t)m);
    for (i = 0; i < n; ++i) {
        int64_t h;
        int s;
        orc_bucket_sign(&P, (uint64_t)(i0 + i), (uint64_t)m, &h, &s);
        for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            SA[h * d + col[k]] += (double)s * (double)val[k];
        if (Sb) Sb[h] += (double)s * (double)b[i];
    }
}

/*
 * The same SA and Sb on all host cores, for the CPU baseline's all-core
 * variant: every row's (h, sigma) is computed in parallel, the rows are
 * counting-sorted by bucket (stable: ascending row order inside a bucket,
 * the permutation P of Section 5.2), and the buckets are summed in parallel,
 * each over its rows in ascending order.  Every entry of SA and Sb is thus the
 * same float64 sum, taken in the same order, as in orc_sketch_csr: the two
 * give bitwise identical results.  `threads` <= 0 uses the OpenMP default.
 */
void orc_sketch_csr_parallel(int64_t n, int64_t d, const int32_t *row_ptr, const int32_t *col,
                             const float *val, const float *b, int64_t m, uint64_t seed, int64_t i0,
                             int threads, double *SA, double *Sb)
{
    orc_poly P;
    int64_t i, j;
    int64_t *h = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int *sg = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int64_t *start = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (threads <= 0) threads = omp_get_max_threads();
    orc_coefficients(seed, &P);
    memset(SA, 0, sizeof(double) * (size_t)m * (size_t)d);
    if (Sb) memset(Sb, 0, sizeof(double) * (size_t)m);
#pragma omp parallel for num_threads(threads) schedule(static)
    for (i = 0; i < n; ++i) orc_bucket_sign(&P, (uint64_t)(i0 + i), (uint64_t)m, &h[i], &sg[i]);
    for (i = 0; i < n; ++i) ++start[h[i] + 1];
    for (j = 0; j < m; ++j) start[j + 1] += start[j];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        memcpy(fill, start, sizeof(int64_t) * (size_t)m);
        for (i = 0; i < n; ++i) order[fill[h[i]]++] = i;
        free(fill);
    }
#pragma omp parallel for num_threads(threads) schedule(dynamic, 64)
    for (j = 0; j < m; ++j) {
        int64_t q, k;
        for (q = start[j]; q < start[j + 1]; ++q) {
            const int64_t r = order[q];
            for (k = row_ptr[r]; k < row_ptr[r + 1]; ++k)
                SA[j * d + col[k]] += (double)sg[r] * (double)val[k];
            if (Sb) Sb[j] += (double)sg[r] * (double)b[r];
        }
    }
    free(h);
    free(sg);
    free(start);
    free(order);
}

/*
 * Seeds of the inner sketches of a generalized sparse embedding: the `count`
 * raw SplitMix64 outputs that follow the eight accepted coefficient draws of
 * `seed` in its stream (this build's reading; the paper only asks the inner
 * sketches B^(i) to be independent of h and of each other).
 */
void orc_seeds_after_coeffs(uint64_t seed, int64_t count, uint64_t *out)
{
    uint64_t state = seed;
    int64_t k;
    int taken = 0;
    while (taken < 8) {
        if ((orc_splitmix_next(&state) & ORC_P) != ORC_P) ++taken;
    }
    for (k = 0; k < count; ++k) out[k] = orc_splitmix_next(&state);
}

/*
 * Generalized sparse embedding (Section "Generalized Sparse Embedding
 * Matrices", "The construction"), row by row: row i lies in block h(i) of q
 * (h = the bucket map of `seed` over q buckets); inner sketch b (seed_b, v
 * buckets) sends it, with sign sigma_b(i) and weight 1 / sqrt(kappa), to row
 * h(i) * v * kappa + b * v + h_b(i) of the t = q * v * kappa output rows.
 * SA: t x d float64, Sb: t float64 (skipped when b == NULL), overwritten.
 */
void orc_sketch_csr_general(int64_t n, int64_t d, const int32_t *row_ptr, const int32_t *col,
                            const float *val, const float *b, int64_t q, int64_t v, int64_t kappa,
                            uint64_t seed, double *SA, double *Sb)
{
    orc_poly Pout;
    int64_t i, k, j;
    const int64_t t = q * v * kappa;
    const double w = 1.0 / sqrt((double)kappa);
    uint64_t *seeds = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)kappa);
    orc_poly *inner = (orc_poly *)malloc(sizeof(orc_poly) * (size_t)kappa);
    orc_coefficients(seed, &Pout);
    orc_seeds_after_coeffs(seed, kappa, seeds);
    for (j = 0; j < kappa; ++j) orc_coefficients(seeds[j], &inner[j]);
    memset(SA, 0, sizeof(double) * (size_t)t * (size_t)d);
    if (Sb) memset(Sb, 0, sizeof(double) * (size_t)t);
    for (i = 0; i < n; ++i) {
        int64_t blk, hb;
        int s0, sb;
        orc_bucket_sign(&Pout, (uint64_t)i, (uint64_t)q, &blk, &s0);
        for (j = 0; j < kappa; ++j) {
            int64_t row;
            orc_bucket_sign(&inner[j], (uint64_t)i, (uint64_t)v, &hb, &sb);
            row = blk * v * kappa + j * v + hb;
            for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                SA[row * d + col[k]] += w * (double)sb * (double)val[k];
            if (Sb) Sb[row] += w * (double)sb * (double)b[i];
        }
    }
    free(seeds);
    free(inner);
}

/*
 * The sketch with values v_i in place of the signs (S(v)[h(i), i] = v_i):
 * SA[h(i), :] += v_i A_i and Sb[h(i)] += v_i b_i, rows in ascending order.
 */
void orc_sketch_csr_values(int64_t n, int64_t d, const int32_t *row_ptr, const int32_t *col,
                           const float *val, const float *b, int64_t m, uint64_t seed, const float *v,
                           double *SA, double *Sb)
{
    orc_poly P;
    int64_t i, k;
    orc_coefficients(seed, &P);
    memset(SA, 0, sizeof(double) * (size_t)m * (size_t)d);
    if (Sb) memset(Sb, 0, sizeof(double) * (size_t)m);
    for (i = 0; i < n; ++i) {
        int64_t h;
        int s;
        orc_bucket_sign(&P, (uint64_t)i, (uint64_t)m, &h, &s);
        for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            SA[h * d + col[k]] += (double)v[i] * (double)val[k];
        if (Sb) Sb[h] += (double)v[i] * (double)b[i];
    }
}

/*
 * Gradient of a loss through SA(v), Sb(v): gv_i = sum_k gSA[h(i), col_k] val_k
 * + gSb[h(i)] b_i (gSb or b NULL: first term only).
 */
void orc_sketch_values_backward_csr(int64_t n, int64_t d, const int32_t *row_ptr, const int32_t *col,
                                    const float *val, const float *b, int64_t m, uint64_t seed,
                                    const double *gSA, const double *gSb, double *gv)
{
    orc_poly P;
    int64_t i, k;
    orc_coefficients(seed, &P);
    for (i = 0; i < n; ++i) {
        int64_t h;
        int s;
        double acc = 0.0;
        orc_bucket_sign(&P, (uint64_t)i, (uint64_t)m, &h, &s);
        for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k) acc += gSA[h * d + col[k]] * (double)val[k];
        if (gSb && b) acc += gSb[h] * (double)b[i];
        gv[i] = acc;
    }
}

/* Same for dense row-major A (n x d, leading dimension lda). */
void orc_sketch_dense(int64_t n, int64_t d, int64_t lda, const float *A, const float *b,
                      int64_t m, uint64_t seed, int64_t i0, double *SA, double *Sb)
{
    orc_poly P;
    int64_t i, j;
    orc_coefficients(seed, &P);
    memset(SA, 0, sizeof(double) * (size_t)m * (size_t)d);
    if (Sb) memset(Sb, 0, sizeof(double) * (size_t)m);
    for (i = 0; i < n; ++i) {
        int64_t h;
        int s;
        orc_bucket_sign(&P, (uint64_t)(i0 + i), (uint64_t)m, &h, &s);
        for (j = 0; j < d; ++j)
            SA[h * d + j] += (double)s * (double)A[i * lda + j];
        if (Sb) Sb[h] += (double)s * (double)b[i];
    }
}

/* y = A x (float64) for CSR A: used for exact residuals of returned solutions. */
void orc_csr_matvec(int64_t n, const int32_t *row_ptr, const int32_t *col, const float *val,
                    const double *x, double *y)
{
    int64_t i, k;
    for (i = 0; i < n; ++i) {
        double acc = 0.0;
        for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            acc += (double)val[k] * x[col[k]];
        y[i] = acc;
    }
}

/* g = A^T z (float64) for CSR A. */
void orc_csr_rmatvec(int64_t n, int64_t d, const int32_t *row_ptr, const int32_t *col,
                     const float *val, const double *z, double *g)
{
    int64_t i, k;
    memset(g, 0, sizeof(double) * (size_t)d);
    for (i = 0; i < n; ++i)
        for (k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            g[col[k]] += (double)val[k] * z[i];
}
