/*
 * Oracle tile routines: plain, slow, sequential CPU arithmetic.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it (through oracle/__init__.py).  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes comes from the task-programming model of the paper:
 * tasks are functions over registered buffers with R / W / RW access modes
 * (Section 2), and a program with the annotations removed is a valid
 * sequential program (Section 3), so executing every task at submission, in
 * submission order, is a legal schedule and gives the reference result.
 *
 * The task bodies are the paper's vector-scaling example (Section 2: each
 * element of the buffer is multiplied by a scalar factor) and the tile
 * kernels of a right-looking tiled Cholesky factorisation, the
 * "common idiom" the paper gives for partitioned matrices (Section 5.1).
 * The paper states no Cholesky arithmetic; the tile bodies below are the
 * textbook definitions, written out loop by loop:
 *   POTRF : A_kk = L_kk L_kk^T          (Cholesky-Crout, column by column)
 *   TRSM  : A_ik <- A_ik L_kk^{-T}       (right side, lower, transposed)
 *   SYRK  : A_ii <- A_ii - A_ik A_ik^T   (lower triangle only)
 *   GEMM  : A_ij <- A_ij - A_ik A_jk^T
 * Layout: a tile is a contiguous b x b block, column-major inside the tile
 * (element (r, c) at r + c*b).  Only the lower triangle of diagonal tiles is
 * read or written.
 *
 * Compiled with -O2 -ffp-contract=off -fno-fast-math: every multiply and add
 * is a separately rounded IEEE-754 operation, subnormals are honoured.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define AT(A, ld, r, c) (A)[(size_t)(r) + (size_t)(c) * (size_t)(ld)]

/* ---------------------------------------------------------------- vector */

/* Vector-scaling task body (Section 2 example): val[i] *= factor, binary32,
 * one rounding per multiply. */
void orc_scal_f32(float *x, int64_t n, float f)
{
    for (int64_t i = 0; i < n; ++i) {
        float v = x[i] * f;
        x[i] = v;
    }
}

/* ------------------------------------------------------------------ FP64 */

/* Cholesky-Crout on an n x n column-major block with leading dimension ld.
 * Returns 0, or the 1-based column j at which the pivot d_j is <= 0 or NaN
 * (LAPACK's info convention); columns before it hold the factor, the rest
 * is left as partially updated. */
int orc_potrf(double *A, int n, int ld)
{
    for (int j = 0; j < n; ++j) {
        double d = AT(A, ld, j, j);
        for (int p = 0; p < j; ++p) d -= AT(A, ld, j, p) * AT(A, ld, j, p);
        if (!(d > 0.0)) return j + 1;
        double ljj = sqrt(d);
        AT(A, ld, j, j) = ljj;
        for (int i = j + 1; i < n; ++i) {
            double s = AT(A, ld, i, j);
            for (int p = 0; p < j; ++p) s -= AT(A, ld, i, p) * AT(A, ld, j, p);
            AT(A, ld, i, j) = s / ljj;
        }
    }
    return 0;
}

/* X L^T = A solved for X in place of A: A is m x n (ld lda), L is n x n lower
 * (ld ldl).  Row r: X(r,c) = (A(r,c) - sum_{q<c} X(r,q) L(c,q)) / L(c,c). */
void orc_trsm(const double *L, int ldl, double *A, int m, int n, int lda)
{
    for (int r = 0; r < m; ++r) {
        for (int c = 0; c < n; ++c) {
            double s = AT(A, lda, r, c);
            for (int q = 0; q < c; ++q) s -= AT(A, lda, r, q) * AT(L, ldl, c, q);
            AT(A, lda, r, c) = s / AT(L, ldl, c, c);
        }
    }
}

/* C <- C - A A^T on the lower triangle of the n x n block C; A is n x k. */
void orc_syrk(const double *A, int n, int k, int lda, double *C, int ldc)
{
    for (int c = 0; c < n; ++c) {
        for (int r = c; r < n; ++r) {
            double s = 0.0;
            for (int p = 0; p < k; ++p) s += AT(A, lda, r, p) * AT(A, lda, c, p);
            AT(C, ldc, r, c) = AT(C, ldc, r, c) - s;
        }
    }
}

/* C <- C - A B^T; C is m x n, A is m x k, B is n x k. */
void orc_gemm(const double *A, int lda, const double *B, int ldb, double *C,
              int m, int n, int k, int ldc)
{
    for (int c = 0; c < n; ++c) {
        for (int r = 0; r < m; ++r) {
            double s = 0.0;
            for (int p = 0; p < k; ++p) s += AT(A, lda, r, p) * AT(B, ldb, c, p);
            AT(C, ldc, r, c) = AT(C, ldc, r, c) - s;
        }
    }
}

/* ------------------------------------------------------- low precision */

/* Round a value to the nearest value of a binary format with `p`
 * significant bits (implicit bit included) and minimum normal exponent
 * `emin`, ties to even: ONE rounding, straight from FP64.  Values whose
 * magnitude rounds above `maxval` become +-maxval when `satfinite` is set,
 * +-inf otherwise.  NaN stays NaN.
 *   bfloat16 : p = 8, emin = -126, maxval = (2 - 2^-7) * 2^127
 *   E4M3     : p = 4, emin = -6,   maxval = 448 (no infinities; saturating)
 * The quantum (spacing of the format's grid around x) is 2^(e - p + 1), e
 * the exponent of x's leading bit clamped below at emin (the format's
 * subnormals share the quantum of its smallest binade).  x / quantum is exact
 * in FP64 (a power-of-two scaling of a finite double), rint() rounds it to
 * the nearest integer with ties to even in the default rounding mode, and
 * the product with the quantum is exact again. */
double orc_round_format(double x, int p, int emin, double maxval, int satfinite)
{
    if (x != x || x == 0.0) return x;
    if (isinf(x)) {
        if (satfinite) return x > 0 ? maxval : -maxval;
        return x;
    }
    int e2;
    frexp(x, &e2);             /* |x| = m 2^e2, m in [0.5, 1) */
    int e = e2 - 1;            /* exponent of the leading bit */
    if (e < emin) e = emin;    /* subnormal range: fixed quantum */
    double quantum = ldexp(1.0, e - p + 1);
    double y = rint(x / quantum) * quantum;
    if (fabs(y) > maxval) {
        if (satfinite) return y > 0 ? maxval : -maxval;
        return y > 0 ? INFINITY : -INFINITY;
    }
    return y;
}

/* Smallest integer e with amax <= fmt_max * 2^e (exact comparisons), the
 * exponent of the per-tile power-of-two scale s = 2^e.  amax = 0 gives 0. */
int orc_scale_exponent(double amax, double fmt_max)
{
    if (!(amax > 0.0)) return 0;
    int e2;
    frexp(amax / fmt_max, &e2);
    int e = e2 + 1;
    while (e > -1074 && amax <= ldexp(fmt_max, e - 1)) --e;
    while (amax > ldexp(fmt_max, e)) ++e;
    return e;
}

/* Quantise n FP64 values: q[i] = round_format(x[i] / s), s = 2^e.  x / s is
 * exact (a power-of-two scaling), so each value is rounded once, from FP64
 * to the format.  q holds the format values as doubles. */
void orc_quantise(const double *x, int64_t n, int e, int p, int emin,
                  double maxval, int satfinite, double *q)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = ldexp(x[i], -e);
        q[i] = orc_round_format(v, p, emin, maxval, satfinite);
    }
}

/* Mixed-precision update C <- fl32(C - s * sum_p QA(r,p) QB(c,p)) for an m x n
 * binary32 block C (lower triangle only when lower != 0).  QA, QB hold
 * low-precision values (exactly representable), s is the product of the two
 * tiles' power-of-two scales.  The sum of the exact products is accumulated
 * in FP64; the device accumulates in binary32, so the comparison uses a
 * bound on binary32 accumulation error. */
void orc_gemm_lowp(const double *QA, int lda, const double *QB, int ldb,
                   double s, float *C, int m, int n, int k, int ldc, int lower)
{
    for (int c = 0; c < n; ++c) {
        for (int r = lower ? c : 0; r < m; ++r) {
            double acc = 0.0;
            for (int p = 0; p < k; ++p) acc += AT(QA, lda, r, p) * AT(QB, ldb, c, p);
            double v = (double)AT(C, ldc, r, c) - s * acc;
            AT(C, ldc, r, c) = (float)v;
        }
    }
}

/* sum_p |QA(r,p) QB(c,p)| for the same block, the scale of the binary32
 * accumulation error bound used by the parity tests. */
void orc_gemm_abs(const double *QA, int lda, const double *QB, int ldb,
                  double *out, int m, int n, int k, int ldo)
{
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < m; ++r) {
            double acc = 0.0;
            for (int p = 0; p < k; ++p) acc += fabs(AT(QA, lda, r, p) * AT(QB, ldb, c, p));
            AT(out, ldo, r, c) = acc;
        }
}
