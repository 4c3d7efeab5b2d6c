/*
 * ORACLE -- test infrastructure only.  Plain FP64 complex mode-j product
 * (Section 1): for an n_1 x ... x n_N tensor X in column-major order, viewed
 * as (L, n, R) with L = n_1 ... n_{j-1}, n = n_j, R = n_{j+1} ... n_N (times
 * any trailing right-hand-side extent),
 *
 *   Y[l, i, r] = sum_{k=0}^{n-1} M[i, k] * X[l, k, r],
 *
 * M column-major n x n (m_{ik} at M[2 (i + k n)]), complex numbers interleaved
 * (re, im).  The sum runs over k in ascending order with a plain complex
 * multiply-add (no fused multiply-add: compiled with -ffp-contract=off).
 * The (i, r) fibres are independent; OpenMP spreads them over threads, which
 * changes no entry's arithmetic.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use this file.
 */
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Returns 0 on success, 2 on bad arguments.  Y must not alias X. */
int oracle_mode_product(int64_t L, int64_t n, int64_t R, const double *M, const double *X,
                        double *Y)
{
    if (L < 1 || n < 1 || R < 0 || !M || !X || !Y) return 2;
    const int64_t fibres = n * R;
    #pragma omp parallel for schedule(static) if (L * fibres >= 65536)
    for (int64_t f = 0; f < fibres; ++f) {
        const int64_t i = f % n, r = f / n;
        double *y = Y + 2 * (L * (i + n * r));
        for (int64_t l = 0; l < L; ++l) {
            y[2 * l] = 0.0;
            y[2 * l + 1] = 0.0;
        }
        for (int64_t k = 0; k < n; ++k) {
            const double m_re = M[2 * (i + k * n)], m_im = M[2 * (i + k * n) + 1];
            const double *x = X + 2 * (L * (k + n * r));
            for (int64_t l = 0; l < L; ++l) {
                const double x_re = x[2 * l], x_im = x[2 * l + 1];
                y[2 * l] += m_re * x_re - m_im * x_im;
                y[2 * l + 1] += m_re * x_im + m_im * x_re;
            }
        }
    }
    return 0;
}

/* Threads of the fibre loop when called from the calling thread (1 keeps the
 * mode product on that thread, for callers that run several solves at once). */
void oracle_set_threads(int k)
{
#ifdef _OPENMP
    if (k >= 1) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
