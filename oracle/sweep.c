/*
 * ORACLE -- test infrastructure only.  Plain, sequential FP64 triangular sweep
 * of the non-recursive N-dimensional Bartels-Stewart method.  Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark use this file; the
 * CUDA library never links it.
 *
 * What it computes (Section 2, Eq. (yi1i2iN)): given upper-triangular T_j and
 * the transformed right-hand side C, the tensor Y with
 *
 *   y_i = ( c_i - sum_j sum_{k > i_j} t_{j, i_j k} y_{i with i_j -> k} )
 *         / sum_j t_{j, i_j i_j}.
 *
 * Order (Algorithm 3, with the index generator of Algorithm 2): the linear
 * index runs from n_1*...*n_N down to 1 while the multi-index (i_1, ..., i_N)
 * is decremented as a mixed-radix counter with i_1 fastest.  The numerator
 * accumulates mode j = 1..N in ascending order and, inside a mode, k
 * ascending.  Y overwrites C in place because c_i is read once, before y_i is
 * written (remark after Algorithm 2).
 *
 * Layout (Section 2.2, Eq. (index)): column-major, zero-based
 * index = sum_j i_j * S_j with S_1 = 1, S_{j+1} = S_j * n_j; the entry that
 * differs only in mode j (i_j -> k) sits at index + (k - i_j) * S_j.
 * Complex numbers are interleaved (re, im) doubles; T_j is column-major, so
 * t_{j, a b} is at T_j[2 * (a + b * n_j)].
 *
 * Complex division: Smith's algorithm (R. L. Smith, CACM 5(8), 1962).
 */
#include <stdint.h>
#include <stdlib.h>

static void smith_div(double a, double b, double c, double d, double *re, double *im)
{
    /* (a + ib) / (c + id) */
    double ac = c < 0 ? -c : c;
    double ad = d < 0 ? -d : d;
    if (ad <= ac) {
        double r = d / c;
        double den = c + d * r;
        *re = (a + b * r) / den;
        *im = (b - a * r) / den;
    } else {
        double r = c / d;
        double den = c * r + d;
        *re = (a * r + b) / den;
        *im = (b * r - a) / den;
    }
}

/* Returns 0 on success, 1 if some denominator was exactly zero, 2 on bad args. */
int oracle_sweep(int N, const int64_t *n, const double *const *T, double *Y)
{
    if (N < 1 || !n || !T || !Y) return 2;
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *ii = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!S || !ii) { free(S); free(ii); return 2; }
    int64_t total = 1;
    for (int j = 0; j < N; ++j) {
        S[j] = total;
        total *= n[j];
        ii[j] = n[j] - 1;               /* Algorithm 2 starts at (n_1, ..., n_N) */
    }
    int status = 0;
    for (int64_t index = total - 1; index >= 0; --index) {
        double num_re = Y[2 * index], num_im = Y[2 * index + 1];
        double den_re = 0.0, den_im = 0.0;
        for (int j = 0; j < N; ++j) {
            const double *Tj = T[j];
            int64_t nj = n[j], ij = ii[j];
            den_re += Tj[2 * (ij + ij * nj)];
            den_im += Tj[2 * (ij + ij * nj) + 1];
            for (int64_t k = ij + 1; k < nj; ++k) {
                double t_re = Tj[2 * (ij + k * nj)], t_im = Tj[2 * (ij + k * nj) + 1];
                int64_t o = index + (k - ij) * S[j];
                double y_re = Y[2 * o], y_im = Y[2 * o + 1];
                num_re -= t_re * y_re - t_im * y_im;
                num_im -= t_re * y_im + t_im * y_re;
            }
        }
        if (den_re == 0.0 && den_im == 0.0) status = 1;
        smith_div(num_re, num_im, den_re, den_im, &Y[2 * index], &Y[2 * index + 1]);
        /* mixed-radix decrement, i_1 fastest (Algorithm 2) */
        for (int k = 0; k < N; ++k) {
            if (ii[k] > 0) { ii[k] -= 1; break; }
            ii[k] = n[k] - 1;
        }
    }
    free(S);
    free(ii);
    return status;
}

/* Mixed-radix generator of Algorithm 2 on its own: writes the 1-based tuples in
 * generation order into out[count * N] (for checking the traversal order). */
int oracle_counter_order(int N, const int64_t *n, int64_t count, int64_t *out)
{
    if (N < 1) return 2;
    int64_t *ii = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!ii) return 2;
    for (int j = 0; j < N; ++j) ii[j] = n[j];
    for (int64_t t = 0; t < count; ++t) {
        for (int j = 0; j < N; ++j) out[t * N + j] = ii[j];
        int k = 0;
        while (k < N) {
            if (ii[k] > 1) { ii[k] -= 1; break; }
            ii[k] = n[k];
            ++k;
        }
    }
    free(ii);
    return 0;
}
