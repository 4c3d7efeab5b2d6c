// Host matrix exponential exp(M) for the ODE solution of Theorem 1 (Section 3,
// Eq. (C)), which applies exp(t A_j) along every mode.
//
// Method: scaling and squaring with the [13/13] Pade approximant (N. J. Higham,
// "The scaling and squaring method for the matrix exponential revisited",
// SIAM J. Matrix Anal. Appl. 26(4), 2005): M is scaled by 2^-s so that
// ||2^-s M||_1 <= theta_13 = 5.37..., r_13(X) = (V - U)^-1 (V + U) with U the
// odd and V the even part of the Pade numerator, then squared s times.  The
// Pade coefficients come from their closed form
//   b_k = (2m - k)! m! / ((2m)! k! (m - k)!),  m = 13.
// All arithmetic is std::complex<double>; matrices are column-major.
#include "sylv_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace sylv {

using cd = std::complex<double>;

namespace {

using Mat = std::vector<cd>;

void matmul(int64_t n, const Mat &A, const Mat &B, Mat &C) {
    C.assign((size_t)(n * n), cd(0.0, 0.0));
    for (int64_t c = 0; c < n; ++c)
        for (int64_t k = 0; k < n; ++k) {
            const cd b = B[(size_t)(k + c * n)];
            if (b == cd(0.0, 0.0)) continue;
            const cd *a = &A[(size_t)(k * n)];
            cd *out = &C[(size_t)(c * n)];
            for (int64_t r = 0; r < n; ++r) out[r] += a[r] * b;
        }
}

double norm1(int64_t n, const Mat &A) {
    double best = 0.0;
    for (int64_t c = 0; c < n; ++c) {
        double s = 0.0;
        for (int64_t r = 0; r < n; ++r) s += std::abs(A[(size_t)(r + c * n)]);
        best = std::max(best, s);
    }
    return best;
}

// Solve P X = Q in place (X overwrites Q) by LU with partial pivoting.
bool solve_lu(int64_t n, Mat P, Mat &Q) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k;
        double best = std::abs(P[(size_t)(k + k * n)]);
        for (int64_t r = k + 1; r < n; ++r) {
            const double v = std::abs(P[(size_t)(r + k * n)]);
            if (v > best) { best = v; p = r; }
        }
        if (!(best > 0.0)) return false;
        if (p != k) {
            for (int64_t c = 0; c < n; ++c) std::swap(P[(size_t)(k + c * n)], P[(size_t)(p + c * n)]);
            for (int64_t c = 0; c < n; ++c) std::swap(Q[(size_t)(k + c * n)], Q[(size_t)(p + c * n)]);
        }
        const cd d = P[(size_t)(k + k * n)];
        for (int64_t r = k + 1; r < n; ++r) {
            const cd f = P[(size_t)(r + k * n)] / d;
            P[(size_t)(r + k * n)] = f;
            if (f == cd(0.0, 0.0)) continue;
            for (int64_t c = k + 1; c < n; ++c) P[(size_t)(r + c * n)] -= f * P[(size_t)(k + c * n)];
            for (int64_t c = 0; c < n; ++c) Q[(size_t)(r + c * n)] -= f * Q[(size_t)(k + c * n)];
        }
    }
    // back substitution with the upper factor, every column of Q
    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = n - 1; r >= 0; --r) {
            cd s = Q[(size_t)(r + c * n)];
            for (int64_t k = r + 1; k < n; ++k) s -= P[(size_t)(r + k * n)] * Q[(size_t)(k + c * n)];
            Q[(size_t)(r + c * n)] = s / P[(size_t)(r + r * n)];
        }
    return true;
}

}  // namespace

sylv_status expm_host(int64_t n, const double *Min, double *Eout) {
    if (n < 1) return SYLV_ERR_SHAPE;
    const size_t nn = (size_t)(n * n);
    Mat M(nn);
    for (size_t k = 0; k < nn; ++k) {
        M[k] = cd(Min[2 * k], Min[2 * k + 1]);
        if (!std::isfinite(M[k].real()) || !std::isfinite(M[k].imag())) return SYLV_ERR_INVALID_ARG;
    }
    constexpr int m = 13;
    constexpr double theta13 = 5.371920351148152;
    double b[m + 1];
    b[0] = 1.0;
    for (int k = 1; k <= m; ++k) b[k] = b[k - 1] * (double)(m - k + 1) / ((double)(2 * m - k + 1) * k);

    const double nrm = norm1(n, M);
    int s = 0;
    if (nrm > theta13) s = (int)std::ceil(std::log2(nrm / theta13));
    if (s > 0) {
        const double f = std::ldexp(1.0, -s);
        for (auto &z : M) z *= f;
    }
    Mat M2, M4, M6, tmp, tmp2;
    matmul(n, M, M, M2);
    matmul(n, M2, M2, M4);
    matmul(n, M4, M2, M6);
    // U = M [M6 (b13 M6 + b11 M4 + b9 M2) + b7 M6 + b5 M4 + b3 M2 + b1 I]
    // V =    M6 (b12 M6 + b10 M4 + b8 M2) + b6 M6 + b4 M4 + b2 M2 + b0 I
    Mat inner(nn), V(nn), U(nn);
    for (size_t k = 0; k < nn; ++k) inner[k] = b[13] * M6[k] + b[11] * M4[k] + b[9] * M2[k];
    matmul(n, M6, inner, tmp);
    for (size_t k = 0; k < nn; ++k) tmp[k] += b[7] * M6[k] + b[5] * M4[k] + b[3] * M2[k];
    for (int64_t i = 0; i < n; ++i) tmp[(size_t)(i + i * n)] += b[1];
    matmul(n, M, tmp, U);
    for (size_t k = 0; k < nn; ++k) inner[k] = b[12] * M6[k] + b[10] * M4[k] + b[8] * M2[k];
    matmul(n, M6, inner, V);
    for (size_t k = 0; k < nn; ++k) V[k] += b[6] * M6[k] + b[4] * M4[k] + b[2] * M2[k];
    for (int64_t i = 0; i < n; ++i) V[(size_t)(i + i * n)] += b[0];
    // r13 = (V - U)^-1 (V + U)
    Mat P(nn), R(nn);
    for (size_t k = 0; k < nn; ++k) {
        P[k] = V[k] - U[k];
        R[k] = V[k] + U[k];
    }
    if (!solve_lu(n, P, R)) return SYLV_ERR_SINGULAR;
    for (int i = 0; i < s; ++i) {
        matmul(n, R, R, tmp2);
        R.swap(tmp2);
    }
    for (size_t k = 0; k < nn; ++k) {
        Eout[2 * k] = R[k].real();
        Eout[2 * k + 1] = R[k].imag();
        if (!std::isfinite(R[k].real()) || !std::isfinite(R[k].imag())) return SYLV_ERR_INVALID_ARG;
    }
    return SYLV_OK;
}

}  // namespace sylv
