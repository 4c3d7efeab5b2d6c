// Host complex Schur decomposition A = Q T Q^* (the setup step of Section 2:
// each A_j is reduced to upper-triangular T_j by a unitary U_j).
//
// Method (textbook; Golub & Van Loan, "Matrix Computations", ch. 7):
//   1. Householder reduction to upper Hessenberg form, H = Q0^* A Q0.
//   2. Implicit single-shift QR sweeps (bulge chasing with complex Givens
//      rotations) on the active window, Wilkinson shift from the trailing
//      2x2 block, exceptional shifts after 10 and 20 stalled sweeps, and
//      deflation when a subdiagonal entry falls below eps times its
//      neighbouring diagonal entries.
// All arithmetic is std::complex<double>; matrices are column-major.
#include "sylv_internal.h"

#include <cmath>
#include <complex>
#include <vector>

namespace sylv {

using cd = std::complex<double>;

namespace {

struct Mat {
    int64_t n;
    std::vector<cd> v;
    explicit Mat(int64_t n_) : n(n_), v((size_t)(n_ * n_)) {}
    cd &operator()(int64_t r, int64_t c) { return v[(size_t)(r + c * n)]; }
    const cd &operator()(int64_t r, int64_t c) const { return v[(size_t)(r + c * n)]; }
};

// Givens rotation G = [[c, s], [-conj(s), c]] (c real) with G [a; b] = [r; 0].
void givens(cd a, cd b, double &c, cd &s) {
    double aa = std::abs(a), bb = std::abs(b);
    if (bb == 0.0) { c = 1.0; s = 0.0; return; }
    if (aa == 0.0) { c = 0.0; s = std::conj(b) / bb; return; }
    double rho = std::hypot(aa, bb);
    c = aa / rho;
    s = (a / aa) * std::conj(b) / rho;
}

// rows r, r+1 of M, columns [c0, c1):  [x; y] <- G [x; y]
void rot_rows(Mat &M, int64_t r, int64_t c0, int64_t c1, double c, cd s) {
    for (int64_t k = c0; k < c1; ++k) {
        cd x = M(r, k), y = M(r + 1, k);
        M(r, k) = c * x + s * y;
        M(r + 1, k) = -std::conj(s) * x + c * y;
    }
}

// columns q, q+1 of M, rows [r0, r1):  [x, y] <- [x, y] G^*
void rot_cols(Mat &M, int64_t q, int64_t r0, int64_t r1, double c, cd s) {
    for (int64_t k = r0; k < r1; ++k) {
        cd x = M(k, q), y = M(k, q + 1);
        M(k, q) = c * x + std::conj(s) * y;
        M(k, q + 1) = -s * x + c * y;
    }
}

// eigenvalue of [[a, b], [c, d]] closest to d
cd wilkinson(cd a, cd b, cd c, cd d) {
    cd tr_half = 0.5 * (a - d);
    cd disc = std::sqrt(tr_half * tr_half + b * c);
    cd m1 = d - (b * c) / (tr_half + disc);
    cd m2 = d - (b * c) / (tr_half - disc);
    bool ok1 = std::isfinite(m1.real()) && std::isfinite(m1.imag());
    bool ok2 = std::isfinite(m2.real()) && std::isfinite(m2.imag());
    if (ok1 && ok2) return std::abs(m1 - d) <= std::abs(m2 - d) ? m1 : m2;
    if (ok1) return m1;
    if (ok2) return m2;
    return d;
}

}  // namespace

sylv_status schur_host(int64_t n, const double *A, double *Qout, double *Tout) {
    if (n < 1 || !A || !Qout || !Tout) return SYLV_ERR_INVALID_ARG;
    Mat H(n), Q(n);
    for (int64_t k = 0; k < n * n; ++k) H.v[(size_t)k] = cd(A[2 * k], A[2 * k + 1]);
    for (int64_t k = 0; k < n; ++k) Q(k, k) = 1.0;
    for (int64_t k = 0; k < n * n; ++k)
        if (!std::isfinite(H.v[(size_t)k].real()) || !std::isfinite(H.v[(size_t)k].imag()))
            return SYLV_ERR_INVALID_ARG;

    // 1. Householder reduction to Hessenberg form.
    std::vector<cd> v((size_t)n);
    for (int64_t k = 0; k + 2 < n; ++k) {
        double xnorm2 = 0.0;
        for (int64_t i = k + 1; i < n; ++i) xnorm2 += std::norm(H(i, k));
        double xnorm = std::sqrt(xnorm2);
        if (xnorm == 0.0) continue;
        cd x0 = H(k + 1, k);
        cd phase = std::abs(x0) == 0.0 ? cd(1.0, 0.0) : x0 / std::abs(x0);
        cd alpha = -phase * xnorm;                 // H x = alpha e1
        for (int64_t i = k + 1; i < n; ++i) v[(size_t)i] = H(i, k);
        v[(size_t)(k + 1)] -= alpha;
        double vnorm2 = 0.0;
        for (int64_t i = k + 1; i < n; ++i) vnorm2 += std::norm(v[(size_t)i]);
        if (vnorm2 == 0.0) continue;
        double beta = 2.0 / vnorm2;                // P = I - beta v v^*
        for (int64_t c = k; c < n; ++c) {          // H <- P H
            cd dot = 0.0;
            for (int64_t i = k + 1; i < n; ++i) dot += std::conj(v[(size_t)i]) * H(i, c);
            dot *= beta;
            for (int64_t i = k + 1; i < n; ++i) H(i, c) -= v[(size_t)i] * dot;
        }
        for (int64_t r = 0; r < n; ++r) {          // H <- H P, Q <- Q P
            cd dh = 0.0, dq = 0.0;
            for (int64_t i = k + 1; i < n; ++i) {
                dh += H(r, i) * v[(size_t)i];
                dq += Q(r, i) * v[(size_t)i];
            }
            dh *= beta;
            dq *= beta;
            for (int64_t i = k + 1; i < n; ++i) {
                H(r, i) -= dh * std::conj(v[(size_t)i]);
                Q(r, i) -= dq * std::conj(v[(size_t)i]);
            }
        }
        for (int64_t i = k + 2; i < n; ++i) H(i, k) = 0.0;
    }

    // 2. Shifted QR on the Hessenberg matrix.
    const double eps = 2.220446049250313e-16;
    double hnorm = 0.0;
    for (auto &z : H.v) hnorm = std::max(hnorm, std::abs(z));
    int64_t hi = n - 1;
    int iter = 0, total = 0;
    const int max_total = (int)(60 * n + 60);
    while (hi > 0) {
        int64_t l = hi;
        while (l > 0) {
            double s = std::abs(H(l - 1, l - 1)) + std::abs(H(l, l));
            if (s == 0.0) s = hnorm;
            if (std::abs(H(l, l - 1)) <= eps * s) { H(l, l - 1) = 0.0; break; }
            --l;
        }
        if (l == hi) { --hi; iter = 0; continue; }
        if (++total > max_total) return SYLV_ERR_SCHUR;
        ++iter;
        cd mu;
        if (iter % 10 == 0) {
            // exceptional shift to break cycles
            mu = H(hi, hi) + cd(0.75 * std::abs(H(hi, hi - 1)), 0.4375 * std::abs(H(hi, hi - 1)));
        } else {
            mu = wilkinson(H(hi - 1, hi - 1), H(hi - 1, hi), H(hi, hi - 1), H(hi, hi));
        }
        cd x = H(l, l) - mu, y = H(l + 1, l);
        for (int64_t k = l; k < hi; ++k) {
            double c;
            cd s;
            givens(x, y, c, s);
            int64_t c0 = (k > l) ? k - 1 : l;
            rot_rows(H, k, c0, n, c, s);
            int64_t r1 = std::min<int64_t>(k + 3, hi + 1);
            rot_cols(H, k, 0, r1, c, s);
            rot_cols(Q, k, 0, n, c, s);
            if (k > l) H(k + 1, k - 1) = 0.0;
            if (k + 1 < hi) { x = H(k + 1, k); y = H(k + 2, k); }
        }
    }

    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = 0; r < n; ++r) {
            cd t = (r <= c) ? H(r, c) : cd(0.0, 0.0);
            Tout[2 * (r + c * n)] = t.real();
            Tout[2 * (r + c * n) + 1] = t.imag();
            Qout[2 * (r + c * n)] = Q(r, c).real();
            Qout[2 * (r + c * n) + 1] = Q(r, c).imag();
        }
    return SYLV_OK;
}

}  // namespace sylv
