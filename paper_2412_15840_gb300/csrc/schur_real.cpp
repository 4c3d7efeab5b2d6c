// Host real Schur decomposition A = Q T Q^T of a real matrix (the setup step of
// Section 2 in real arithmetic): Q orthogonal, T quasi-upper-triangular with
// 1 x 1 blocks (real eigenvalues) and 2 x 2 blocks (complex-conjugate pairs).
//
// Method (textbook; Golub & Van Loan, "Matrix Computations", ch. 7):
//   1. Householder reduction to upper Hessenberg form.
//   2. Francis double-shift QR steps (3 x 3 Householder bulge chasing) on the
//      active window, shifts from the trailing 2 x 2 block, exceptional shifts
//      after 10 stalled steps, deflation when a subdiagonal entry falls below
//      eps times its neighbouring diagonal entries.  A deflated 2 x 2 block with
//      real eigenvalues is split by a rotation onto one of its eigenvectors.
//   3. Reordering so that every 2 x 2 block starts at an even index: a block at
//      an odd index k is preceded by a 1 x 1 block, and the two are swapped by
//      the direct method of Bai & Demmel (1993): with a = T[k-1, k-1] and B the
//      2 x 2 block, X solves a X - X B = T[k-1, k:k+2], the columns of [-X; I]
//      span the invariant subspace of B's eigenvalues, and the orthogonal
//      factor of their QR decomposition moves B ahead of a.
// Blocks at even offsets let a tiling with even block extents keep every
// coupled pair inside one tile.  Matrices are column-major.
#include "sylv_internal.h"

#include <cmath>
#include <vector>

namespace sylv {

namespace {

struct RMat {
    int64_t n;
    std::vector<double> v;
    explicit RMat(int64_t n_) : n(n_), v((size_t)(n_ * n_), 0.0) {}
    double &operator()(int64_t r, int64_t c) { return v[(size_t)(r + c * n)]; }
    double operator()(int64_t r, int64_t c) const { return v[(size_t)(r + c * n)]; }
};

// Householder vector of x (length m <= 3): (I - tau v v^T) x = beta e_1, v[0] = 1
void house(const double *x, int m, double *v, double &tau) {
    double sig = 0.0;
    for (int i = 1; i < m; ++i) sig += x[i] * x[i];
    v[0] = 1.0;
    for (int i = 1; i < m; ++i) v[i] = x[i];
    if (sig == 0.0) { tau = 0.0; return; }
    const double mu = std::sqrt(x[0] * x[0] + sig);
    const double v0 = x[0] <= 0.0 ? x[0] - mu : -sig / (x[0] + mu);
    tau = 2.0 * v0 * v0 / (sig + v0 * v0);
    for (int i = 1; i < m; ++i) v[i] /= v0;
}

// rows r0 .. r0+m-1 of M, columns [c0, c1): (I - tau v v^T) applied from the left
void refl_rows(RMat &M, int64_t r0, int m, int64_t c0, int64_t c1, const double *v, double tau) {
    if (tau == 0.0) return;
    for (int64_t c = c0; c < c1; ++c) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += v[i] * M(r0 + i, c);
        s *= tau;
        for (int i = 0; i < m; ++i) M(r0 + i, c) -= s * v[i];
    }
}

// columns c0 .. c0+m-1 of M, rows [r0, r1): applied from the right
void refl_cols(RMat &M, int64_t c0, int m, int64_t r0, int64_t r1, const double *v, double tau) {
    if (tau == 0.0) return;
    for (int64_t r = r0; r < r1; ++r) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += M(r, c0 + i) * v[i];
        s *= tau;
        for (int i = 0; i < m; ++i) M(r, c0 + i) -= s * v[i];
    }
}

// plane rotation [c s; -s c] on rows k, k+1 (left) and columns k, k+1 (right)
void rot_both(RMat &H, RMat &Q, int64_t k, double c, double s) {
    const int64_t n = H.n;
    for (int64_t j = 0; j < n; ++j) {
        const double x = H(k, j), y = H(k + 1, j);
        H(k, j) = c * x + s * y;
        H(k + 1, j) = -s * x + c * y;
    }
    for (int64_t i = 0; i < n; ++i) {
        const double x = H(i, k), y = H(i, k + 1);
        H(i, k) = c * x + s * y;
        H(i, k + 1) = -s * x + c * y;
        const double qx = Q(i, k), qy = Q(i, k + 1);
        Q(i, k) = c * qx + s * qy;
        Q(i, k + 1) = -s * qx + c * qy;
    }
}

// a deflated 2 x 2 block at (k, k): if its eigenvalues are real, rotate onto an
// eigenvector so that the block becomes upper triangular (two 1 x 1 blocks)
void split_2x2(RMat &H, RMat &Q, int64_t k) {
    const double a = H(k, k), b = H(k, k + 1), c = H(k + 1, k), d = H(k + 1, k + 1);
    const double p = 0.5 * (a - d);
    const double disc = p * p + b * c;
    if (disc < 0.0) return;                       // complex pair: keep the block
    const double r = std::sqrt(disc);
    const double lam = 0.5 * (a + d) + (p >= 0.0 ? r : -r);
    // eigenvector of lam: (b, lam - a) or (lam - d, c), the larger one
    double x = b, y = lam - a;
    const double x2 = lam - d, y2 = c;
    if (std::hypot(x2, y2) > std::hypot(x, y)) { x = x2; y = y2; }
    const double h = std::hypot(x, y);
    if (h == 0.0) return;
    rot_both(H, Q, k, x / h, y / h);
    H(k + 1, k) = 0.0;
}

// swap the 1 x 1 block at k - 1 with the 2 x 2 block at k (direct method)
bool swap_1_2(RMat &T, RMat &Q, int64_t k) {
    const int64_t n = T.n;
    const int64_t k0 = k - 1;
    const double a = T(k0, k0);
    const double b11 = T(k, k), b12 = T(k, k + 1), b21 = T(k + 1, k), b22 = T(k + 1, k + 1);
    // X (a I - B) = t, X a row of 2
    const double m11 = a - b11, m12 = -b12, m21 = -b21, m22 = a - b22;
    const double det = m11 * m22 - m12 * m21;
    if (det == 0.0 || !std::isfinite(det)) return false;
    const double t1 = T(k0, k), t2 = T(k0, k + 1);
    // [x1 x2] [m11 m12; m21 m22] = [t1 t2]
    const double x1 = (t1 * m22 - t2 * m21) / det;
    const double x2 = (t2 * m11 - t1 * m12) / det;
    // QR of M = [-x1 -x2; 1 0; 0 1] by two reflections
    double col1[3] = {-x1, 1.0, 0.0}, col2[3] = {-x2, 0.0, 1.0};
    double v1[3], tau1, v2[3], tau2;
    house(col1, 3, v1, tau1);
    {   // apply H1 to col2
        double s = tau1 * (v1[0] * col2[0] + v1[1] * col2[1] + v1[2] * col2[2]);
        for (int i = 0; i < 3; ++i) col2[i] -= s * v1[i];
    }
    house(col2 + 1, 2, v2, tau2);
    // T <- Q^T T Q on the 3 x 3 window (rows k0..k0+2 from column k0, columns
    // k0..k0+2 for rows 0..k0+2), Q <- Q Qs with Qs = H1 H2 (H2 acting on 1..2)
    refl_rows(T, k0, 3, k0, n, v1, tau1);
    refl_rows(T, k0 + 1, 2, k0, n, v2, tau2);
    refl_cols(T, k0, 3, 0, n, v1, tau1);
    refl_cols(T, k0 + 1, 2, 0, n, v2, tau2);
    refl_cols(Q, k0, 3, 0, n, v1, tau1);
    refl_cols(Q, k0 + 1, 2, 0, n, v2, tau2);
    // the moved 2 x 2 block now leads; the entries below it are rounding
    const double scale = std::fabs(a) + std::fabs(b11) + std::fabs(b22) + std::fabs(b12) +
                         std::fabs(b21);
    const double below = std::fabs(T(k0 + 2, k0)) + std::fabs(T(k0 + 2, k0 + 1));
    if (!(below <= 1e-10 * scale)) return false;
    T(k0 + 2, k0) = 0.0;
    T(k0 + 2, k0 + 1) = 0.0;
    return true;
}

}  // namespace

sylv_status schur_real_host(int64_t n, const double *A, double *Qout, double *Tout) {
    if (n < 1) return SYLV_ERR_INVALID_ARG;
    RMat H(n), Q(n);
    for (int64_t i = 0; i < n * n; ++i) {
        if (!std::isfinite(A[i])) return SYLV_ERR_INVALID_ARG;
        H.v[(size_t)i] = A[i];
    }
    for (int64_t i = 0; i < n; ++i) Q(i, i) = 1.0;

    // 1. Hessenberg reduction
    std::vector<double> x((size_t)n), v((size_t)n);
    for (int64_t k = 0; k + 2 < n; ++k) {
        const int64_t m = n - k - 1;
        double sig = 0.0;
        for (int64_t i = 1; i < m; ++i) sig += H(k + 1 + i, k) * H(k + 1 + i, k);
        if (sig == 0.0) continue;
        const double x0 = H(k + 1, k);
        const double mu = std::sqrt(x0 * x0 + sig);
        const double v0 = x0 <= 0.0 ? x0 - mu : -sig / (x0 + mu);
        const double tau = 2.0 * v0 * v0 / (sig + v0 * v0);
        v[0] = 1.0;
        for (int64_t i = 1; i < m; ++i) v[(size_t)i] = H(k + 1 + i, k) / v0;
        for (int64_t c = k; c < n; ++c) {
            double s = 0.0;
            for (int64_t i = 0; i < m; ++i) s += v[(size_t)i] * H(k + 1 + i, c);
            s *= tau;
            for (int64_t i = 0; i < m; ++i) H(k + 1 + i, c) -= s * v[(size_t)i];
        }
        for (int64_t r = 0; r < n; ++r) {
            double s = 0.0, sq = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                s += H(r, k + 1 + i) * v[(size_t)i];
                sq += Q(r, k + 1 + i) * v[(size_t)i];
            }
            s *= tau;
            sq *= tau;
            for (int64_t i = 0; i < m; ++i) {
                H(r, k + 1 + i) -= s * v[(size_t)i];
                Q(r, k + 1 + i) -= sq * v[(size_t)i];
            }
        }
        for (int64_t i = k + 2; i < n; ++i) H(i, k) = 0.0;
    }

    // 2. Francis double-shift QR
    const double eps = 2.220446049250313e-16;
    int64_t hi = n - 1;
    int stall = 0;
    int64_t steps = 0;
    while (hi >= 0) {
        int64_t l = hi;
        while (l > 0) {
            const double s = std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l));
            if (std::fabs(H(l, l - 1)) <= eps * (s == 0.0 ? 1.0 : s)) break;
            --l;
        }
        if (l > 0) H(l, l - 1) = 0.0;
        if (l == hi) { --hi; stall = 0; continue; }
        if (l == hi - 1) { split_2x2(H, Q, hi - 1); hi -= 2; stall = 0; continue; }
        if (++steps > 60 * n) return SYLV_ERR_SCHUR;
        double s, t;
        if (++stall % 11 == 10) {
            const double w = std::fabs(H(hi, hi - 1)) + std::fabs(H(hi - 1, hi - 2));
            s = 1.5 * w;
            t = w * w;
        } else {
            s = H(hi - 1, hi - 1) + H(hi, hi);
            t = H(hi - 1, hi - 1) * H(hi, hi) - H(hi - 1, hi) * H(hi, hi - 1);
        }
        double xv[3];
        xv[0] = H(l, l) * H(l, l) + H(l, l + 1) * H(l + 1, l) - s * H(l, l) + t;
        xv[1] = H(l + 1, l) * (H(l, l) + H(l + 1, l + 1) - s);
        xv[2] = H(l + 1, l) * H(l + 2, l + 1);
        for (int64_t k = l; k + 2 <= hi; ++k) {
            double vv[3], tau;
            house(xv, 3, vv, tau);
            const int64_t q = k > l ? k - 1 : l;
            refl_rows(H, k, 3, q, n, vv, tau);
            const int64_t r = std::min<int64_t>(k + 3, hi);
            refl_cols(H, k, 3, 0, r + 1, vv, tau);
            refl_cols(Q, k, 3, 0, n, vv, tau);
            xv[0] = H(k + 1, k);
            xv[1] = H(k + 2, k);
            if (k + 3 <= hi) xv[2] = H(k + 3, k);
            if (k > l) { H(k + 1, k - 1) = 0.0; H(k + 2, k - 1) = 0.0; }
        }
        {
            double vv[2], tau;
            house(xv, 2, vv, tau);
            refl_rows(H, hi - 1, 2, hi - 2, n, vv, tau);
            refl_cols(H, hi - 1, 2, 0, hi + 1, vv, tau);
            refl_cols(Q, hi - 1, 2, 0, n, vv, tau);
            H(hi, hi - 2) = 0.0;
        }
    }
    // clean the entries below the first subdiagonal
    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = c + 2; r < n; ++r) H(r, c) = 0.0;

    // 3. move every 2 x 2 block to an even offset
    for (int64_t k = 0; k + 1 < n;) {
        if (H(k + 1, k) == 0.0) { ++k; continue; }
        if (k % 2 == 1) {
            if (!swap_1_2(H, Q, k)) return SYLV_ERR_SCHUR;
            k += 1;          // the block now starts at k - 1 (even); next after it
        } else {
            k += 2;
        }
    }
    for (int64_t c = 0; c < n; ++c)
        for (int64_t r = c + 1; r < n; ++r)
            if (!(r == c + 1 && c % 2 == 0)) H(r, c) = 0.0;
    for (int64_t i = 0; i < n * n; ++i) {
        Qout[i] = Q.v[(size_t)i];
        Tout[i] = H.v[(size_t)i];
    }
    return SYLV_OK;
}

}  // namespace sylv

extern "C" sylv_status sylv_schur_real(int64_t n, const double *A, double *Q, double *T) {
    if (!A || !Q || !T) return SYLV_ERR_INVALID_ARG;
    return sylv::schur_real_host(n, A, Q, T);
}
