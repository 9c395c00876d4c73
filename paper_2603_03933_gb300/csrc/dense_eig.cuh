// Small dense symmetric eigen-solvers on the host (FP64), used by the Lanczos driver.
//
// smallest_generalized(T, G): smallest eigenpair of the pencil T y = theta G y with G
// symmetric positive definite, by Cholesky G = L L^T, C = L^{-1} T L^{-T},
// Householder reduction of C to tridiagonal form, Sturm-sequence bisection for the
// smallest eigenvalue, inverse iteration on the tridiagonal for its eigenvector, and
// back-transformation y = L^{-T} Q z.  O(k^3) for a k x k pencil.
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace lbtr {
namespace dense {

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x (Sturm count).
inline int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
    int cnt = 0;
    double q = 1.0;
    const int n = (int)d.size();
    for (int i = 0; i < n; ++i) {
        double off = i > 0 ? e[i - 1] * e[i - 1] : 0.0;
        q = d[i] - x - (i > 0 ? off / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Smallest eigenvalue of a symmetric tridiagonal matrix by bisection.
inline double tridiag_smallest(const std::vector<double>& d, const std::vector<double>& e) {
    const int n = (int)d.size();
    double lo = d[0], hi = d[0];
    for (int i = 0; i < n; ++i) {
        double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(d, e, mid) >= 1) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Eigenvector of the tridiagonal (d, e) for eigenvalue theta by inverse iteration.
inline std::vector<double> tridiag_vector(const std::vector<double>& d, const std::vector<double>& e, double theta) {
    const int n = (int)d.size();
    std::vector<double> x(n, 1.0 / std::sqrt((double)n)), y(n);
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale = std::max(scale, std::fabs(d[i]) + (i < n - 1 ? std::fabs(e[i]) : 0.0));
    const double shift = theta - 1e-13 * std::max(scale, 1e-300);
    for (int it = 0; it < 4; ++it) {
        // solve (T - shift I) y = x with Gaussian elimination and partial pivoting
        std::vector<double> a(n), b(n), c(n), f(n), rhs = x;   // sub, diag, super, second super
        for (int i = 0; i < n; ++i) {
            b[i] = d[i] - shift;
            a[i] = i > 0 ? e[i - 1] : 0.0;
            c[i] = i < n - 1 ? e[i] : 0.0;
            f[i] = 0.0;
        }
        for (int i = 0; i < n - 1; ++i) {
            if (std::fabs(a[i + 1]) > std::fabs(b[i])) {   // swap rows i and i+1
                std::swap(b[i], a[i + 1]);
                std::swap(c[i], b[i + 1]);
                std::swap(f[i], c[i + 1]);
                std::swap(rhs[i], rhs[i + 1]);
            }
            double piv = b[i] != 0.0 ? b[i] : 1e-300;
            double m = a[i + 1] / piv;
            b[i + 1] -= m * c[i];
            c[i + 1] -= m * f[i];
            rhs[i + 1] -= m * rhs[i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = rhs[i];
            if (i + 1 < n) s -= c[i] * y[i + 1];
            if (i + 2 < n) s -= f[i] * y[i + 2];
            y[i] = s / (b[i] != 0.0 ? b[i] : 1e-300);
        }
        double nrm = 0.0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        for (int i = 0; i < n; ++i) x[i] = y[i] / nrm;
    }
    return x;
}

// Smallest eigenpair of (T, G); T, G row-major k x k.  Returns false if G is not SPD.
inline bool smallest_generalized(int k, const std::vector<double>& Tm, const std::vector<double>& G,
                                 double& theta, std::vector<double>& yout) {
    // Cholesky G = L L^T
    std::vector<double> L(k * k, 0.0);
    for (int j = 0; j < k; ++j) {
        double s = G[j * k + j];
        for (int p = 0; p < j; ++p) s -= L[j * k + p] * L[j * k + p];
        if (!(s > 0.0)) return false;
        L[j * k + j] = std::sqrt(s);
        for (int i = j + 1; i < k; ++i) {
            double t = G[i * k + j];
            for (int p = 0; p < j; ++p) t -= L[i * k + p] * L[j * k + p];
            L[i * k + j] = t / L[j * k + j];
        }
    }
    // W = L^{-1} T (forward substitution on columns), C = W L^{-T} = L^{-1} (L^{-1} T)^T
    std::vector<double> W(k * k), C(k * k);
    for (int col = 0; col < k; ++col)
        for (int i = 0; i < k; ++i) {
            double s = Tm[i * k + col];
            for (int p = 0; p < i; ++p) s -= L[i * k + p] * W[p * k + col];
            W[i * k + col] = s / L[i * k + i];
        }
    // C = L^{-1} W^T, then symmetrise
    for (int col = 0; col < k; ++col)
        for (int i = 0; i < k; ++i) {
            double s = W[col * k + i];
            for (int p = 0; p < i; ++p) s -= L[i * k + p] * C[p * k + col];
            C[i * k + col] = s / L[i * k + i];
        }
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j) {
            double a = 0.5 * (C[i * k + j] + C[j * k + i]);
            C[i * k + j] = C[j * k + i] = a;
        }
    // Householder tridiagonalisation: C = Q Tri Q^T, reflectors kept in V
    std::vector<std::vector<double>> V;
    std::vector<double> p(k), q(k);
    for (int i = 0; i + 2 < k; ++i) {
        const int m = k - i - 1;
        std::vector<double> v(m);
        double alpha = 0.0;
        for (int r = 0; r < m; ++r) { v[r] = C[(i + 1 + r) * k + i]; alpha += v[r] * v[r]; }
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) { V.push_back(std::vector<double>()); continue; }
        if (v[0] > 0) alpha = -alpha;
        v[0] -= alpha;
        double vn = 0.0;
        for (double t : v) vn += t * t;
        vn = std::sqrt(vn);
        if (vn == 0.0) { V.push_back(std::vector<double>()); continue; }
        for (double& t : v) t /= vn;
        // A' = H A H on the trailing block rows/cols i+1.. (and column/row i)
        // p = 2 A v over the sub-block (rows i.., cols i+1..)
        for (int r = i; r < k; ++r) {
            double s = 0.0;
            for (int c2 = 0; c2 < m; ++c2) s += C[r * k + (i + 1 + c2)] * v[c2];
            p[r] = 2.0 * s;
        }
        double K = 0.0;
        for (int c2 = 0; c2 < m; ++c2) K += v[c2] * p[i + 1 + c2];
        for (int r = i; r < k; ++r) q[r] = p[r] - (r > i ? K * v[r - i - 1] : 0.0);
        for (int r = i; r < k; ++r)
            for (int c2 = i; c2 < k; ++c2) {
                double vr = r > i ? v[r - i - 1] : 0.0, vc = c2 > i ? v[c2 - i - 1] : 0.0;
                C[r * k + c2] -= vr * q[c2] + q[r] * vc;
            }
        V.push_back(v);
    }
    std::vector<double> d(k), e(k > 1 ? k - 1 : 1, 0.0);
    for (int i = 0; i < k; ++i) d[i] = C[i * k + i];
    for (int i = 0; i + 1 < k; ++i) e[i] = 0.5 * (C[(i + 1) * k + i] + C[i * k + i + 1]);
    if (k == 1) { theta = d[0]; yout.assign(1, 1.0 / L[0]); return true; }
    theta = tridiag_smallest(d, e);
    std::vector<double> z = tridiag_vector(d, e, theta);
    // back-transform z <- H_0 H_1 ... z (apply reflectors in reverse order)
    for (int i = (int)V.size() - 1; i >= 0; --i) {
        const std::vector<double>& v = V[i];
        if (v.empty()) continue;
        double s = 0.0;
        for (size_t r = 0; r < v.size(); ++r) s += v[r] * z[i + 1 + r];
        for (size_t r = 0; r < v.size(); ++r) z[i + 1 + r] -= 2.0 * s * v[r];
    }
    // y = L^{-T} z
    yout.assign(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
        double s = z[i];
        for (int p2 = i + 1; p2 < k; ++p2) s -= L[p2 * k + i] * yout[p2];
        yout[i] = s / L[i * k + i];
    }
    return true;
}

}  // namespace dense
}  // namespace lbtr
