// Eigen-decomposition of a dense symmetric matrix on the host (set-up of the Matern KL, once
// per process): Householder reduction to tridiagonal form, then the implicit symmetric QR
// iteration with Wilkinson shifts (Golub & Van Loan, Matrix Computations, Algorithms 8.3.1 and
// 8.3.3). About 8 n^3 flops with the eigenvectors; both phases are backward stable.
#include <cmath>
#include <vector>

#include "internal.h"

namespace mls2mc {

namespace {

// Householder reduction A = Q T Q^T. On return d (n) and e (n-1) hold the diagonal and the
// off-diagonal of T, and qt the rows of Q^T (row-major n x n).
void tridiagonalise(int n, std::vector<double>& a, std::vector<double>& d, std::vector<double>& e,
                    std::vector<double>& qt) {
    auto A = [&](int i, int j) -> double& { return a[(size_t)i * n + j]; };
    std::vector<std::vector<double>> vs(n > 2 ? n - 2 : 0);
    std::vector<double> beta(n > 2 ? n - 2 : 0, 0.0), p(n), q(n);
    d.assign(n, 0.0);
    e.assign(n > 1 ? n - 1 : 0, 0.0);
    for (int k = 0; k + 2 < n; ++k) {
        // x = A(k+1:n, k); the reflector H = I - b v v^T maps x onto alpha e_1
        const int s = n - k - 1;
        std::vector<double>& v = vs[k];
        v.resize(s);
        double xx = 0.0;
        for (int i = 0; i < s; ++i) {
            v[i] = A(k, k + 1 + i);
            xx += v[i] * v[i];
        }
        const double xn = std::sqrt(xx);
        const double alpha = v[0] > 0.0 ? -xn : xn;
        d[k] = A(k, k);
        e[k] = alpha;
        const double vv = xx - v[0] * v[0] + (v[0] - alpha) * (v[0] - alpha);
        v[0] -= alpha;
        if (xn == 0.0 || vv == 0.0) {   // column already reduced
            e[k] = v[0] + alpha;
            beta[k] = 0.0;
            continue;
        }
        const double b = 2.0 / vv;
        beta[k] = b;
        // A22 <- H A22 H = A22 - v w^T - w v^T,  p = b A22 v,  w = p - (b/2)(p . v) v
        double pv = 0.0;
        for (int i = 0; i < s; ++i) {
            const double* row = &A(k + 1 + i, k + 1);
            double acc = 0.0;
            for (int j = 0; j < s; ++j) acc += row[j] * v[j];
            p[i] = b * acc;
            pv += p[i] * v[i];
        }
        const double kk = 0.5 * b * pv;
        for (int i = 0; i < s; ++i) q[i] = p[i] - kk * v[i];
        for (int i = 0; i < s; ++i) {
            double* row = &A(k + 1 + i, k + 1);
            const double vi = v[i], qi = q[i];
            for (int j = 0; j < s; ++j) row[j] -= vi * q[j] + qi * v[j];
        }
    }
    if (n >= 2) {
        d[n - 2] = A(n - 2, n - 2);
        e[n - 2] = A(n - 2, n - 1);
    }
    if (n >= 1) d[n - 1] = A(n - 1, n - 1);

    // Q = H_0 H_1 ... H_{n-3}, accumulated backwards (each H_k acts on indices k+1 .. n-1, where
    // the product of the later reflectors is already confined)
    std::vector<double> Q((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    std::vector<double> r(n);
    for (int k = n - 3; k >= 0; --k) {
        if (beta[k] == 0.0) continue;
        const std::vector<double>& v = vs[k];
        const int s = n - k - 1, o = k + 1;
        // rows o.. of Q: Q <- Q - b v (v^T Q), columns o.. only
        for (int j = 0; j < s; ++j) r[j] = 0.0;
        for (int i = 0; i < s; ++i) {
            const double* row = &Q[(size_t)(o + i) * n + o];
            const double vi = v[i];
            for (int j = 0; j < s; ++j) r[j] += vi * row[j];
        }
        for (int i = 0; i < s; ++i) {
            double* row = &Q[(size_t)(o + i) * n + o];
            const double f = beta[k] * v[i];
            for (int j = 0; j < s; ++j) row[j] -= f * r[j];
        }
    }
    qt.resize((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) qt[(size_t)j * n + i] = Q[(size_t)i * n + j];
}

}  // namespace

bool symmetric_eigen(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>& vt) {
    std::vector<double> d, e;
    tridiagonalise(n, a, d, e, vt);
    double tnorm = 0.0;
    for (int i = 0; i < n; ++i) tnorm = std::fmax(tnorm, std::fabs(d[i]) + (i ? std::fabs(e[i - 1]) : 0.0) +
                                                          (i + 1 < n ? std::fabs(e[i]) : 0.0));
    const double eps = 2.220446049250313e-16, floor_ = 1e-2 * eps * tnorm;
    auto negligible = [&](int i) {   // e[i] couples d[i] and d[i+1]
        return std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1])) || std::fabs(e[i]) <= floor_;
    };
    long steps = 0;
    int m = n - 1;
    while (m > 0) {
        if (negligible(m - 1)) {   // d[m] has converged
            e[m - 1] = 0.0;
            --m;
            continue;
        }
        int l = m - 1;   // the unreduced block is l .. m
        while (l > 0 && !negligible(l - 1)) --l;
        if (++steps > 30L * n) return false;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer to d[m]
        const double dl = 0.5 * (d[m - 1] - d[m]), b = e[m - 1];
        const double mu = d[m] - b * b / (dl + std::copysign(std::hypot(dl, b), dl));
        double x = d[l] - mu, z = e[l];
        for (int k = l; k < m; ++k) {
            // rotation R in the plane (k, k+1) with R [x; z] = [r; 0]; T <- R T R^T
            const double rr = std::hypot(x, z);
            const double c = rr > 0.0 ? x / rr : 1.0, s = rr > 0.0 ? z / rr : 0.0;
            if (k > l) e[k - 1] = rr;
            const double a0 = d[k], b0 = e[k], g0 = d[k + 1];
            d[k] = c * c * a0 + 2.0 * c * s * b0 + s * s * g0;
            d[k + 1] = s * s * a0 - 2.0 * c * s * b0 + c * c * g0;
            e[k] = c * s * (g0 - a0) + (c * c - s * s) * b0;
            if (k + 1 < m) {   // the bulge at (k, k+2)
                x = e[k];
                z = s * e[k + 1];
                e[k + 1] *= c;
            }
            // eigenvector rows: V^T <- R V^T
            double* r0 = &vt[(size_t)k * n];
            double* r1 = &vt[(size_t)(k + 1) * n];
            for (int j = 0; j < n; ++j) {
                const double u0 = r0[j], u1 = r1[j];
                r0[j] = c * u0 + s * u1;
                r1[j] = -s * u0 + c * u1;
            }
        }
    }
    w = d;
    return true;
}

}  // namespace mls2mc
