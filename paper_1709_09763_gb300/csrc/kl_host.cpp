// KL table of the prior log-diffusion field (host set-up, runs once per handle).
//
// Sec. 5, Eq. truncKL: u(x) = sum_k sqrt(lambda_k) phi_k(x) theta_k with theta_k
// standard normal and m0 = 0. The covariance is the separable exponential
// sigma^2 exp(-|x1-y1|/lc) exp(-|x2-y2|/lc); its 1-D eigenpairs on [0,1] solve,
// with a = 1/2, c = 1/lc and x = omega*a,
//   even (cos) modes: omega*tan(omega a) = c,   odd (sin) modes: omega + c*tan(omega a) = 0,
//   lambda = 2c / (omega^2 + c^2),
// and mode m has x in (m pi/2, (m+1) pi/2). 2-D modes are products phi_m(x1) phi_n(x2)
// with eigenvalue sigma^2 lambda_m lambda_n, ordered by eigenvalue descending, ties
// (the symmetric pairs (m,n), (n,m)) broken by smaller max(m,n), then smaller m.
// The field is evaluated at triangle centroids.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace mls2mc {

namespace {

// g(x) whose root in (lo, hi) gives mode m; both forms are the tan-equations
// multiplied through by cos(x), so g is smooth on the bracket.
double mode_eq(int m, double x, double a, double c) {
    if ((m & 1) == 0) return (x / a) * std::sin(x) - c * std::cos(x);
    return (x / a) * std::cos(x) + c * std::sin(x);
}

double find_root(int m, double a, double c) {
    const double pi = 3.14159265358979323846;
    double lo = m * pi / 2.0, hi = (m + 1) * pi / 2.0;
    double glo = mode_eq(m, lo, a, c);
    // bisection to a tight bracket, then secant polishing inside it
    for (int it = 0; it < 200 && (hi - lo) > 4e-16 * hi; ++it) {
        double mid = 0.5 * (lo + hi);
        double gm = mode_eq(m, mid, a, c);
        if (gm == 0.0) return mid;
        if ((gm < 0) == (glo < 0)) { lo = mid; glo = gm; } else { hi = mid; }
    }
    return 0.5 * (lo + hi);
}

}  // namespace

void kl_eig_1d(double corr_len, int n_modes, std::vector<double>& lam,
               std::vector<double>& omega) {
    const double a = 0.5, c = 1.0 / corr_len;
    lam.resize(n_modes);
    omega.resize(n_modes);
    for (int m = 0; m < n_modes; ++m) {
        double w = find_root(m, a, c) / a;
        omega[m] = w;
        lam[m] = 2.0 * c / (w * w + c * c);
    }
}

static double phi_1d(int m, double w, double s) {
    const double a = 0.5;
    if ((m & 1) == 0) return std::cos(w * (s - 0.5)) / std::sqrt(a + std::sin(2.0 * w * a) / (2.0 * w));
    return std::sin(w * (s - 0.5)) / std::sqrt(a - std::sin(2.0 * w * a) / (2.0 * w));
}

void kl_table(int N, double corr_len, double variance, int K, std::vector<double>& psi,
              std::vector<double>& lambda) {
    std::vector<double> lam1, om1;
    kl_eig_1d(corr_len, K, lam1, om1);
    struct Pair { double lam; int m, n; };
    std::vector<Pair> pairs;
    pairs.reserve((size_t)K * K);
    for (int m = 0; m < K; ++m)
        for (int n = 0; n < K; ++n) pairs.push_back({variance * (lam1[m] * lam1[n]), m, n});
    std::stable_sort(pairs.begin(), pairs.end(), [](const Pair& p, const Pair& q) {
        if (p.lam != q.lam) return p.lam > q.lam;
        int mp = std::max(p.m, p.n), mq = std::max(q.m, q.n);
        if (mp != mq) return mp < mq;
        return p.m < q.m;
    });
    const int E = 2 * N * N;
    const double h = 1.0 / N;
    psi.assign((size_t)K * E, 0.0);
    lambda.resize(K);
    // 1-D eigenfunction values at the centroid coordinates (i + 1/3) h and (i + 2/3) h
    std::vector<double> f13((size_t)K * N), f23((size_t)K * N);
    for (int m = 0; m < K; ++m)
        for (int i = 0; i < N; ++i) {
            f13[(size_t)m * N + i] = phi_1d(m, om1[m], (i + 1.0 / 3.0) * h);
            f23[(size_t)m * N + i] = phi_1d(m, om1[m], (i + 2.0 / 3.0) * h);
        }
    for (int k = 0; k < K; ++k) {
        const Pair& p = pairs[k];
        lambda[k] = p.lam;
        const double s = std::sqrt(p.lam);
        double* row = psi.data() + (size_t)k * E;
        for (int j = 0; j < N; ++j)
            for (int i = 0; i < N; ++i) {
                const size_t e = 2 * ((size_t)j * N + i);
                // lower triangle centroid ((i+2/3)h, (j+1/3)h), upper ((i+1/3)h, (j+2/3)h)
                row[e] = s * f23[(size_t)p.m * N + i] * f13[(size_t)p.n * N + j];
                row[e + 1] = s * f13[(size_t)p.m * N + i] * f23[(size_t)p.n * N + j];
            }
    }
}

void obs_table(int N, int n_obs, const double* xy, std::vector<int>& idx, std::vector<double>& wts) {
    // P1 interpolation: locate the cell, then the triangle (lower when dx >= dy),
    // then barycentric weights of its three vertices (node index j * fem_row_stride(N) + i).
    const double h = 1.0 / N;
    idx.resize((size_t)n_obs * 3);
    wts.resize((size_t)n_obs * 3);
    for (int r = 0; r < n_obs; ++r) {
        const double x = xy[2 * r], y = xy[2 * r + 1];
        int i = (int)std::floor(x / h), j = (int)std::floor(y / h);
        i = std::min(std::max(i, 0), N - 1);
        j = std::min(std::max(j, 0), N - 1);
        const double dx = x / h - i, dy = y / h - j;   // local coordinates in [0,1]^2
        const int SR = fem_row_stride(N);
        const int v00 = j * SR + i, v10 = v00 + 1, v01 = v00 + SR, v11 = v01 + 1;
        if (dx >= dy) {  // lower triangle (0,0),(1,0),(1,1): weights 1-dx, dx-dy, dy
            idx[3 * r] = v00; wts[3 * r] = 1.0 - dx;
            idx[3 * r + 1] = v10; wts[3 * r + 1] = dx - dy;
            idx[3 * r + 2] = v11; wts[3 * r + 2] = dy;
        } else {         // upper triangle (0,0),(1,1),(0,1): weights 1-dy, dx, dy-dx
            idx[3 * r] = v00; wts[3 * r] = 1.0 - dy;
            idx[3 * r + 1] = v11; wts[3 * r + 1] = dx;
            idx[3 * r + 2] = v01; wts[3 * r + 2] = dy - dx;
        }
    }
}

}  // namespace mls2mc
