// Matern prior (smoothness 3/2) KL table and the nine-source load vector of Sec. 5 (host
// set-up, once per handle; the eigen-decomposition once per process and correlation length).
//
// Covariance (Minasny & McBratney 2005, the parametrisation cited in Sec. 5):
//   C(r) = sigma^2 (1 + z) exp(-z),  z = sqrt(6) r / lc,
// with which N_sto = 10 terms at lc = 0.65 carry the 94.5 % of the variance stated for
// Example 5.1. KL pairs by the Nystrom method on the midpoint rule of a 32 x 32 cell grid
// (weight w = 1/32^2): W C u = lambda u, extended to any point by
//   phi(x) = (1/lambda) sum_q w C(x, q) u(q).
// The grid and C are invariant under x -> 1-x (Sx), y -> 1-y (Sy) and x <-> y (R). Every
// eigenvector has a definite parity (sx, sy) under (Sx, Sy); each parity sector is solved on
// the quarter grid (x, y < 1/2) with the kernel folded over the four mirror images,
//   A_s(p, q) = w [C(p, q) + sx C(p, Sx q) + sy C(p, Sy q) + sx sy C(p, Sx Sy q)].
// R maps sector (+,-) onto (-,+): their eigenvalues coincide, and the (-,+) eigenvectors are
// taken as the mirror images of the (+,-) ones. Order: eigenvalue descending; eigenvalues
// within a relative 1e-9 count as equal and are ordered by sector (+,+), (+,-), (-,+), (-,-).
// Sign: sum over the full grid of w u g > 0 with g(x, y) = exp(0.7 x + 1.3 y), except for
// (-,+) members, which carry the sign of their mirror partner.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

namespace mls2mc {

namespace {

constexpr int kM = 32;            // quadrature cells per side
constexpr int kH = kM / 2;        // quarter grid side
constexpr int kQ = kH * kH;       // quarter grid points
constexpr double kW = 1.0 / (kM * kM);

double matern32(double r, double lc, double var) {
    const double z = std::sqrt(6.0) * r / lc;
    return var * (1.0 + z) * std::exp(-z);
}

double qcoord(int i) { return (i + 0.5) / kM; }   // quarter-grid index i (x or y) -> coordinate

// kernel at p summed over the four mirror images of q with the parity signs of sector (sx, sy)
double folded(double px, double py, double qx, double qy, int sx, int sy, double lc, double var) {
    const double c1 = matern32(std::hypot(px - qx, py - qy), lc, var);
    const double c2 = matern32(std::hypot(px - (1.0 - qx), py - qy), lc, var);
    const double c3 = matern32(std::hypot(px - qx, py - (1.0 - qy)), lc, var);
    const double c4 = matern32(std::hypot(px - (1.0 - qx), py - (1.0 - qy)), lc, var);
    return c1 + sx * c2 + sy * c3 + sx * sy * c4;
}

// Eigen-decomposition of a symmetric n x n matrix a (row-major, overwritten) by the cyclic
// Jacobi method (Golub & Van Loan, Sec. 8.5): each rotation J(p, q) zeroes a_pq; sweeps until the
// off-diagonal mass is below (1e-15)^2 of the diagonal's. Eigenvalues to w, eigenvectors to the
// columns of v.
void jacobi_eigen(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>& v) {
    v.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            diag += a[(size_t)p * n + p] * a[(size_t)p * n + p];
            for (int q = p + 1; q < n; ++q) off += a[(size_t)p * n + q] * a[(size_t)p * n + q];
        }
        if (off <= 1e-30 * diag) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double tau = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
                const double t = tau >= 0.0 ? 1.0 / (tau + std::sqrt(1.0 + tau * tau))
                                            : -1.0 / (-tau + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {   // columns p, q: A J
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // rows p, q: J^T A
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                a[(size_t)p * n + q] = a[(size_t)q * n + p] = 0.0;
                for (int k = 0; k < n; ++k) {   // V J
                    const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
                    v[(size_t)k * n + p] = c * vkp - s * vkq;
                    v[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
}

struct Mode {
    double lam;
    int sector;                // 0 (+,+), 1 (+,-), 2 (-,+), 3 (-,-)
    int sx, sy;
    std::vector<double> u;     // quarter-grid values, full-grid normalisation sum w u^2 = 1
};

std::vector<Mode> compute_modes(double lc, double var) {
    static const int SX[4] = {1, 1, -1, -1}, SY[4] = {1, -1, 1, -1};
    std::vector<Mode> all;
    for (int sec : {0, 1, 3}) {
        const int sx = SX[sec], sy = SY[sec];
        std::vector<double> A((size_t)kQ * kQ);
        for (int p = 0; p < kQ; ++p)
            for (int q = 0; q < kQ; ++q)
                A[(size_t)p * kQ + q] = kW * folded(qcoord(p / kH), qcoord(p % kH), qcoord(q / kH), qcoord(q % kH),
                                                    sx, sy, lc, var);
        std::vector<double> w, V;
        jacobi_eigen(kQ, A, w, V);
        for (int k = 0; k < kQ; ++k) {
            Mode m{w[k], sec, sx, sy, std::vector<double>(kQ)};
            const double scale = 1.0 / std::sqrt(4.0 * kW);
            double sg = 0.0;
            for (int q = 0; q < kQ; ++q) {
                m.u[q] = V[(size_t)q * kQ + k] * scale;
                const double x = qcoord(q / kH), y = qcoord(q % kH);
                const double g = std::exp(0.7 * x + 1.3 * y) + sx * std::exp(0.7 * (1.0 - x) + 1.3 * y) +
                                 sy * std::exp(0.7 * x + 1.3 * (1.0 - y)) +
                                 sx * sy * std::exp(0.7 * (1.0 - x) + 1.3 * (1.0 - y));
                sg += kW * m.u[q] * g;
            }
            if (sg < 0.0)
                for (double& x : m.u) x = -x;
            if (sec == 1) {   // its mirror image x <-> y, in sector (-,+)
                Mode r{m.lam, 2, -1, 1, std::vector<double>(kQ)};
                for (int ix = 0; ix < kH; ++ix)
                    for (int iy = 0; iy < kH; ++iy) r.u[ix * kH + iy] = m.u[iy * kH + ix];
                all.push_back(std::move(m));
                all.push_back(std::move(r));
            } else {
                all.push_back(std::move(m));
            }
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const Mode& a, const Mode& b) { return a.lam > b.lam; });
    for (size_t i = 0; i < all.size();) {
        size_t j = i;
        while (j + 1 < all.size() && all[i].lam - all[j + 1].lam <= 1e-9 * all[i].lam) ++j;
        std::stable_sort(all.begin() + i, all.begin() + j + 1,
                         [](const Mode& a, const Mode& b) { return a.sector < b.sector; });
        i = j + 1;
    }
    return all;
}

// the ordered modes of (lc, variance), computed once per process
const std::vector<Mode>& modes(double lc, double var) {
    static std::mutex mu;
    static std::map<std::pair<double, double>, std::vector<Mode>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(lc, var);
    auto it = cache.find(key);
    if (it == cache.end()) it = cache.emplace(key, compute_modes(lc, var)).first;
    return it->second;
}

double nine_sources(double x, double y) {
    const double var = 0.001, norm = 1.0 / std::sqrt(2.0 * 3.14159265358979323846 * var);
    double gx = 0.0, gy = 0.0;
    for (int n = 1; n <= 3; ++n) {
        gx += norm * std::exp(-(x - 0.25 * n) * (x - 0.25 * n) / (2.0 * var));
        gy += norm * std::exp(-(y - 0.25 * n) * (y - 0.25 * n) / (2.0 * var));
    }
    return gx * gy;
}

}  // namespace

int matern_max_terms() { return 64; }

void matern_kl_table(int N, double corr_len, double variance, int K, std::vector<double>& psi,
                     std::vector<double>& lambda) {
    const std::vector<Mode>& ms = modes(corr_len, variance);
    const int E = 2 * N * N;
    const double h = 1.0 / N;
    psi.assign((size_t)K * E, 0.0);
    lambda.resize(K);
    for (int k = 0; k < K; ++k) lambda[k] = ms[k].lam;
    std::vector<double> acc(K);
    for (int e = 0; e < E; ++e) {
        const int cell = e / 2, i = cell % N, j = cell / N;
        // lower triangle centroid ((i+2/3)h, (j+1/3)h), upper ((i+1/3)h, (j+2/3)h)
        const double x = (e & 1) ? (i + 1.0 / 3.0) * h : (i + 2.0 / 3.0) * h;
        const double y = (e & 1) ? (j + 2.0 / 3.0) * h : (j + 1.0 / 3.0) * h;
        std::fill(acc.begin(), acc.end(), 0.0);
        for (int q = 0; q < kQ; ++q) {
            const double qx = qcoord(q / kH), qy = qcoord(q % kH);
            const double c1 = matern32(std::hypot(x - qx, y - qy), corr_len, variance);
            const double c2 = matern32(std::hypot(x - (1.0 - qx), y - qy), corr_len, variance);
            const double c3 = matern32(std::hypot(x - qx, y - (1.0 - qy)), corr_len, variance);
            const double c4 = matern32(std::hypot(x - (1.0 - qx), y - (1.0 - qy)), corr_len, variance);
            for (int k = 0; k < K; ++k) {
                const Mode& m = ms[k];
                acc[k] += (c1 + m.sx * c2 + m.sy * c3 + m.sx * m.sy * c4) * m.u[q];
            }
        }
        for (int k = 0; k < K; ++k)   // sqrt(lambda) phi = sqrt(lambda) (1/lambda) sum w C u
            psi[(size_t)k * E + e] = kW * acc[k] / std::sqrt(ms[k].lam);
    }
}

void nine_source_load(int N, std::vector<double>& b, double& bnorm2) {
    const int S = fem_row_stride(N);
    const double h = 1.0 / N, area = 0.5 * h * h;
    b.assign((size_t)(N + 1) * S, 0.0);
    auto node = [&](int i, int j) { return (size_t)j * S + i; };
    for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
            // lower (i,j),(i+1,j),(i+1,j+1) and upper (i,j),(i+1,j+1),(i,j+1): each vertex takes
            // area/3 times the mean of f at the midpoints of its two edges (phi_a = 1/2 there)
            const int tri[2][3][2] = {{{i, j}, {i + 1, j}, {i + 1, j + 1}}, {{i, j}, {i + 1, j + 1}, {i, j + 1}}};
            for (const auto& t : tri) {
                double fm[3];   // midpoints of the edges (0,1), (1,2), (2,0)
                for (int a = 0; a < 3; ++a) {
                    const int c = (a + 1) % 3;
                    fm[a] = nine_sources(0.5 * (t[a][0] + t[c][0]) * h, 0.5 * (t[a][1] + t[c][1]) * h);
                }
                b[node(t[0][0], t[0][1])] += area / 3.0 * 0.5 * (fm[0] + fm[2]);
                b[node(t[1][0], t[1][1])] += area / 3.0 * 0.5 * (fm[0] + fm[1]);
                b[node(t[2][0], t[2][1])] += area / 3.0 * 0.5 * (fm[1] + fm[2]);
            }
        }
    bnorm2 = 0.0;
    for (int j = 0; j <= N; ++j)
        for (int i = 0; i <= S - 1; ++i) {
            double& v = b[node(i, j)];
            if (i == 0 || j == 0 || i >= N || j == N) v = 0.0;   // Dirichlet nodes and padding
            else bnorm2 += v * v;
        }
}

}  // namespace mls2mc
