// Matern prior (smoothness 3/2) KL table and the nine-source load vector of Sec. 5 (host
// set-up, once per handle; the eigen-decomposition once per process, correlation length and
// grid).
//
// Covariance (Minasny & McBratney 2005, the parametrisation cited in Sec. 5):
//   C(r) = sigma^2 (1 + z) exp(-z),  z = sqrt(6) r / lc,
// with which N_sto = 10 terms at lc = 0.65 carry the 94.5 % of the variance stated for
// Example 5.1, and 320 terms at lc = 0.1 the 95 % stated for Example 5.3. KL pairs by the
// Nystrom method on the midpoint rule of an M x M cell grid (weight w = 1/M^2; M = 32 for up to
// 64 terms, 64 beyond): W C u = lambda u, extended to any point by
//   phi(x) = (1/lambda) sum_q w C(x, q) u(q).
// The grid and C are invariant under x -> 1-x (Sx), y -> 1-y (Sy) and x <-> y (R). Every
// eigenvector has a definite parity (sx, sy) under (Sx, Sy); each parity sector is solved on
// the quarter grid (x, y < 1/2) with the kernel folded over the four mirror images,
//   A_s(p, q) = w [C(p, q) + sx C(p, Sx q) + sy C(p, Sy q) + sx sy C(p, Sx Sy q)].
// R maps sector (+,-) onto (-,+): their eigenvalues coincide, and the (-,+) eigenvectors are
// taken as the mirror images of the (+,-) ones. R maps (+,+) and (-,-) onto themselves; each is
// split into the vectors even and odd under R, solved on an orthonormal basis of each (R-even
// and R-odd eigenvalues can lie within a relative 1e-8, and the split keeps such pairs from
// mixing by rounding). Order: eigenvalue descending; eigenvalues within a relative 1e-9 count as
// equal and are ordered by sector (+,+), (+,-), (-,+), (-,-), R-even first. Sign: sum over the
// full grid of w u g > 0 with g(x, y) = exp(0.7 x + 1.3 y), except for (-,+) members, which
// carry the sign of their mirror partner.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <utility>
#include <vector>

#include "internal.h"

namespace mls2mc {

namespace {

constexpr int kMaxTerms = 512;

int nystrom_cells(int K) { return K <= 64 ? 32 : 64; }

double matern32(double r, double lc, double var) {
    const double z = std::sqrt(6.0) * r / lc;
    return var * (1.0 + z) * std::exp(-z);
}

// C(p, .) at q and its three mirror images Sx q, Sy q, SxSy q
void mirror_cov(double px, double py, double qx, double qy, double lc, double var, double c[4]) {
    const double ax = px - qx, bx = px - (1.0 - qx), ay = py - qy, by = py - (1.0 - qy);
    c[0] = matern32(std::sqrt(ax * ax + ay * ay), lc, var);
    c[1] = matern32(std::sqrt(bx * bx + ay * ay), lc, var);
    c[2] = matern32(std::sqrt(ax * ax + by * by), lc, var);
    c[3] = matern32(std::sqrt(bx * bx + by * by), lc, var);
}

double fold(const double c[4], int sx, int sy) { return c[0] + sx * c[1] + sy * c[2] + sx * sy * c[3]; }

struct Mode {
    double lam;
    int sector;                // 0 (+,+), 1 (+,-), 2 (-,+), 3 (-,-)
    int sub;                   // -1 R-even, +1 R-odd, 0 no split
    int sx, sy;
    std::vector<double> u;     // quarter-grid values (index ix * m + iy), full-grid sum w u^2 = 1
};

struct Sub {
    int sector, sx, sy, parity;   // parity under R: +1, -1, or 0 (sector not split)
};
constexpr Sub kSubs[5] = {{0, 1, 1, 1}, {0, 1, 1, -1}, {1, 1, -1, 0}, {3, -1, -1, 1}, {3, -1, -1, -1}};

// eigenpairs of one sub-problem on the quarter grid of an M x M grid
bool solve_sub(int M, const Sub& s, double lc, double var, std::vector<Mode>& out) {
    const int m = M / 2, Q = m * m;
    const double w = 1.0 / ((double)M * M);
    auto coord = [M](int i) { return (i + 0.5) / M; };
    std::vector<double> A((size_t)Q * Q);
    for (int p = 0; p < Q; ++p)
        for (int q = p; q < Q; ++q) {
            double c[4];
            mirror_cov(coord(p / m), coord(p % m), coord(q / m), coord(q % m), lc, var, c);
            A[(size_t)p * Q + q] = A[(size_t)q * Q + p] = w * fold(c, s.sx, s.sy);
        }
    // basis: vector b has up to two entries (index, coefficient)
    struct Vec { int i0, i1; double c0, c1; };
    std::vector<Vec> B;
    if (s.parity == 0) {
        for (int p = 0; p < Q; ++p) B.push_back({p, -1, 1.0, 0.0});
    } else {
        const double h = 1.0 / std::sqrt(2.0);
        for (int ix = 0; ix < m; ++ix)
            for (int iy = ix; iy < m; ++iy) {
                if (ix == iy) {
                    if (s.parity > 0) B.push_back({ix * m + iy, -1, 1.0, 0.0});
                } else {
                    B.push_back({ix * m + iy, iy * m + ix, h, s.parity * h});
                }
            }
    }
    const int n = (int)B.size();
    std::vector<double> R((size_t)n * n);
    auto at = [&](int i, int j) { return A[(size_t)i * Q + j]; };
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            const Vec &x = B[a], &y = B[b];
            double v = x.c0 * y.c0 * at(x.i0, y.i0);
            if (y.i1 >= 0) v += x.c0 * y.c1 * at(x.i0, y.i1);
            if (x.i1 >= 0) v += x.c1 * y.c0 * at(x.i1, y.i0);
            if (x.i1 >= 0 && y.i1 >= 0) v += x.c1 * y.c1 * at(x.i1, y.i1);
            R[(size_t)a * n + b] = v;
        }
    std::vector<double>().swap(A);
    std::vector<double> lam, vt;
    if (!symmetric_eigen(n, R, lam, vt)) return false;
    const double scale = 1.0 / std::sqrt(4.0 * w);
    out.clear();
    for (int k = 0; k < n; ++k) {
        Mode md{lam[k], s.sector, -s.parity, s.sx, s.sy, std::vector<double>(Q, 0.0)};
        const double* v = &vt[(size_t)k * n];
        for (int a = 0; a < n; ++a) {
            md.u[B[a].i0] += B[a].c0 * v[a] * scale;
            if (B[a].i1 >= 0) md.u[B[a].i1] += B[a].c1 * v[a] * scale;
        }
        double sg = 0.0;
        for (int q = 0; q < Q; ++q) {
            const double x = coord(q / m), y = coord(q % m);
            const double g = std::exp(0.7 * x + 1.3 * y) + s.sx * std::exp(0.7 * (1.0 - x) + 1.3 * y) +
                             s.sy * std::exp(0.7 * x + 1.3 * (1.0 - y)) +
                             s.sx * s.sy * std::exp(0.7 * (1.0 - x) + 1.3 * (1.0 - y));
            sg += w * md.u[q] * g;
        }
        if (sg < 0.0)
            for (double& x : md.u) x = -x;
        if (s.sector == 1) {   // its mirror image x <-> y, in sector (-,+)
            Mode r{md.lam, 2, 0, -1, 1, std::vector<double>(Q)};
            for (int ix = 0; ix < m; ++ix)
                for (int iy = 0; iy < m; ++iy) r.u[ix * m + iy] = md.u[iy * m + ix];
            out.push_back(std::move(md));
            out.push_back(std::move(r));
        } else {
            out.push_back(std::move(md));
        }
    }
    return true;
}

// run f(0) .. f(n-1) on up to `threads` threads (inline when threads cannot be started)
template <typename F>
void parallel_for(int n, int threads, F f) {
    threads = std::max(1, std::min(threads, n));
    if (threads == 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> pool;
    try {
        for (int t = 0; t < threads; ++t)
            pool.emplace_back([=] {
                for (int i = t; i < n; i += threads) f(i);
            });
    } catch (...) {
        for (auto& th : pool) th.join();
        for (int i = 0; i < n; ++i) f(i);   // thread start failed: finish inline (f is idempotent)
        return;
    }
    for (auto& th : pool) th.join();
}

int host_threads() {
    const unsigned h = std::thread::hardware_concurrency();
    return h == 0 ? 1 : (int)std::min(h, 32u);
}

// all modes in order (the leading kMaxTerms kept); empty if an eigen-solve failed
std::vector<Mode> compute_modes(double lc, double var, int M) {
    std::vector<std::vector<Mode>> parts(5);
    std::vector<char> ok(5, 0);
    parallel_for(5, 5, [&](int i) { ok[i] = solve_sub(M, kSubs[i], lc, var, parts[i]); });
    std::vector<Mode> all;
    for (int i = 0; i < 5; ++i) {
        if (!ok[i]) return {};
        for (Mode& md : parts[i]) all.push_back(std::move(md));
    }
    std::stable_sort(all.begin(), all.end(), [](const Mode& a, const Mode& b) { return a.lam > b.lam; });
    for (size_t i = 0; i < all.size();) {
        size_t j = i;
        while (j + 1 < all.size() && all[i].lam - all[j + 1].lam <= 1e-9 * all[i].lam) ++j;
        std::stable_sort(all.begin() + i, all.begin() + j + 1, [](const Mode& a, const Mode& b) {
            return std::make_pair(a.sector, a.sub) < std::make_pair(b.sector, b.sub);
        });
        i = j + 1;
    }
    if (all.size() > (size_t)kMaxTerms) all.resize(kMaxTerms);
    return all;
}

// the ordered modes of (lc, variance, M), computed once per process
const std::vector<Mode>& modes(double lc, double var, int M) {
    static std::mutex mu;
    static std::map<std::tuple<double, double, int>, std::vector<Mode>> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_tuple(lc, var, M);
    auto it = cache.find(key);
    if (it == cache.end()) it = cache.emplace(key, compute_modes(lc, var, M)).first;
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

int matern_max_terms() { return kMaxTerms; }

bool matern_kl_table(int N, double corr_len, double variance, int K, std::vector<double>& psi,
                     std::vector<double>& lambda) {
    const int M = nystrom_cells(K), m = M / 2, Q = m * m;
    const std::vector<Mode>& ms = modes(corr_len, variance, M);
    if ((int)ms.size() < K) return false;
    const int E = 2 * N * N;
    const double h = 1.0 / N, w = 1.0 / ((double)M * M);
    psi.assign((size_t)K * E, 0.0);
    lambda.resize(K);
    for (int k = 0; k < K; ++k) lambda[k] = ms[k].lam;
    // blocks of kB elements: the folded kernel of the four sectors at each quarter-grid point
    // (layout [sector][q][element of the block]), then per mode kB independent dot products
    constexpr int kB = 8;
    const int nblk = (E + kB - 1) / kB;
    const long long work = (long long)E * Q * (4 + K);
    const int threads = work < (1LL << 22) ? 1 : host_threads();
    parallel_for(nblk, threads, [&](int blk) {
        std::vector<double> f((size_t)4 * Q * kB, 0.0);
        const int e0 = blk * kB, nb = std::min(kB, E - e0);
        for (int b = 0; b < nb; ++b) {
            const int e = e0 + b, cell = e / 2, i = cell % N, j = cell / N;
            // lower triangle centroid ((i+2/3)h, (j+1/3)h), upper ((i+1/3)h, (j+2/3)h)
            const double x = (e & 1) ? (i + 1.0 / 3.0) * h : (i + 2.0 / 3.0) * h;
            const double y = (e & 1) ? (j + 2.0 / 3.0) * h : (j + 1.0 / 3.0) * h;
            for (int q = 0; q < Q; ++q) {
                double c[4];
                mirror_cov(x, y, (q / m + 0.5) / M, (q % m + 0.5) / M, corr_len, variance, c);
                f[((size_t)0 * Q + q) * kB + b] = fold(c, 1, 1);
                f[((size_t)1 * Q + q) * kB + b] = fold(c, 1, -1);
                f[((size_t)2 * Q + q) * kB + b] = fold(c, -1, 1);
                f[((size_t)3 * Q + q) * kB + b] = fold(c, -1, -1);
            }
        }
        for (int k = 0; k < K; ++k) {
            const Mode& md = ms[k];
            const double* u = md.u.data();
            const double* fs = &f[(size_t)md.sector * Q * kB];
            double acc[kB] = {};
            for (int q = 0; q < Q; ++q) {
                const double uq = u[q];
                for (int b = 0; b < kB; ++b) acc[b] += fs[(size_t)q * kB + b] * uq;
            }
            // sqrt(lambda) phi = sqrt(lambda) (1/lambda) sum w C u
            const double sc = w / std::sqrt(md.lam);
            for (int b = 0; b < nb; ++b) psi[(size_t)k * E + e0 + b] = sc * acc[b];
        }
    });
    return true;
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
