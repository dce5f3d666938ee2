// Sampler kernels, all FP64: linear test forward model, Philox draws, adaptive increment
// search (cv target), evidence increment, systematic resampling, pCN propose/accept.
//
// Sources: cv and ESS of the incremental weights (Sec. 3.4, Eq. EQ:ESS:SMC_Update, population
// moments); the next inverse temperature / bridging temperature minimises (cv - tau*)^2 over
// [min(beta + eps, 1), 1] (Eqs. Eq_ESS_opt, Eq_cv_opt); ITU weights exp(-(beta_k - beta_{k-1}) Phi)
// and bridging weights exp(-beta (zeta_m - zeta_{m-1}) (Phi_l - Phi_{l-1})) (Secs. 3.2, 4.1);
// resampling before the Markov move (Sec. 2.4); evidence as the product of mean incremental
// weights (Sec. 5.1.3). Random numbers: Philox4x32-10 (Salmon et al., SC 2011), counter =
// (block, particle, event, purpose), key = the 64-bit seed; uniforms with 53 random bits;
// normals by the Box-Muller transform.
#include <cuda_runtime.h>

#include <cstdint>

#include "handle.h"
#include "smc_device.h"

namespace mls2mc {

namespace {

// one warp per particle: G[o] = sum_k A[o][k] theta[k], Phi = 1/2 sum ((y - G)/sigma)^2 (Eq. phi)
__global__ void linear_eval_kernel(const double* __restrict__ A, int n, int K, int n_obs,
                                   const double* __restrict__ theta, const double* __restrict__ y,
                                   double inv_sigma2, double* G, double* Phi, int* iters) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double* th = theta + (size_t)warp * K;
    double m = 0.0;
    for (int o = lane; o < n_obs; o += 32) {
        double g = 0.0;
        for (int k = 0; k < K; ++k) g = fma(A[(size_t)o * K + k], th[k], g);
        if (G) G[(size_t)warp * n_obs + o] = g;
        const double r = y[o] - g;
        m += r * r;
    }
    for (int off = 16; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
    if (lane == 0) {
        Phi[warp] = 0.5 * m * inv_sigma2;
        if (iters) iters[warp] = 0;
    }
}

// ---- Philox4x32-10 ---------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint64_t seed) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        if (r < 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    return c;
}

// uniform in [0, 1) with 53 random bits: 27 high bits of hi, 26 of lo
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
    return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6)) * (1.0 / 9007199254740992.0);
}

// normals for entries 2b, 2b+1 of particle j (Box-Muller on two 53-bit uniforms)
__device__ __forceinline__ void normal_pair(uint32_t b, uint32_t j, uint32_t event, uint32_t purpose,
                                            uint64_t seed, double& z0, double& z1) {
    const uint4 x = philox(make_uint4(b, j, event, purpose), seed);
    const double v1 = u53(x.x, x.y), v2 = u53(x.z, x.w);
    const double r = sqrt(-2.0 * log(1.0 - v1));
    const double ang = 2.0 * 3.141592653589793 * v2;
    z0 = r * cos(ang);
    z1 = r * sin(ang);
}

__global__ void normals_kernel(double* out, int J, int K, uint32_t event, uint32_t purpose, uint64_t seed,
                               const double* base, double c0, double c1) {
    // out[j][k] = c0 * base[j][k] + c1 * xi[j][k]  (base == null: out = xi)
    const int nb = (K + 1) / 2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)J * nb) return;
    const int j = (int)(t / nb), b = (int)(t - (long long)j * nb);
    double z0, z1;
    normal_pair((uint32_t)b, (uint32_t)j, event, purpose, seed, z0, z1);
    const size_t o = (size_t)j * K + 2 * b;
    if (base) {
        out[o] = __dadd_rn(__dmul_rn(c0, base[o]), __dmul_rn(c1, z0));
        if (2 * b + 1 < K) out[o + 1] = __dadd_rn(__dmul_rn(c0, base[o + 1]), __dmul_rn(c1, z1));
    } else {
        out[o] = z0;
        if (2 * b + 1 < K) out[o + 1] = z1;
    }
}

__global__ void uniforms_kernel(double* out, int J, uint32_t event, uint32_t purpose, uint64_t seed) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= J) return;
    const uint4 x = philox(make_uint4(0u, (uint32_t)j, event, purpose), seed);
    out[j] = 1.0 - u53(x.x, x.y);
}

// ---- block reduction helpers -----------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_reduce_sum(double (&v)[NV], double* sh /*[NV][32]*/) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
        for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[i * 32 + w] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double s = 0.0;
        for (int k = 0; k < nw; ++k) s += sh[i * 32 + k];
        v[i] = s;
    }
    __syncthreads();
}

// ---- adaptive increment (Eq. Eq_cv_opt) --------------------------------------------------
__global__ void inc_min_kernel(const double* a, int n, double* pmin) {
    __shared__ double sh[32];
    double m = INFINITY;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) m = fmin(m, a[j]);
    for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = INFINITY;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) r = fmin(r, sh[k]);
        pmin[blockIdx.x] = r;
    }
}

__global__ void inc_init_kernel(const double* pmin, int nblk, IncState* st, double dmax, double tau, double eps) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = INFINITY;
    for (int k = 0; k < nblk; ++k) m = fmin(m, pmin[k]);
    st->amin = m;
    st->dmax = dmax;
    st->dmin = fmin(eps, dmax);
    st->target = log1p(tau * tau);   // log(1 + tau^2)
    st->tau = tau;
    st->x = dmax;                     // first test: the whole remaining step
    st->phase = 0;
    st->iter = 0;
    st->done = (m == INFINITY || !(m == m)) ? -1 : 0;   // -1: empty or NaN potentials
}

// sums at x = st->x over w_j = exp(-x (a_j - amin)): S1, S2, T1 = sum a~ w, T2 = sum a~ w^2
__global__ void inc_eval_kernel(const double* a, int n, const IncState* st, double* partials) {
    __shared__ double sh[4 * 32];
    if (st->done) return;
    const double x = st->x, amin = st->amin;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double at = a[j] - amin;
        const double w = exp(-x * at);
        const double w2 = w * w;
        v[0] += w;
        v[1] += w2;
        v[2] += at * w;
        v[3] += at * w2;
    }
    block_reduce_sum<4>(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) partials[blockIdx.x * 4 + i] = v[i];
}

// one decision of the search: boundary tests first, then Newton steps on
// g(x) = log(1 + cv(x)^2) - log(1 + tau^2) in t = log x (the increment spans decades),
// safeguarded by geometric bisection of the bracket [lo, hi] (lo >= eps > 0)
__global__ void inc_decide_kernel(const double* partials, int nblk, IncState* st, int n, int max_iter) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (st->done) return;
    double S1 = 0, S2 = 0, T1 = 0, T2 = 0;
    for (int k = 0; k < nblk; ++k) {
        S1 += partials[4 * k];
        S2 += partials[4 * k + 1];
        T1 += partials[4 * k + 2];
        T2 += partials[4 * k + 3];
    }
    const double x = st->x;
    const double ratio = (double)n * S2 / (S1 * S1);      // 1 + cv^2
    const double g = log(ratio) - st->target;
    st->iter += 1;
    bool finish = false;
    if (st->phase == 0) {                    // x = dmax
        if (!(g > 0.0)) finish = true;       // cv(dmax) <= tau (also: all a equal)
        else {
            st->phase = 1;
            st->x = st->dmin;
            st->hi = x;
        }
    } else if (st->phase == 1) {             // x = dmin
        if (g >= 0.0 || st->dmin >= st->dmax) finish = true;
        else {
            st->phase = 2;
            st->lo = x;
            st->x = sqrt(st->lo * st->hi);
        }
    } else {
        if (g > 0.0) st->hi = x; else st->lo = x;
        const double lo = st->lo, hi = st->hi;
        const double gp = 2.0 * (T1 / S1 - T2 / S2);       // dg/dx >= 0
        double xn = x * exp(-g / (x * gp));                 // Newton step in log x
        if (!(xn > lo && xn < hi)) xn = sqrt(lo * hi);
        if (g == 0.0 || hi <= lo * (1.0 + 4e-16) || fabs(xn - x) <= 1e-15 * x || st->iter >= max_iter) finish = true;
        else st->x = xn;
    }
    if (finish) {
        st->delta = x;
        st->S1 = S1;
        st->log_mean_w = -x * st->amin + log(S1 / (double)n);
        const double c2 = ratio - 1.0;
        st->cv = c2 > 0.0 ? sqrt(c2) : 0.0;
        st->done = 1;
    }
}

// ---- systematic resampling -----------------------------------------------------------------
// Inclusive prefix sums of the normalised weights W_j = w_j / sum w, w_j = exp(-delta (a_j - amin))
// (or given weights), one block of 1024 threads: each thread owns a contiguous chunk; chunk
// totals are scanned with warp shuffles (fixed order), then each chunk is rescanned. The last
// entry is set to 1 exactly.
__global__ void __launch_bounds__(1024) cdf_kernel(const double* a, const double* w_in, int n,
                                                   const IncState* st, double* cdf) {
    __shared__ double warp_tot[32];
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int chunk = (n + T - 1) / T;
    const int j0 = min(n, t * chunk), j1 = min(n, j0 + chunk);
    double s = 0.0;
    for (int j = j0; j < j1; ++j) {
        const double w = w_in ? w_in[j] : exp(-st->delta * (a[j] - st->amin));
        cdf[j] = w;
        s += w;
    }
    // inclusive scan of chunk totals inside the warp
    double incl = s;
    for (int off = 1; off < 32; off <<= 1) {
        const double v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = T >> 5;
        double v = lane < nw ? warp_tot[lane] : 0.0;
        for (int off = 1; off < 32; off <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += u;
        }
        if (lane < nw) warp_tot[lane] = v;   // inclusive warp totals
    }
    __syncthreads();
    const double total = warp_tot[(T >> 5) - 1];
    double run = (incl - s) + (wid > 0 ? warp_tot[wid - 1] : 0.0);   // exclusive offset of the chunk
    const double inv = 1.0 / total;
    for (int j = j0; j < j1; ++j) {
        run += cdf[j];
        cdf[j] = run * inv;
    }
    __syncthreads();
    if (t == 0 && n > 0) cdf[n - 1] = 1.0;
}

// ancestor(i) = min{ j : cdf_j > (U + i)/n }; U from Philox (or given, U >= 0)
__global__ void ancestors_kernel(const double* cdf, int n, double U, uint32_t event, uint64_t seed, int* anc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (U < 0.0) {
        const uint4 x = philox(make_uint4(0u, 0u, event, (uint32_t)kPurposeResample), seed);
        U = u53(x.x, x.y);
    }
    const double pos = (U + (double)i) / (double)n;
    int lo = 0, hi = n - 1;                 // cdf[n-1] = 1 > pos always
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cdf[mid] > pos) hi = mid; else lo = mid + 1;
    }
    anc[i] = lo;
}

// gather theta rows and up to two potential caches by ancestor index
__global__ void gather_kernel(const int* anc, int n, int K, const double* th_in, double* th_out,
                              const double* p0_in, double* p0_out, const double* p1_in, double* p1_out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * K) return;
    const int i = (int)(t / K), k = (int)(t - (long long)i * K);
    const int src = anc[i];
    th_out[t] = th_in[(size_t)src * K + k];
    if (k == 0) {
        if (p0_in) p0_out[i] = p0_in[src];
        if (p1_in) p1_out[i] = p1_in[src];
    }
}

// ---- increments of a level update and the cv^LU predictor ------------------------------------
__global__ void lu_increment_kernel(const double* phi_c, const double* phi_f, int n, double beta, double* a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) a[j] = beta * (phi_f[j] - phi_c[j]);
}

// cv of exp(-beta (d_j - min d)), d_j = phi_f[j] - phi_c[j], j < n (one block)
__global__ void cv_lu_kernel(const double* phi_c, const double* phi_f, int n, double beta, double* out) {
    __shared__ double sh[2 * 32];
    __shared__ double smin[32];
    double m = INFINITY;
    for (int j = threadIdx.x; j < n; j += blockDim.x) m = fmin(m, phi_f[j] - phi_c[j]);
    for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) smin[threadIdx.x >> 5] = m;
    __syncthreads();
    double dmin = INFINITY;
    for (int k = 0; k < (int)(blockDim.x + 31) / 32; ++k) dmin = fmin(dmin, smin[k]);
    double v[2] = {0.0, 0.0};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double w = exp(-beta * ((phi_f[j] - phi_c[j]) - dmin));
        v[0] += w;
        v[1] += w * w;
    }
    block_reduce_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        const double mean = v[0] / n, c2 = v[1] / n - mean * mean;
        out[0] = c2 > 0.0 ? sqrt(c2) / mean : 0.0;
    }
}

// ---- pCN acceptance ---------------------------------------------------------------------------
// target potential beta * ((1 - zeta) Phi_c + zeta Phi_f) (zeta < 0: beta * Phi_c), with explicit
// rounding so the comparison with log U is evaluated exactly as written
__device__ __forceinline__ double target_potential(double beta, double zeta, double pc, double pf) {
    if (zeta < 0.0) return __dmul_rn(beta, pc);
    return __dmul_rn(beta, __dadd_rn(__dmul_rn(1.0 - zeta, pc), __dmul_rn(zeta, pf)));
}

__global__ void pcn_accept_kernel(int n, int K, double beta, double zeta, uint32_t event, uint64_t seed,
                                  double* theta, const double* theta_p, double* phi_c, const double* phi_cp,
                                  double* phi_f, const double* phi_fp, unsigned long long* n_acc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = false;
    if (j < n) {
        const uint4 x = philox(make_uint4(0u, (uint32_t)j, event, (uint32_t)kPurposePcnU), seed);
        const double U = 1.0 - u53(x.x, x.y);
        const double t_old = target_potential(beta, zeta, phi_c[j], zeta < 0.0 ? 0.0 : phi_f[j]);
        const double t_new = target_potential(beta, zeta, phi_cp[j], zeta < 0.0 ? 0.0 : phi_fp[j]);
        ok = log(U) < -(t_new - t_old);
        if (ok) {
            for (int k = 0; k < K; ++k) theta[(size_t)j * K + k] = theta_p[(size_t)j * K + k];
            phi_c[j] = phi_cp[j];
            if (zeta >= 0.0) phi_f[j] = phi_fp[j];
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, ok);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(n_acc, (unsigned long long)__popc(ballot));
}

// ---- delayed acceptance (Christen & Fox 2005) ----------------------------------------------------
// stage 1 on the surrogate potentials: pass with probability min(1, exp(-(t~(theta') - t~(theta))));
// survivors are compacted (index list, proposal rows) for the exact solve
__global__ void da_stage1_kernel(int n, int K, double beta, double zeta, uint32_t event, uint64_t seed,
                                 const double* ps_c, const double* ps_f, const double* psp_c, const double* psp_f,
                                 const double* theta_p, int* surv_idx, int* n_surv, double* theta_s) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint4 x = philox(make_uint4(0u, (uint32_t)j, event, (uint32_t)kPurposeDaU), seed);
    const double U = 1.0 - u53(x.x, x.y);
    const bool br = zeta >= 0.0;
    const double t_old = target_potential(beta, zeta, ps_c[j], br ? ps_f[j] : 0.0);
    const double t_new = target_potential(beta, zeta, psp_c[j], br ? psp_f[j] : 0.0);
    if (log(U) < -(t_new - t_old)) {
        const int slot = atomicAdd(n_surv, 1);
        surv_idx[slot] = j;
        for (int k = 0; k < K; ++k) theta_s[(size_t)slot * K + k] = theta_p[(size_t)j * K + k];
    }
}

// stage 2 on the exact potentials of the survivors, corrected by the surrogate ratio:
// accept with probability min(1, exp(-(t(theta') - t(theta)) + (t~(theta') - t~(theta))))
__global__ void da_stage2_kernel(int ns, int K, double beta, double zeta, uint32_t event, uint64_t seed,
                                 const int* surv_idx, const double* theta_s, const double* phi_cs,
                                 const double* phi_fs, double* theta, double* phi_c, double* phi_f, double* ps_c,
                                 double* ps_f, const double* psp_c, const double* psp_f,
                                 unsigned long long* n_acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = false;
    if (i < ns) {
        const int j = surv_idx[i];
        const uint4 x = philox(make_uint4(0u, (uint32_t)j, event, (uint32_t)kPurposePcnU), seed);
        const double U = 1.0 - u53(x.x, x.y);
        const bool br = zeta >= 0.0;
        const double t_old = target_potential(beta, zeta, phi_c[j], br ? phi_f[j] : 0.0);
        const double t_new = target_potential(beta, zeta, phi_cs[i], br ? phi_fs[i] : 0.0);
        const double s_old = target_potential(beta, zeta, ps_c[j], br ? ps_f[j] : 0.0);
        const double s_new = target_potential(beta, zeta, psp_c[j], br ? psp_f[j] : 0.0);
        ok = log(U) < -(t_new - t_old) + (s_new - s_old);
        if (ok) {
            for (int k = 0; k < K; ++k) theta[(size_t)j * K + k] = theta_s[(size_t)i * K + k];
            phi_c[j] = phi_cs[i];
            ps_c[j] = psp_c[j];
            if (br) {
                phi_f[j] = phi_fs[i];
                ps_f[j] = psp_f[j];
            }
        }
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, ok);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(n_acc, (unsigned long long)__popc(ballot));
}

// number of negative iteration counts (solves that did not converge), accumulated into *bad
__global__ void count_bad_kernel(const int* iters, int n, unsigned* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool b = i < n && iters[i] < 0;
    const unsigned ballot = __ballot_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(bad, (unsigned)__popc(ballot));
}

// ---- posterior moments over equally weighted particles ----------------------------------------
__global__ void moments_kernel(const double* theta, int n, int K, double* mean, double* var) {
    __shared__ double sh[32];
    const int k = blockIdx.x;
    double m[1] = {0.0};
    for (int j = threadIdx.x; j < n; j += blockDim.x) m[0] += theta[(size_t)j * K + k];
    block_reduce_sum<1>(m, sh);
    const double mu = m[0] / n;
    double q[1] = {0.0};
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double t = theta[(size_t)j * K + k] - mu;
        q[0] += t * t;
    }
    block_reduce_sum<1>(q, sh);
    if (threadIdx.x == 0) {
        mean[k] = mu;
        var[k] = q[0] / n;
    }
}

}  // namespace

// ---- launch wrappers ----------------------------------------------------------------------------
static int grid_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

cudaError_t linear_eval_launch(const double* A, int n, int K, int n_obs, const double* theta, const double* y,
                               double inv_sigma2, double* G, double* Phi, int* iters, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    linear_eval_kernel<<<grid_for((long long)n * 32, 256), 256, 0, st>>>(A, n, K, n_obs, theta, y, inv_sigma2, G,
                                                                         Phi, iters);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t normals_launch(double* out, int J, int K, uint32_t event, uint32_t purpose, uint64_t seed,
                           const double* base, double c0, double c1, cudaStream_t st) {
    if (J <= 0) return cudaSuccess;
    const long long work = (long long)J * ((K + 1) / 2);
    normals_kernel<<<grid_for(work, 256), 256, 0, st>>>(out, J, K, event, purpose, seed, base, c0, c1);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t uniforms_launch(double* out, int J, uint32_t event, uint32_t purpose, uint64_t seed, cudaStream_t st) {
    if (J <= 0) return cudaSuccess;
    uniforms_kernel<<<grid_for(J, 256), 256, 0, st>>>(out, J, event, purpose, seed);
    count_launches(1);
    return cudaGetLastError();
}

int inc_blocks(int n) { return std::min(kIncMaxBlocks, std::max(1, (n + 255) / 256)); }

cudaError_t inc_start(const double* a, int n, double dmax, double tau, double eps, IncWork& w, cudaStream_t st) {
    const int nb = inc_blocks(n);
    inc_min_kernel<<<nb, 256, 0, st>>>(a, n, w.partials);
    count_launches(1);
    inc_init_kernel<<<1, 32, 0, st>>>(w.partials, nb, w.state, dmax, tau, eps);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t inc_iterate(const double* a, int n, int iters, IncWork& w, cudaStream_t st) {
    const int nb = inc_blocks(n);
    for (int i = 0; i < iters; ++i) {
        inc_eval_kernel<<<nb, 256, 0, st>>>(a, n, w.state, w.partials);
        count_launches(1);
        inc_decide_kernel<<<1, 32, 0, st>>>(w.partials, nb, w.state, n, kIncMaxIter);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t resample_launch(const double* a, const double* w_in, int n, const IncState* state, double U,
                            uint32_t event, uint64_t seed, double* cdf, int* anc, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cdf_kernel<<<1, 1024, 0, st>>>(a, w_in, n, state, cdf);
    count_launches(1);
    ancestors_kernel<<<grid_for(n, 256), 256, 0, st>>>(cdf, n, U, event, seed, anc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t gather_launch(const int* anc, int n, int K, const double* th_in, double* th_out, const double* p0_in,
                          double* p0_out, const double* p1_in, double* p1_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    gather_kernel<<<grid_for((long long)n * K, 256), 256, 0, st>>>(anc, n, K, th_in, th_out, p0_in, p0_out, p1_in,
                                                                   p1_out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t lu_increment_launch(const double* phi_c, const double* phi_f, int n, double beta, double* a,
                                cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    lu_increment_kernel<<<grid_for(n, 256), 256, 0, st>>>(phi_c, phi_f, n, beta, a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t cv_lu_launch(const double* phi_c, const double* phi_f, int n, double beta, double* out, cudaStream_t st) {
    cv_lu_kernel<<<1, 256, 0, st>>>(phi_c, phi_f, n, beta, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t pcn_accept_launch(int n, int K, double beta, double zeta, uint32_t event, uint64_t seed, double* theta,
                              const double* theta_p, double* phi_c, const double* phi_cp, double* phi_f,
                              const double* phi_fp, unsigned long long* n_acc, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    pcn_accept_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, K, beta, zeta, event, seed, theta, theta_p, phi_c, phi_cp,
                                                        phi_f, phi_fp, n_acc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t da_stage1_launch(int n, int K, double beta, double zeta, uint32_t event, uint64_t seed, const double* ps_c,
                             const double* ps_f, const double* psp_c, const double* psp_f, const double* theta_p,
                             int* surv_idx, int* n_surv, double* theta_s, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    da_stage1_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, K, beta, zeta, event, seed, ps_c, ps_f, psp_c, psp_f, theta_p,
                                                       surv_idx, n_surv, theta_s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t da_stage2_launch(int ns, int K, double beta, double zeta, uint32_t event, uint64_t seed, const int* surv_idx,
                             const double* theta_s, const double* phi_cs, const double* phi_fs, double* theta,
                             double* phi_c, double* phi_f, double* ps_c, double* ps_f, const double* psp_c,
                             const double* psp_f, unsigned long long* n_acc, cudaStream_t st) {
    if (ns <= 0) return cudaSuccess;
    da_stage2_kernel<<<grid_for(ns, 256), 256, 0, st>>>(ns, K, beta, zeta, event, seed, surv_idx, theta_s, phi_cs, phi_fs,
                                                        theta, phi_c, phi_f, ps_c, ps_f, psp_c, psp_f, n_acc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t count_bad_launch(const int* iters, int n, unsigned* bad, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    count_bad_kernel<<<grid_for(n, 256), 256, 0, st>>>(iters, n, bad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t moments_launch(const double* theta, int n, int K, double* mean, double* var, cudaStream_t st) {
    moments_kernel<<<K, 256, 0, st>>>(theta, n, K, mean, var);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace mls2mc
