// Sampler kernels, all FP64: linear test forward model, Philox draws, adaptive increment
// search (cv target), evidence increment, systematic resampling, pCN / random-walk propose and
// accept, the two stages of delayed acceptance.
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

// the task (problem) of this block in a multi-problem launch: start[p] <= blockIdx.x < start[p + 1]
__device__ __forceinline__ int task_of_block(const int* start, int count) {
    __shared__ int p_s;
    if (threadIdx.x == 0) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (start[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        p_s = lo;
    }
    __syncthreads();
    return p_s;
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

// many problems' proposals or draws (256-thread blocks, a contiguous block range per problem)
__global__ void normals_multi_kernel(const __grid_constant__ NormTasks T) {
    const int p = task_of_block(T.start, T.count);
    const NormTask& k = T.t[p];
    const int nb = (k.K + 1) / 2;
    const long long t = (long long)(blockIdx.x - (unsigned)T.start[p]) * blockDim.x + threadIdx.x;
    if (t >= (long long)k.J * nb) return;
    const int j = (int)(t / nb), b = (int)(t - (long long)j * nb);
    double z0, z1;
    normal_pair((uint32_t)b, (uint32_t)j, k.event, k.purpose, k.seed, z0, z1);
    const size_t o = (size_t)j * k.K + 2 * b;
    if (k.base) {
        k.out[o] = __dadd_rn(__dmul_rn(k.c0, k.base[o]), __dmul_rn(k.c1, z0));
        if (2 * b + 1 < k.K) k.out[o + 1] = __dadd_rn(__dmul_rn(k.c0, k.base[o + 1]), __dmul_rn(k.c1, z1));
    } else {
        k.out[o] = z0;
        if (2 * b + 1 < k.K) k.out[o + 1] = z1;
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
// One cooperative launch runs the whole search. Every block sums its slice of the particles, the
// blocks meet at a grid barrier, and then every block reduces all partial sums in the same fixed
// order and takes the same decision on its own copy of the search state, so one barrier per
// decision suffices. Partial sums are double-buffered by decision parity: a block can be at most
// one decision ahead of the slowest one.
//
// The search solves g(x) = log(1 + cv(x)^2) - log(1 + tau^2) = 0 for the increment x, where
// cv(x) is the coefficient of variation of w_j = exp(-x a~_j), a~_j = a_j - min a (population
// moments: 1 + cv^2 = n S2 / S1^2 with S1 = sum w, S2 = sum w^2); g is non-decreasing in x.
// Decision 1 evaluates both ends of [dmin, dmax] (dmin = min(eps, dmax)): g(dmax) <= 0 takes
// the whole remaining step, g(dmin) >= 0 the smallest one (the constrained minimiser of
// (cv - tau)^2, Eqs. Eq_ESS_opt, Eq_cv_opt). Otherwise the root is bracketed and found in
// t = log x (the increment spans decades) from a regula-falsi start by Halley steps, kept inside
// the bracket (Newton, then bisection in t, as fallbacks). Only g itself needs FP64: the step is
// a correction, computed in FP32 (FP64 instructions are expensive on this part).
//
// Sums at a point x: S1, S2, T1 = sum a~ w, T2 = sum a~ w^2, U1 = sum a~^2 w, U2 = sum a~^2 w^2;
// dS1/dx = -T1, dS2/dx = -2 T2, d2S1/dx2 = U1, d2S2/dx2 = 4 U2.

// state after the minimum of the potentials is known
__device__ void inc_init(IncState& st, double amin, double dmax, double tau, double eps, double base, double top) {
    st.amin = amin;
    st.base = base;
    st.top = top;
    st.dmax = dmax;
    st.dmin = fmin(eps, dmax);
    st.target = log1p(tau * tau);   // log(1 + tau^2)
    st.tau = tau;
    st.x = dmax;
    st.phase = 0;
    st.iter = 0;
    st.done = (amin == INFINITY || !(amin == amin)) ? -1 : 0;   // -1: empty or NaN potentials
}

__device__ void inc_finish(IncState& st, double x, double S1, double ratio, int n) {
    st.delta = x;
    st.next = x >= st.dmax ? st.top : st.base + x;
    st.S1 = S1;
    st.log_mean_w = -x * st.amin + log(S1 / (double)n);
    const double c2 = ratio - 1.0;
    st.cv = c2 > 0.0 ? sqrt(c2) : 0.0;
    st.done = 1;
}

// one decision from the block-reduced sums v[kIncSums]. Decision 1: S1, S2 at dmax, S1, S2 at
// dmin, then sum a~ and sum a~^2 (unweighted, for the starting point). Later decisions: the six
// sums at x.
__device__ void inc_decide(IncState& st, const double* v, int n, int max_iter) {
    st.iter += 1;
    if (st.phase == 0) {
        const double r_hi = (double)n * v[1] / (v[0] * v[0]);
        const double g_hi = log(r_hi) - st.target;
        if (!(g_hi > 0.0)) {                                   // cv(dmax) <= tau (also: all a equal)
            inc_finish(st, st.dmax, v[0], r_hi, n);
            return;
        }
        const double r_lo = (double)n * v[3] / (v[2] * v[2]);
        const double g_lo = log(r_lo) - st.target;
        if (g_lo >= 0.0 || st.dmin >= st.dmax) {
            inc_finish(st, st.dmin, v[2], r_lo, n);
            return;
        }
        st.phase = 1;
        st.lo = st.dmin;
        st.hi = st.dmax;
        st.tlo = log(st.lo);
        st.thi = log(st.hi);
        st.glo = g_lo;
        st.ghi = g_hi;
        // small increments: w ~ 1 - x a~, so cv(x)^2 ~ x^2 var(a~) and the root is near tau / sd(a~)
        const double mean = v[4] / n, var = v[5] / n - mean * mean;
        const double x0 = var > 0.0 ? st.tau / sqrt(var) : 0.0;
        double t0 = x0 > st.lo && x0 < st.hi ? log(x0) : st.tlo + (st.thi - st.tlo) * (-g_lo / (g_hi - g_lo));
        if (!(t0 > st.tlo && t0 < st.thi)) t0 = 0.5 * (st.tlo + st.thi);   // regula falsi in t, bisection
        st.t = t0;
        st.x = exp(t0);
        return;
    }
    const double x = st.x, S1 = v[0], S2 = v[1];
    const double ratio = (double)n * S2 / (S1 * S1);
    const double g = log(ratio) - st.target;
    const double t = st.t;
    if (g > 0.0) {
        st.hi = x;
        st.thi = t;
        st.ghi = g;
    } else {
        st.lo = x;
        st.tlo = t;
        st.glo = g;
    }
    if (g == 0.0 || st.hi <= st.lo * (1.0 + 4e-16) || st.iter >= max_iter) {
        inc_finish(st, x, S1, ratio, n);
        return;
    }
    // derivatives in t = log x, in FP32
    const float fx = (float)x;
    const float m1 = (float)v[2] / (float)S1, m2 = (float)v[3] / (float)S2;     // T1/S1, T2/S2
    const float q1 = (float)v[4] / (float)S1, q2 = (float)v[5] / (float)S2;     // U1/S1, U2/S2
    const float gp = 2.f * (m1 - m2);                                          // dg/dx
    const float gpp = 4.f * (q2 - m2 * m2) - 2.f * (q1 - m1 * m1);             // d2g/dx2
    const float G = (float)g, Gp = fx * gp, Gpp = fx * gp + fx * fx * gpp;
    const double tlo = st.tlo, thi = st.thi;
    bool local = true;
    float dt = -2.f * G * Gp / (2.f * Gp * Gp - G * Gpp);                      // Halley
    if (!(t + dt > tlo && t + dt < thi)) dt = -G / Gp;                          // Newton
    double tn = t + (double)dt;
    if (!(tn > tlo && tn < thi)) {                                              // secant on the bracket
        local = false;
        tn = tlo + (thi - tlo) * (-st.glo / (st.ghi - st.glo));
        if (!(tn > tlo && tn < thi)) tn = 0.5 * (tlo + thi);
    }
    const double xn = exp(tn);
    if (local && fabs(tn - t) <= 1e-7) {
        // the step lands within rounding of the root (the next Halley correction would be of
        // order dt^3): finish at xn, its sums extrapolated to second order in xn - x (the
        // neglected terms are of order ((xn - x) a~)^3)
        const double d = xn - x;
        const double S1n = S1 - v[2] * d + 0.5 * v[4] * d * d;
        const double S2n = S2 - 2.0 * v[3] * d + 2.0 * v[5] * d * d;
        inc_finish(st, xn, S1n, (double)n * S2n / (S1n * S1n), n);
        return;
    }
    st.t = tn;
    st.x = xn;
}

// grid barrier on a counter zeroed before the launch (thread 0 of each block; the caller
// synchronises the block around it). Bounded: after about a second of waiting (or once another
// block has given up) it raises *err and returns false.
__device__ bool grid_barrier(unsigned* bar, int* err, unsigned nblocks, unsigned& generation) {
    __threadfence();
    const unsigned target = (++generation) * nblocks;
    atomicAdd(bar, 1u);
    const long long t0 = clock64();
    while (true) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
        if (v >= target) break;
        if (*(volatile int*)err) return false;
        if (clock64() - t0 > 2000000000LL) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// sum of v[kIncSums] over the block into thread 0 (warp shuffles, then warp 0 over the warps)
__device__ __forceinline__ void inc_block_sum(double (&v)[kIncSums], double* sh /*[kIncSums][32]*/) {
#pragma unroll
    for (int i = 0; i < kIncSums; ++i)
        for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
    constexpr int nw = kIncThreads / 32;
    if (nw > 1) {
        if ((threadIdx.x & 31) == 0 && threadIdx.x > 0)
#pragma unroll
            for (int i = 0; i < kIncSums; ++i) sh[i * 32 + (threadIdx.x >> 5)] = v[i];
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 1; k < nw; ++k)
#pragma unroll
                for (int i = 0; i < kIncSums; ++i) v[i] += sh[i * 32 + k];
    }
}

// The search of one problem by the blocks bid = 0 .. nb - 1 that a launch gives it (the whole grid
// of a single-problem launch, or a contiguous range of a multi-problem launch); the result depends
// on n and nb only, not on the rest of the grid.
__device__ __forceinline__ void inc_search_blocks(const double* a, int n, double dmax, double tau, double eps,
                                                  int max_iter, double base, double top, const IncWork& w,
                                                  const unsigned bid, const unsigned nb) {
    __shared__ double sh[kIncSums * 32];
    __shared__ IncState st;
    __shared__ int ok_s;
    const int lane = threadIdx.x & 31;
    unsigned generation = 0;
    // minimum of the potentials (the weights are formed relative to it)
    double m = INFINITY;
    for (int j = bid * blockDim.x + threadIdx.x; j < n; j += nb * blockDim.x) m = fmin(m, a[j]);
    for (int off = 16; off > 0; off >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kIncThreads / 32; ++k) m = fmin(m, sh[k]);
        w.partials[bid] = m;
        ok_s = grid_barrier(w.bar, w.err, nb, generation);
    }
    __syncthreads();
    if (!ok_s) return;
    if (threadIdx.x < 32) {   // warp 0: minimum over the blocks
        double mm = INFINITY;
        for (unsigned k = lane; k < nb; k += 32) mm = fmin(mm, __ldcg(&w.partials[k]));
        for (int off = 16; off > 0; off >>= 1) mm = fmin(mm, __shfl_xor_sync(0xffffffffu, mm, off));
        if (lane == 0) inc_init(st, mm, dmax, tau, eps, base, top);
    }
    __syncthreads();
    for (int dec = 0; st.done == 0; ++dec) {
        double* part = w.partials + kIncMaxBlocks + (dec & 1) * kIncSums * kIncMaxBlocks;
        const double amin = st.amin;
        double v[kIncSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (st.phase == 0) {   // both ends of the interval
            const double xh = st.dmax, xl = st.dmin;
            for (int j = bid * blockDim.x + threadIdx.x; j < n; j += nb * blockDim.x) {
                const double at = a[j] - amin;
                const double wh = exp(-xh * at), wl = exp(-xl * at);
                v[0] += wh;
                v[1] += wh * wh;
                v[2] += wl;
                v[3] += wl * wl;
                v[4] += at;
                v[5] += at * at;
            }
        } else {
            const double x = st.x;
            for (int j = bid * blockDim.x + threadIdx.x; j < n; j += nb * blockDim.x) {
                const double at = a[j] - amin;
                const double wj = exp(-x * at);
                const double w2 = wj * wj;
                v[0] += wj;
                v[1] += w2;
                v[2] += at * wj;
                v[3] += at * w2;
                v[4] += at * at * wj;
                v[5] += at * at * w2;
            }
        }
        inc_block_sum(v, sh);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int i = 0; i < kIncSums; ++i) part[bid * kIncSums + i] = v[i];
            ok_s = grid_barrier(w.bar, w.err, nb, generation);
        }
        __syncthreads();
        if (!ok_s) return;
        if (threadIdx.x < 32) {   // warp 0: sums over the blocks in a fixed order, then the decision
            double t[kIncSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (unsigned k = lane; k < nb; k += 32)
#pragma unroll
                for (int i = 0; i < kIncSums; ++i) t[i] += __ldcg(&part[k * kIncSums + i]);
#pragma unroll
            for (int i = 0; i < kIncSums; ++i)
                for (int off = 16; off > 0; off >>= 1) t[i] += __shfl_xor_sync(0xffffffffu, t[i], off);
            if (lane == 0) inc_decide(st, t, n, max_iter);
        }
        __syncthreads();
    }
    if (bid == 0 && threadIdx.x == 0) *w.state = st;
}

__global__ void __launch_bounds__(kIncThreads) inc_search_kernel(const double* a, int n, double dmax, double tau,
                                                                 double eps, int max_iter, double base, double top,
                                                                 IncWork w) {
    inc_search_blocks(a, n, dmax, tau, eps, max_iter, base, top, w, blockIdx.x, gridDim.x);
}

// many problems' searches in one cooperative launch: problem p takes inc_blocks(n_p) blocks and
// its own barrier counter, so every problem's result is the single-problem launch's, bit for bit
__global__ void __launch_bounds__(kIncThreads) inc_search_multi_kernel(const __grid_constant__ IncTasks T) {
    const int p = task_of_block(T.start, T.count);
    const IncTask& k = T.t[p];
    inc_search_blocks(k.a, k.n, k.dmax, k.tau, k.eps, k.max_iter, k.base, k.top, k.w,
                      blockIdx.x - (unsigned)T.start[p], (unsigned)(T.start[p + 1] - T.start[p]));
}



// ---- systematic resampling with the gather, one cooperative launch ------------------------------
// The weights w_j = exp(-delta (a_j - amin)) of the increment just found, their normalised inclusive
// prefix sums (cdf, last entry 1 exactly), the ancestors min{j : cdf_j > (U + i)/n} and the gather
// of theta rows and potential caches, with the FP64 work spread over the blocks: each block scans a
// contiguous range, and after a grid barrier adds the prefix of the block totals (summed in the same
// fixed order by every block). Deterministic for given n and grid.
constexpr int kRsThreads = 128;

// the resampling of one problem by the blocks bid = 0 .. nb - 1 that a launch gives it; *distinct
// (if given) receives the number of distinct ancestors
__device__ __forceinline__ void resample_gather_blocks(
    const double* a, int n, const IncState* state, uint32_t event, uint64_t seed, int K, const double* th_in,
    double* th_out, const double* p0_in, double* p0_out, const double* p1_in, double* p1_out, double* cdf, int* anc,
    double* btot, unsigned* bar, int* err, unsigned* distinct, const unsigned bid, const unsigned nb) {
    __shared__ double warp_tot[kRsThreads / 32];
    __shared__ double run_s, off_s, inv_s;
    __shared__ int ok_s;
    __shared__ unsigned distinct_s;
    // zeroed before the first grid barrier, added to after the last one
    if (distinct && bid == 0 && threadIdx.x == 0) *distinct = 0u;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned generation = 0;
    const int chunk = (n + (int)nb - 1) / (int)nb;
    const int j0 = min(n, (int)bid * chunk), j1 = min(n, j0 + chunk);
    const double delta = state->delta, amin = state->amin;
    if (tid == 0) run_s = 0.0;
    __syncthreads();
    for (int base = j0; base < j1; base += kRsThreads) {
        const int j = base + tid;
        const double w = j < j1 ? exp(-delta * (a[j] - amin)) : 0.0;
        double incl = w;
        for (int off = 1; off < 32; off <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += u;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        double before = run_s;
        for (int k = 0; k < wid; ++k) before += warp_tot[k];
        if (j < j1) cdf[j] = before + incl;
        __syncthreads();
        if (tid == kRsThreads - 1) run_s = before + incl;
        __syncthreads();
    }
    if (tid == 0) {
        btot[bid] = run_s;
        ok_s = grid_barrier(bar, err, nb, generation);
    }
    __syncthreads();
    if (!ok_s) return;
    if (wid == 0) {   // offset of this block and the total, in a fixed order
        double off = 0.0, tot = 0.0;
        for (unsigned k = lane; k < nb; k += 32) {
            const double v = __ldcg(&btot[k]);
            tot += v;
            if (k < bid) off += v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (lane == 0) {
            off_s = off;
            inv_s = 1.0 / tot;
        }
    }
    __syncthreads();
    for (int j = j0 + tid; j < j1; j += kRsThreads) cdf[j] = j == n - 1 ? 1.0 : (cdf[j] + off_s) * inv_s;
    __syncthreads();   // every thread's entries written before thread 0 arrives at the grid barrier
    if (tid == 0) ok_s = grid_barrier(bar, err, nb, generation);
    __syncthreads();
    if (!ok_s) return;
    const uint4 x = philox(make_uint4(0u, 0u, event, (uint32_t)kPurposeResample), seed);
    const double U = u53(x.x, x.y);
    for (int i = bid * kRsThreads + tid; i < n; i += nb * kRsThreads) {
        const double pos = (U + (double)i) / (double)n;
        int lo = 0, hi = n - 1;   // cdf[n-1] = 1 > pos always
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__ldcg(&cdf[mid]) > pos) hi = mid; else lo = mid + 1;
        }
        anc[i] = lo;
    }
    __syncthreads();
    if (tid == 0) ok_s = grid_barrier(bar, err, nb, generation);
    __syncthreads();
    if (!ok_s) return;
    // gather: one warp per particle row (coalesced over k), rows spread over every warp of the grid;
    // a row starts a new ancestor when its index differs from the previous row's (sorted ancestors)
    if (tid == 0) distinct_s = 0u;
    __syncthreads();
    const int n_warps = (int)nb * (kRsThreads / 32);
    unsigned fresh = 0u;
    for (int i = (int)bid * (kRsThreads / 32) + wid; i < n; i += n_warps) {
        const int src = __ldcg(&anc[i]);
        for (int k = lane; k < K; k += 32) th_out[(size_t)i * K + k] = th_in[(size_t)src * K + k];
        if (lane == 0) {
            if (p0_in) p0_out[i] = p0_in[src];
            if (p1_in) p1_out[i] = p1_in[src];
            fresh += (i == 0 || __ldcg(&anc[i - 1]) != src) ? 1u : 0u;
        }
    }
    if (distinct) {
        if (lane == 0 && fresh) atomicAdd(&distinct_s, fresh);
        __syncthreads();
        if (tid == 0 && distinct_s) atomicAdd(distinct, distinct_s);
    }
}

__global__ void __launch_bounds__(kRsThreads) resample_gather_kernel(
    const double* a, int n, const IncState* state, uint32_t event, uint64_t seed, int K, const double* th_in,
    double* th_out, const double* p0_in, double* p0_out, const double* p1_in, double* p1_out, double* cdf, int* anc,
    double* btot, unsigned* bar, int* err, unsigned* distinct) {
    resample_gather_blocks(a, n, state, event, seed, K, th_in, th_out, p0_in, p0_out, p1_in, p1_out, cdf, anc, btot,
                           bar, err, distinct, blockIdx.x, gridDim.x);
}

// many problems' resamplings in one cooperative launch (rs_blocks(n_p) blocks and a barrier counter
// per problem: each result is the single-problem launch's, bit for bit)
__global__ void __launch_bounds__(kRsThreads) resample_gather_multi_kernel(const __grid_constant__ RsTasks T) {
    const int p = task_of_block(T.start, T.count);
    const RsTask& k = T.t[p];
    resample_gather_blocks(k.a, k.n, k.state, k.event, k.seed, k.K, k.th_in, k.th_out, k.p0_in, k.p0_out, k.p1_in,
                           k.p1_out, k.cdf, k.anc, k.btot, k.bar, k.err, k.distinct, blockIdx.x - (unsigned)T.start[p],
                           (unsigned)(T.start[p + 1] - T.start[p]));
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

// ---- increments of a level update and the cv^LU predictor ------------------------------------
__global__ void lu_increment_kernel(const double* phi_c, const double* phi_f, int n, double beta, double* a) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) a[j] = beta * (phi_f[j] - phi_c[j]);
}

__global__ void lu_increment_multi_kernel(const __grid_constant__ LuTasks T) {
    const int p = task_of_block(T.start, T.count);
    const LuTask& k = T.t[p];
    const int j = (int)(blockIdx.x - (unsigned)T.start[p]) * blockDim.x + threadIdx.x;
    if (j < k.n) k.a[j] = k.beta * (k.phi_f[j] - k.phi_c[j]);
}

// cv of exp(-beta (d_j - min d)), d_j = phi_f[j] - phi_c[j], j < n (one block)
__device__ __forceinline__ void cv_lu_block(const double* phi_c, const double* phi_f, int n, double beta, double* out) {
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

__global__ void cv_lu_kernel(const double* phi_c, const double* phi_f, int n, double beta, double* out) {
    cv_lu_block(phi_c, phi_f, n, beta, out);
}

// one block per problem, each the single-problem kernel's arithmetic
__global__ void cv_lu_multi_kernel(const __grid_constant__ CvTasks T) {
    const CvTask& k = T.t[blockIdx.x];
    cv_lu_block(k.phi_c, k.phi_f, k.n, k.beta, k.out);
}

// ---- pCN acceptance ---------------------------------------------------------------------------
// target potential beta * ((1 - zeta) Phi_c + zeta Phi_f) (zeta < 0: beta * Phi_c), with explicit
// rounding so the comparison with log U is evaluated exactly as written
__device__ __forceinline__ double target_potential(double beta, double zeta, double pc, double pf) {
    if (zeta < 0.0) return __dmul_rn(beta, pc);
    return __dmul_rn(beta, __dadd_rn(__dmul_rn(1.0 - zeta, pc), __dmul_rn(zeta, pf)));
}

// the Metropolis decision of particle j (j >= n: none); true if the proposal was taken
__device__ __forceinline__ bool pcn_accept_one(int j, int n, int K, double beta, double zeta, uint32_t event,
                                               uint64_t seed, double* theta, const double* theta_p, double* phi_c,
                                               const double* phi_cp, double* phi_f, const double* phi_fp, int rwm) {
    bool ok = false;
    if (j < n) {
        const uint4 x = philox(make_uint4(0u, (uint32_t)j, event, (uint32_t)kPurposePcnU), seed);
        const double U = 1.0 - u53(x.x, x.y);
        const double t_old = target_potential(beta, zeta, phi_c[j], zeta < 0.0 ? 0.0 : phi_f[j]);
        const double t_new = target_potential(beta, zeta, phi_cp[j], zeta < 0.0 ? 0.0 : phi_fp[j]);
        double log_prior = 0.0;   // random walk: log mu0(theta') - log mu0(theta), mu0 = N(0, I)
        if (rwm) {
            double sn = 0.0, so = 0.0;
            for (int k = 0; k < K; ++k) {
                const double a = theta_p[(size_t)j * K + k], b = theta[(size_t)j * K + k];
                sn += a * a;
                so += b * b;
            }
            log_prior = -0.5 * (sn - so);
        }
        ok = log(U) < -(t_new - t_old) + log_prior;
        if (ok) {
            for (int k = 0; k < K; ++k) theta[(size_t)j * K + k] = theta_p[(size_t)j * K + k];
            phi_c[j] = phi_cp[j];
            if (zeta >= 0.0) phi_f[j] = phi_fp[j];
        }
    }
    return ok;
}

__global__ void pcn_accept_kernel(int n, int K, double beta, const double* beta_p, double zeta, const double* zeta_p,
                                  uint32_t event, uint64_t seed, double* theta, const double* theta_p, double* phi_c,
                                  const double* phi_cp, double* phi_f, const double* phi_fp,
                                  unsigned long long* n_acc, int rwm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (beta_p) beta = *beta_p;
    if (zeta_p) zeta = *zeta_p;
    const bool ok = pcn_accept_one(j, n, K, beta, zeta, event, seed, theta, theta_p, phi_c, phi_cp, phi_f, phi_fp, rwm);
    const unsigned ballot = __ballot_sync(0xffffffffu, ok);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(n_acc, (unsigned long long)__popc(ballot));
}

// many problems' acceptances (64-thread blocks, a contiguous block range per problem); beta and
// zeta read from the device where a pointer is given (the value an increment search left there)
__global__ void pcn_accept_multi_kernel(const __grid_constant__ AccTasks T) {
    const int p = task_of_block(T.start, T.count);
    const AccTask& k = T.t[p];
    const int j = (int)(blockIdx.x - (unsigned)T.start[p]) * blockDim.x + threadIdx.x;
    const double beta = k.beta_p ? *k.beta_p : k.beta;
    const double zeta = k.zeta_p ? *k.zeta_p : k.zeta;
    const bool ok = pcn_accept_one(j, k.n, k.K, beta, zeta, k.event, k.seed, k.theta, k.theta_p, k.phi_c, k.phi_cp,
                                   k.phi_f, k.phi_fp, k.rwm);
    const unsigned ballot = __ballot_sync(0xffffffffu, ok);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(k.n_acc, (unsigned long long)__popc(ballot));
}

// ---- delayed acceptance (Christen & Fox 2005) ----------------------------------------------------
// stage 1 on the surrogate potentials: pass with probability min(1, exp(-(t~(theta') - t~(theta))));
// the survivors are then compacted in particle order (deterministic: the exact solves, and the
// training pairs they add to the surrogate's set, come in the same order on every run)
// (random walk, rwm != 0: the prior ratio of N(0, I) enters stage 1; stage 2 divides the exact
// target ratio by the surrogate one, in which the prior ratio cancels)
__global__ void da_stage1_kernel(int n, int K, double beta, double zeta, uint32_t event, uint64_t seed,
                                 const double* ps_c, const double* ps_f, const double* psp_c, const double* psp_f,
                                 const double* theta, const double* theta_p, int rwm, int* pass) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint4 x = philox(make_uint4(0u, (uint32_t)j, event, (uint32_t)kPurposeDaU), seed);
    const double U = 1.0 - u53(x.x, x.y);
    const bool br = zeta >= 0.0;
    const double t_old = target_potential(beta, zeta, ps_c[j], br ? ps_f[j] : 0.0);
    const double t_new = target_potential(beta, zeta, psp_c[j], br ? psp_f[j] : 0.0);
    double log_prior = 0.0;
    if (rwm) {
        double sn = 0.0, so = 0.0;
        for (int k = 0; k < K; ++k) {
            const double a = theta_p[(size_t)j * K + k], b = theta[(size_t)j * K + k];
            sn += a * a;
            so += b * b;
        }
        log_prior = -0.5 * (sn - so);
    }
    pass[j] = log(U) < -(t_new - t_old) + log_prior;
}

// surv_idx = the indices j with pass[j] set, increasing; *n_surv = their number (one block of
// 1024 threads: warp ballots, warp totals scanned by warp 0, a running base per chunk)
__global__ void __launch_bounds__(1024) compact_kernel(const int* pass, int n, int* surv_idx, int* n_surv) {
    __shared__ int warp_off[32];
    __shared__ int base_s, total_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) base_s = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int j = base + tid;
        const bool f = j < n && pass[j];
        const unsigned ballot = __ballot_sync(0xffffffffu, f);
        if (lane == 0) warp_off[wid] = __popc(ballot);
        __syncthreads();
        if (wid == 0) {
            const int c = warp_off[lane];
            int incl = c;
            for (int off = 1; off < 32; off <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += u;
            }
            warp_off[lane] = incl - c;          // exclusive offset of each warp
            if (lane == 31) total_s = incl;
        }
        __syncthreads();
        if (f) surv_idx[base_s + warp_off[wid] + __popc(ballot & ((1u << lane) - 1u))] = j;
        __syncthreads();
        if (tid == 0) base_s += total_s;
        __syncthreads();
    }
    if (tid == 0) *n_surv = base_s;
}

// rows dst[i] = src[idx[i]] (K doubles) for i < *n_rows (grid over nmax rows)
__global__ void gather_rows_kernel(const int* idx, const int* n_rows, int nmax, int K, const double* src,
                                   double* dst) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nmax * K) return;
    const int i = (int)(t / K), k = (int)(t - (long long)i * K);
    if (i < *n_rows) dst[t] = src[(size_t)idx[i] * K + k];
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

__global__ void count_bad_multi_kernel(const __grid_constant__ BadTasks T) {
    const int p = task_of_block(T.start, T.count);
    const BadTask& k = T.t[p];
    const int i = (int)(blockIdx.x - (unsigned)T.start[p]) * blockDim.x + threadIdx.x;
    const bool b = i < k.n && k.iters[i] < 0;
    const unsigned ballot = __ballot_sync(0xffffffffu, b);
    if ((threadIdx.x & 31) == 0 && ballot) atomicAdd(k.bad, (unsigned)__popc(ballot));
}

// zero words[i] words at ptr[i] (barrier counters, error flags, accept counters of many problems)
__global__ void zero_words_kernel(const __grid_constant__ ZeroList Z) {
    for (int i = threadIdx.x; i < Z.count; i += blockDim.x)
        for (int w = 0; w < Z.words[i]; ++w) Z.ptr[i][w] = 0u;
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

// ---- covariance-shaped random walk (not in the paper) ----------------------------------------
// The population mean (one block per coordinate, fixed-order block sum).
__global__ void pop_mean_kernel(const double* theta, int n, int K, double* mean) {
    __shared__ double sh[32];
    const int k = blockIdx.x;
    double m[1] = {0.0};
    for (int j = threadIdx.x; j < n; j += blockDim.x) m[0] += theta[(size_t)j * K + k];
    block_reduce_sum<1>(m, sh);
    if (threadIdx.x == 0) mean[k] = m[0] / n;
}

// Partial sums of (theta_j - mean)(theta_j - mean)^T over chunks of kCovRows particles: block
// (tile pair, chunk) sums its rows in order for a 16 x 16 tile (a-tile <= b-tile) of the upper
// triangle into part[chunk][a][b].
constexpr int kCovTile = 16, kCovRows = 1024;
__global__ void __launch_bounds__(256) pop_cov_partial_kernel(const double* theta, int n, int K, const double* mean,
                                                              double* part) {
    __shared__ double ta[32][kCovTile + 1], tb[32][kCovTile + 1];
    const int nt = (K + kCovTile - 1) / kCovTile;
    int pair = blockIdx.x, ai = 0;   // pair index -> (ai, bi) with ai <= bi
    while (pair >= nt - ai) {
        pair -= nt - ai;
        ++ai;
    }
    const int bi = ai + pair;
    const int chunk = blockIdx.y;
    const int j0 = chunk * kCovRows, j1 = min(n, j0 + kCovRows);
    const int tx = threadIdx.x % kCovTile, ty = threadIdx.x / kCovTile;   // entry (a0 + ty, b0 + tx)
    const int a0 = ai * kCovTile, b0 = bi * kCovTile;
    double acc = 0.0;
    for (int jb = j0; jb < j1; jb += 32) {
        // stage 32 rows of both tiles' coordinates, centred
        for (int q = threadIdx.x; q < 32 * kCovTile; q += 256) {
            const int r = q / kCovTile, c = q % kCovTile, j = jb + r;
            const int ka = a0 + c, kb = b0 + c;
            ta[r][c] = (j < j1 && ka < K) ? theta[(size_t)j * K + ka] - mean[ka] : 0.0;
            tb[r][c] = (j < j1 && kb < K) ? theta[(size_t)j * K + kb] - mean[kb] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) acc = fma(ta[r][ty], tb[r][tx], acc);
        __syncthreads();
    }
    const int a = a0 + ty, b = b0 + tx;
    if (a < K && b < K && a <= b) part[((size_t)chunk * K + a) * K + b] = acc;
}

// C[a][b] = C[b][a] = (sum of the chunks' partials in chunk order) / n, for a <= b
__global__ void pop_cov_finish_kernel(const double* part, int chunks, int n, int K, double* cov) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)K * K) return;
    const int a = (int)(t / K), b = (int)(t - (long long)a * K);
    if (a > b) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[((size_t)c * K + a) * K + b];
    s /= n;
    cov[(size_t)a * K + b] = s;
    cov[(size_t)b * K + a] = s;
}

// theta'_j = theta_j + s L xi_j, xi_j read from and theta'_j written to out (row j): one warp per
// particle, the row of xi staged in shared memory, lane k sums L[k][m] xi[m] for m <= k in order
constexpr int kStepWarps = 4;
__global__ void __launch_bounds__(32 * kStepWarps) cov_step_kernel(const double* theta, double* out,
                                                                   const double* L, int n, int K, double s) {
    extern __shared__ double xs[];   // [kStepWarps][K]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * kStepWarps + w;
    if (j >= n) return;              // whole warps leave together
    double* x = xs + (size_t)w * K;
    for (int k = lane; k < K; k += 32) x[k] = out[(size_t)j * K + k];
    __syncwarp();
    for (int k = lane; k < K; k += 32) {
        const double* Lk = L + (size_t)k * K;
        double acc = 0.0;
        for (int m = 0; m <= k; ++m) acc = fma(Lk[m], x[m], acc);
        out[(size_t)j * K + k] = fma(s, acc, theta[(size_t)j * K + k]);
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

int inc_blocks(int n) { return std::min(kIncMaxBlocks, std::max(1, (n + 63) / 64)); }

cudaError_t inc_search_launch(const double* a, int n, double dmax, double tau, double eps, int max_iter, double base,
                              double top, IncWork& w, cudaStream_t st) {
    const int nb = inc_blocks(n);
    cudaError_t e = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st);   // barrier counter, error flag
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a,        (void*)&n,    (void*)&dmax, (void*)&tau, (void*)&eps,
                    (void*)&max_iter, (void*)&base, (void*)&top,  (void*)&w};
    e = cudaLaunchCooperativeKernel((const void*)inc_search_kernel, dim3(nb), dim3(kIncThreads), args, 0, st);
    count_launches(1);
    return e;
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

cudaError_t resample_gather_launch(const double* a, int n, const IncState* state, uint32_t event, uint64_t seed,
                                   int K, const double* th_in, double* th_out, const double* p0_in, double* p0_out,
                                   const double* p1_in, double* p1_out, double* cdf, int* anc, IncWork& w,
                                   unsigned* distinct, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    // one block per 32 particles (up to kIncMaxBlocks): the searches and the row gather are
    // latency-bound, so they want many warps in flight
    const int nb = std::min(kIncMaxBlocks, std::max(1, (n + 31) / 32));
    cudaError_t e = cudaMemsetAsync(w.bar, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    double* btot = w.partials;   // the search is finished: its scratch is free
    void* args[] = {(void*)&a,     (void*)&n,      (void*)&state,  (void*)&event, (void*)&seed, (void*)&K,
                    (void*)&th_in, (void*)&th_out, (void*)&p0_in,  (void*)&p0_out, (void*)&p1_in,
                    (void*)&p1_out, (void*)&cdf,   (void*)&anc,    (void*)&btot,  (void*)&w.bar, (void*)&w.err,
                    (void*)&distinct};
    e = cudaLaunchCooperativeKernel((const void*)resample_gather_kernel, dim3(nb), dim3(kRsThreads), args, 0, st);
    count_launches(1);
    return e;
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

cudaError_t pcn_accept_launch(int n, int K, double beta, const double* beta_p, double zeta, const double* zeta_p,
                              uint32_t event, uint64_t seed, double* theta, const double* theta_p, double* phi_c,
                              const double* phi_cp, double* phi_f, const double* phi_fp, unsigned long long* n_acc,
                              int rwm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    // 64-thread blocks: the FP64 work (log U, target potentials) spread over many SMs
    pcn_accept_kernel<<<grid_for(n, 64), 64, 0, st>>>(n, K, beta, beta_p, zeta, zeta_p, event, seed, theta, theta_p,
                                                      phi_c, phi_cp, phi_f, phi_fp, n_acc, rwm);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t da_stage1_launch(int n, int K, double beta, double zeta, uint32_t event, uint64_t seed, const double* ps_c,
                             const double* ps_f, const double* psp_c, const double* psp_f, const double* theta,
                             const double* theta_p, int rwm, int* pass, int* surv_idx, int* n_surv, double* theta_s,
                             cudaStream_t st) {
    if (n <= 0) return cudaMemsetAsync(n_surv, 0, sizeof(int), st);
    da_stage1_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, K, beta, zeta, event, seed, ps_c, ps_f, psp_c, psp_f, theta,
                                                       theta_p, rwm, pass);
    compact_kernel<<<1, 1024, 0, st>>>(pass, n, surv_idx, n_surv);
    gather_rows_kernel<<<grid_for((long long)n * K, 256), 256, 0, st>>>(surv_idx, n_surv, n, K, theta_p, theta_s);
    count_launches(3);
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

// ---- multi-problem launchers -------------------------------------------------------------------
int rs_blocks(int n) { return std::min(kIncMaxBlocks, std::max(1, (n + 31) / 32)); }

namespace {

// co-resident blocks of a cooperative kernel on this device
int coop_capacity(const void* kern, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    return std::max(1, sms * per_sm);
}

// split tasks into launches of at most kMaxTasks tasks and `cap` blocks (blocks_of(task) each) and
// call launch(list) for each
template <typename Task, typename BlocksOf, typename Launch>
cudaError_t for_task_lists(const std::vector<Task>& tasks, int cap, BlocksOf blocks_of, Launch launch) {
    size_t i = 0;
    while (i < tasks.size()) {
        TaskList<Task> L;
        L.count = 0;
        int blocks = 0;
        while (i < tasks.size() && L.count < kMaxTasks) {
            const int b = blocks_of(tasks[i]);
            if (L.count > 0 && blocks + b > cap) break;
            L.t[L.count] = tasks[i];
            L.start[L.count] = blocks;
            blocks += b;
            ++L.count;
            ++i;
        }
        L.start[L.count] = blocks;
        if (blocks > 0) {
            cudaError_t e = launch(L, blocks);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t zero_bars(const IncTasks& L, cudaStream_t st) {
    std::vector<std::pair<unsigned*, int>> z;
    for (int i = 0; i < L.count; ++i) z.push_back({L.t[i].w.bar, 2});
    return zero_words_launch(z, st);
}

}  // namespace

cudaError_t zero_words_launch(const std::vector<std::pair<unsigned*, int>>& list, cudaStream_t st) {
    for (size_t i = 0; i < list.size(); i += 2 * kMaxTasks) {
        ZeroList Z;
        Z.count = 0;
        for (size_t k = i; k < list.size() && Z.count < 2 * kMaxTasks; ++k) {
            Z.ptr[Z.count] = list[k].first;
            Z.words[Z.count] = list[k].second;
            ++Z.count;
        }
        zero_words_kernel<<<1, 128, 0, st>>>(Z);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t inc_search_multi_launch(const std::vector<IncTask>& tasks, cudaStream_t st) {
    static int cap = 0;
    if (!cap) cap = coop_capacity((const void*)inc_search_multi_kernel, kIncThreads);
    return for_task_lists(tasks, cap, [](const IncTask& t) { return inc_blocks(t.n); },
                          [&](const IncTasks& L, int blocks) {
                              cudaError_t e = zero_bars(L, st);
                              if (e != cudaSuccess) return e;
                              void* args[] = {(void*)&L};
                              e = cudaLaunchCooperativeKernel((const void*)inc_search_multi_kernel, dim3(blocks),
                                                              dim3(kIncThreads), args, 0, st);
                              count_launches(1);
                              return e;
                          });
}

cudaError_t resample_gather_multi_launch(const std::vector<RsTask>& tasks, cudaStream_t st) {
    static int cap = 0;
    if (!cap) cap = coop_capacity((const void*)resample_gather_multi_kernel, kRsThreads);
    return for_task_lists(tasks, cap, [](const RsTask& t) { return rs_blocks(t.n); },
                          [&](const RsTasks& L, int blocks) {
                              std::vector<std::pair<unsigned*, int>> z;
                              for (int i = 0; i < L.count; ++i) z.push_back({L.t[i].bar, 2});
                              cudaError_t e = zero_words_launch(z, st);
                              if (e != cudaSuccess) return e;
                              void* args[] = {(void*)&L};
                              e = cudaLaunchCooperativeKernel((const void*)resample_gather_multi_kernel, dim3(blocks),
                                                              dim3(kRsThreads), args, 0, st);
                              count_launches(1);
                              return e;
                          });
}

cudaError_t normals_multi_launch(const std::vector<NormTask>& tasks, cudaStream_t st) {
    return for_task_lists(tasks, 1 << 30, [](const NormTask& t) { return grid_for((long long)t.J * ((t.K + 1) / 2), 256); },
                          [&](const NormTasks& L, int blocks) {
                              normals_multi_kernel<<<blocks, 256, 0, st>>>(L);
                              count_launches(1);
                              return cudaGetLastError();
                          });
}

cudaError_t pcn_accept_multi_launch(const std::vector<AccTask>& tasks, cudaStream_t st) {
    return for_task_lists(tasks, 1 << 30, [](const AccTask& t) { return grid_for(t.n, 64); },
                          [&](const AccTasks& L, int blocks) {
                              pcn_accept_multi_kernel<<<blocks, 64, 0, st>>>(L);
                              count_launches(1);
                              return cudaGetLastError();
                          });
}

cudaError_t lu_increment_multi_launch(const std::vector<LuTask>& tasks, cudaStream_t st) {
    return for_task_lists(tasks, 1 << 30, [](const LuTask& t) { return grid_for(t.n, 256); },
                          [&](const LuTasks& L, int blocks) {
                              lu_increment_multi_kernel<<<blocks, 256, 0, st>>>(L);
                              count_launches(1);
                              return cudaGetLastError();
                          });
}

cudaError_t cv_lu_multi_launch(const std::vector<CvTask>& tasks, cudaStream_t st) {
    return for_task_lists(tasks, 1 << 30, [](const CvTask&) { return 1; },
                          [&](const CvTasks& L, int blocks) {
                              cv_lu_multi_kernel<<<blocks, 256, 0, st>>>(L);
                              count_launches(1);
                              return cudaGetLastError();
                          });
}

cudaError_t count_bad_multi_launch(const std::vector<BadTask>& tasks, cudaStream_t st) {
    return for_task_lists(tasks, 1 << 30, [](const BadTask& t) { return grid_for(t.n, 256); },
                          [&](const BadTasks& L, int blocks) {
                              count_bad_multi_kernel<<<blocks, 256, 0, st>>>(L);
                              count_launches(1);
                              return cudaGetLastError();
                          });
}

// population covariance of theta (n x K) into cov (K x K, symmetric); mean (K) and part
// (pop_cov_partial_doubles(n, K)) are scratch
size_t pop_cov_partial_doubles(int n, int K) { return (size_t)((n + kCovRows - 1) / kCovRows) * K * K; }

cudaError_t pop_cov_launch(const double* theta, int n, int K, double* mean, double* part, double* cov, cudaStream_t st) {
    if (n <= 0 || K <= 0) return cudaSuccess;
    pop_mean_kernel<<<K, 256, 0, st>>>(theta, n, K, mean);
    const int nt = (K + kCovTile - 1) / kCovTile, chunks = (n + kCovRows - 1) / kCovRows;
    pop_cov_partial_kernel<<<dim3(nt * (nt + 1) / 2, chunks), 256, 0, st>>>(theta, n, K, mean, part);
    pop_cov_finish_kernel<<<grid_for((long long)K * K, 256), 256, 0, st>>>(part, chunks, n, K, cov);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t cov_step_launch(const double* theta, double* out, const double* L, int n, int K, double s, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const size_t smem = (size_t)kStepWarps * K * sizeof(double);
    cov_step_kernel<<<(n + kStepWarps - 1) / kStepWarps, 32 * kStepWarps, smem, st>>>(theta, out, L, n, K, s);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t moments_launch(const double* theta, int n, int K, double* mean, double* var, cudaStream_t st) {
    moments_kernel<<<K, 256, 0, st>>>(theta, n, K, mean, var);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace mls2mc
