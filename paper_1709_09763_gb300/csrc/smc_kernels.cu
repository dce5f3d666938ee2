// Sampler kernels (FP64): linear test forward model; more below as they are added.
#include <cuda_runtime.h>

#include "handle.h"

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

}  // namespace

cudaError_t linear_eval_launch(const double* A, int n, int K, int n_obs, const double* theta, const double* y,
                               double inv_sigma2, double* G, double* Phi, int* iters, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)(((size_t)n * 32 + threads - 1) / threads);
    linear_eval_kernel<<<blocks, threads, 0, st>>>(A, n, K, n_obs, theta, y, inv_sigma2, G, Phi, iters);
    return cudaGetLastError();
}

}  // namespace mls2mc
