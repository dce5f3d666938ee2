// Surrogate network theta -> G_l(theta), one per level: training and inference on the device.
//
// The paper has no surrogate. The library adds one as the first stage of a delayed-acceptance
// pCN move (Christen & Fox 2005): only proposals that pass the cheap surrogate screen are solved
// exactly, and the exact potential still decides every accepted move, so the target is unchanged.
//
// Network: K inputs -> 4 hidden layers of 256 (exact GELU z Phi(z)) -> n_obs outputs (padded to a
// multiple of 16 with zero rows). It predicts standardised observations z = (G - mu) / s with mu,
// s the per-output mean and standard deviation of the training targets; the loss is the mean
// squared error over batch and outputs. Weights and activations are BF16, accumulation FP32 (the
// tcgen05 GEMM), master weights and Adam moments FP32 (Kingma & Ba 2015). Layer l stores its
// weights W[out][in] and a transposed copy Wt[in][out] so every product of the forward and
// backward passes is a K-major GEMM:
//   forward      X_{l+1} = GELU(X_l W_l^T + b_l)          A = X_l,     B = W_l
//   input grad   dZ_{l-1} = (dZ_l W_l) * GELU'(pre_{l-1})  A = dZ_l,    B = Wt_l
//   weight grad  dW_l = dZ_l^T X_l                          A = dZ_l^T,  B = X_l^T (transposed copies
//                                                           written by the epilogues)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "handle.h"
#include "mlp.h"
#include "smc_device.h"
#include "umma_gemm.h"

namespace mls2mc {

namespace {

__device__ __forceinline__ uint4 philox_m(uint4 c, uint64_t seed) {
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

// X0 = bf16(theta) [B][Kp] (zero padded) and optionally its transpose X0t [Kp][ldt]
__global__ void input_kernel(const double* theta, int B, int K, int Kp, __nv_bfloat16* X, __nv_bfloat16* Xt,
                             int ldt) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B * Kp) return;
    const int b = (int)(t / Kp), k = (int)(t - (long long)b * Kp);
    const __nv_bfloat16 v = __float2bfloat16_rn(k < K ? (float)theta[(size_t)b * K + k] : 0.0f);
    X[t] = v;
    if (Xt) Xt[(size_t)k * ldt + b] = v;
}

// G = mu + s z and Phi~ = 1/2 sum ((y - G)/sigma)^2, one warp per row
__global__ void predict_kernel(const float* Z, int B, int NOp, int n_obs, const float* mu, const float* sd,
                               const double* y, double inv_sigma2, double* G, double* phi) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= B) return;
    double m = 0.0;
    for (int o = lane; o < n_obs; o += 32) {
        const double g = (double)mu[o] + (double)sd[o] * (double)Z[(size_t)row * NOp + o];
        if (G) G[(size_t)row * n_obs + o] = g;
        const double r = y[o] - g;
        m += r * r;
    }
    for (int off = 16; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
    if (lane == 0 && phi) phi[row] = 0.5 * m * inv_sigma2;
}

// minibatch: rows idx of the training ring; targets standardised and padded
__global__ void batch_kernel(const double* ring_th, const double* ring_G, const int* idx, int B, int K, int n_obs,
                             int NOp, const float* mu, const float* sd, double* th_out, float* tgt) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = K > NOp ? K : NOp;
    if (t >= (long long)B * W) return;
    const int b = (int)(t / W), c = (int)(t - (long long)b * W);
    const int src = idx[b];
    if (c < K) th_out[(size_t)b * K + c] = ring_th[(size_t)src * K + c];
    if (c < NOp)
        tgt[(size_t)b * NOp + c] =
            c < n_obs ? (float)((ring_G[(size_t)src * n_obs + c] - (double)mu[c]) / (double)sd[c]) : 0.0f;
}

__global__ void sample_indices_kernel(int* idx, int B, int count, uint32_t step, uint32_t level, uint64_t seed) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint4 x = philox_m(make_uint4((uint32_t)b, step, level, 6u), seed);
    idx[b] = (int)(((uint64_t)x.x * (uint64_t)count) >> 32);
}

// dZ = 2 (Z - z) / (B n_obs) on real outputs, 0 on padding; bf16 row-major and transposed;
// per-block partial sums of squared errors
__global__ void loss_grad_kernel(const float* Z, const float* tgt, int B, int NOp, int n_obs, __nv_bfloat16* dZ,
                                 __nv_bfloat16* dZt, int ldt, double* partial) {
    __shared__ double sh[32];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double e2 = 0.0;
    if (t < (long long)B * NOp) {
        const int b = (int)(t / NOp), c = (int)(t - (long long)b * NOp);
        float g = 0.0f;
        if (c < n_obs) {
            const float d = Z[t] - tgt[t];
            e2 = (double)d * d;
            g = 2.0f * d / ((float)B * (float)n_obs);
        }
        const __nv_bfloat16 v = __float2bfloat16_rn(g);
        dZ[t] = v;
        dZt[(size_t)c * ldt + b] = v;
    }
    for (int off = 16; off > 0; off >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = e2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        partial[blockIdx.x] = s;
    }
}

// bias gradient: row sums of dZ^T [rows][ld] over the first B columns, one block of kRowsumThreads
// per row: each thread sums eight columns per 16-byte load (ld is a multiple of 8), then a fixed
// warp-shuffle and per-warp order (deterministic)
constexpr int kRowsumThreads = 256;
__global__ void __launch_bounds__(kRowsumThreads) rowsum_kernel(const __nv_bfloat16* Xt, int B, int ld, float* out) {
    __shared__ float sh[kRowsumThreads / 32];
    const __nv_bfloat16* x = Xt + (size_t)blockIdx.x * ld;
    const int B8 = B & ~7;
    float s = 0.0f;
    for (int b = threadIdx.x * 8; b < B8; b += kRowsumThreads * 8) {
        const uint4 u = *reinterpret_cast<const uint4*>(x + b);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(h[k]);
            s += f.x;
            s += f.y;
        }
    }
    for (int b = B8 + threadIdx.x; b < B; b += kRowsumThreads) s += __bfloat162float(x[b]);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < kRowsumThreads / 32; ++w) t += sh[w];
        out[blockIdx.x] = t;
    }
}

// the ten parameter tensors of one network (weights and biases of five layers) for one Adam launch
struct AdamSet {
    float* w[10];
    const float* g[10];
    float* m[10];
    float* v[10];
    __nv_bfloat16* wb[10];   // BF16 copy and its transpose [cols][ld_t] (weights only)
    __nv_bfloat16* wt[10];
    int cols[10];
    int ld_t[10];
    int start[11];           // element offsets of the tensors in the launch's index space
};

// one Adam step of every tensor of a network (Kingma & Ba 2015): element i of the launch belongs to
// the tensor whose [start, next start) holds it; per element the arithmetic of a single-tensor step
__global__ void adam_all_kernel(AdamSet a, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int gi_ = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi_ >= a.start[10]) return;
    int t = 0;
#pragma unroll
    for (int k = 1; k < 10; ++k) t += gi_ >= a.start[k];
    const int i = gi_ - a.start[t];
    float* w = a.w[t];
    float* m = a.m[t];
    float* v = a.v[t];
    const float gi = a.g[t][i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (a.wb[t]) {
        const __nv_bfloat16 h = __float2bfloat16_rn(wi);
        a.wb[t][i] = h;
        const int r = i / a.cols[t], c = i - r * a.cols[t];
        a.wt[t][(size_t)c * a.ld_t[t] + r] = h;
    }
}

__global__ void to_bf16_kernel(const float* w, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const __nv_bfloat16 h = __float2bfloat16_rn(w[i]);
    wb[i] = h;
    const int r = i / cols, c = i - r * cols;
    wt[(size_t)c * rows + r] = h;
}

// per-output mean and standard deviation of the ring's targets (FP64 sums), one block per output
__global__ void norm_kernel(const double* ring_G, int count, int n_obs, int NOp, float* mu, float* sd) {
    __shared__ double sh[2][32];
    const int o = blockIdx.x;
    if (o >= NOp) return;
    if (o >= n_obs) {
        if (threadIdx.x == 0) {
            mu[o] = 0.0f;
            sd[o] = 1.0f;
        }
        return;
    }
    double s1 = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const double g = ring_G[(size_t)i * n_obs + o];
        s1 += g;
        s2 += g * g;
    }
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = s1;
        sh[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
        const double m = a / count, var = b / count - m * m;
        mu[o] = (float)m;
        sd[o] = (float)(var > 1e-300 ? sqrt(var) : 1.0);
    }
}

__global__ void ring_append_kernel(double* ring_th, double* ring_G, int cap, int head, const double* th,
                                   const double* G, int n, int K, int n_obs) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int W = K + n_obs;
    if (t >= (long long)n * W) return;
    const int i = (int)(t / W), c = (int)(t - (long long)i * W);
    const int dst = (head + i) % cap;
    if (c < K) ring_th[(size_t)dst * K + c] = th[(size_t)i * K + c];
    else ring_G[(size_t)dst * n_obs + (c - K)] = G[(size_t)i * n_obs + (c - K)];
}

int grid_of(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ---- host side ---------------------------------------------------------------------------------
static int round_up(int x, int m) { return (x + m - 1) / m * m; }

// the ring of training pairs of a level (two buffers, nothing initialised: count says what is valid);
// collecting pairs needs nothing else, so a level whose screen is never used costs two allocations
int Handle::mlp_ring(int level) {
    if ((int)mlps.size() < (int)levels.size()) mlps.resize(levels.size());
    Mlp& S = mlps[level];
    if (S.ring_th) return SMC_OK;
    const int cap = std::max(4 * std::max(opts.J, 1), 8192);
    cudaError_t e = cudaMalloc((void**)&S.ring_th, (size_t)cap * K * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&S.ring_G, (size_t)cap * n_obs * 8);
    if (e != cudaSuccess) return fail(SMC_ENOMEM, "surrogate pair ring: %s", cudaGetErrorString(e));
    S.cap = cap;
    return SMC_OK;
}

// the network of a level: weights (He-normal from the library's Philox stream), Adam state,
// standardisation; set up on first training or prediction
int Handle::mlp_setup(int level) {
    RC_CHECK(mlp_ring(level));
    Mlp& S = mlps[level];
    if (S.ready) return SMC_OK;
    S.d[0] = round_up(K, 8);
    for (int l = 1; l <= 4; ++l) S.d[l] = kMlpWidth;
    S.d[5] = round_up(n_obs, 16);
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    for (int l = 0; l < 5; ++l) {
        const size_t n = (size_t)S.d[l + 1] * S.d[l];
        A((void**)&S.Wm[l], n * 4);
        A((void**)&S.mW[l], n * 4);
        A((void**)&S.vW[l], n * 4);
        A((void**)&S.gW[l], n * 4);
        A((void**)&S.W[l], n * 2);
        A((void**)&S.Wt[l], n * 2);
        A((void**)&S.bm[l], (size_t)S.d[l + 1] * 4);
        A((void**)&S.mb[l], (size_t)S.d[l + 1] * 4);
        A((void**)&S.vb[l], (size_t)S.d[l + 1] * 4);
        A((void**)&S.gb[l], (size_t)S.d[l + 1] * 4);
    }
    A((void**)&S.mu, (size_t)S.d[5] * 4);
    A((void**)&S.sd, (size_t)S.d[5] * 4);
    A((void**)&S.err, 4);
    if (e != cudaSuccess) return fail(SMC_ENOMEM, "surrogate buffers: %s", cudaGetErrorString(e));
    // He-normal initial weights from the library's Philox stream (purpose 7, event = level * 8 + layer)
    for (int l = 0; l < 5; ++l) {
        const int rows = S.d[l + 1], cols = S.d[l];
        double* tmp = nullptr;
        e = cudaMalloc((void**)&tmp, (size_t)rows * cols * 8);
        if (e != cudaSuccess) return fail(SMC_ENOMEM, "surrogate init");
        normals_launch(tmp, rows, cols, (uint32_t)(level * 8 + l), 7u, opts.seed, nullptr, 0.0, 0.0, stream);
        std::vector<double> h((size_t)rows * cols);
        cudaMemcpyAsync(h.data(), tmp, h.size() * 8, cudaMemcpyDeviceToHost, stream);
        e = cudaStreamSynchronize(stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate init");
        std::vector<float> w(h.size());
        const double sc = std::sqrt(2.0 / (l == 0 ? std::max(K, 1) : cols));
        for (size_t i = 0; i < h.size(); ++i) {
            const int r = (int)(i / cols), c = (int)(i % cols);
            const bool pad = (l == 0 && c >= K) || (l == 4 && r >= n_obs);
            w[i] = pad ? 0.0f : (float)(sc * h[i]);
        }
        cudaMemcpyAsync(S.Wm[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice, stream);
    }
    S.ready = true;
    S.t = 0;
    return mlp_sync_bf16(level);
}

int Handle::mlp_sync_bf16(int level) {
    Mlp& S = mlps[level];
    for (int l = 0; l < 5; ++l) {
        const int rows = S.d[l + 1], cols = S.d[l];
        to_bf16_kernel<<<grid_of((long long)rows * cols, 256), 256, 0, stream>>>(S.Wm[l], rows, cols, S.W[l], S.Wt[l]);
        count_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "surrogate weight copy");
}

int Handle::mlp_work(int B) {
    if (B <= mwork.cap) return SMC_OK;
    mwork.release();
    const int ldt = round_up(B, 8);
    const int dmax = std::max(kMlpWidth, std::max(round_up(K, 8), round_up(n_obs, 16)));
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    for (int l = 0; l < 6; ++l) {
        A((void**)&mwork.X[l], (size_t)B * dmax * 2);
        A((void**)&mwork.Xt[l], (size_t)dmax * ldt * 2);
    }
    for (int l = 0; l < 5; ++l) {
        A((void**)&mwork.pre[l], (size_t)B * dmax * 4);
        A((void**)&mwork.dZ[l], (size_t)B * dmax * 2);
        A((void**)&mwork.dZt[l], (size_t)dmax * ldt * 2);
    }
    A((void**)&mwork.Z, (size_t)B * dmax * 4);
    A((void**)&mwork.tgt, (size_t)B * dmax * 4);
    A((void**)&mwork.th, (size_t)B * K * 8);
    A((void**)&mwork.idx, (size_t)B * 4);
    A((void**)&mwork.partial, (size_t)grid_of((long long)B * dmax, 256) * 8);
    // up to 64 split-K slices of a dmax x dmax weight gradient
    const size_t sk = (size_t)64 * dmax * dmax;
    if (e == cudaSuccess) e = cudaMalloc((void**)&mwork.splitk, sk * 4);
    if (e == cudaSuccess) mwork.splitk_floats = sk;
    if (e != cudaSuccess) {
        mwork.release();
        return fail(SMC_ENOMEM, "surrogate work buffers for batch %d: %s", B, cudaGetErrorString(e));
    }
    mwork.cap = B;
    mwork.ldt = ldt;
    return SMC_OK;
}

void MlpWork::release() {
    for (auto& p : X) { cudaFree(p); p = nullptr; }
    for (auto& p : Xt) { cudaFree(p); p = nullptr; }
    for (auto& p : pre) { cudaFree(p); p = nullptr; }
    for (auto& p : dZ) { cudaFree(p); p = nullptr; }
    for (auto& p : dZt) { cudaFree(p); p = nullptr; }
    cudaFree(Z); cudaFree(tgt); cudaFree(th); cudaFree(idx); cudaFree(partial); cudaFree(splitk);
    Z = tgt = nullptr; th = nullptr; idx = nullptr; partial = nullptr; splitk = nullptr;
    splitk_floats = 0;
    cap = 0;
}

void Mlp::release() {
    for (int l = 0; l < 5; ++l) {
        for (void* p : {(void*)Wm[l], (void*)mW[l], (void*)vW[l], (void*)gW[l], (void*)W[l], (void*)Wt[l],
                        (void*)bm[l], (void*)mb[l], (void*)vb[l], (void*)gb[l]})
            cudaFree(p);
    }
    cudaFree(mu); cudaFree(sd); cudaFree(ring_th); cudaFree(ring_G); cudaFree(err);
}

// forward pass of B rows of theta (device FP64 [B][K]); training = keep activations for backward
int Handle::mlp_forward(int level, int B, const double* theta, bool training) {
    Mlp& S = mlps[level];
    RC_CHECK(mlp_work(B));
    const int ldt = mwork.ldt;
    input_kernel<<<grid_of((long long)B * S.d[0], 256), 256, 0, stream>>>(theta, B, K, S.d[0], mwork.X[0],
                                                                         training ? mwork.Xt[0] : nullptr, ldt);
    count_launches(1);
    for (int l = 0; l < 5; ++l) {
        GemmEpi epi;
        if (l < 4) {
            epi.kind = kEpiBiasGelu;
            epi.bias = S.bm[l];
            epi.pre = training ? mwork.pre[l] : nullptr;
            epi.ld_pre = S.d[l + 1];
            epi.act = mwork.X[l + 1];
            epi.ld_act = S.d[l + 1];
            epi.act_t = training ? mwork.Xt[l + 1] : nullptr;
            epi.ld_act_t = ldt;
        } else {
            epi.kind = kEpiStoreF32;
            epi.bias = S.bm[l];
            epi.out_f32 = mwork.Z;
            epi.ld_out = S.d[5];
        }
        cudaError_t e = umma_gemm(mwork.X[l], S.d[l], S.W[l], S.d[l], B, S.d[l + 1], S.d[l], epi, S.err, stream);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate forward GEMM");
    }
    return SMC_OK;
}

int Handle::mlp_predict(int level, int B, const double* theta, double* G, double* phi) {
    if (B <= 0) return SMC_OK;
    RC_CHECK(mlp_forward(level, B, theta, false));
    Mlp& S = mlps[level];
    predict_kernel<<<grid_of((long long)B * 32, 256), 256, 0, stream>>>(mwork.Z, B, S.d[5], n_obs, S.mu, S.sd, d_y,
                                                                        1.0 / (sigma * sigma), G, phi);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "surrogate prediction");
}

// one forward + backward on B rows (theta, standardised targets already in mwork.th / mwork.tgt);
// gradients land in S.gW / S.gb; returns the mean squared error
int Handle::mlp_backward(int level, int B, double* loss) {
    Mlp& S = mlps[level];
    const int ldt = mwork.ldt;
    RC_CHECK(mlp_forward(level, B, mwork.th, true));
    const int NOp = S.d[5];
    const int nb = grid_of((long long)B * NOp, 256);
    loss_grad_kernel<<<nb, 256, 0, stream>>>(mwork.Z, mwork.tgt, B, NOp, n_obs, mwork.dZ[4], mwork.dZt[4], ldt,
                                             mwork.partial);
    count_launches(1);
    for (int l = 4; l >= 0; --l) {
        // weight gradient dW_l = dZ_l^T X_l  (M = out, N = in, K = batch)
        GemmEpi ew;
        ew.kind = kEpiStoreF32;
        ew.out_f32 = S.gW[l];
        ew.ld_out = S.d[l];
        ew.ws = mwork.splitk;
        ew.ws_floats = mwork.splitk_floats;
        cudaError_t e = umma_gemm(mwork.dZt[l], ldt, mwork.Xt[l], ldt, S.d[l + 1], S.d[l], B, ew, S.err, stream);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate weight-gradient GEMM");
        rowsum_kernel<<<S.d[l + 1], kRowsumThreads, 0, stream>>>(mwork.dZt[l], B, ldt, S.gb[l]);
        count_launches(1);
        if (l > 0) {
            // input gradient through the GELU of layer l-1: dZ_{l-1} = (dZ_l W_l) * GELU'(pre_{l-1})
            GemmEpi ex;
            ex.kind = kEpiGeluBackward;
            ex.pre_in = mwork.pre[l - 1];
            ex.ld_pre = S.d[l];
            ex.act = mwork.dZ[l - 1];
            ex.ld_act = S.d[l];
            ex.act_t = mwork.dZt[l - 1];
            ex.ld_act_t = ldt;
            e = umma_gemm(mwork.dZ[l], S.d[l + 1], S.Wt[l], S.d[l + 1], B, S.d[l], S.d[l + 1], ex, S.err, stream);
            if (e != cudaSuccess) return cuda_fail(e, "surrogate input-gradient GEMM");
        }
    }
    if (loss) {
        std::vector<double> part((size_t)nb);
        cudaError_t e = cudaMemcpyAsync(part.data(), mwork.partial, (size_t)nb * 8, cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "surrogate loss");
        double s = 0.0;
        for (double v : part) s += v;
        *loss = s / ((double)B * n_obs);
    }
    return SMC_OK;
}

int Handle::mlp_adam(int level) {
    Mlp& S = mlps[level];
    S.t += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - std::pow(b1, (float)S.t), c2 = 1.0f - std::pow(b2, (float)S.t);
    AdamSet a;
    int off = 0;
    for (int l = 0; l < 5; ++l) {
        const int rows = S.d[l + 1], cols = S.d[l];
        const int tw = 2 * l, tb = 2 * l + 1;
        a.w[tw] = S.Wm[l], a.g[tw] = S.gW[l], a.m[tw] = S.mW[l], a.v[tw] = S.vW[l];
        a.wb[tw] = S.W[l], a.wt[tw] = S.Wt[l], a.cols[tw] = cols, a.ld_t[tw] = rows;
        a.start[tw] = off;
        off += rows * cols;
        a.w[tb] = S.bm[l], a.g[tb] = S.gb[l], a.m[tb] = S.mb[l], a.v[tb] = S.vb[l];
        a.wb[tb] = nullptr, a.wt[tb] = nullptr, a.cols[tb] = 1, a.ld_t[tb] = 0;
        a.start[tb] = off;
        off += rows;
    }
    a.start[10] = off;
    adam_all_kernel<<<grid_of(off, 256), 256, 0, stream>>>(a, mlp_lr, b1, b2, eps, c1, c2);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "surrogate Adam step");
}

int Handle::mlp_add_pairs(int level, int n, const double* theta, const double* G) {
    RC_CHECK(mlp_ring(level));
    Mlp& S = mlps[level];
    if (n <= 0) return SMC_OK;
    if (n > S.cap) {   // keep the most recent cap pairs
        theta += (size_t)(n - S.cap) * K;
        G += (size_t)(n - S.cap) * n_obs;
        n = S.cap;
    }
    ring_append_kernel<<<grid_of((long long)n * (K + n_obs), 256), 256, 0, stream>>>(S.ring_th, S.ring_G, S.cap,
                                                                                     S.head, theta, G, n, K, n_obs);
    count_launches(1);
    S.head = (S.head + n) % S.cap;
    S.count = std::min(S.cap, S.count + n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "surrogate pair append");
}

int Handle::mlp_train(int level, int steps, int batch, double* last_loss) {
    RC_CHECK(mlp_setup(level));
    Mlp& S = mlps[level];
    if (S.count <= 0) return fail(SMC_EINVAL, "no training pairs for level %d", level);
    if (!S.norm_set) {
        norm_kernel<<<S.d[5], 256, 0, stream>>>(S.ring_G, S.count, n_obs, S.d[5], S.mu, S.sd);
        count_launches(1);
        S.norm_set = true;
    }
    RC_CHECK(mlp_work(batch));
    double loss = 0.0;
    for (int s = 0; s < steps; ++s) {
        sample_indices_kernel<<<grid_of(batch, 256), 256, 0, stream>>>(mwork.idx, batch, S.count,
                                                                       (uint32_t)(S.t + 1), (uint32_t)level, opts.seed);
        const int W = std::max(K, S.d[5]);
        batch_kernel<<<grid_of((long long)batch * W, 256), 256, 0, stream>>>(S.ring_th, S.ring_G, mwork.idx, batch, K,
                                                                           n_obs, S.d[5], S.mu, S.sd, mwork.th,
                                                                           mwork.tgt);
        count_launches(2);
        RC_CHECK(mlp_backward(level, batch, (s == steps - 1) ? &loss : nullptr));
        RC_CHECK(mlp_adam(level));
    }
    int herr = 0;
    cudaError_t e = cudaMemcpyAsync(&herr, S.err, 4, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "surrogate training");
    if (herr) return fail(SMC_ETIMEOUT, "tensor-core GEMM wait timed out");
    if (last_loss) *last_loss = loss;
    return SMC_OK;
}

}  // namespace mls2mc

// ---- C ABI ---------------------------------------------------------------------------------
using namespace mls2mc;

namespace {
Handle* H(smc_handle* h) { return reinterpret_cast<Handle*>(h); }

int stage_in(Handle* h, const double* src, size_t count, double** dev) {
    *dev = nullptr;
    if (count == 0) return SMC_OK;
    cudaError_t e = cudaMalloc((void**)dev, count * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(*dev, src, count * 8, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "stage host array");
    return SMC_OK;
}
}  // namespace

extern "C" {

int smc_surrogate_add_pairs(smc_handle* hh, int level, int n, const double* theta, const double* G) {
    if (!hh || n < 0 || (n > 0 && (!theta || !G))) return SMC_EINVAL;
    Handle* h = H(hh);
    if (level < 0 || level >= (int)h->levels.size()) return h->fail(SMC_EINVAL, "level out of range");
    double *dt = nullptr, *dg = nullptr;
    int rc = stage_in(h, theta, (size_t)n * h->K, &dt);
    if (rc == SMC_OK) rc = stage_in(h, G, (size_t)n * h->n_obs, &dg);
    if (rc == SMC_OK) rc = h->mlp_add_pairs(level, n, dt, dg);
    cudaStreamSynchronize(h->stream);
    cudaFree(dt);
    cudaFree(dg);
    return rc;
}

int smc_surrogate_train(smc_handle* hh, int level, int steps, int batch, double* loss) {
    if (!hh || steps < 0 || batch < 1) return SMC_EINVAL;
    Handle* h = H(hh);
    if (level < 0 || level >= (int)h->levels.size()) return h->fail(SMC_EINVAL, "level out of range");
    return h->mlp_train(level, steps, batch, loss);
}

int smc_surrogate_predict(smc_handle* hh, int level, int n, const double* theta, double* G, double* phi) {
    if (!hh || n < 0 || (n > 0 && !theta)) return SMC_EINVAL;
    Handle* h = H(hh);
    if (level < 0 || level >= (int)h->levels.size()) return h->fail(SMC_EINVAL, "level out of range");
    if (n == 0) return SMC_OK;
    int rc = h->mlp_setup(level);
    if (rc != SMC_OK) return rc;
    double *dt = nullptr, *dg = nullptr, *dp = nullptr;
    rc = stage_in(h, theta, (size_t)n * h->K, &dt);
    cudaError_t e = cudaSuccess;
    if (rc == SMC_OK) {
        e = cudaMalloc((void**)&dg, (size_t)n * h->n_obs * 8);
        if (e == cudaSuccess) e = cudaMalloc((void**)&dp, (size_t)n * 8);
        if (e != cudaSuccess) rc = h->cuda_fail(e, "prediction buffers");
    }
    if (rc == SMC_OK) rc = h->mlp_predict(level, n, dt, dg, dp);
    if (rc == SMC_OK && G) e = cudaMemcpyAsync(G, dg, (size_t)n * h->n_obs * 8, cudaMemcpyDeviceToHost, h->stream);
    if (rc == SMC_OK && e == cudaSuccess && phi) e = cudaMemcpyAsync(phi, dp, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream);
    if (rc == SMC_OK && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (rc == SMC_OK && e != cudaSuccess) rc = h->cuda_fail(e, "surrogate prediction");
    cudaFree(dt);
    cudaFree(dg);
    cudaFree(dp);
    return rc;
}

// layout of the flat parameter arrays: for l = 0..4, W_l [d(l+1)][d(l)] then b_l [d(l+1)]
int smc_surrogate_dims(smc_handle* hh, int* dims6) {
    if (!hh || !dims6) return SMC_EINVAL;
    Handle* h = H(hh);
    const int d[6] = {(h->K + 7) / 8 * 8, kMlpWidth, kMlpWidth, kMlpWidth, kMlpWidth, (h->n_obs + 15) / 16 * 16};
    for (int i = 0; i < 6; ++i) dims6[i] = d[i];
    return SMC_OK;
}

int smc_surrogate_params(smc_handle* hh, int level, int direction, float* params, float* mu_sd) {
    if (!hh || !params) return SMC_EINVAL;
    Handle* h = H(hh);
    if (level < 0 || level >= (int)h->levels.size()) return h->fail(SMC_EINVAL, "level out of range");
    int rc = h->mlp_setup(level);
    if (rc != SMC_OK) return rc;
    Mlp& S = h->mlps[level];
    cudaMemcpyKind kind = direction ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < 5 && e == cudaSuccess; ++l) {
        const size_t nw = (size_t)S.d[l + 1] * S.d[l], nb = (size_t)S.d[l + 1];
        e = direction ? cudaMemcpyAsync(params + off, S.Wm[l], nw * 4, kind, h->stream)
                      : cudaMemcpyAsync(S.Wm[l], params + off, nw * 4, kind, h->stream);
        off += nw;
        if (e == cudaSuccess)
            e = direction ? cudaMemcpyAsync(params + off, S.bm[l], nb * 4, kind, h->stream)
                          : cudaMemcpyAsync(S.bm[l], params + off, nb * 4, kind, h->stream);
        off += nb;
    }
    if (e == cudaSuccess && mu_sd) {
        const size_t no = (size_t)S.d[5];
        if (direction) {
            e = cudaMemcpyAsync(mu_sd, S.mu, no * 4, kind, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(mu_sd + no, S.sd, no * 4, kind, h->stream);
        } else {
            e = cudaMemcpyAsync(S.mu, mu_sd, no * 4, kind, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(S.sd, mu_sd + no, no * 4, kind, h->stream);
            S.norm_set = true;
        }
    }
    if (e == cudaSuccess && !direction) {
        rc = h->mlp_sync_bf16(level);
        if (rc != SMC_OK) return rc;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "surrogate parameters");
    return SMC_OK;
}

int smc_surrogate_grads(smc_handle* hh, int level, int n, const double* theta, const double* G, float* grads,
                        double* loss) {
    if (!hh || n < 1 || !theta || !G || !grads) return SMC_EINVAL;
    Handle* h = H(hh);
    if (level < 0 || level >= (int)h->levels.size()) return h->fail(SMC_EINVAL, "level out of range");
    int rc = h->mlp_setup(level);
    if (rc != SMC_OK) return rc;
    Mlp& S = h->mlps[level];
    rc = h->mlp_work(n);
    if (rc != SMC_OK) return rc;
    // standardised targets computed on the host side of this test entry point from the set mu, sd
    std::vector<float> musd((size_t)2 * S.d[5]);
    cudaMemcpy(musd.data(), S.mu, (size_t)S.d[5] * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(musd.data() + S.d[5], S.sd, (size_t)S.d[5] * 4, cudaMemcpyDeviceToHost);
    std::vector<float> tgt((size_t)n * S.d[5], 0.0f);
    for (int i = 0; i < n; ++i)
        for (int o = 0; o < h->n_obs; ++o)
            tgt[(size_t)i * S.d[5] + o] = (float)((G[(size_t)i * h->n_obs + o] - musd[o]) / musd[S.d[5] + o]);
    cudaError_t e = cudaMemcpyAsync(h->mwork.th, theta, (size_t)n * h->K * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->mwork.tgt, tgt.data(), tgt.size() * 4, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "stage gradient inputs");
    rc = h->mlp_backward(level, n, loss);
    if (rc != SMC_OK) return rc;
    size_t off = 0;
    for (int l = 0; l < 5 && e == cudaSuccess; ++l) {
        const size_t nw = (size_t)S.d[l + 1] * S.d[l], nb = (size_t)S.d[l + 1];
        e = cudaMemcpyAsync(grads + off, S.gW[l], nw * 4, cudaMemcpyDeviceToHost, h->stream);
        off += nw;
        if (e == cudaSuccess) e = cudaMemcpyAsync(grads + off, S.gb[l], nb * 4, cudaMemcpyDeviceToHost, h->stream);
        off += nb;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "copy gradients");
    return SMC_OK;
}

}  // extern "C"
