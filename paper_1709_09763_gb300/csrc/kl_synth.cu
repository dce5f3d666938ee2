// KL synthesis on the tensor cores (mixed path): kappa[j][e] = exp(sum_k theta_jk Psi_ke)
// (Sec. 5, Eq. truncKL, kappa = exp(u)).
//
// The contraction particles x K by K x triangles runs as one BF16 GEMM with FP32 accumulation.
// To keep u at FP32 accuracy, theta and Psi are each split into three BF16 pieces
// (x = x1 + x2 + x3, each piece the BF16 rounding of what the previous ones left), and the six
// cross products whose size is above 2^-24 relative -- (1,1), (1,2), (2,1), (2,2), (1,3), (3,1) --
// are concatenated along K: A' = [t1 t1 t2 t2 t1 t3], B' = [P1 P2 P1 P2 P3 P1], K' = 6K (padded to
// a multiple of 8 with zeros). The epilogue applies exp and writes kappa as FP32 [n][E], which the
// solve kernel reads instead of forming u itself.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <cstdint>
#include <vector>

#include "handle.h"
#include "umma_gemm.h"

namespace mls2mc {

namespace {

__global__ void theta_split_kernel(const double* theta, int n, int K, int Kp, __nv_bfloat16* out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * Kp) return;
    const int j = (int)(t / Kp), c = (int)(t - (long long)j * Kp);
    const int blk = c / K, k = c - blk * K;
    float v = 0.0f;
    if (blk < 6) {
        // split of theta rounded to FP32 (24 bits, all that three BF16 pieces carry); each remainder
        // is exact in FP32, so no FP64 arithmetic is needed
        const float x = (float)theta[(size_t)j * K + k];
        const __nv_bfloat16 p1 = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(p1);
        const __nv_bfloat16 p2 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(p2);
        const __nv_bfloat16 p3 = __float2bfloat16_rn(r2);
        // A' blocks: t1 t1 t2 t2 t1 t3
        const __nv_bfloat16 sel[6] = {p1, p1, p2, p2, p1, p3};
        out[t] = sel[blk];
        return;
    }
    out[t] = __float2bfloat16_rn(v);
}

uint16_t bf16_bits_host(double x) {
    const __nv_bfloat16 b = __float2bfloat16_rn((float)x);
    uint16_t u;
    std::memcpy(&u, &b, 2);
    return u;
}

double bf16_value_host(uint16_t u) {
    uint32_t w = (uint32_t)u << 16;
    float f;
    std::memcpy(&f, &w, 4);
    return (double)f;
}

}  // namespace

int kl_split_width(int K) { return (6 * K + 7) / 8 * 8; }

// B' = [P1 P2 P1 P2 P3 P1] as BF16 bits, [E][Kp] (K-major rows, one per triangle)
std::vector<uint16_t> kl_split_table(const std::vector<double>& psi, int K, int E) {
    const int Kp = kl_split_width(K);
    std::vector<uint16_t> out((size_t)E * Kp, 0);
    for (int e = 0; e < E; ++e)
        for (int k = 0; k < K; ++k) {
            const double x = psi[(size_t)k * E + e];
            const uint16_t p1 = bf16_bits_host(x);
            const double r1 = x - bf16_value_host(p1);
            const uint16_t p2 = bf16_bits_host(r1);
            const double r2 = r1 - bf16_value_host(p2);
            const uint16_t p3 = bf16_bits_host(r2);
            const uint16_t sel[6] = {p1, p2, p1, p2, p3, p1};
            for (int b = 0; b < 6; ++b) out[(size_t)e * Kp + b * K + k] = sel[b];
        }
    return out;
}

int Handle::synth_kappa(int level, int n, const double* theta, cudaStream_t st) {
    const Level& L = levels[level];
    const int E = 2 * L.N * L.N, Kp = kl_split_width(K);
    const size_t need_k = (size_t)n * E, need_t = (size_t)n * Kp;
    if (need_k > synth_kappa_cap || need_t > synth_theta_cap) {
        cudaFree(synth_kappa_buf);
        cudaFree(synth_theta_buf);
        synth_kappa_buf = nullptr;
        synth_theta_buf = nullptr;
        synth_kappa_cap = synth_theta_cap = 0;
        cudaError_t e = cudaMalloc((void**)&synth_kappa_buf, need_k * 4);
        if (e == cudaSuccess) e = cudaMalloc((void**)&synth_theta_buf, need_t * 2);
        if (e != cudaSuccess) return fail(SMC_ENOMEM, "synthesis buffers for %d particles: %s", n, cudaGetErrorString(e));
        synth_kappa_cap = need_k;
        synth_theta_cap = need_t;
    }
    if (!synth_err) {
        cudaError_t e = cudaMalloc((void**)&synth_err, 4);
        if (e == cudaSuccess) e = cudaMemset(synth_err, 0, 4);
        if (e != cudaSuccess) return fail(SMC_ENOMEM, "synthesis flag");
    }
    const long long work = (long long)n * Kp;
    theta_split_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(theta, n, K, Kp,
                                                                 reinterpret_cast<__nv_bfloat16*>(synth_theta_buf));
    count_launches(1);
    GemmEpi epi;
    epi.kind = kEpiExp;
    epi.out_f32 = synth_kappa_buf;
    epi.ld_out = E;
    cudaError_t e = umma_gemm(synth_theta_buf, Kp, L.psi_split, Kp, n, E, Kp, epi, synth_err, st);
    if (e != cudaSuccess) return cuda_fail(e, "KL synthesis GEMM");
    return SMC_OK;
}

}  // namespace mls2mc
