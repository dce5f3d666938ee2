// KL synthesis on the tensor cores (mixed path): kappa[j][e] = exp(sum_k theta_jk Psi_ke)
// (Sec. 5, Eq. truncKL, kappa = exp(u)).
//
// The contraction particles x K by K x triangles runs as one BF16 GEMM with FP32 accumulation.
// To keep u at FP32 accuracy, theta and Psi are each split into three BF16 pieces
// (x = x1 + x2 + x3, each piece the BF16 rounding of what the previous ones left), and the six
// cross products whose size is above 2^-24 relative are concatenated along K, smallest first:
// (2,2), (1,3), (3,1), (1,2), (2,1), (1,1), i.e. A' = [t2 t1 t3 t1 t2 t1], B' = [P2 P3 P1 P2 P1 P1],
// K' = 6K (padded to a multiple of 8 with zeros). The accumulator then stays small while the small
// products enter and the truncation of its last steps acts at the size of u only: measured on the
// GB300, G within 5.3e-8 of the FP64 oracle for 32 terms (1/16 .. 1/64) and 2.9e-8 for the 320-term
// flow cell (1/16, 1/32), against 2.6e-7 and 1.8e-7 with the largest products first. The epilogue
// applies exp and writes kappa as FP32 [n][E], which the solve kernel reads instead of forming u
// itself.
//
// Expansions beyond 256 terms are synthesised in groups of 64. The error of u from the tensor cores'
// FP32 accumulation follows a round-toward-zero model of the accumulator, one rounding per K = 16
// step (measured: at K = 320 the G errors of a single 1920-wide contraction correlate 1.00 with
// that model and reach 1.6e-6), which shrinks |u| systematically. One contraction stays within
// 1e-6 up to K = 256 (measured at 256 and 128 terms); beyond, each group of 64 terms is its own
// GEMM (the layout above, per group) into an FP32 partial, and the partials are summed in FP64
// before exp (measured at K = 320 on 1/16: G within 3.0e-7; the model gave 2.7e-7).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
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
        // A' blocks: t2 t1 t3 t1 t2 t1
        const __nv_bfloat16 sel[6] = {p2, p1, p3, p1, p2, p1};
        out[t] = sel[blk];
        return;
    }
    out[t] = __float2bfloat16_rn(v);
}

// theta split of the group of Kg terms starting at k0 (the layout of theta_split_kernel, blocks of
// width Kg): out [n][Kp]
__global__ void theta_split_group_kernel(const double* theta, int n, int K, int k0, int Kg, int Kp,
                                         __nv_bfloat16* out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * Kp) return;
    const int j = (int)(t / Kp), c = (int)(t - (long long)j * Kp);
    const int blk = c / Kg, k = c - blk * Kg;
    if (blk < 6) {
        const float x = (float)theta[(size_t)j * K + k0 + k];
        const __nv_bfloat16 p1 = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(p1);
        const __nv_bfloat16 p2 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(p2);
        const __nv_bfloat16 p3 = __float2bfloat16_rn(r2);
        const __nv_bfloat16 sel[6] = {p2, p1, p3, p1, p2, p1};
        out[t] = sel[blk];
        return;
    }
    out[t] = __float2bfloat16_rn(0.0f);
}

// kappa[t] = exp(sum over groups of part[g][t]), the sum and exp in FP64
__global__ void sum_exp_kernel(const float* part, int groups, long long nE, float* kappa) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nE; t += stride) {
        double u = 0.0;
        for (int g = 0; g < groups; ++g) u += (double)part[(size_t)g * nE + t];
        kappa[t] = (float)exp(u);
    }
}

constexpr int kSynthGroup = 64;     // terms per accumulation of a grouped synthesis
constexpr int kSingleMax = 256;     // up to this many terms: one contraction (measured within 1e-6)

// terms of group g (the whole expansion when it is synthesised in one contraction)
int group_terms(int K, int g) {
    if (K <= kSingleMax) return K;
    return K - g * kSynthGroup < kSynthGroup ? K - g * kSynthGroup : kSynthGroup;
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

int kl_groups(int K) { return K <= kSingleMax ? 1 : (K + kSynthGroup - 1) / kSynthGroup; }

int kl_split_total(int K) {
    int s = 0;
    for (int g = 0; g < kl_groups(K); ++g) s += kl_split_width(group_terms(K, g));
    return s;
}

// B' = [P2 P3 P1 P2 P1 P1] as BF16 bits, per group of terms an [E][Kp] block (K-major rows, one
// per triangle), the groups one after the other (one group, the whole table, for K <= 256)
std::vector<uint16_t> kl_split_table(const std::vector<double>& psi, int K, int E) {
    std::vector<uint16_t> out((size_t)E * kl_split_total(K), 0);
    size_t base = 0;
    for (int g = 0; g < kl_groups(K); ++g) {
        const int k0 = g * kSynthGroup, Kg = group_terms(K, g), Kp = kl_split_width(Kg);
        for (int e = 0; e < E; ++e)
            for (int k = 0; k < Kg; ++k) {
                const double x = psi[(size_t)(k0 + k) * E + e];
                const uint16_t p1 = bf16_bits_host(x);
                const double r1 = x - bf16_value_host(p1);
                const uint16_t p2 = bf16_bits_host(r1);
                const double r2 = r1 - bf16_value_host(p2);
                const uint16_t p3 = bf16_bits_host(r2);
                const uint16_t sel[6] = {p2, p3, p1, p2, p1, p1};
                for (int b = 0; b < 6; ++b) out[base + (size_t)e * Kp + b * Kg + k] = sel[b];
            }
        base += (size_t)E * Kp;
    }
    return out;
}

// grow the synthesis buffers to hold n particles on `level` (no launch); a no-op when they do
int Handle::synth_reserve(int level, int n) {
    const Level& L = levels[level];
    const int E = 2 * L.N * L.N, Kt = kl_split_total(K), G = kl_groups(K);
    const size_t need_k = (size_t)n * E, need_t = (size_t)n * Kt;
    if (need_k > synth_kappa_cap || need_t > synth_theta_cap) {
        // both buffers grow to at least their previous size: alternating shapes never shrink them
        const size_t cap_k = std::max(need_k, synth_kappa_cap), cap_t = std::max(need_t, synth_theta_cap);
        cudaFree(synth_kappa_buf);
        cudaFree(synth_theta_buf);
        synth_kappa_buf = nullptr;
        synth_theta_buf = nullptr;
        synth_kappa_cap = synth_theta_cap = 0;
        cudaError_t e = cudaMalloc((void**)&synth_kappa_buf, cap_k * 4);
        if (e == cudaSuccess) e = cudaMalloc((void**)&synth_theta_buf, cap_t * 2);
        if (e != cudaSuccess) return fail(SMC_ENOMEM, "synthesis buffers for %d particles: %s", n, cudaGetErrorString(e));
        synth_kappa_cap = cap_k;
        synth_theta_cap = cap_t;
    }
    const size_t need_p = G > 1 ? (size_t)G * n * E : 0;   // FP32 partials of the term groups
    if (need_p > synth_part_cap) {
        cudaFree(synth_part_buf);
        synth_part_buf = nullptr;
        synth_part_cap = 0;
        cudaError_t e = cudaMalloc((void**)&synth_part_buf, need_p * 4);
        if (e != cudaSuccess) return fail(SMC_ENOMEM, "synthesis partials for %d particles: %s", n, cudaGetErrorString(e));
        synth_part_cap = need_p;
    }
    if (!synth_err) {
        cudaError_t e = cudaMalloc((void**)&synth_err, 4);
        if (e == cudaSuccess) e = cudaMemset(synth_err, 0, 4);
        if (e != cudaSuccess) return fail(SMC_ENOMEM, "synthesis flag");
    }
    return SMC_OK;
}

int Handle::synth_kappa(int level, int n, const double* theta, cudaStream_t st) {
    const Level& L = levels[level];
    const int E = 2 * L.N * L.N, Kt = kl_split_total(K), G = kl_groups(K);
    RC_CHECK(synth_reserve(level, n));
    if (G == 1) {
        const long long work = (long long)n * Kt;
        theta_split_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(
            theta, n, K, Kt, reinterpret_cast<__nv_bfloat16*>(synth_theta_buf));
        count_launches(1);
        GemmEpi epi;
        epi.kind = kEpiExp;
        epi.out_f32 = synth_kappa_buf;
        epi.ld_out = E;
        cudaError_t e = umma_gemm(synth_theta_buf, Kt, L.psi_split, Kt, n, E, Kt, epi, synth_err, st);
        if (e != cudaSuccess) return cuda_fail(e, "KL synthesis GEMM");
        return SMC_OK;
    }
    size_t off_t = 0, off_b = 0;   // group offsets in the theta split and in the table (elements)
    for (int g = 0; g < G; ++g) {
        const int Kg = group_terms(K, g), Kp = kl_split_width(Kg);
        const long long work = (long long)n * Kp;
        theta_split_group_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(
            theta, n, K, g * kSynthGroup, Kg, Kp, reinterpret_cast<__nv_bfloat16*>(synth_theta_buf + off_t));
        count_launches(1);
        GemmEpi epi;
        epi.kind = kEpiStoreF32;
        epi.out_f32 = synth_part_buf + (size_t)g * n * E;
        epi.ld_out = E;
        cudaError_t e = umma_gemm(synth_theta_buf + off_t, Kp, L.psi_split + off_b, Kp, n, E, Kp, epi, synth_err, st);
        if (e != cudaSuccess) return cuda_fail(e, "KL synthesis GEMM of a term group");
        off_t += (size_t)n * Kp;
        off_b += (size_t)E * Kp;
    }
    const long long nE = (long long)n * E;
    const int blocks = (int)std::min<long long>((nE + 255) / 256, 152LL * 8);
    sum_exp_kernel<<<blocks, 256, 0, st>>>(synth_part_buf, G, nE, synth_kappa_buf);
    count_launches(1);
    return SMC_OK;
}

}  // namespace mls2mc
