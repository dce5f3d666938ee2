// Surrogate network state per level and shared work buffers (internal).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mls2mc {

constexpr int kMlpWidth = 256;   // hidden width (4 hidden layers)

#define RC_CHECK(expr)                  \
    do {                                \
        int _r = (expr);                \
        if (_r != SMC_OK) return _r;    \
    } while (0)

struct Mlp {
    bool ready = false, norm_set = false;
    int d[6] = {0, 0, 0, 0, 0, 0};          // layer widths: K padded, 256 x 4, n_obs padded
    int t = 0;                               // Adam steps taken
    float *Wm[5] = {}, *bm[5] = {};          // FP32 master weights
    float *mW[5] = {}, *vW[5] = {}, *mb[5] = {}, *vb[5] = {};
    float *gW[5] = {}, *gb[5] = {};
    __nv_bfloat16 *W[5] = {}, *Wt[5] = {};   // BF16 copies [out][in] and [in][out]
    float *mu = nullptr, *sd = nullptr;      // standardisation of the targets
    double *ring_th = nullptr, *ring_G = nullptr;   // training pairs (theta, G_l(theta))
    int cap = 0, count = 0, head = 0;
    int* err = nullptr;                      // tensor-core wait time-out flag
    void release();
};

struct MlpWork {
    int cap = 0, ldt = 0;
    __nv_bfloat16 *X[6] = {}, *Xt[6] = {};
    float* pre[5] = {};
    __nv_bfloat16 *dZ[5] = {}, *dZt[5] = {};
    float *Z = nullptr, *tgt = nullptr;
    double* th = nullptr;
    int* idx = nullptr;
    double* partial = nullptr;
    float* splitk = nullptr;                 // split-K partial tiles of the weight gradients
    size_t splitk_floats = 0;
    void release();
};

}  // namespace mls2mc
