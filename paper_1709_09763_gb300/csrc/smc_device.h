// Device state and launch wrappers of the sampler kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

namespace mls2mc {

// Philox counter word 3: what the draw is for (the library's draw layout)
constexpr uint32_t kPurposePrior = 1;
constexpr uint32_t kPurposePcnXi = 2;
constexpr uint32_t kPurposePcnU = 3;
constexpr uint32_t kPurposeResample = 4;
constexpr uint32_t kPurposeDaU = 5;

constexpr int kIncMaxBlocks = 128;    // blocks of the increment search (one cooperative launch)
constexpr int kIncThreads = 64;       // two warps a block: short FP64 reductions
constexpr int kIncSums = 6;           // sums per block and decision
constexpr int kIncMaxIter = 200;      // cap on decisions of one search

// state of one adaptive-increment search, resident in device memory
struct IncState {
    double amin, dmin, dmax, target, tau;
    double lo, hi, x;                 // bracket and current point
    double tlo, thi, t;               // their logarithms
    double glo, ghi;                  // g at the bracket ends
    double base, top;                 // next = delta >= dmax ? top : base + delta
    int phase, iter, done, pad;
    // results
    double delta, log_mean_w, cv, S1, next;
};

struct IncWork {
    IncState* state = nullptr;   // device: the result
    double* partials = nullptr;  // device [kIncMaxBlocks] minima, then [2][kIncMaxBlocks][kIncSums] sums
    unsigned* bar = nullptr;     // device: grid-barrier counter, then (as int) the error flag
    int* err = nullptr;          // = (int*)(bar + 1): a block gave up waiting at the grid barrier
};
constexpr size_t kIncPartials = (size_t)kIncMaxBlocks * (1 + 2 * kIncSums);

int inc_blocks(int n);
// the whole search on a[0..n) into *w.state (w.err set if a grid barrier timed out)
cudaError_t inc_search_launch(const double* a, int n, double dmax, double tau, double eps, int max_iter, double base,
                              double top, IncWork& w, cudaStream_t st);

cudaError_t normals_launch(double* out, int J, int K, uint32_t event, uint32_t purpose, uint64_t seed,
                           const double* base, double c0, double c1, cudaStream_t st);
cudaError_t uniforms_launch(double* out, int J, uint32_t event, uint32_t purpose, uint64_t seed, cudaStream_t st);
// U >= 0: use it as the offset; U < 0: draw it from Philox (event, kPurposeResample)
cudaError_t resample_launch(const double* a, const double* w_in, int n, const IncState* state, double U,
                            uint32_t event, uint64_t seed, double* cdf, int* anc, cudaStream_t st);
// weights of the increment in *state, systematic resampling (U from Philox (event, kPurposeResample))
// and the gather of theta rows and up to two potential caches, in one cooperative launch; uses
// w's barrier and scratch (w.err set if a grid barrier timed out); *distinct (if given) receives the
// number of distinct ancestors
cudaError_t resample_gather_launch(const double* a, int n, const IncState* state, uint32_t event, uint64_t seed,
                                   int K, const double* th_in, double* th_out, const double* p0_in, double* p0_out,
                                   const double* p1_in, double* p1_out, double* cdf, int* anc, IncWork& w,
                                   unsigned* distinct, cudaStream_t st);
cudaError_t lu_increment_launch(const double* phi_c, const double* phi_f, int n, double beta, double* a,
                                cudaStream_t st);
cudaError_t cv_lu_launch(const double* phi_c, const double* phi_f, int n, double beta, double* out, cudaStream_t st);
// zeta < 0: tempering target beta * Phi_c; else bridging target beta ((1 - zeta) Phi_c + zeta Phi_f)
// beta_p (device, or null): read beta there instead (the tempering parameter the increment search
// left on the device, so the host need not wait for it); rwm: random-walk proposal, whose
// acceptance includes the prior ratio of N(0, I)
cudaError_t pcn_accept_launch(int n, int K, double beta, const double* beta_p, double zeta, const double* zeta_p,
                              uint32_t event, uint64_t seed, double* theta, const double* theta_p, double* phi_c,
                              const double* phi_cp, double* phi_f, const double* phi_fp, unsigned long long* n_acc,
                              int rwm, cudaStream_t st);
cudaError_t da_stage1_launch(int n, int K, double beta, double zeta, uint32_t event, uint64_t seed, const double* ps_c,
                             const double* ps_f, const double* psp_c, const double* psp_f, const double* theta,
                             const double* theta_p, int rwm, int* pass, int* surv_idx, int* n_surv, double* theta_s,
                             cudaStream_t st);
cudaError_t da_stage2_launch(int ns, int K, double beta, double zeta, uint32_t event, uint64_t seed, const int* surv_idx,
                             const double* theta_s, const double* phi_cs, const double* phi_fs, double* theta,
                             double* phi_c, double* phi_f, double* ps_c, double* ps_f, const double* psp_c,
                             const double* psp_f, unsigned long long* n_acc, cudaStream_t st);
cudaError_t count_bad_launch(const int* iters, int n, unsigned* bad, cudaStream_t st);

// ---- many problems in one launch (the batched sampler) ------------------------------------------
// Task tables travel as kernel parameters (__grid_constant__, at most kMaxTasks problems per launch;
// the launchers split longer lists). Each problem gets the block count its single-problem launch
// would use and its own barrier counter and scratch, so its results equal that launch's bit for bit.
constexpr int kMaxTasks = 64;

struct IncTask {
    const double* a;
    int n, max_iter;
    double dmax, tau, eps, base, top;
    IncWork w;
};
struct RsTask {
    const double* a;
    int n, K;
    const IncState* state;
    uint32_t event, pad;
    uint64_t seed;
    const double *th_in, *p0_in, *p1_in;
    double *th_out, *p0_out, *p1_out, *cdf, *btot;
    int* anc;
    unsigned* bar;
    int* err;
    unsigned* distinct;   // distinct ancestors (may be null)
};
struct NormTask {
    double* out;
    const double* base;
    uint64_t seed;
    int J, K;
    uint32_t event, purpose;
    double c0, c1;
};
struct AccTask {
    int n, K, rwm;
    uint32_t event;
    uint64_t seed;
    double beta, zeta;
    const double *beta_p, *zeta_p;   // read on the device instead, where given
    double *theta, *phi_c, *phi_f;
    const double *theta_p, *phi_cp, *phi_fp;
    unsigned long long* n_acc;
};
struct LuTask {
    const double *phi_c, *phi_f;
    double* a;
    int n;
    double beta;
};
struct CvTask {
    const double *phi_c, *phi_f;
    double* out;
    int n;
    double beta;
};
struct BadTask {
    const int* iters;
    unsigned* bad;
    int n;
};
template <typename Task>
struct TaskList {
    Task t[kMaxTasks];
    int start[kMaxTasks + 1];   // first block of each task; start[count] = the grid
    int count;
};
using IncTasks = TaskList<IncTask>;
using RsTasks = TaskList<RsTask>;
using NormTasks = TaskList<NormTask>;
using AccTasks = TaskList<AccTask>;
using LuTasks = TaskList<LuTask>;
using CvTasks = TaskList<CvTask>;
using BadTasks = TaskList<BadTask>;
struct ZeroList {
    unsigned* ptr[2 * kMaxTasks];
    int words[2 * kMaxTasks];
    int count;
};

int rs_blocks(int n);   // blocks of one problem's resampling launch
cudaError_t inc_search_multi_launch(const std::vector<IncTask>& tasks, cudaStream_t st);
cudaError_t resample_gather_multi_launch(const std::vector<RsTask>& tasks, cudaStream_t st);
cudaError_t normals_multi_launch(const std::vector<NormTask>& tasks, cudaStream_t st);
cudaError_t pcn_accept_multi_launch(const std::vector<AccTask>& tasks, cudaStream_t st);
cudaError_t lu_increment_multi_launch(const std::vector<LuTask>& tasks, cudaStream_t st);
cudaError_t cv_lu_multi_launch(const std::vector<CvTask>& tasks, cudaStream_t st);
cudaError_t count_bad_multi_launch(const std::vector<BadTask>& tasks, cudaStream_t st);
// words (unsigned) to zero: (pointer, count) pairs
cudaError_t zero_words_launch(const std::vector<std::pair<unsigned*, int>>& list, cudaStream_t st);
cudaError_t moments_launch(const double* theta, int n, int K, double* mean, double* var, cudaStream_t st);
// covariance-shaped random walk: the population covariance (scratch: mean K doubles, partials
// pop_cov_partial_doubles(n, K) doubles) and the step out = theta + s L out (out holds xi on entry)
size_t pop_cov_partial_doubles(int n, int K);
cudaError_t pop_cov_launch(const double* theta, int n, int K, double* mean, double* part, double* cov, cudaStream_t st);
cudaError_t cov_step_launch(const double* theta, double* out, const double* L, int n, int K, double s, cudaStream_t st);

}  // namespace mls2mc
