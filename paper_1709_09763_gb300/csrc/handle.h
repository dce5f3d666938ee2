// The opaque smc_handle behind the C ABI (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "mlp.h"

namespace mls2mc {

struct Level {
    int N = 0;                   // 1/h
    double* psi64 = nullptr;     // [K][2N^2]
    float* psi32 = nullptr;      // [K][2N^2]
    int* obs_idx = nullptr;      // [n_obs][3]
    double* obs_w = nullptr;     // [n_obs][3]
    double* linA = nullptr;      // linear forward model [n_obs][K]
    uint16_t* psi_split = nullptr;   // mixed path: BF16 three-way split of Psi^T, [2N^2][kl_split_width(K)],
                                     // or per group of 64 terms such a block when K > 256 (kl_split_table)
    std::vector<double> lambda;  // KL eigenvalues
    std::vector<double> psi_host;
    void* rhs = nullptr;         // load vector (FemArgs::rhs), null for f = 1
    double bnorm2 = 0.0;
};

struct Handle {
    int K = 0, n_obs = 0, forward_kind = SMC_FWD_FEM, precision = SMC_FP64;
    int flow_cell = 0;           // SMC_BC_FLOW_CELL
    double sigma = 1.0, rtol = 1e-13;
    int max_iter = 100;
    smc_sampler_opts opts{};
    cudaStream_t stream = nullptr;
    std::vector<Level> levels;
    std::vector<double> y_host;
    double* d_y = nullptr;
    std::string last_error;

    // staging buffers of the host-pointer entry points
    double* scratch_theta = nullptr;
    double* scratch_G = nullptr;
    double* scratch_phi = nullptr;
    int* scratch_iters = nullptr;
    int scratch_cap = 0;

    // sampler state (smc_kernels.cu / controller.cpp)
    struct Sampler* smp = nullptr;

    // large levels: per-block hierarchy slices in global memory (fem_solve.cu)
    float* big_scratch = nullptr;
    float* cp_scratch = nullptr;   // refinement state of the compact form's blocks
    size_t cp_cap = 0;
    size_t big_cap = 0;
    int* big_counter = nullptr;

    // tensor-core KL synthesis buffers (kl_synth.cu)
    float* synth_kappa_buf = nullptr;
    uint16_t* synth_theta_buf = nullptr;
    size_t synth_kappa_cap = 0, synth_theta_cap = 0;
    float* synth_part_buf = nullptr;   // K > 256: FP32 partial fields of the term groups [groups][n][E]
    size_t synth_part_cap = 0;
    int* synth_err = nullptr;
    int synth_kappa(int level, int n, const double* theta, cudaStream_t st);
    int synth_reserve(int level, int n);

    // opt-in CUDA-event timing of forward-solve launches, per level
    bool timing = false;
    struct TimedLaunch {
        int level;
        cudaEvent_t start, stop;
    };
    std::vector<TimedLaunch> timed;
    std::vector<TimedLaunch> timed_phase;   // level = phase of smc_get_phase_timing
    std::vector<cudaEvent_t> event_pool;
    cudaEvent_t take_event();

    // surrogate networks (mlp.cu)
    std::vector<Mlp> mlps;
    MlpWork mwork;
    float mlp_lr = 1e-3f;
    int mlp_ring(int level);
    int mlp_setup(int level);
    int mlp_sync_bf16(int level);
    int mlp_work(int B);
    int mlp_forward(int level, int B, const double* theta, bool training);
    int mlp_predict(int level, int B, const double* theta, double* G, double* phi);
    int mlp_backward(int level, int B, double* loss);
    int mlp_adam(int level);
    int mlp_add_pairs(int level, int n, const double* theta, const double* G);
    int mlp_train(int level, int steps, int batch, double* last_loss);

    ~Handle();
    int fail(int code, const char* fmt, ...);
    int cuda_fail(cudaError_t e, const char* what);
    int ensure_scratch(int n);
    int eval_device(int level, int n, const double* theta, double* G, double* Phi, int* iters, cudaStream_t st);
    FemArgs fem_args(int level, int n, const double* theta, double* G, double* Phi, int* iters) const;
    int block_size(int N) const;
    int alloc_sampler();
    void free_sampler();
    // sampler (controller.cpp)
    int smp_eval(int level, int n, const double* theta, double* phi);
    int check_iters(int n);
    unsigned* bad_counter();
    unsigned* distinct_counter();
    double mcmc_step() const;
    void adapt_step(double rate);
    unsigned last_distinct = 0;   // distinct ancestors of the last resampling (read with the counters)
    double last_step = 0.0;       // the Markov kernel's step of the last moves
    int read_counters(unsigned long long* acc, struct IncState* pending = nullptr);
    int check_increment(const struct IncState& st);
    const double* next_param_device() const;
    int increment(const double* a, int n, double dmax, double base, struct IncState& st, bool wait);
    int reweight_resample(const double* a, double dmax, double base, bool carry_fine, struct IncState& st, bool wait);
    int mcmc(int level, double zeta, double& rate, const double* beta_p = nullptr, struct IncState* pending = nullptr,
             const double* zeta_p = nullptr);
    int mcmc_da(int level, double zeta, double& rate);
    int maybe_train(int level);
    bool da_ready(int level, double zeta) const;
    bool da_worth(int level);
    bool may_screen(int level, double zeta);
    int propose(uint32_t ev, double s);
    int shape_factor();
    std::vector<int> da_gate;   // per level: 0 unknown, 1 screen pays, -1 it does not
    std::vector<float> da_t_solve, da_t_pred;   // per level: the gate's measured device times (ms)
    struct DaSolveEvents {
        cudaEvent_t a = nullptr, b = nullptr;
        int n = 0;   // particles the recorded evaluation solved (0: none recorded)
    };
    std::vector<DaSolveEvents> da_ev;   // per level: the sampler's first large evaluation, timed for the gate
    float da_solve_ms(int level);
    float da_predict_ms(int level);
    double last_da_rate = -1.0;
    void record(int type, double zeta, const struct IncState& st, double rate, double cv_lu, smc_stage_info* info);
    int itu(double cv_lu, smc_stage_info* info);
    int tempering_update(int level, double beta0, int n_mcmc, smc_stage_info* info);
    int bridging_update(int level, double beta, double zeta0, int n_mcmc, smc_stage_info* info);
    int lu(int head, smc_stage_info* info);
    int sampler_start();
    int sampler_restart();
    bool sampler_done() const;
    int step(smc_stage_info* info);
};

int kl_split_width(int K);
int kl_groups(int K);        // term groups the synthesis accumulates separately (1 up to K = 256)
int kl_split_total(int K);   // summed split widths of the groups
std::vector<uint16_t> kl_split_table(const std::vector<double>& psi, int K, int E);

// G = A theta and Phi for the linear test forward model (smc_kernels.cu)
cudaError_t linear_eval_launch(const double* A, int n, int K, int n_obs, const double* theta, const double* y,
                               double inv_sigma2, double* G, double* Phi, int* iters, cudaStream_t st);

}  // namespace mls2mc
