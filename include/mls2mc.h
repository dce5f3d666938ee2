/*
 * mls2mc.h -- C ABI of the GB300 library for the likelihood hot path of the
 * Multilevel Sequential^2 Monte Carlo sampler (Latz, Papaioannou, Ullmann,
 * "Multilevel Sequential^2 Monte Carlo for Bayesian inverse problems",
 * arXiv:1709.09763).
 *
 * Problem (Sec. 2.1, Sec. 5): -div(exp(u(x)) grad p(x)) = 1 on (0,1)^2, p = 0 on
 * the boundary, u a truncated KL expansion of a Gaussian field (Eq. truncKL)
 * with coefficients theta ~ N(0, I_K). Observations are point values of p
 * (Sec. 5), the noise is N(0, sigma^2 I) and the potential is
 * Phi(theta) = 1/2 |(y - G(theta)) / sigma|^2 (Eq. phi). A level l is a
 * uniform mesh of 2 / h_l^2 P1 triangles (Sec. 5).
 *
 * Conventions for every entry point:
 *  - Return value: SMC_OK (0) or a negative SMC_E* code. smc_last_error()
 *    gives a one-line reason for the last failure on a handle.
 *  - Host pointers are owned by the caller and only read or written during
 *    the call. Device pointers ("_device" entry points) must point to memory
 *    of the handle's device and stay valid until the work queued on the
 *    given stream has finished.
 *  - All arrays are dense, row-major, C order. theta is FP64 [n][K].
 *  - Device memory that the library needs is allocated by smc_init and
 *    freed by smc_destroy. A handle is not thread-safe; handles are
 *    independent of each other.
 */
#ifndef MLS2MC_H
#define MLS2MC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SMC_OK          0
#define SMC_EINVAL     -1   /* invalid argument or descriptor */
#define SMC_ENOMEM     -2   /* device or host allocation failed */
#define SMC_ECUDA      -3   /* a CUDA call failed (reason in smc_last_error) */
#define SMC_ENOCONV    -4   /* some linear solve reached its iteration cap */
#define SMC_ESINGULAR  -5   /* all incremental weights underflowed (numerical singularity, Sec. 4.3) */
#define SMC_ETIMEOUT   -6   /* a bounded device wait gave up */

/* precision of the forward solve */
#define SMC_FP64   0   /* FP64 field, FP64 multigrid-preconditioned CG */
#define SMC_MIXED  1   /* FP32 field + FP32 multigrid-PCG, FP64 residual refinement */

/* forward model kind */
#define SMC_FWD_FEM     0  /* the PDE of Sec. 5 */
#define SMC_FWD_LINEAR  1  /* G_l(theta) = A_l theta (linear-Gaussian test problems) */

typedef struct {
    int n_levels;              /* N_L >= 1 */
    const int* inv_h;          /* [n_levels] 1/h_l, coarse to fine; powers of two in [4, 64] */
    int K;                     /* KL terms N_sto, 1 <= K <= 256 */
    double corr_len;           /* correlation length of the separable exponential covariance */
    double variance;           /* prior field variance */
    int n_obs;                 /* observations, 1 <= n_obs <= 1024 */
    const double* obs_xy;      /* [n_obs][2] points in [0,1]^2 */
    const double* y;           /* [n_obs] data */
    double sigma;              /* noise standard deviation, Gamma = sigma^2 I */
    int forward_kind;          /* SMC_FWD_FEM or SMC_FWD_LINEAR */
    const double* linear_A;    /* SMC_FWD_LINEAR only: [n_levels][n_obs][K] */
} smc_problem_desc;

typedef struct {
    int J;                     /* particles */
    int J_tilde;               /* particles used by the cv^LU predictor (Sec. 4.4) */
    int n_mcmc;                /* pCN steps per update */
    double tau_star;           /* target cv of the incremental weights (Eq. Eq_cv_opt) */
    double tau_lu;             /* cv^LU threshold of the update scheme (Eq. eq_updatescheme_final) */
    double eps;                /* minimum increment of beta or zeta (Eq. Eq_ESS_opt) */
    double s_pcn;              /* pCN step size s: theta' = sqrt(1-s^2) theta + s xi */
    int precision;             /* SMC_FP64 or SMC_MIXED */
    uint64_t seed;             /* Philox4x32-10 key */
    int max_iter;              /* cap on inner CG iterations per refinement pass */
    double rtol;               /* FP64 relative residual target of each forward solve */
    void* stream;              /* cudaStream_t used for all work, or NULL for the default stream */
} smc_sampler_opts;

typedef struct smc_handle smc_handle;

/* Build a handle: KL tables and observation operators for every level, device
 * buffers for opts->J particles. The descriptor is copied. Sec. 2.1-2.2. */
int smc_init(const smc_problem_desc* problem, const smc_sampler_opts* opts, smc_handle** out);

/* Free everything the handle owns. NULL is ignored. */
void smc_destroy(smc_handle* h);

/* One-line reason for the last failing call on h (never NULL). */
const char* smc_last_error(const smc_handle* h);

/* Forward map and potential on level `level` (0-based, coarse to fine) for n
 * particles: G_l(theta) (Sec. 2.1, Sec. 5) and Phi_l (Eq. phi). Host arrays:
 * theta [n][K] in, G [n][n_obs] out (may be NULL), Phi [n] out. Copies in and
 * out on the handle's stream and waits for it. n may be 0. Returns
 * SMC_ENOCONV if any solve reached opts.max_iter without meeting opts.rtol
 * (its Phi is still written). */
int smc_eval_likelihood(smc_handle* h, int level, int n, const double* theta,
                        double* G, double* Phi);

/* Same as smc_eval_likelihood on device arrays, queued on `stream` (a
 * cudaStream_t, NULL = the handle's stream); iters [n] (device, may be NULL)
 * receives the inner CG iterations of each solve, negative if it did not
 * converge. Does not wait; convergence is reported by iters only. */
int smc_eval_likelihood_device(smc_handle* h, int level, int n, const double* theta,
                               double* G, double* Phi, int* iters, void* stream);

/* Copy the KL table Psi of level `level` (FP64 [K][2/h^2], triangle order
 * e = 2*(j*N + i) + t, t = 0 lower / 1 upper half of cell (i, j)) to host memory,
 * and the K eigenvalues lambda_k (Eq. truncKL). Either pointer may be NULL. */
int smc_kl_table(const smc_handle* h, int level, double* psi, double* lambda);

/* Sizes of a handle: K, n_obs, number of levels, J. Any pointer may be NULL. */
int smc_sizes(const smc_handle* h, int* K, int* n_obs, int* n_levels, int* J);

#ifdef __cplusplus
}
#endif

#endif /* MLS2MC_H */
