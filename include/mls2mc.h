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
#define SMC_MIXED  1   /* FP32 field + FP32 multigrid-PCG, residual refinement in double-float
                          arithmetic (pairs of FP32 numbers, FP64-grade) */

/* forward model kind */
#define SMC_FWD_FEM     0  /* the PDE of Sec. 5 */
#define SMC_FWD_LINEAR  1  /* G_l(theta) = A_l theta (linear-Gaussian test problems) */

/* prior covariance of the log-diffusion field (Sec. 5, Eq. truncKL) */
#define SMC_COV_SEP_EXP 0  /* variance exp(-|x1-x1'|/lc - |x2-x2'|/lc); analytic KL pairs */
#define SMC_COV_MATERN  1  /* Matern, smoothness 3/2: variance (1 + z) exp(-z), z = sqrt(6) |x - x'| / lc
                              (Minasny & McBratney 2005); KL by the Nystrom method on the midpoint
                              rule of a 32 x 32 cell grid (64 x 64 beyond 64 terms), eigenvectors
                              of definite parity under x -> 1-x and y -> 1-y, and under x <-> y
                              where that maps the parity sector onto itself (the library
                              documentation gives the order and sign rules); K <= 512 */
/* source term f of the PDE */
#define SMC_SRC_ONE     0  /* f = 1 */
#define SMC_SRC_NINE    1  /* the nine smoothed point sources of Example 5.1: products of 1-D Gaussian
                              densities N(x1; 0.25 n, 0.001) N(x2; 0.25 m, 0.001), n, m = 1..3; load
                              vector by the edge-midpoint rule on every triangle */
/* boundary conditions of the PDE */
#define SMC_BC_DIRICHLET 0 /* p = 0 on the whole boundary (Examples 5.1, 5.2) */
#define SMC_BC_FLOW_CELL 1 /* the flow cell of Example 5.3: p = 0 on x = 0, p = 1 on x = 1, no flow on
                              y = 0 and y = 1, f = 0 (source_kind must be SMC_SRC_ONE and is ignored);
                              levels 1/8 .. 1/256 (FP64: .. 1/32); the pressure does not depend on a
                              uniform scale of kappa, so a prior mean m0 of the field has no effect */
/* Markov kernel of the sampler */
#define SMC_PROP_PCN    0  /* theta' = sqrt(1 - s^2) theta + s xi */
#define SMC_PROP_RWM    1  /* theta' = theta + s xi (random walk of Sec. 5; s^2 = 2.38^2 / K there),
                              accepted with the prior ratio N(0, I) included */
#define SMC_PROP_RWM_COV 2 /* theta' = theta + s L xi, accepted as SMC_PROP_RWM: a random walk shaped by
                              the particle population (not in the paper). Before each update's moves,
                              L L^T = C + 1e-4 (tr C / K + 1e-12) I with C the covariance of the
                              population (1/J normalisation); every move of the update uses the same L,
                              so each leaves its target invariant. Not run by the batched sampler */

typedef struct {
    int n_levels;              /* N_L >= 1 */
    const int* inv_h;          /* [n_levels] 1/h_l, coarse to fine; powers of two in [4, 32] (FP64),
                                  [4, 256] (mixed; 1/128 keeps its fine level on chip across the two
                                  CTAs of a thread-block cluster, 1/256 in device memory) */
    int K;                     /* KL terms N_sto: 1 <= K <= 256, or <= 512 with the FEM forward map at
                                  SMC_MIXED (Example 5.3 keeps 320); Matern: K <= 512 */
    double corr_len;           /* correlation length of the separable exponential covariance */
    double variance;           /* prior field variance */
    int n_obs;                 /* observations, 1 <= n_obs <= 1024 */
    const double* obs_xy;      /* [n_obs][2] points in [0,1]^2 */
    const double* y;           /* [n_obs] data */
    double sigma;              /* noise standard deviation, Gamma = sigma^2 I */
    int forward_kind;          /* SMC_FWD_FEM or SMC_FWD_LINEAR */
    const double* linear_A;    /* SMC_FWD_LINEAR only: [n_levels][n_obs][K] */
    int cov_kind;              /* SMC_COV_SEP_EXP (0, the default) or SMC_COV_MATERN */
    int source_kind;           /* SMC_SRC_ONE (0, the default) or SMC_SRC_NINE */
    int bc_kind;               /* SMC_BC_DIRICHLET (0, the default) or SMC_BC_FLOW_CELL */
} smc_problem_desc;

typedef struct {
    int J;                     /* particles */
    int J_tilde;               /* particles used by the cv^LU predictor (Sec. 4.4) */
    int n_mcmc;                /* pCN steps per update */
    double tau_star;           /* target cv of the incremental weights (Eq. Eq_cv_opt) */
    double tau_lu;             /* cv^LU threshold of the update scheme (Eq. eq_updatescheme_final) */
    double eps;                /* minimum increment of beta or zeta (Eq. Eq_ESS_opt) */
    double s_pcn;              /* step size s of the Markov kernel (see proposal) */
    int precision;             /* SMC_FP64 or SMC_MIXED */
    uint64_t seed;             /* Philox4x32-10 key */
    int max_iter;              /* cap on inner CG iterations per refinement pass */
    double rtol;               /* relative residual target of each forward solve (<= 0: 1e-13 on the FP64
                                  path, 2e-7 on the mixed path, where the solve's share of the G error is
                                  then below 1e-8; the KL synthesis in BF16 splits dominates it) */
    int surrogate;             /* 0: plain pCN; 1: delayed-acceptance pCN screened by the surrogate network on
                                  the levels where an exact solve costs more than 8 surrogate passes (measured);
                                  2: screen on every level */
    int surrogate_train_steps; /* Adam steps of the first training round of a level (<= 0: 50; later rounds 1/4) */
    int surrogate_batch;       /* training minibatch, at most the pairs held (<= 0: 8192) */
    void* stream;              /* cudaStream_t used for all work, or NULL for the default stream */
    int proposal;              /* SMC_PROP_PCN (0, the default), SMC_PROP_RWM or SMC_PROP_RWM_COV (step
                                  s = s_pcn); with the surrogate screen the prior ratio of the random
                                  walks enters stage 1 */
    double tau_min;            /* > 0: update scheme u' of Sec. 4.5 (Eq. eq_updatescheme_final_Lmax):
                                  at beta = 1 the level update is assessed by cv^LU on the first
                                  J_tilde particles and the run stops on the current level when it is
                                  below tau_min; 0: scheme u (every level is reached) */
    double accept_target;      /* > 0: adapt the Markov kernel's step between updates: the first update
                                  uses s_pcn, each later one s * exp(a - accept_target), a the previous
                                  update's acceptance rate (clamped to [1e-4, 1] for pCN, [1e-4, 100]
                                  for the random walk). The step of an update depends on earlier updates
                                  only, so each update's kernel still leaves its target invariant. 0: the
                                  step stays s_pcn (not in the paper; Sec. 5 fixes the step) */
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
/* The same table computed on the host without a handle or a GPU (Eq. truncKL; Sec. 5 for the
 * Matern prior): cov_kind SMC_COV_SEP_EXP or SMC_COV_MATERN, 1 <= N <= 256 cells per side,
 * 1 <= K <= 512 terms (the Matern Nystrom grid has 32 x 32 cells up to 64 terms and 64 x 64
 * beyond). psi: host [K][2 N^2] in the triangle order above, lambda: host [K]; either may be
 * NULL. The Matern eigen-decomposition is computed once per process for each (corr_len,
 * variance, grid) and reused by every later call and handle. SMC_EINVAL on invalid arguments
 * or an eigen-solve that did not converge, SMC_ENOMEM if the host table cannot be allocated. */
int smc_kl_table_host(int cov_kind, int N, double corr_len, double variance, int K, double* psi,
                      double* lambda);

/* Opt-in timing (no counterpart in the paper; for measurement): when enabled, every forward-solve
 * launch is bracketed by CUDA events on its stream. smc_get_timing waits for the recorded
 * launches, returns the summed device milliseconds and launch counts per level ([8] arrays,
 * either may be NULL) and forgets them. */
int smc_set_timing(smc_handle* h, int enable);
/* Autotuner of the solve kernel (no counterpart in the paper): for every level, time each compiled
 * block size (threads per particle) on n_tune prior draws and keep the fastest for the process
 * (shared by all handles of the same 1/h and precision). chosen [n_levels] receives the block
 * sizes, best_ms [n_levels] the time per launch (either may be NULL). smc_set_block_size forces a
 * block size for a level (T = 0 restores the default: the compact form on 1/32 and 1/64 of the
 * mixed path, the two-CTA form on 1/128, else the first compiled size); T must be one of the
 * compiled sizes. A negative size -T selects the compact form with T threads per particle (mixed
 * precision: -512 at 1/h = 64, -256 at 1/h = 32): several particles per SM, the fine level in five
 * arrays and each coarse level in four, the refinement state in device memory (same results as the
 * size T, bit for bit). At 1/h = 128, -1024 selects the two-CTA form: one particle per cluster of two
 * CTAs of 1024 threads on two SMs, each keeping half of the fine rows on chip with one halo row from
 * the other through distributed shared memory, the coarse levels 1/64 .. 1/2 in both (the same
 * algorithm as 1024, which keeps the fine level in device memory; potentials agree to rounding).
 * Batched solves on 1/128 run the two-CTA form where a cluster fits; flow-cell solves the
 * device-memory form. */
int smc_autotune(smc_handle* h, int n_tune, int* chosen, float* best_ms);
int smc_set_block_size(smc_handle* h, int level, int T);
/* The block size the solves of `level` run with (set, tuned or the default) into *T. */
int smc_block_size(smc_handle* h, int level, int* T);

/* Phase timing (no counterpart in the paper; for measurement): with smc_set_timing enabled, the parts
 * of the sampler's updates that are not forward solves are bracketed by CUDA events on the handle's
 * stream. ms8 [8] (may be NULL) receives the summed device milliseconds since the last call, by
 * phase: 0 surrogate training, 1 surrogate inference (stage-1 forward passes), 2 stage-1 screening
 * and survivor compaction, 3 increments and resampling (Sec. 3.4, Sec. 2.4), 4 Markov-move
 * proposals and acceptances, 5 the screening gate's calibration, 6-7 unused. The forward solves
 * themselves are in smc_get_timing. Waits for the recorded events. */
int smc_get_phase_timing(smc_handle* h, double* ms8);

/* Number of CUDA kernels this library has launched in the process so far (all handles). */
long long smc_kernel_launches(void);
int smc_get_timing(smc_handle* h, double* ms_per_level, long long* launches_per_level);

/* Sizes of a handle: K, n_obs, number of levels, J. Any pointer may be NULL. */
int smc_sizes(const smc_handle* h, int* K, int* n_obs, int* n_levels, int* J);

/* ---- many independent problems (no counterpart in the paper) -------------------------------
 * A batch groups handles of independent inverse problems (each its own hierarchy, K, data). One
 * batch evaluation runs, for every problem p, the likelihood of n[p] particles (device array
 * theta[p], [n[p]][K_p]) on its level level[p], writing phi[p] [n[p]] (device) and, if iters is
 * not NULL, iters[p] [n[p]] (device, as in smc_eval_likelihood_device): the tensor-core KL
 * syntheses of all mixed-precision problems, then one persistent solve launch per level size
 * whose blocks take (problem, particle) work items from a device counter (1/h = 128 in the two-CTA
 * form, whose clusters take the items, where a cluster fits; 1/h = 256 in the form that keeps its
 * fine levels in device memory). With use_graph = 1 the
 * sequence is captured into a CUDA graph on `stream` (which must not be the default stream) the
 * first time and replayed afterwards, as long as levels, counts and pointers are unchanged. The
 * call queues work on `stream` and does not wait. Handles must be distinct FEM handles and must
 * outlive the batch. */
typedef struct smc_batch smc_batch;
int smc_batch_create(int n_problems, smc_handle* const* handles, smc_batch** out);
int smc_batch_eval(smc_batch* b, const int* level, const int* n, const double* const* theta, double* const* phi,
                   int* const* iters, void* stream, int use_graph);
const char* smc_batch_last_error(const smc_batch* b);
void smc_batch_destroy(smc_batch* b);

/* ---- the sampler (needs opts.J > 0) ------------------------------------------------------- */

/* One record per importance-sampling update: an inverse temperature update (type 0, ITU) or one
 * bridging step of a level update (type 1, LU) (Sec. 4.1). beta, zeta: the temperatures after the
 * update (zeta = -1 for an ITU); delta: the chosen increment (Eq. Eq_cv_opt); cv: cv of its
 * incremental weights (Sec. 3.4); cv_lu: the predictor of Sec. 4.4 when it decided this update
 * (else -1); log_z_inc: log of the mean incremental weight (the evidence factor, Sec. 5.1.3);
 * evals_per_level: cumulative forward solves per level after the update. */
typedef struct {
    int type;
    int level;
    double beta;
    double zeta;
    double delta;
    double cv;
    double cv_lu;
    double log_z_inc;
    double accept_rate;
    double da_stage1_rate;
    long long evals_per_level[8];
    int n_bridge;
    int status;            /* 1: the sampler had already reached beta = 1 on the finest level */
    int n_unique;          /* distinct ancestors the update's resampling kept (of J) */
    int pad;
    double step;           /* the Markov kernel's step s the update's moves used */
} smc_stage_info;

/* One step of the update scheme u of Eq. eq_updatescheme_final (Sec. 4.4): an ITU, or a whole LU
 * with all its bridging steps. The first call draws the prior particles (Philox, see the
 * library documentation) and evaluates Phi_1 on them. info (may be NULL) receives the last
 * update's record; info->status = 1 when there was nothing left to do. A failure of an ITU's
 * increment search (SMC_ESINGULAR, SMC_ETIMEOUT) is reported when the update ends; the particles
 * are then unspecified. */
int smc_step(smc_handle* h, smc_stage_info* info);

/* Steps until beta = 1 on the finest level (under the scheme u', opts.tau_min > 0: on the level
 * where the run stopped, which smc_state reports), or max_updates steps (<= 0: no cap). */
int smc_run(smc_handle* h, int max_updates, smc_stage_info* last);

/* Sampler state: current level (0-based), beta, log of the evidence estimate (Sec. 5.1.3),
 * number of importance-sampling updates so far, forward solves per level [8]. Any pointer may be NULL. */
int smc_state(const smc_handle* h, int* level, double* beta, double* log_evidence, int* n_updates,
              long long* evals_per_level);

/* Copy up to max_records update records (oldest first) into out; *count = records available. */
int smc_path(const smc_handle* h, int max_records, smc_stage_info* out, int* count);

/* Mean and variance (population, 1/J) of each KL coefficient over the current equally weighted
 * particles, and log Z (Sec. 5.1). mean, var: [K] host arrays, each may be NULL. */
int smc_posterior_moments(smc_handle* h, double* mean, double* var, double* log_evidence);

/* Copy the current particles theta [J][K] and their potential Phi on the current level [J]. */
int smc_get_particles(const smc_handle* h, double* theta, double* phi);

/* Replace the particles by theta [J][K] (host), restart the sampler at beta = 0 on level 0 and
 * evaluate Phi_1 there (instead of drawing from the prior). */
int smc_set_particles(smc_handle* h, const double* theta);

/* One tempering update of the current particles on level `level` from inverse temperature beta0
 * (Sec. 3.1 with the adaptive step of Eq. Eq_cv_opt): evaluate Phi_level on all particles, choose
 * delta in [min(eps, 1 - beta0), 1 - beta0], reweight by exp(-delta Phi_level), resample
 * systematically, and run n_mcmc pCN steps for exp(-(beta0 + delta) Phi_level) mu0. The particles
 * change; the update-scheme state of smc_step (level, beta, evidence) does not. This is the building
 * block of single-level SMC on any level (Example example_SMC) and of hand-made update schemes.
 * info (may be NULL): type 0, the level, the new beta, delta, cv, log mean weight, accept rate.
 * Without the surrogate the host does not wait for the increment search: its failures
 * (SMC_ESINGULAR, SMC_ETIMEOUT) are reported when the update ends, the particles then unspecified. */
int smc_tempering_update(smc_handle* h, int level, double beta0, int n_mcmc, smc_stage_info* info);

/* One bridging step between `level` and level + 1 (0 <= level < n_levels - 1) at inverse temperature
 * beta (0 < beta <= 1), from bridging temperature zeta0 in [0, 1) (Sec. 4.1): evaluate Phi_level and
 * Phi_level+1 on all particles, choose dzeta in [min(eps, 1 - zeta0), 1 - zeta0] for the weights
 * exp(-beta dzeta (Phi_level+1 - Phi_level)) (Eq. Eq_cv_opt), resample systematically, and run n_mcmc
 * pCN steps for exp(-beta ((1 - zeta) Phi_level + zeta Phi_level+1)) mu0 with zeta = zeta0 + dzeta
 * (1 when the whole remaining step was taken), each proposal solved on both levels. The particles
 * change; the update-scheme state of smc_step does not. The building block of a level update
 * (smc_step runs these from zeta0 = 0 until zeta = 1). info (may be NULL): type 1, level + 1, beta,
 * the new zeta, dzeta, cv, log mean weight, accept rate. Waits for the increment search. */
int smc_bridging_update(smc_handle* h, int level, double beta, double zeta0, int n_mcmc, smc_stage_info* info);

/* ---- many problems' samplers advanced together ------------------------------------------------
 * smc_init_batch builds n_problems handles (smc_init of problems[p] with opts[p]) and a batch that
 * owns them (smc_batch_destroy destroys them); smc_batch_handle returns problem p's handle (owned
 * by the batch; NULL for a bad index) for smc_state, smc_path, smc_posterior_moments and
 * smc_get_particles. smc_batch_create also makes a batch that a sampler can step, from handles the
 * caller keeps.
 *
 * smc_batch_step performs, for every problem not yet finished, its next importance-sampling update
 * under the update scheme of Eq. eq_updatescheme_final (Sec. 4.4, or the scheme u' of Sec. 4.5 when
 * its opts.tau_min > 0): an ITU, or one bridging step of a level update (Sec. 4.1), with the cv^LU
 * predictor on the first J~ particles where the scheme asks for it. The work of all problems runs
 * phase by phase in shared launches: the likelihoods in one persistent launch per level size, the
 * adaptive increments (Sec. 3.4, Eq. Eq_cv_opt) in one cooperative launch, the resampling with its
 * gather (Sec. 2.4) in another, each pCN step's proposals and acceptances in one launch each. Each
 * problem's path and particles equal those that smc_step on its own handle produces, bit for bit
 * (an LU that smc_step performs in one call takes one batched step per bridging step). The first
 * step of a problem draws its prior particles (as smc_step does). infos (may be NULL): [n_problems]
 * records of this step's update per problem, status 1 where the problem had nothing left to do.
 * Requirements: FEM problems with Dirichlet boundary conditions, the plain sampler (opts.surrogate
 * = 0), one stream shared by all handles (SMC_EINVAL otherwise). On a failure of some problem the
 * step still completes the others' updates and returns the first error (smc_batch_last_error names
 * the problem). Queues work on the handles' stream and waits for it (once at the end, and once after
 * the predictors when some problem needs one).
 * smc_batch_run steps until every problem is finished (beta = 1 on its finest level, or stopped by
 * the scheme u'), or max_steps steps (<= 0: no cap); *steps (may be NULL) receives the steps taken. */
int smc_init_batch(int n_problems, const smc_problem_desc* problems, const smc_sampler_opts* opts,
                   smc_batch** out);
smc_handle* smc_batch_handle(smc_batch* b, int p);
int smc_batch_step(smc_batch* b, smc_stage_info* infos);
int smc_batch_run(smc_batch* b, int max_steps, int* steps);

/* ---- surrogate network (no counterpart in the paper) ------------------------------------------
 * Per level, a network theta -> G_l(theta): K inputs, 4 hidden layers of 256 with the exact GELU
 * z Phi(z), n_obs outputs; BF16 weights and activations, FP32 accumulation (tensor cores), FP32
 * master weights, Adam (lr 1e-3, betas 0.9/0.999, eps 1e-8). It predicts standardised observations
 * (G - mu) / s, mu and s the per-output mean and standard deviation of its training targets (fixed
 * at the first training). It serves as the first stage of delayed-acceptance pCN (Christen & Fox
 * 2005); the exact potential still judges every accepted move. Parameter arrays are flat FP32:
 * for l = 0..4, W_l [d(l+1)][d(l)] row-major then b_l [d(l+1)], with d from smc_surrogate_dims
 * (d0 = K rounded up to 8, d1..d4 = 256, d5 = n_obs rounded up to 16; padding rows/columns 0). */

/* dims6 <- the six layer widths d0..d5. */
int smc_surrogate_dims(smc_handle* h, int* dims6);

/* The screening gate of surrogate = 1 on one level (not in the paper): *decision 0 undecided, 1 the
 * level is screened, -1 it is not; *solve_ms and *predict_ms the device times it compared (an exact
 * solve of J particles against a surrogate forward pass of J particles). A level whose solve costs at
 * most 8 passes is never screened; above that, it is screened from the first update whose own
 * n_mcmc sweeps of exact solves, with those already run on the level, cost twice its first training
 * round (estimated as the round's Adam steps times 4 forward passes of the minibatch); until then
 * the decision stays 0 and its training pairs are collected. Zero times when not measured or when surrogate = 2 forces the screen. Any
 * output pointer may be NULL. SMC_EINVAL for a null handle or a bad level. */
int smc_surrogate_gate(const smc_handle* h, int level, int* decision, double* solve_ms, double* predict_ms);
/* Append n training pairs (theta [n][K], G [n][n_obs], host) to level's ring of recent pairs. */
int smc_surrogate_add_pairs(smc_handle* h, int level, int n, const double* theta, const double* G);
/* steps Adam steps on minibatches of `batch` pairs drawn (Philox) from the ring; *loss (may be NULL)
 * gets the last minibatch's mean squared error in standardised units. */
int smc_surrogate_train(smc_handle* h, int level, int steps, int batch, double* loss);
/* Surrogate G~ [n][n_obs] (may be NULL) and Phi~ [n] (may be NULL) of theta [n][K] (host arrays). */
int smc_surrogate_predict(smc_handle* h, int level, int n, const double* theta, double* G, double* phi);
/* direction 1: copy the FP32 parameters (and mu, s: [2][d5], may be NULL) out; 0: copy them in. */
int smc_surrogate_params(smc_handle* h, int level, int direction, float* params, float* mu_sd);
/* One forward and backward pass on n pairs without an update: gradients of the mean squared error
 * (same flat layout as the parameters) and the loss. */
int smc_surrogate_grads(smc_handle* h, int level, int n, const double* theta, const double* G, float* grads,
                        double* loss);

/* ---- kernel-level entry points of the sampler's device steps -------------------------------- */

/* The adaptive increment of Eq. Eq_cv_opt for incremental log-weights -delta * a_j, j < n <= J:
 * the argmin over delta in [min(eps, dmax), dmax] of (cv(exp(-delta a)) - tau*)^2 (tau*, eps from
 * the options). out3 = {delta, log mean_j exp(-delta a_j), cv at delta}. Host arrays. */
int smc_next_increment(smc_handle* h, int n, const double* a, double dmax, double* out3);

/* Systematic resampling of n <= J particles with unnormalised weights w (> 0) and offset U in
 * [0, 1): anc[i] = min{ j : c_j > (U + i)/n }, c the cumulative normalised weights (c_{n-1} = 1). */
int smc_systematic_resample(smc_handle* h, int n, const double* w, double U, int* anc);

/* Allocation-free systematic resampling. The paper has no counterpart to this: it serves callers
 * that cannot allocate device memory -- code whose device memory is all owned by another
 * framework's pool, hosts that forbid cudaMalloc after start-up (real-time or embedded loops where
 * an allocation could block or fail), plug-ins without a handle of this library. The result is
 * the same as smc_systematic_resample's, but w [n] (unnormalised weights > 0) and anc [n] are
 * DEVICE arrays, the work is queued on `stream` (a cudaStream_t, NULL = default stream) without
 * waiting, and no handle is needed. Its scratch (one double per particle) is a fixed device array
 * of SMC_NOALLOC_MAX_PARTICLES entries (512 KiB) that every GPU loading the library holds until the
 * process exits; n beyond that maximum returns SMC_EINVAL. It calls no cudaMalloc or cudaFree.
 * Every call looks up the array's device address in the current context (nothing is cached, so a
 * device reset or another current context is safe). The first call on a device may load the
 * library's device code: make it before any stream capture (a first call on a capturing stream
 * returns SMC_EINVAL). All calls share the array: calls that overlap on the GPU race on it, so the
 * caller must serialise them. Returns SMC_EINVAL for bad arguments (n < 1, n too large, U outside
 * [0, 1) or NaN, NULL arrays), SMC_ECUDA if the look-up or the launch fails. */
#define SMC_NOALLOC_MAX_PARTICLES 65536
int smc_systematic_resample_noalloc(const double* w, int n, double U, int* anc, void* stream);

/* The library's tensor-core GEMM (tcgen05, BF16 operands, FP32 accumulation) on host arrays:
 * C[M][N] = A[M][K] . B[N][K]^T with A, B BF16 bit patterns (uint16), K a multiple of 8. It is the
 * contraction of the surrogate network and of the KL synthesis u = theta . Psi (Eq. truncKL).
 * Allocates and frees its own device buffers; SMC_ETIMEOUT if a bounded wait gave up. */
int smc_gemm_bf16(int M, int N, int K, const uint16_t* A, const uint16_t* B, float* C);

/* Philox4x32-10 draws of the library's layout with key opts.seed: out [J][K] standard normals
 * (counter (k/2, j, event, purpose), Box-Muller), or out [J] uniforms in (0, 1] (counter (0, j, event,
 * purpose), 1 - 53-bit uniform). */
int smc_philox_normals(smc_handle* h, int J, int K, unsigned event, unsigned purpose, double* out);
int smc_philox_uniforms(smc_handle* h, int J, unsigned event, unsigned purpose, double* out);

#ifdef __cplusplus
}
#endif

#endif /* MLS2MC_H */
