// Host controller of the MLS^2MC sampler (Sec. 4): the update scheme of Eq. eq_updatescheme_final
// with the cv^LU predictor on the first J~ particles (Sec. 4.4), or the scheme u' of Eq.
// eq_updatescheme_final_Lmax (Sec. 4.5) when opts.tau_min > 0. All per-particle work is queued on
// the device (likelihood, increment search, resampling, pCN or random-walk moves); the host reads
// back a few scalars per update (the chosen increment, log mean weight, cv, accept count).
//
// Order of operations and random draws (Philox counter layout) are the library's convention:
//   prior particles              event 0, purpose 1 (normals)
//   resampling offset U          event = importance-sampling update index, purpose 4
//   pCN step m (global counter)  event = m; normals purpose 2, accept uniform purpose 3
// An ITU reweights by exp(-delta Phi_l), resamples, sets beta <- beta + delta (exactly 1 when
// delta took the whole remaining step) and runs n_mcmc pCN steps for exp(-beta Phi_l) mu0. An LU
// evaluates Phi_{l+1} on all particles (reusing the J~ predictor evaluations), then bridges
// zeta = 0 -> 1 with weights exp(-beta dzeta (Phi_{l+1} - Phi_l)), resampling and pCN steps for
// exp(-beta((1 - zeta) Phi_l + zeta Phi_{l+1})) mu0 that solve both levels per proposal. The
// Markov kernel is pCN, or the random walk of Sec. 5 (opts.proposal; the same draws, theta' =
// theta + s xi, with the prior ratio in the acceptance).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "handle.h"
#include "sampler.h"
#include "smc_device.h"

namespace mls2mc {

int Handle::alloc_sampler() {
    const int J = opts.J;
    if (J <= 0) return SMC_OK;
    smp = new Sampler();
    smp->J = J;
    smp->K = K;
    const size_t JK = (size_t)J * K;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    A((void**)&smp->theta, JK * 8);
    A((void**)&smp->theta_p, JK * 8);
    A((void**)&smp->theta_t, JK * 8);
    for (double** p : {&smp->phi_c, &smp->phi_f, &smp->phi_cp, &smp->phi_fp, &smp->phi_t0, &smp->phi_t1, &smp->a,
                       &smp->cdf})
        A((void**)p, (size_t)J * 8);
    A((void**)&smp->anc, (size_t)J * 4);
    A((void**)&smp->iters, (size_t)J * 4);
    A((void**)&smp->scal, 64);
    A((void**)&smp->mom, (size_t)2 * K * 8);
    A((void**)&smp->n_acc, 16);   // [0] accepted moves (u64), [8] non-converged solves (u32)
    A((void**)&smp->inc.state, sizeof(IncState));
    A((void**)&smp->inc.partials, kIncPartials * 8);
    A((void**)&smp->inc.bar, 2 * sizeof(unsigned));
    smp->inc.err = reinterpret_cast<int*>(smp->inc.bar + 1);
    if (opts.surrogate) {
        A((void**)&smp->G_buf, (size_t)J * n_obs * 8);
        for (double** p : {&smp->ps_c, &smp->ps_f, &smp->psp_c, &smp->psp_f, &smp->phi_cs, &smp->phi_fs})
            A((void**)p, (size_t)J * 8);
        A((void**)&smp->theta_s, JK * 8);
        A((void**)&smp->surv_idx, (size_t)J * 4);
        A((void**)&smp->da_pass, (size_t)J * 4);
        A((void**)&smp->n_surv, 4);
    }
    if (opts.proposal == SMC_PROP_RWM_COV) {
        A((void**)&smp->cmean, (size_t)K * 8);
        A((void**)&smp->cpart, pop_cov_partial_doubles(J, K) * 8);
        A((void**)&smp->cov, (size_t)K * K * 8);
        A((void**)&smp->chol, (size_t)K * K * 8);
    }
    if (e == cudaSuccess) e = cudaMemset(smp->n_acc, 0, 16);
    if (e != cudaSuccess) return fail(SMC_ENOMEM, "sampler buffers for J = %d: %s", J, cudaGetErrorString(e));
    return SMC_OK;
}

void Handle::free_sampler() {
    if (!smp) return;
    for (void* p : {(void*)smp->theta, (void*)smp->theta_p, (void*)smp->theta_t, (void*)smp->phi_c,
                    (void*)smp->phi_f, (void*)smp->phi_cp, (void*)smp->phi_fp, (void*)smp->phi_t0,
                    (void*)smp->phi_t1, (void*)smp->a, (void*)smp->cdf, (void*)smp->scal, (void*)smp->mom,
                    (void*)smp->anc, (void*)smp->iters, (void*)smp->n_acc, (void*)smp->inc.state,
                    (void*)smp->inc.partials, (void*)smp->inc.bar, (void*)smp->G_buf, (void*)smp->ps_c, (void*)smp->ps_f,
                    (void*)smp->psp_c, (void*)smp->psp_f, (void*)smp->theta_s, (void*)smp->phi_cs,
                    (void*)smp->phi_fs, (void*)smp->surv_idx, (void*)smp->n_surv,
                    (void*)smp->da_pass, (void*)smp->cmean, (void*)smp->cpart, (void*)smp->cov, (void*)smp->chol})
        cudaFree(p);
    delete smp;
    smp = nullptr;
}

#define CK(expr)                                              \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, #expr);   \
    } while (0)
#define RC(expr)                        \
    do {                                \
        int _r = (expr);                \
        if (_r != SMC_OK) return _r;    \
    } while (0)

// Opt-in phase timing (smc_set_timing): CUDA events on the handle's stream around the parts of an
// update that are not forward solves (those are timed per level by eval_device); the phases of
// smc_get_phase_timing.
enum Phase { kPhTrain = 0, kPhInfer = 1, kPhScreen = 2, kPhReweight = 3, kPhMove = 4, kPhGate = 5 };
struct PhaseTimer {
    Handle* h;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseTimer(Handle* h_, int ph) : h(h_), phase(ph) {
        if (h->timing) {
            a = h->take_event();
            cudaEventRecord(a, h->stream);
        }
    }
    ~PhaseTimer() {
        if (!a) return;
        cudaEvent_t b = h->take_event();
        cudaEventRecord(b, h->stream);
        h->timed_phase.push_back({phase, a, b});
    }
};

// exact likelihood of n particles on one level, counted; with the surrogate enabled the
// observations are kept as training pairs (theta, G_l(theta)) of that level's network
int Handle::smp_eval(int level, int n, const double* theta, double* phi) {
    if (n <= 0) return SMC_OK;
    // no pairs for a level whose screening gate has been measured and said no
    const bool collect = opts.surrogate && forward_kind == SMC_FWD_FEM &&
                         !(level < (int)da_gate.size() && da_gate[level] < 0);
    // the screening gate's solve time: events around the first evaluation of at least half the
    // particles on a level whose gate is still open
    const bool gate_open = opts.surrogate == 1 && forward_kind == SMC_FWD_FEM && 2 * n >= smp->J &&
                           !(level < (int)da_gate.size() && da_gate[level] != 0) &&
                           !(level < (int)da_ev.size() && da_ev[level].n > 0);
    if (gate_open) {
        if ((int)da_ev.size() < (int)levels.size()) da_ev.resize(levels.size());
        da_ev[level].a = take_event();
        da_ev[level].b = take_event();
        cudaEventRecord(da_ev[level].a, stream);
    }
    RC(eval_device(level, n, theta, collect ? smp->G_buf : nullptr, phi, smp->iters, stream));
    if (gate_open) {
        cudaEventRecord(da_ev[level].b, stream);
        da_ev[level].n = n;
    }
    smp->evals[level] += n;
    if (collect) {
        RC(mlp_add_pairs(level, n, theta, smp->G_buf));
        smp->pairs_new[level] += n;
    }
    // non-converged solves are counted on the device and checked when the update reads its counters
    CK(count_bad_launch(smp->iters, n, bad_counter(), stream));
    return SMC_OK;
}

unsigned* Handle::bad_counter() { return reinterpret_cast<unsigned*>(reinterpret_cast<char*>(smp->n_acc) + 8); }
unsigned* Handle::distinct_counter() { return reinterpret_cast<unsigned*>(reinterpret_cast<char*>(smp->n_acc) + 12); }

// the Markov kernel's step for the coming moves, and its adaptation from their acceptance rate
// (opts.accept_target > 0: s <- s exp(a - target), clamped; the next update's step depends only on
// updates that are finished, so every update's kernel is fixed when it runs)
double Handle::mcmc_step() const { return opts.accept_target > 0.0 ? smp->step : opts.s_pcn; }
void Handle::adapt_step(double rate) {
    if (!(opts.accept_target > 0.0)) return;
    const double hi = opts.proposal == SMC_PROP_PCN ? 1.0 : 100.0;
    smp->step = std::min(hi, std::max(1e-4, smp->step * std::exp(rate - opts.accept_target)));
}

// read the accept and non-convergence counters and the grid-barrier flag of the last increment
// search and resampling, and (pending != null) the state of a search whose result the host has
// not waited for (one wait)
int Handle::read_counters(unsigned long long* acc, IncState* pending) {
    unsigned char buf[16];
    int rs_err = 0;
    CK(cudaMemcpyAsync(buf, smp->n_acc, 16, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(&rs_err, smp->inc.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    if (pending) CK(cudaMemcpyAsync(pending, smp->inc.state, sizeof(IncState), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (rs_err) return fail(SMC_ETIMEOUT, "increment search or resampling: a block gave up at a grid barrier");
    if (pending) RC(check_increment(*pending));
    unsigned long long a;
    unsigned bad;
    std::memcpy(&a, buf, 8);
    std::memcpy(&bad, buf + 8, 4);
    std::memcpy(&last_distinct, buf + 12, 4);
    if (acc) *acc = a;
    if (bad) {
        CK(cudaMemsetAsync(bad_counter(), 0, 4, stream));
        return fail(SMC_ENOCONV, "%u forward solves did not reach rtol", bad);
    }
    return SMC_OK;
}

// Whether screening pays on a level (not in the paper). Measured once per level (events on the
// handle's stream): the device time of an exact solve of J particles against a surrogate forward
// pass of J particles; a level whose solve costs at most kDaCostRatio forward passes is never
// screened (the screen adds a forward pass, a compaction and a host read per Markov step). A level
// above that ratio is screened from the first update whose own Markov steps' exact solves, with
// those already run on the level, cost kDaAmortize times the level's first training round (rent or
// buy over the work known so far: a level the sampler passes through with little work never pays
// for a network, one it stays on pays a bounded multiple of the best choice in hindsight). The
// first round is estimated as its Adam steps times kDaTrainStepPasses forward passes of the
// minibatch (one step measured 0.30 ms against about 0.075 ms for a forward pass of 8000 rows at
// K = 64).
constexpr double kDaCostRatio = 8.0;
constexpr double kDaAmortize = 2.0;
constexpr double kDaTrainStepPasses = 4.0;

namespace {
// a surrogate forward pass of J particles has the same shapes on every level (K -> 4 x 256 -> n_obs):
// its device time is measured once per process for each (K, n_obs, J)
std::mutex g_pred_mu;
std::map<std::tuple<int, int, int>, float> g_pred_ms;
}  // namespace

// device time of an exact solve of J particles on `level`: from the sampler's own first evaluation
// of (most of) its particles there (events recorded by smp_eval), else measured now
float Handle::da_solve_ms(int level) {
    Sampler* S = smp;
    if (level < (int)da_ev.size() && da_ev[level].n > 0) {
        float t = 0.f;
        const DaSolveEvents& d = da_ev[level];
        if (cudaEventSynchronize(d.b) == cudaSuccess && cudaEventElapsedTime(&t, d.a, d.b) == cudaSuccess)
            return t * (float)S->J / (float)d.n;
    }
    cudaEvent_t a = take_event(), b = take_event();
    cudaEventRecord(a, stream);
    const int rc = eval_device(level, S->J, S->theta, nullptr, S->phi_t1, S->iters, stream);
    cudaEventRecord(b, stream);
    float t = 0.f;
    if (rc != SMC_OK || cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess)
        t = -1.f;
    event_pool.push_back(a);
    event_pool.push_back(b);
    return t;
}

float Handle::da_predict_ms(int level) {
    Sampler* S = smp;
    const auto key = std::make_tuple(K, n_obs, S->J);
    {
        std::lock_guard<std::mutex> lock(g_pred_mu);
        auto it = g_pred_ms.find(key);
        if (it != g_pred_ms.end()) return it->second;
    }
    if (mlp_setup(level) != SMC_OK) return -1.f;
    // untimed pass first: buffers allocated on first use must not fall inside the measurement
    if (mlp_predict(level, S->J, S->theta, nullptr, S->phi_t0) != SMC_OK) return -1.f;
    cudaEvent_t a = take_event(), b = take_event();
    cudaEventRecord(a, stream);
    const int rc = mlp_predict(level, S->J, S->theta, nullptr, S->phi_t0);
    cudaEventRecord(b, stream);
    float t = 0.f;
    if (rc != SMC_OK || cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&t, a, b) != cudaSuccess)
        t = -1.f;
    event_pool.push_back(a);
    event_pool.push_back(b);
    if (t > 0.f) {
        std::lock_guard<std::mutex> lock(g_pred_mu);
        g_pred_ms[key] = t;
    }
    return t;
}

bool Handle::da_worth(int level) {
    if ((int)da_gate.size() < (int)levels.size()) {
        da_gate.assign(levels.size(), 0);
        da_t_solve.assign(levels.size(), 0.f);
        da_t_pred.assign(levels.size(), 0.f);
    }
    if (da_gate[level] != 0) return da_gate[level] > 0;
    if (opts.surrogate == 2) {   // screen every level, no cost measurement
        da_gate[level] = 1;
        return true;
    }
    if (!(da_t_solve[level] > 0.f)) {   // the cost ratio, measured once
        PhaseTimer pt(this, kPhGate);
        const float t_solve = da_solve_ms(level);
        const float t_pred = t_solve > 0.f ? da_predict_ms(level) : -1.f;
        da_t_solve[level] = std::max(t_solve, 0.f);
        da_t_pred[level] = std::max(t_pred, 0.f);
        if (!(t_solve > 0.f && t_pred > 0.f && t_solve > kDaCostRatio * t_pred)) {
            da_gate[level] = -1;
            return false;
        }
    }
    // amortization: the exact-solve time spent on the level so far and the coming update's Markov
    // steps against the level's first training round
    const int steps = opts.surrogate_train_steps > 0 ? opts.surrogate_train_steps : 50;
    const int batch = opts.surrogate_batch > 0 ? opts.surrogate_batch : 8192;
    const double t_train = steps * kDaTrainStepPasses * (double)da_t_pred[level] * batch / smp->J;
    const double work = ((double)smp->evals[level] / smp->J + opts.n_mcmc) * da_t_solve[level];
    if (work < kDaAmortize * t_train) return false;   // not yet: the gate stays undecided
    da_gate[level] = 1;
    return true;
}

// training schedule: once the level has J pairs, then again after every 4 J new pairs (50 Adam
// steps the first time, a quarter of that afterwards) on minibatches of up to 8192 pairs: the
// small GEMMs of a step are latency-bound, so few large steps train for less than many small ones
int Handle::maybe_train(int level) {
    if (!opts.surrogate || forward_kind != SMC_FWD_FEM) return SMC_OK;
    if ((int)mlps.size() <= level) return SMC_OK;
    Mlp& M = mlps[level];
    if (M.count < smp->J) return SMC_OK;
    if (M.t > 0 && smp->pairs_new[level] < 4LL * smp->J) return SMC_OK;
    const int base = opts.surrogate_train_steps > 0 ? opts.surrogate_train_steps : 50;
    const int steps = M.t == 0 ? base : std::max(1, base / 4);
    const int batch = std::min(opts.surrogate_batch > 0 ? opts.surrogate_batch : 8192, M.count);
    double loss = 0.0;
    PhaseTimer pt(this, kPhTrain);
    RC(mlp_train(level, steps, batch, &loss));
    smp->pairs_new[level] = 0;
    return SMC_OK;
}

// whether the moves of a target on level (and level + 1 when bridging, zeta >= 0) can be screened:
// every level involved is worth it (its gate is measured here if it is still open)
bool Handle::may_screen(int level, double zeta) {
    return opts.surrogate && forward_kind == SMC_FWD_FEM && da_worth(level) && (zeta < 0.0 || da_worth(level + 1));
}

bool Handle::da_ready(int level, double zeta) const {
    if (!opts.surrogate || forward_kind != SMC_FWD_FEM) return false;
    auto on = [&](int l) {
        return (int)mlps.size() > l && mlps[l].ready && mlps[l].t > 0 && (int)da_gate.size() > l && da_gate[l] > 0;
    };
    return on(level) && (zeta < 0.0 || on(level + 1));
}

int Handle::check_iters(int n) {
    // cheap host check of the first slot only would miss failures; copy the counts (n ints)
    std::vector<int> its((size_t)n);
    CK(cudaMemcpyAsync(its.data(), smp->iters, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    for (int i = 0; i < n; ++i)
        if (its[i] < 0) return fail(SMC_ENOCONV, "forward solve of particle %d did not converge", i);
    return SMC_OK;
}

int Handle::check_increment(const IncState& st) {
    if (st.done == -1) return fail(SMC_ESINGULAR, "non-finite incremental weights (numerical singularity)");
    if (st.done != 1) return fail(SMC_ENOCONV, "increment search did not finish");
    return SMC_OK;
}

// adaptive increment on a[0..n): Eq. Eq_cv_opt, one cooperative launch. The device state also
// holds the next parameter, next = delta >= dmax ? 1 : base + delta. wait: copy the state to st
// and check it now; otherwise the caller resolves it later (read_counters with pending = &st).
int Handle::increment(const double* a, int n, double dmax, double base, IncState& st, bool wait) {
    Sampler* S = smp;
    CK(inc_search_launch(a, n, dmax, opts.tau_star, opts.eps, kIncMaxIter, base, 1.0, S->inc, stream));
    if (!wait) return SMC_OK;
    int err = 0;
    CK(cudaMemcpyAsync(&err, S->inc.err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(&st, S->inc.state, sizeof(IncState), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (err) return fail(SMC_ETIMEOUT, "increment search: a block gave up waiting at the grid barrier");
    return check_increment(st);
}

// increment, evidence factor (when waited for), resampling and gather
int Handle::reweight_resample(const double* a, double dmax, double base, bool carry_fine, IncState& st, bool wait) {
    Sampler* S = smp;
    PhaseTimer pt(this, kPhReweight);
    RC(increment(a, S->J, dmax, base, st, wait));
    if (wait) S->log_z += st.log_mean_w;
    CK(resample_gather_launch(a, S->J, S->inc.state, (uint32_t)S->stage, opts.seed, K, S->theta, S->theta_t,
                              S->phi_c, S->phi_t0, carry_fine ? S->phi_f : nullptr, S->phi_t1, S->cdf, S->anc,
                              S->inc, distinct_counter(), stream));
    std::swap(S->theta, S->theta_t);
    std::swap(S->phi_c, S->phi_t0);
    if (carry_fine) std::swap(S->phi_f, S->phi_t1);
    return SMC_OK;
}

const double* Handle::next_param_device() const {
    return reinterpret_cast<const double*>(reinterpret_cast<const char*>(smp->inc.state) + offsetof(IncState, next));
}

// the proposals of one Markov step into theta_p: pCN sqrt(1 - s^2) theta + s xi, the random walk
// theta + s xi, or the covariance-shaped walk theta + s L xi (xi from the library's Philox layout)
int Handle::propose(uint32_t ev, double s) {
    Sampler* S = smp;
    if (opts.proposal == SMC_PROP_RWM_COV) {
        CK(normals_launch(S->theta_p, S->J, K, ev, kPurposePcnXi, opts.seed, nullptr, 0.0, 0.0, stream));
        CK(cov_step_launch(S->theta, S->theta_p, S->chol, S->J, K, s, stream));
        return SMC_OK;
    }
    const double c0 = opts.proposal == SMC_PROP_RWM ? 1.0 : std::sqrt(1.0 - s * s);
    CK(normals_launch(S->theta_p, S->J, K, ev, kPurposePcnXi, opts.seed, S->theta, c0, s, stream));
    return SMC_OK;
}

// the covariance-shaped walk's factor L for the coming moves (not in the paper): L L^T = C +
// 1e-4 (tr C / K + 1e-12) I with C the covariance of the population before the moves, computed on
// the device (FP64, fixed summation order), factored on the host (Cholesky, FP64) and sent back
int Handle::shape_factor() {
    Sampler* S = smp;
    CK(pop_cov_launch(S->theta, S->J, K, S->cmean, S->cpart, S->cov, stream));
    std::vector<double> C((size_t)K * K), L((size_t)K * K, 0.0);
    CK(cudaMemcpyAsync(C.data(), S->cov, C.size() * 8, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    double tr = 0.0;
    for (int k = 0; k < K; ++k) tr += C[(size_t)k * K + k];
    const double ridge = 1e-4 * (tr / K + 1e-12);
    for (int k = 0; k < K; ++k) C[(size_t)k * K + k] += ridge;
    for (int i = 0; i < K; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = C[(size_t)i * K + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * K + k] * L[(size_t)j * K + k];
            if (i == j) {
                if (!(v > 0.0)) return fail(SMC_ESINGULAR, "population covariance is not positive definite");
                L[(size_t)i * K + i] = std::sqrt(v);
            } else {
                L[(size_t)i * K + j] = v / L[(size_t)j * K + j];
            }
        }
    CK(cudaMemcpyAsync(S->chol, L.data(), L.size() * 8, cudaMemcpyHostToDevice, stream));
    CK(cudaStreamSynchronize(stream));   // L's host storage is released on return
    return SMC_OK;
}

// n_mcmc pCN (or random-walk) Metropolis steps; zeta < 0: tempering target on `level`, else
// bridging target on level, level+1. beta_p / zeta_p: read beta / zeta on the device (where the
// increment search left it) instead of the host value; pending: the search state to read back
// with the counters
int Handle::mcmc(int level, double zeta, double& rate, const double* beta_p, IncState* pending, const double* zeta_p) {
    // The moves may be screened only where the host holds the target (the update waited for its
    // increment); an update that reads beta or zeta on the device, with the search state still to
    // be read back, keeps exact moves even when the screening gate opens during it (its solves can
    // complete the gate's amortization), and the next update screens. Networks are trained only
    // for targets whose every level is worth screening.
    const bool host_target = !beta_p && !pending && !zeta_p;
    if (host_target && may_screen(level, zeta)) {
        RC(maybe_train(level));
        if (zeta >= 0.0) RC(maybe_train(level + 1));
    }
    if (host_target && da_ready(level, zeta)) return mcmc_da(level, zeta, rate);
    Sampler* S = smp;
    const bool rwm = opts.proposal != SMC_PROP_PCN;
    const double s = mcmc_step();
    last_step = s;
    if (opts.proposal == SMC_PROP_RWM_COV) RC(shape_factor());
    CK(cudaMemsetAsync(S->n_acc, 0, 8, stream));
    for (int m = 0; m < opts.n_mcmc; ++m) {
        const uint32_t ev = (uint32_t)S->mcmc_event;
        {
            PhaseTimer pt(this, kPhMove);
            RC(propose(ev, s));
        }
        RC(smp_eval(level, S->J, S->theta_p, S->phi_cp));
        if (zeta >= 0.0) RC(smp_eval(level + 1, S->J, S->theta_p, S->phi_fp));
        PhaseTimer pt(this, kPhMove);
        CK(pcn_accept_launch(S->J, K, S->beta, beta_p, zeta, zeta_p, ev, opts.seed, S->theta, S->theta_p, S->phi_c,
                             S->phi_cp, S->phi_f, S->phi_fp, S->n_acc, rwm ? 1 : 0, stream));
        S->mcmc_event += 1;
    }
    unsigned long long acc = 0;
    RC(read_counters(&acc, pending));
    rate = opts.n_mcmc > 0 ? (double)acc / ((double)opts.n_mcmc * S->J) : 0.0;
    adapt_step(rate);
    return SMC_OK;
}

// delayed-acceptance pCN (Christen & Fox 2005): stage 1 on the surrogate potentials of every
// proposal, exact solves only for the stage-1 survivors, stage 2 with the surrogate-corrected
// exact ratio; the target is unchanged
int Handle::mcmc_da(int level, double zeta, double& rate) {
    Sampler* S = smp;
    const int J = S->J;
    const bool br = zeta >= 0.0;
    const bool rwm = opts.proposal != SMC_PROP_PCN;
    const double s = mcmc_step();
    last_step = s;
    if (opts.proposal == SMC_PROP_RWM_COV) RC(shape_factor());
    CK(cudaMemsetAsync(S->n_acc, 0, 8, stream));
    {
        PhaseTimer pt(this, kPhInfer);
        RC(mlp_predict(level, J, S->theta, nullptr, S->ps_c));
        if (br) RC(mlp_predict(level + 1, J, S->theta, nullptr, S->ps_f));
    }
    long long passed = 0;
    for (int m = 0; m < opts.n_mcmc; ++m) {
        const uint32_t ev = (uint32_t)S->mcmc_event;
        {
            PhaseTimer pt(this, kPhMove);
            RC(propose(ev, s));
        }
        {
            PhaseTimer pt(this, kPhInfer);
            RC(mlp_predict(level, J, S->theta_p, nullptr, S->psp_c));
            if (br) RC(mlp_predict(level + 1, J, S->theta_p, nullptr, S->psp_f));
        }
        int ns = 0;
        {
            PhaseTimer pt(this, kPhScreen);
            CK(da_stage1_launch(J, K, S->beta, zeta, ev, opts.seed, S->ps_c, S->ps_f, S->psp_c, S->psp_f, S->theta,
                                S->theta_p, rwm ? 1 : 0,
                                S->da_pass, S->surv_idx, S->n_surv, S->theta_s, stream));
            CK(cudaMemcpyAsync(&ns, S->n_surv, 4, cudaMemcpyDeviceToHost, stream));
        }
        CK(cudaStreamSynchronize(stream));
        passed += ns;
        if (ns > 0) {
            RC(smp_eval(level, ns, S->theta_s, S->phi_cs));
            if (br) RC(smp_eval(level + 1, ns, S->theta_s, S->phi_fs));
            PhaseTimer pt(this, kPhMove);
            CK(da_stage2_launch(ns, K, S->beta, zeta, ev, opts.seed, S->surv_idx, S->theta_s, S->phi_cs, S->phi_fs,
                                S->theta, S->phi_c, S->phi_f, S->ps_c, S->ps_f, S->psp_c, S->psp_f, S->n_acc,
                                stream));
        }
        S->mcmc_event += 1;
    }
    unsigned long long acc = 0;
    RC(read_counters(&acc));
    const double props = (double)opts.n_mcmc * J;
    rate = props > 0 ? (double)acc / props : 0.0;
    adapt_step(rate);
    S->da_proposals += (long long)props;
    S->da_pass1 += passed;
    last_da_rate = props > 0 ? (double)passed / props : 0.0;
    return SMC_OK;
}

void Handle::record(int type, double zeta, const IncState& st, double rate, double cv_lu, smc_stage_info* info) {
    Sampler* S = smp;
    smc_stage_info r;
    std::memset(&r, 0, sizeof r);
    r.type = type;
    r.level = S->level + (type == 1 ? 1 : 0);
    r.beta = S->beta;
    r.zeta = zeta;
    r.delta = st.delta;
    r.cv = st.cv;
    r.cv_lu = cv_lu;
    r.log_z_inc = st.log_mean_w;
    r.accept_rate = rate;
    r.n_unique = (int)last_distinct;
    r.step = last_step;
    r.da_stage1_rate = last_da_rate;
    last_da_rate = -1.0;
    for (int l = 0; l < 8; ++l) r.evals_per_level[l] = S->evals[l];
    S->path.push_back(r);
    if (info) *info = r;
}

// The plain sampler does not wait for the increment search: the pCN accept reads the new beta
// from the device and the search state comes back with the update's counters (one host wait per
// update). Where the surrogate may screen the moves, the host needs beta earlier, so it waits.
int Handle::tempering_update(int level, double beta0, int n_mcmc, smc_stage_info* info) {
    Sampler* S = smp;
    RC(smp_eval(level, S->J, S->theta, S->phi_c));
    IncState st;
    const double log_z = S->log_z, beta = S->beta, step0 = S->step;
    const int nm = opts.n_mcmc;
    const bool wait = may_screen(level, -1.0);
    S->beta = beta0;
    RC(reweight_resample(S->phi_c, 1.0 - beta0, beta0, false, st, wait));
    if (wait) S->beta = st.next;
    opts.n_mcmc = n_mcmc;
    double rate = 0.0;
    const int rc = mcmc(level, -1.0, rate, wait ? nullptr : next_param_device(), wait ? nullptr : &st);
    opts.n_mcmc = nm;
    S->beta = beta;
    S->log_z = log_z;
    S->step = step0;
    if (rc != SMC_OK) return rc;
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->n_unique = (int)last_distinct;
        info->step = last_step;
        info->type = 0;
        info->level = level;
        info->beta = st.next;
        info->zeta = -1.0;
        info->delta = st.delta;
        info->cv = st.cv;
        info->cv_lu = -1.0;
        info->log_z_inc = st.log_mean_w;
        info->accept_rate = rate;
        for (int l = 0; l < 8; ++l) info->evals_per_level[l] = S->evals[l];
    }
    S->stage += 1;
    return SMC_OK;
}

// One bridging step between `level` and level + 1 at inverse temperature beta, from bridging
// temperature zeta0 (Sec. 4.1): Phi_level and Phi_level+1 of every particle, the adaptive increment of
// zeta for the weights exp(-beta dzeta (Phi_level+1 - Phi_level)) (Eq. Eq_cv_opt), resampling with both
// potentials carried, and n_mcmc Markov steps for exp(-beta ((1 - zeta) Phi_level + zeta Phi_level+1))
// mu0, each proposal solved on both levels. Like tempering_update it leaves the update scheme's
// state (level, beta, evidence) unchanged.
int Handle::bridging_update(int level, double beta, double zeta0, int n_mcmc, smc_stage_info* info) {
    Sampler* S = smp;
    RC(smp_eval(level, S->J, S->theta, S->phi_c));
    RC(smp_eval(level + 1, S->J, S->theta, S->phi_f));
    CK(lu_increment_launch(S->phi_c, S->phi_f, S->J, beta, S->a, stream));
    IncState st;
    const double log_z = S->log_z, beta_s = S->beta, step0 = S->step;
    const int nm = opts.n_mcmc;
    // the moves read zeta on the device unless they may be screened (then the host needs it)
    const bool wait = may_screen(level, 0.0);
    S->beta = beta;
    int rc = reweight_resample(S->a, 1.0 - zeta0, zeta0, true, st, wait);
    double rate = 0.0;
    if (rc == SMC_OK) {
        opts.n_mcmc = n_mcmc;
        rc = wait ? mcmc(level, st.next, rate) : mcmc(level, 0.0, rate, nullptr, &st, next_param_device());
        opts.n_mcmc = nm;
    }
    S->beta = beta_s;
    S->log_z = log_z;
    S->step = step0;
    if (rc != SMC_OK) return rc;
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->n_unique = (int)last_distinct;
        info->step = last_step;
        info->type = 1;
        info->level = level + 1;
        info->beta = beta;
        info->zeta = st.next;
        info->delta = st.delta;
        info->cv = st.cv;
        info->cv_lu = -1.0;
        info->log_z_inc = st.log_mean_w;
        info->accept_rate = rate;
        info->n_bridge = 1;
        for (int l = 0; l < 8; ++l) info->evals_per_level[l] = S->evals[l];
    }
    S->stage += 1;
    return SMC_OK;
}

int Handle::itu(double cv_lu, smc_stage_info* info) {
    Sampler* S = smp;
    IncState st;
    const bool wait = may_screen(S->level, -1.0);
    RC(reweight_resample(S->phi_c, 1.0 - S->beta, S->beta, false, st, wait));
    if (wait) S->beta = st.next;
    double rate = 0.0;
    RC(mcmc(S->level, -1.0, rate, wait ? nullptr : next_param_device(), wait ? nullptr : &st));
    if (!wait) {
        S->beta = st.next;
        S->log_z += st.log_mean_w;
    }
    record(0, -1.0, st, rate, cv_lu, info);
    S->stage += 1;
    S->prev_lu = false;
    return SMC_OK;
}

int Handle::lu(int head, smc_stage_info* info) {
    Sampler* S = smp;
    const int l = S->level;
    RC(smp_eval(l + 1, S->J - head, S->theta + (size_t)head * K, S->phi_f + head));
    double zeta = 0.0;
    int nb = 0;
    IncState st;
    double rate = 0.0;
    while (zeta < 1.0) {
        // the moves read zeta on the device unless they may be screened; the search state comes
        // back with the moves' counters (one host wait per bridging step). Decided per bridging
        // step: the solves of one step can open the screening gate for the next.
        const bool wait = may_screen(l, 0.0);
        CK(lu_increment_launch(S->phi_c, S->phi_f, S->J, S->beta, S->a, stream));
        RC(reweight_resample(S->a, 1.0 - zeta, zeta, true, st, wait));
        if (wait) {
            zeta = st.next;
            RC(mcmc(l, zeta, rate));
        } else {
            RC(mcmc(l, 0.0, rate, nullptr, &st, next_param_device()));
            zeta = st.next;
            S->log_z += st.log_mean_w;
        }
        record(1, zeta, st, rate, -1.0, info);
        S->path.back().n_bridge = ++nb;
        if (info) info->n_bridge = nb;
        S->stage += 1;
    }
    S->level = l + 1;
    std::swap(S->phi_c, S->phi_f);
    S->prev_lu = true;
    return SMC_OK;
}

int Handle::sampler_start() {
    Sampler* S = smp;
    CK(normals_launch(S->theta, S->J, K, 0u, kPurposePrior, opts.seed, nullptr, 0.0, 0.0, stream));
    return sampler_restart();
}

int Handle::sampler_restart() {
    Sampler* S = smp;
    S->level = 0;
    S->beta = 0.0;
    S->log_z = 0.0;
    S->prev_lu = true;
    S->terminated = false;
    S->stage = 0;
    S->mcmc_event = 0;
    S->step = opts.s_pcn;
    for (auto& v : S->evals) v = 0;
    S->path.clear();
    S->started = true;
    return smp_eval(0, S->J, S->theta, S->phi_c);
}

bool Handle::sampler_done() const {
    return smp && smp->started && smp->beta >= 1.0 && (smp->level == (int)levels.size() - 1 || smp->terminated);
}

int Handle::step(smc_stage_info* info) {
    if (!smp) return fail(SMC_EINVAL, "handle was created with J = 0");
    Sampler* S = smp;
    if (!S->started) RC(sampler_start());
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->status = 1;
    }
    if (sampler_done()) return SMC_OK;
    const int L = (int)levels.size();
    if (S->level == L - 1) return itu(-1.0, info);
    // beta = 1: only the level can be raised. Under the scheme u' of Sec. 4.5 (tau_min > 0) the
    // level update is first assessed by cv^LU on the first J~ particles, and the sampler stops on
    // this level when it is below tau_min (no update is recorded).
    if (S->beta >= 1.0 && !(opts.tau_min > 0.0)) return lu(0, info);
    if (S->beta < 1.0 && S->prev_lu) return itu(-1.0, info);
    const int jt = std::min(opts.J_tilde, S->J);
    RC(smp_eval(S->level + 1, jt, S->theta, S->phi_f));
    CK(cv_lu_launch(S->phi_c, S->phi_f, jt, S->beta, S->scal, stream));
    double cv_lu = 0.0;
    CK(cudaMemcpyAsync(&cv_lu, S->scal, 8, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (S->beta >= 1.0) {
        if (cv_lu < opts.tau_min) {
            S->terminated = true;
            return SMC_OK;   // info->status stays 1: nothing was done
        }
        return lu(jt, info);
    }
    if (cv_lu < opts.tau_lu) return itu(cv_lu, info);
    return lu(jt, info);
}

}  // namespace mls2mc

using namespace mls2mc;

extern "C" {

int smc_step(smc_handle* hh, smc_stage_info* info) {
    if (!hh) return SMC_EINVAL;
    return reinterpret_cast<Handle*>(hh)->step(info);
}

int smc_run(smc_handle* hh, int max_updates, smc_stage_info* last) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->smp) return h->fail(SMC_EINVAL, "handle was created with J = 0");
    smc_stage_info info;
    std::memset(&info, 0, sizeof info);
    for (int u = 0; (max_updates <= 0 || u < max_updates); ++u) {
        if (h->smp->started && h->sampler_done()) break;
        int rc = h->step(&info);
        if (rc != SMC_OK) return rc;
    }
    if (last) *last = info;
    return SMC_OK;
}

int smc_state(const smc_handle* hh, int* level, double* beta, double* log_evidence, int* n_updates,
              long long* evals_per_level) {
    if (!hh) return SMC_EINVAL;
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h->smp) return SMC_EINVAL;
    const Sampler* S = h->smp;
    if (level) *level = S->level;
    if (beta) *beta = S->beta;
    if (log_evidence) *log_evidence = S->log_z;
    if (n_updates) *n_updates = (int)S->path.size();
    if (evals_per_level)
        for (int l = 0; l < 8; ++l) evals_per_level[l] = S->evals[l];
    return SMC_OK;
}

int smc_surrogate_gate(const smc_handle* hh, int level, int* decision, double* solve_ms, double* predict_ms) {
    if (!hh) return SMC_EINVAL;
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (level < 0 || level >= (int)h->levels.size()) return SMC_EINVAL;
    const bool known = level < (int)h->da_gate.size();
    if (decision) *decision = known ? h->da_gate[level] : 0;
    if (solve_ms) *solve_ms = known ? (double)h->da_t_solve[level] : 0.0;
    if (predict_ms) *predict_ms = known ? (double)h->da_t_pred[level] : 0.0;
    return SMC_OK;
}

int smc_path(const smc_handle* hh, int max_records, smc_stage_info* out, int* count) {
    if (!hh) return SMC_EINVAL;
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (!h->smp) return SMC_EINVAL;
    const int n = (int)h->smp->path.size();
    if (count) *count = n;
    if (out)
        for (int i = 0; i < n && i < max_records; ++i) out[i] = h->smp->path[i];
    return SMC_OK;
}

int smc_posterior_moments(smc_handle* hh, double* mean, double* var, double* log_evidence) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->smp || !h->smp->started) return h->fail(SMC_EINVAL, "sampler has not run");
    Sampler* S = h->smp;
    cudaError_t e = moments_launch(S->theta, S->J, h->K, S->mom, S->mom + h->K, h->stream);
    std::vector<double> m((size_t)2 * h->K);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m.data(), S->mom, m.size() * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "posterior moments");
    if (mean) std::memcpy(mean, m.data(), 8 * (size_t)h->K);
    if (var) std::memcpy(var, m.data() + h->K, 8 * (size_t)h->K);
    if (log_evidence) *log_evidence = S->log_z;
    return SMC_OK;
}

int smc_get_particles(const smc_handle* hh, double* theta, double* phi) {
    if (!hh) return SMC_EINVAL;
    Handle* h = const_cast<Handle*>(reinterpret_cast<const Handle*>(hh));
    if (!h->smp || !h->smp->started) return h->fail(SMC_EINVAL, "sampler has not run");
    Sampler* S = h->smp;
    cudaError_t e = cudaSuccess;
    if (theta) e = cudaMemcpyAsync(theta, S->theta, (size_t)S->J * h->K * 8, cudaMemcpyDeviceToHost, h->stream);
    if (phi && e == cudaSuccess) e = cudaMemcpyAsync(phi, S->phi_c, (size_t)S->J * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "copy particles");
    return SMC_OK;
}

int smc_set_particles(smc_handle* hh, const double* theta) {
    if (!hh || !theta) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->smp) return h->fail(SMC_EINVAL, "handle was created with J = 0");
    Sampler* S = h->smp;
    cudaError_t e = cudaMemcpyAsync(S->theta, theta, (size_t)S->J * h->K * 8, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "copy particles");
    return h->sampler_restart();
}

int smc_tempering_update(smc_handle* hh, int level, double beta0, int n_mcmc, smc_stage_info* info) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->smp) return h->fail(SMC_EINVAL, "handle was created with J = 0");
    if (level < 0 || level >= (int)h->levels.size()) return h->fail(SMC_EINVAL, "level %d out of range", level);
    if (!(beta0 >= 0.0 && beta0 < 1.0) || n_mcmc < 0) return h->fail(SMC_EINVAL, "need 0 <= beta0 < 1, n_mcmc >= 0");
    if (!h->smp->started) {
        int rc = h->sampler_start();
        if (rc != SMC_OK) return rc;
    }
    return h->tempering_update(level, beta0, n_mcmc, info);
}

int smc_bridging_update(smc_handle* hh, int level, double beta, double zeta0, int n_mcmc, smc_stage_info* info) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->smp) return h->fail(SMC_EINVAL, "handle was created with J = 0");
    if (level < 0 || level + 1 >= (int)h->levels.size())
        return h->fail(SMC_EINVAL, "level %d has no finer level", level);
    if (!(beta > 0.0 && beta <= 1.0) || !(zeta0 >= 0.0 && zeta0 < 1.0) || n_mcmc < 0)
        return h->fail(SMC_EINVAL, "need 0 < beta <= 1, 0 <= zeta0 < 1, n_mcmc >= 0");
    if (!h->smp->started) {
        int rc = h->sampler_start();
        if (rc != SMC_OK) return rc;
    }
    return h->bridging_update(level, beta, zeta0, n_mcmc, info);
}

// ---- kernel-level entry points -----------------------------------------------------------------
int smc_next_increment(smc_handle* hh, int n, const double* a, double dmax, double* out3) {
    if (!hh || !a || !out3 || n <= 0) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->smp || n > h->smp->J) return h->fail(SMC_EINVAL, "n must be in [1, J]");
    Sampler* S = h->smp;
    cudaError_t e = cudaMemcpyAsync(S->a, a, (size_t)n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "copy a");
    IncState st;
    int rc = h->increment(S->a, n, dmax, 0.0, st, true);
    if (rc != SMC_OK) return rc;
    out3[0] = st.delta;
    out3[1] = st.log_mean_w;
    out3[2] = st.cv;
    return SMC_OK;
}

int smc_systematic_resample(smc_handle* hh, int n, const double* w, double U, int* anc) {
    if (!hh || !w || !anc || n <= 0 || !(U >= 0.0 && U < 1.0)) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h->smp || n > h->smp->J) return h->fail(SMC_EINVAL, "n must be in [1, J]");
    Sampler* S = h->smp;
    cudaError_t e = cudaMemcpyAsync(S->a, w, (size_t)n * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = resample_launch(nullptr, S->a, n, S->inc.state, U, 0u, h->opts.seed, S->cdf, S->anc, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(anc, S->anc, (size_t)n * 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return h->cuda_fail(e, "systematic resampling");
    return SMC_OK;
}

int smc_philox_normals(smc_handle* hh, int J, int K, unsigned event, unsigned purpose, double* out) {
    if (!hh || !out || J <= 0 || K <= 0) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    double* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, (size_t)J * K * 8);
    if (e == cudaSuccess) e = normals_launch(d, J, K, event, purpose, h->opts.seed, nullptr, 0.0, 0.0, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)J * K * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return h->cuda_fail(e, "philox normals");
    return SMC_OK;
}

int smc_philox_uniforms(smc_handle* hh, int J, unsigned event, unsigned purpose, double* out) {
    if (!hh || !out || J <= 0) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    double* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, (size_t)J * 8);
    if (e == cudaSuccess) e = uniforms_launch(d, J, event, purpose, h->opts.seed, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, (size_t)J * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess) return h->cuda_fail(e, "philox uniforms");
    return SMC_OK;
}

}  // extern "C"
