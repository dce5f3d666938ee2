// Many problems' samplers advanced together (C ABI smc_init_batch, smc_batch_step, smc_batch_run).
//
// Every problem of a batch is its own handle with its own sampler (hierarchy, K, data, J, seed). One
// batched step performs, for every problem that is not finished, its next importance-sampling
// update under the update scheme of Eq. eq_updatescheme_final (Sec. 4.4): an ITU, or one bridging
// step of an LU (Sec. 4.1), with the cv^LU predictor on the first J~ particles where the scheme asks
// for it. The work of all problems runs phase by phase in shared launches:
//   - the likelihoods: the tensor-core syntheses of the mixed-precision problems, then one persistent
//     solve launch per level size whose blocks take (problem, particle) items from a device counter;
//   - the adaptive increments (Sec. 3.4, Eq. Eq_cv_opt): one cooperative launch, each problem on its
//     own range of blocks with its own grid barrier;
//   - systematic resampling with the gather of particles and potentials (Sec. 2.4): one cooperative
//     launch, likewise;
//   - each pCN step: one proposal launch, the likelihood launches, one acceptance launch, the new
//     inverse temperature or bridging temperature read on the device where the search left it.
// The host waits once per step (after the predictors, when any problem needs one, and at the end).
// Each problem gets the block counts and arithmetic of its own single-handle launches, so its path
// and particles equal those of smc_step on its handle, bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "batch.h"
#include "handle.h"
#include "sampler.h"
#include "smc_device.h"

namespace mls2mc {

namespace {

// the launch arguments of up to kMaxTasks likelihood requests, grouped by level size, as a kernel
// parameter; item_start[r] is the first work item of request r in the concatenated item space of
// all groups and rel[r] its index within its group
struct EvalUpload {
    FemArgs args[kMaxTasks];
    int offsets[kMaxTasks];
    int rel[kMaxTasks];
    int item_start[kMaxTasks + 1];
    int count, n_groups, total_items;
};

// copies the tables to device memory: the argument and offset arrays, the per-item group table
// (request index within its group), zeroed work counters
__global__ void eval_tables_kernel(const __grid_constant__ EvalUpload U, FemArgs* d_args, int* d_offsets,
                                   int* d_item_group, int* d_counters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < U.count) {
        d_args[t] = U.args[t];
        d_offsets[t] = U.offsets[t];
    }
    if (t < U.n_groups) d_counters[t] = 0;
    for (int i = t; i < U.total_items; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = U.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (U.item_start[mid] <= i) lo = mid; else hi = mid - 1;
        }
        d_item_group[i] = U.rel[lo];
    }
}

}  // namespace

struct BatchSampler {
    // device tables of the multi-problem likelihood launches
    FemArgs* d_args = nullptr;
    int* d_offsets = nullptr;
    int* d_counters = nullptr;
    int* d_item_group = nullptr;
    size_t item_cap = 0;
    float* big_scratch = nullptr;
    size_t big_cap = 0;
    // host-side state per problem: in a level update (bridging), its zeta and bridging count
    std::vector<int> in_lu, nb;
    std::vector<double> zeta;
    // pinned read-back area per problem: counters (accepts u64, non-converged u32), the search's
    // barrier error flag, the search state, the predictor's cv
    struct Back {
        unsigned long long acc;
        unsigned bad, distinct;
        int inc_err, pad2;
        double cv_lu;
        IncState st;
    };
    Back* back = nullptr;
    size_t back_cap = 0;
    // the update phase of a step (increments, resampling, moves) as a CUDA graph: captured every step
    // from the second on (kernel arguments change with the particle buffers and counters), the
    // executable graph updated in place when the captured graph has the same shape
    long long steps = 0;
    cudaGraphExec_t exec = nullptr;
    bool graph_ok = true;
    long long graph_updates = 0, graph_instantiations = 0;

    ~BatchSampler() {
        if (exec) cudaGraphExecDestroy(exec);
        cudaFree(d_args);
        cudaFree(d_offsets);
        cudaFree(d_counters);
        cudaFree(d_item_group);
        cudaFree(big_scratch);
        cudaFreeHost(back);
    }
};

void batch_sampler_free(BatchSampler* s) { delete s; }

namespace {

struct EvalReq {
    int p, level, n;
    const double* theta;
    double* phi;
};

int bfail(Batch* b, int code, const std::string& msg) {
    b->last_error = msg;
    return code;
}

// likelihoods of all requests (at most one per problem): syntheses, table upload, one persistent
// launch per level size; then the non-converged counts and the evaluation counters, as smp_eval does
int multi_eval(Batch* b, const std::vector<EvalReq>& reqs, cudaStream_t st) {
    BatchSampler* S = b->smp;
    for (size_t i0 = 0; i0 < reqs.size(); i0 += kMaxTasks) {
        const size_t i1 = std::min(reqs.size(), i0 + kMaxTasks);
        // order by (level size, precision): each group is contiguous
        std::vector<size_t> idx;
        for (size_t i = i0; i < i1; ++i)
            if (reqs[i].n > 0) idx.push_back(i);
        if (idx.empty()) continue;
        auto key = [&](size_t i) {
            const Handle* h = b->h[reqs[i].p];
            return std::make_pair(h->levels[reqs[i].level].N, h->precision);
        };
        std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return key(x) < key(y); });
        EvalUpload U;
        std::memset(&U, 0, sizeof U);
        struct G {
            int N, precision, T, first, count, total, item_base;
        };
        std::vector<G> groups;
        int items = 0;
        for (size_t r = 0; r < idx.size(); ++r) {
            const EvalReq& q = reqs[idx[r]];
            Handle* h = b->h[q.p];
            const auto k = key(idx[r]);
            if (groups.empty() || groups.back().N != k.first || groups.back().precision != k.second) {
                // the persistent form has no compact variant: a compact size -T runs with T threads
                groups.push_back({k.first, k.second, std::abs(h->block_size(k.first)), (int)r, 0, 0, items});
            }
            G& g = groups.back();
            FemArgs a = h->fem_args(q.level, q.n, q.theta, nullptr, q.phi, h->smp->iters);
            if (h->precision == SMC_MIXED) {
                const int rc = h->synth_kappa(q.level, q.n, q.theta, st);
                if (rc != SMC_OK) return bfail(b, rc, h->last_error);
                a.kappa = h->synth_kappa_buf;
            }
            U.args[r] = a;
            U.offsets[r] = g.total;
            U.rel[r] = g.count;
            U.item_start[r] = items;
            g.count += 1;
            g.total += q.n;
            items += q.n;
        }
        U.count = (int)idx.size();
        U.item_start[U.count] = items;
        U.n_groups = (int)groups.size();
        U.total_items = items;
        if ((size_t)items > S->item_cap) {
            cudaFree(S->d_item_group);
            S->d_item_group = nullptr;
            S->item_cap = 0;
            if (cudaMalloc((void**)&S->d_item_group, sizeof(int) * (size_t)items) != cudaSuccess)
                return bfail(b, SMC_ENOMEM, "batched sampler: item table");
            S->item_cap = (size_t)items;
        }
        size_t big_need = 0;
        for (const G& g : groups)
            if (g.N >= 128) big_need = std::max(big_need, fem_large_multi_scratch(g.N));
        if (big_need > S->big_cap) {
            cudaFree(S->big_scratch);
            S->big_scratch = nullptr;
            S->big_cap = 0;
            if (cudaMalloc((void**)&S->big_scratch, big_need * sizeof(float)) != cudaSuccess)
                return bfail(b, SMC_ENOMEM, "batched sampler: large-level scratch");
            S->big_cap = big_need;
        }
        const int threads = 256, blocks = std::max(1, std::min(1024, (items + threads - 1) / threads));
        eval_tables_kernel<<<blocks, threads, 0, st>>>(U, S->d_args, S->d_offsets, S->d_item_group, S->d_counters);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        for (size_t gi = 0; gi < groups.size() && e == cudaSuccess; ++gi) {
            const G& g = groups[gi];
            if (g.N >= 128)   // the form single solves default to (two-CTA on 1/128)
                e = fem_eval_large_multi_launch(g.N, S->d_args + g.first, S->d_offsets + g.first,
                                                S->d_item_group + g.item_base, g.total, S->big_scratch,
                                                S->d_counters + gi, st);
            else
                e = fem_eval_persistent_launch(g.N, g.precision, g.T, S->d_args + g.first, S->d_offsets + g.first,
                                               S->d_item_group + g.item_base, g.total, S->d_counters + gi, st);
        }
        if (e != cudaSuccess) return bfail(b, SMC_ECUDA, std::string("batched likelihood launch: ") + cudaGetErrorString(e));
    }
    std::vector<BadTask> bad;
    for (const EvalReq& q : reqs) {
        if (q.n <= 0) continue;
        Handle* h = b->h[q.p];
        h->smp->evals[q.level] += q.n;
        bad.push_back({h->smp->iters, h->bad_counter(), q.n});
    }
    cudaError_t e = count_bad_multi_launch(bad, st);
    if (e != cudaSuccess) return bfail(b, SMC_ECUDA, cudaGetErrorString(e));
    return SMC_OK;
}

enum Act { kNone = 0, kItu, kPredict, kLuStart, kBridge };

}  // namespace

// one importance-sampling update of every unfinished problem (see the file comment)
int batch_step(Batch* b, smc_stage_info* infos) {
    const int P = (int)b->h.size();
    cudaStream_t st = b->h[0]->stream;
    for (int p = 0; p < P; ++p) {
        Handle* h = b->h[p];
        if (!h->smp) return bfail(b, SMC_EINVAL, "problem " + std::to_string(p) + ": handle created with J = 0");
        if (h->forward_kind != SMC_FWD_FEM || h->flow_cell || h->opts.surrogate ||
            h->opts.proposal == SMC_PROP_RWM_COV)
            return bfail(b, SMC_EINVAL, "problem " + std::to_string(p) +
                                            ": the batched sampler runs the plain sampler of the Dirichlet problem "
                                            "(pCN or the random walk)");
        if (h->stream != st) return bfail(b, SMC_EINVAL, "all handles of a batched sampler must share one stream");
    }
    if (!b->smp) {
        b->smp = new BatchSampler();
        BatchSampler* S = b->smp;
        S->in_lu.assign(P, 0);
        S->nb.assign(P, 0);
        S->zeta.assign(P, 0.0);
        cudaError_t e = cudaMalloc((void**)&S->d_args, sizeof(FemArgs) * kMaxTasks);
        if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_offsets, sizeof(int) * kMaxTasks);
        if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_counters, sizeof(int) * kMaxTasks);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&S->back, sizeof(BatchSampler::Back) * (size_t)P);
        // the largest item table and large-level scratch a step can need, allocated now: the update
        // phase is captured into a graph, where nothing may be allocated
        size_t items = 0, big = 0;
        for (Handle* h : b->h) {
            items += (size_t)h->smp->J;
            for (const Level& L : h->levels)
                if (L.N >= 128) big = std::max(big, fem_large_multi_scratch(L.N));
            // the syntheses' buffers at their largest (J particles on the finest level): a buffer that
            // grew inside a captured update would free memory that earlier captured launches use
            if (h->precision == SMC_MIXED) {
                const int rc = h->synth_reserve((int)h->levels.size() - 1, h->smp->J);
                if (rc != SMC_OK) return bfail(b, rc, h->last_error);
            }
        }
        if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_item_group, sizeof(int) * std::max<size_t>(items, 1));
        if (e == cudaSuccess && big) e = cudaMalloc((void**)&S->big_scratch, big * sizeof(float));
        if (e != cudaSuccess) return bfail(b, SMC_ENOMEM, "batched sampler tables");
        S->item_cap = std::max<size_t>(items, 1);
        S->big_cap = big;
        S->back_cap = (size_t)P;
    }
    BatchSampler* S = b->smp;
    for (int p = 0; p < P; ++p) {
        Handle* h = b->h[p];
        if (!h->smp->started) {
            const int rc = h->sampler_start();
            if (rc != SMC_OK) return bfail(b, rc, h->last_error);
            S->in_lu[p] = 0;
        }
        if (infos) {
            std::memset(&infos[p], 0, sizeof(smc_stage_info));
            infos[p].status = 1;
        }
    }
    // the next action of every problem (Handle::step's order of tests)
    std::vector<int> act(P, kNone), head(P, 0);
    std::vector<double> cvlu(P, -1.0);
    for (int p = 0; p < P; ++p) {
        Handle* h = b->h[p];
        Sampler* s = h->smp;
        const int L = (int)h->levels.size();
        if (S->in_lu[p]) act[p] = kBridge;
        else if (h->sampler_done()) act[p] = kNone;
        else if (s->level == L - 1) act[p] = kItu;
        else if (s->beta >= 1.0 && !(h->opts.tau_min > 0.0)) act[p] = kLuStart;
        else if (s->beta < 1.0 && s->prev_lu) act[p] = kItu;
        else act[p] = kPredict;
    }
    // cv^LU predictors on the first J~ particles (Sec. 4.4), one host wait for all of them
    {
        std::vector<EvalReq> reqs;
        std::vector<CvTask> cv;
        for (int p = 0; p < P; ++p) {
            if (act[p] != kPredict) continue;
            Handle* h = b->h[p];
            Sampler* s = h->smp;
            const int jt = std::min(h->opts.J_tilde, s->J);
            head[p] = jt;
            reqs.push_back({p, s->level + 1, jt, s->theta, s->phi_f});
            cv.push_back({s->phi_c, s->phi_f, s->scal, jt, s->beta});
        }
        if (!reqs.empty()) {
            int rc = multi_eval(b, reqs, st);
            if (rc != SMC_OK) return rc;
            cudaError_t e = cv_lu_multi_launch(cv, st);
            for (int p = 0; p < P && e == cudaSuccess; ++p)
                if (act[p] == kPredict)
                    e = cudaMemcpyAsync(&S->back[p].cv_lu, b->h[p]->smp->scal, 8, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return bfail(b, SMC_ECUDA, std::string("cv^LU predictors: ") + cudaGetErrorString(e));
            for (int p = 0; p < P; ++p) {
                if (act[p] != kPredict) continue;
                Handle* h = b->h[p];
                Sampler* s = h->smp;
                const double c = S->back[p].cv_lu;
                if (s->beta >= 1.0) {
                    if (c < h->opts.tau_min) {
                        s->terminated = true;   // scheme u': stops on this level, no update
                        act[p] = kNone;
                    } else {
                        act[p] = kLuStart;
                    }
                } else if (c < h->opts.tau_lu) {
                    act[p] = kItu;
                    cvlu[p] = c;
                } else {
                    act[p] = kLuStart;
                }
            }
        }
    }
    // level updates begin: Phi_{l+1} of the particles the predictor did not evaluate
    {
        std::vector<EvalReq> reqs;
        for (int p = 0; p < P; ++p) {
            if (act[p] != kLuStart) continue;
            Sampler* s = b->h[p]->smp;
            const int K = b->h[p]->K;
            reqs.push_back({p, s->level + 1, s->J - head[p], s->theta + (size_t)head[p] * K, s->phi_f + head[p]});
            S->in_lu[p] = 1;
            S->zeta[p] = 0.0;
            S->nb[p] = 0;
            act[p] = kBridge;
        }
        if (!reqs.empty()) {
            const int rc = multi_eval(b, reqs, st);
            if (rc != SMC_OK) return rc;
        }
    }
    // one importance-sampling update per problem: increments, resampling, pCN steps
    std::vector<int> live;
    for (int p = 0; p < P; ++p)
        if (act[p] == kItu || act[p] == kBridge) live.push_back(p);
    if (live.empty()) return SMC_OK;
    // capture the update phase (the first step runs eagerly: buffers that grow on first use, such as
    // the syntheses', reach their size there); a capture that fails falls back to eager launches
    const bool capture = S->graph_ok && S->steps > 0 && st != nullptr;
    S->steps += 1;
    if (capture && cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        S->graph_ok = false;
        return bfail(b, SMC_ECUDA, "batched sampler: stream capture could not begin");
    }
    int phase_rc = SMC_OK;
    auto end_capture = [&](bool launch) -> int {
        if (!capture) return SMC_OK;
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (ce != cudaSuccess || !g || !launch) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            S->graph_ok = false;
            return ce == cudaSuccess ? SMC_OK : bfail(b, SMC_ECUDA, std::string("batched sampler capture: ") +
                                                                      cudaGetErrorString(ce));
        }
        if (S->exec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(S->exec, g, &info) == cudaSuccess) {
                S->graph_updates += 1;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(S->exec);
                S->exec = nullptr;
            }
        }
        if (!S->exec) {
            ce = cudaGraphInstantiate(&S->exec, g, 0);
            if (ce != cudaSuccess) {
                cudaGraphDestroy(g);
                S->exec = nullptr;
                S->graph_ok = false;
                return bfail(b, SMC_ECUDA, std::string("batched sampler graph: ") + cudaGetErrorString(ce));
            }
            S->graph_instantiations += 1;
        }
        cudaGraphDestroy(g);
        ce = cudaGraphLaunch(S->exec, st);
        if (ce != cudaSuccess) return bfail(b, SMC_ECUDA, std::string("batched sampler graph launch: ") +
                                                            cudaGetErrorString(ce));
        return SMC_OK;
    };
    std::vector<LuTask> lut;
    std::vector<IncTask> inc;
    for (int p : live) {
        Handle* h = b->h[p];
        Sampler* s = h->smp;
        const bool br = act[p] == kBridge;
        if (br) lut.push_back({s->phi_c, s->phi_f, s->a, s->J, s->beta});
        IncTask t;
        t.a = br ? s->a : s->phi_c;
        t.n = s->J;
        t.max_iter = kIncMaxIter;
        t.dmax = br ? 1.0 - S->zeta[p] : 1.0 - s->beta;
        t.tau = h->opts.tau_star;
        t.eps = h->opts.eps;
        t.base = br ? S->zeta[p] : s->beta;
        t.top = 1.0;
        t.w = s->inc;
        inc.push_back(t);
    }
    cudaError_t e = lu_increment_multi_launch(lut, st);
    if (e == cudaSuccess) e = inc_search_multi_launch(inc, st);
    std::vector<RsTask> rs;
    for (int p : live) {
        Handle* h = b->h[p];
        Sampler* s = h->smp;
        const bool br = act[p] == kBridge;
        RsTask t;
        std::memset(&t, 0, sizeof t);
        t.a = br ? s->a : s->phi_c;
        t.n = s->J;
        t.K = h->K;
        t.state = s->inc.state;
        t.event = (uint32_t)s->stage;
        t.seed = h->opts.seed;
        t.th_in = s->theta;
        t.th_out = s->theta_t;
        t.p0_in = s->phi_c;
        t.p0_out = s->phi_t0;
        t.p1_in = br ? s->phi_f : nullptr;
        t.p1_out = s->phi_t1;
        t.cdf = s->cdf;
        t.anc = s->anc;
        t.btot = s->inc.partials;
        t.bar = s->inc.bar;
        t.err = s->inc.err;
        t.distinct = h->distinct_counter();
        rs.push_back(t);
    }
    if (e == cudaSuccess) e = resample_gather_multi_launch(rs, st);
    if (e != cudaSuccess) {
        end_capture(false);
        return bfail(b, SMC_ECUDA, std::string("batched resampling: ") + cudaGetErrorString(e));
    }
    for (int p : live) {
        Sampler* s = b->h[p]->smp;
        std::swap(s->theta, s->theta_t);
        std::swap(s->phi_c, s->phi_t0);
        if (act[p] == kBridge) std::swap(s->phi_f, s->phi_t1);
    }
    // pCN (or random-walk) steps for the new targets; beta (ITU) or zeta (bridging) from the device
    std::vector<std::pair<unsigned*, int>> zero;
    int steps = 0;
    for (int p : live) {
        zero.push_back({reinterpret_cast<unsigned*>(b->h[p]->smp->n_acc), 2});
        steps = std::max(steps, b->h[p]->opts.n_mcmc);
    }
    e = zero_words_launch(zero, st);
    if (e != cudaSuccess) {
        end_capture(false);
        return bfail(b, SMC_ECUDA, cudaGetErrorString(e));
    }
    for (int m = 0; m < steps; ++m) {
        std::vector<NormTask> nt;
        std::vector<EvalReq> rc0, rc1;
        std::vector<AccTask> at;
        for (int p : live) {
            Handle* h = b->h[p];
            if (m >= h->opts.n_mcmc) continue;
            Sampler* s = h->smp;
            const bool rwm = h->opts.proposal == SMC_PROP_RWM;
            const double sp = h->mcmc_step(), c0 = rwm ? 1.0 : std::sqrt(1.0 - sp * sp);
            h->last_step = sp;
            const uint32_t ev = (uint32_t)(s->mcmc_event + m);
            nt.push_back({s->theta_p, s->theta, h->opts.seed, s->J, h->K, ev, kPurposePcnXi, c0, sp});
            rc0.push_back({p, s->level, s->J, s->theta_p, s->phi_cp});
            const bool br = act[p] == kBridge;
            if (br) rc1.push_back({p, s->level + 1, s->J, s->theta_p, s->phi_fp});
            AccTask a;
            std::memset(&a, 0, sizeof a);
            a.n = s->J;
            a.K = h->K;
            a.rwm = rwm ? 1 : 0;
            a.event = ev;
            a.seed = h->opts.seed;
            a.beta = s->beta;
            a.zeta = -1.0;
            if (br) a.zeta_p = h->next_param_device();
            else a.beta_p = h->next_param_device();
            a.theta = s->theta;
            a.theta_p = s->theta_p;
            a.phi_c = s->phi_c;
            a.phi_cp = s->phi_cp;
            a.phi_f = s->phi_f;
            a.phi_fp = s->phi_fp;
            a.n_acc = s->n_acc;
            at.push_back(a);
        }
        e = normals_multi_launch(nt, st);
        int rc = e == cudaSuccess ? multi_eval(b, rc0, st) : bfail(b, SMC_ECUDA, cudaGetErrorString(e));
        if (rc == SMC_OK && !rc1.empty()) rc = multi_eval(b, rc1, st);
        if (rc == SMC_OK) {
            e = pcn_accept_multi_launch(at, st);
            if (e != cudaSuccess) rc = bfail(b, SMC_ECUDA, cudaGetErrorString(e));
        }
        if (rc != SMC_OK) {
            end_capture(false);
            return rc;
        }
    }
    phase_rc = end_capture(true);
    if (phase_rc != SMC_OK) return phase_rc;
    // read back every problem's counters and search state, one wait
    for (int p : live) {
        Sampler* s = b->h[p]->smp;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&S->back[p].acc, s->n_acc, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&S->back[p].inc_err, s->inc.err, 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&S->back[p].st, s->inc.state, sizeof(IncState), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bfail(b, SMC_ECUDA, std::string("batched step: ") + cudaGetErrorString(e));
    int first_rc = SMC_OK;
    for (int p : live) {
        Handle* h = b->h[p];
        Sampler* s = h->smp;
        const BatchSampler::Back& r = S->back[p];
        int rc = SMC_OK;
        if (r.inc_err) rc = h->fail(SMC_ETIMEOUT, "increment search or resampling: a block gave up at a grid barrier");
        else if (r.st.done == -1) rc = h->fail(SMC_ESINGULAR, "non-finite incremental weights (numerical singularity)");
        else if (r.st.done != 1) rc = h->fail(SMC_ENOCONV, "increment search did not finish");
        else if (r.bad) {
            cudaMemsetAsync(h->bad_counter(), 0, 4, st);
            rc = h->fail(SMC_ENOCONV, "%u forward solves did not reach rtol", r.bad);
        }
        if (rc != SMC_OK) {
            if (first_rc == SMC_OK) {
                first_rc = rc;
                b->last_error = "problem " + std::to_string(p) + ": " + h->last_error;
            }
            continue;
        }
        const double rate = h->opts.n_mcmc > 0 ? (double)r.acc / ((double)h->opts.n_mcmc * s->J) : 0.0;
        h->last_distinct = r.distinct;
        if (h->opts.n_mcmc <= 0) h->last_step = h->mcmc_step();
        h->adapt_step(rate);
        smc_stage_info* info = infos ? &infos[p] : nullptr;
        if (act[p] == kItu) {
            s->beta = r.st.next;
            s->log_z += r.st.log_mean_w;
            h->record(0, -1.0, r.st, rate, cvlu[p], info);
            s->stage += 1;
            s->prev_lu = false;
        } else {
            s->log_z += r.st.log_mean_w;
            S->zeta[p] = r.st.next;
            h->record(1, S->zeta[p], r.st, rate, -1.0, info);
            s->path.back().n_bridge = ++S->nb[p];
            if (info) info->n_bridge = S->nb[p];
            s->stage += 1;
            if (S->zeta[p] >= 1.0) {
                s->level += 1;
                std::swap(s->phi_c, s->phi_f);
                s->prev_lu = true;
                S->in_lu[p] = 0;
            }
        }
        s->mcmc_event += h->opts.n_mcmc;
    }
    return first_rc;
}

bool batch_done(const Batch* b) {
    for (const Handle* h : b->h)
        if (!h->smp || !h->smp->started || !h->sampler_done()) return false;
    return true;
}

}  // namespace mls2mc

using namespace mls2mc;

extern "C" {

int smc_init_batch(int n_problems, const smc_problem_desc* problems, const smc_sampler_opts* opts,
                   smc_batch** out) {
    if (!out || n_problems < 1 || !problems || !opts) return SMC_EINVAL;
    *out = nullptr;
    std::vector<smc_handle*> hs;
    for (int p = 0; p < n_problems; ++p) {
        smc_handle* h = nullptr;
        const int rc = smc_init(&problems[p], &opts[p], &h);
        if (rc != SMC_OK) {
            for (smc_handle* x : hs) smc_destroy(x);
            return rc;
        }
        hs.push_back(h);
    }
    const int rc = smc_batch_create(n_problems, hs.data(), out);
    if (rc != SMC_OK) {
        for (smc_handle* x : hs) smc_destroy(x);
        return rc;
    }
    reinterpret_cast<Batch*>(*out)->owns_handles = true;
    return SMC_OK;
}

smc_handle* smc_batch_handle(smc_batch* bb, int p) {
    if (!bb) return nullptr;
    Batch* b = reinterpret_cast<Batch*>(bb);
    if (p < 0 || p >= (int)b->h.size()) return nullptr;
    return reinterpret_cast<smc_handle*>(b->h[p]);
}

int smc_batch_step(smc_batch* bb, smc_stage_info* infos) {
    if (!bb) return SMC_EINVAL;
    return batch_step(reinterpret_cast<Batch*>(bb), infos);
}

int smc_batch_run(smc_batch* bb, int max_steps, int* steps) {
    if (!bb) return SMC_EINVAL;
    Batch* b = reinterpret_cast<Batch*>(bb);
    int n = 0;
    int rc = SMC_OK;
    while (max_steps <= 0 || n < max_steps) {
        bool started = true;
        for (Handle* h : b->h) started = started && h->smp && h->smp->started;
        if (started && batch_done(b)) break;
        rc = batch_step(b, nullptr);
        ++n;
        if (rc != SMC_OK) break;
    }
    if (steps) *steps = n;
    return rc;
}

}  // extern "C"
