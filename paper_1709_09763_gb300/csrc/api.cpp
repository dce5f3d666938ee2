// C ABI of the library: handle set-up and the likelihood entry points.
//
// The handle owns all device memory: per level the KL table Psi (FP64 and FP32
// copies, Eq. truncKL), the observation interpolation table (3 nodes and P1
// weights per point) and the data y; plus particle buffers for the sampler.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.h"
#include "smc_device.h"
#include "internal.h"

using namespace mls2mc;

namespace mls2mc {

static std::atomic<long long> g_launches{0};

// autotuned block size of the solve kernel per (1/h, precision), process-wide
static std::mutex g_tune_mu;
static std::map<std::pair<int, int>, int> g_block;

static int tuned_block(int N, int precision) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_block.find({N, precision});
    return it == g_block.end() ? 0 : it->second;
}

// T = 0: the default; T < 0: the compact form with -T threads (where compiled)
static void set_block(int N, int precision, int T) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (T == 0) g_block.erase({N, precision});
    else g_block[{N, precision}] = T;
}
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int Handle::fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    last_error = buf;
    return code;
}

int Handle::cuda_fail(cudaError_t e, const char* what) {
    return fail(SMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

template <typename T>
static cudaError_t upload(T** dst, const T* src, size_t count) {
    *dst = nullptr;
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)dst, count * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

Handle::~Handle() {
    for (auto& L : levels) {
        cudaFree(L.psi64);
        cudaFree(L.psi32);
        cudaFree(L.obs_idx);
        cudaFree(L.obs_w);
        cudaFree(L.linA);
        cudaFree(L.psi_split);
        cudaFree(L.rhs);
    }
    cudaFree(synth_kappa_buf);
    cudaFree(synth_theta_buf);
    cudaFree(synth_part_buf);
    cudaFree(synth_err);
    cudaFree(big_scratch);
    cudaFree(cp_scratch);
    cudaFree(big_counter);
    cudaFree(d_y);
    free_sampler();
    for (auto* v : {&timed, &timed_phase})
        for (auto& t : *v) {
            cudaEventDestroy(t.start);
            cudaEventDestroy(t.stop);
        }
    for (auto& d : da_ev) {
        if (d.a) cudaEventDestroy(d.a);
        if (d.b) cudaEventDestroy(d.b);
    }
    for (auto ev : event_pool) cudaEventDestroy(ev);
    for (auto& m : mlps) m.release();
    mwork.release();
    cudaFree(scratch_theta);
    cudaFree(scratch_G);
    cudaFree(scratch_phi);
    cudaFree(scratch_iters);
}

int Handle::ensure_scratch(int n) {
    if (n <= scratch_cap) return SMC_OK;
    cudaFree(scratch_theta);
    cudaFree(scratch_G);
    cudaFree(scratch_phi);
    cudaFree(scratch_iters);
    scratch_theta = nullptr;
    scratch_G = nullptr;
    scratch_phi = nullptr;
    scratch_iters = nullptr;
    scratch_cap = 0;
    cudaError_t e = cudaMalloc((void**)&scratch_theta, sizeof(double) * (size_t)n * K);
    if (e == cudaSuccess) e = cudaMalloc((void**)&scratch_G, sizeof(double) * (size_t)n * n_obs);
    if (e == cudaSuccess) e = cudaMalloc((void**)&scratch_phi, sizeof(double) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&scratch_iters, sizeof(int) * (size_t)n);
    if (e != cudaSuccess) return fail(SMC_ENOMEM, "scratch allocation for %d particles: %s", n, cudaGetErrorString(e));
    scratch_cap = n;
    return SMC_OK;
}

cudaEvent_t Handle::take_event() {
    if (!event_pool.empty()) {
        cudaEvent_t e = event_pool.back();
        event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int Handle::block_size(int N) const { return tuned_block(N, precision); }

long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

FemArgs Handle::fem_args(int level, int n, const double* theta, double* G, double* Phi, int* iters) const {
    const Level& L = levels[level];
    FemArgs a{};
    a.N = L.N;
    a.precision = precision;
    a.n = n;
    a.K = K;
    a.theta = theta;
    a.psi = precision == SMC_MIXED ? (const void*)L.psi32 : (const void*)L.psi64;
    a.kappa = nullptr;
    a.obs_idx = L.obs_idx;
    a.obs_w = L.obs_w;
    a.n_obs = n_obs;
    a.y = d_y;
    a.inv_sigma2 = 1.0 / (sigma * sigma);
    a.G = G;
    a.Phi = Phi;
    a.iters = iters;
    a.rtol = rtol;
    a.rtol_in = precision == SMC_MIXED ? 1e-4 : std::max(0.5 * rtol, 1e-14);
    a.max_outer = precision == SMC_MIXED ? 8 : 3;
    a.max_inner = max_iter;
    a.rhs = L.rhs;
    a.bnorm2 = L.bnorm2;
    a.flow_cell = flow_cell;
    return a;
}

int Handle::eval_device(int level, int n, const double* theta, double* G, double* Phi, int* iters,
                        cudaStream_t st) {
    if (level < 0 || level >= (int)levels.size()) return fail(SMC_EINVAL, "level %d out of range", level);
    if (n < 0) return fail(SMC_EINVAL, "negative particle count");
    if (n == 0) return SMC_OK;
    if (!theta || !Phi) return fail(SMC_EINVAL, "theta and Phi must not be NULL");
    const Level& L = levels[level];
    cudaError_t e;
    if (forward_kind == SMC_FWD_LINEAR) {
        e = linear_eval_launch(L.linA, n, K, n_obs, theta, d_y, 1.0 / (sigma * sigma), G, Phi, iters, st);
    } else {
        FemArgs a = fem_args(level, n, theta, G, Phi, iters);
        if (precision == SMC_MIXED) {
            int rc = synth_kappa(level, n, theta, st);
            if (rc != SMC_OK) return rc;
            a.kappa = synth_kappa_buf;
        }
        if (L.N == 128 && !flow_cell && precision == SMC_MIXED) {
            int T = tuned_block(L.N, precision);
            if (T == 0) T = fem_default_block(L.N, precision);
            if (T == -1024) {   // two-CTA cluster form: refinement state of its CTAs in device memory
                const int blocks = fem_cluster_blocks();
                if (blocks < 2) return fail(SMC_ECUDA, "no two-CTA cluster fits on this device");
                const size_t need = (size_t)blocks * fem_cluster_ref_floats();
                if (need > cp_cap) {
                    cudaFree(cp_scratch);
                    cp_scratch = nullptr;
                    cp_cap = 0;
                    cudaError_t ea = cudaMalloc((void**)&cp_scratch, need * sizeof(float));
                    if (ea != cudaSuccess) return fail(SMC_ENOMEM, "cluster-form scratch: %s", cudaGetErrorString(ea));
                    cp_cap = need;
                }
                if (!big_counter && cudaMalloc((void**)&big_counter, sizeof(int)) != cudaSuccess)
                    return fail(SMC_ENOMEM, "work counter");
                TimedLaunch t{level, nullptr, nullptr};
                if (timing) {
                    t.start = take_event();
                    t.stop = take_event();
                    cudaEventRecord(t.start, st);
                }
                e = fem_eval_cluster_launch(a, cp_scratch, blocks, big_counter, st);
                if (timing) {
                    cudaEventRecord(t.stop, st);
                    timed.push_back(t);
                }
                if (e != cudaSuccess) return cuda_fail(e, "forward-solve launch");
                return SMC_OK;
            }
        }
        if (L.N >= 128) {
            // large level: hierarchy in global memory, persistent blocks
            const int blocks = fem_global_blocks(L.N);
            const size_t need = (size_t)blocks * fem_global_slice(L.N, flow_cell != 0);
            if (need > big_cap) {
                cudaFree(big_scratch);
                big_scratch = nullptr;
                big_cap = 0;
                cudaError_t ea = cudaMalloc((void**)&big_scratch, need * sizeof(float));
                if (ea != cudaSuccess) return fail(SMC_ENOMEM, "large-level scratch: %s", cudaGetErrorString(ea));
                big_cap = need;
            }
            if (!big_counter && cudaMalloc((void**)&big_counter, sizeof(int)) != cudaSuccess)
                return fail(SMC_ENOMEM, "large-level counter");
            TimedLaunch t{level, nullptr, nullptr};
            if (timing) {
                t.start = take_event();
                t.stop = take_event();
                cudaEventRecord(t.start, st);
            }
            e = fem_eval_global_launch(a, big_scratch, blocks, big_counter, st);
            if (timing) {
                cudaEventRecord(t.stop, st);
                timed.push_back(t);
            }
            if (e != cudaSuccess) return cuda_fail(e, "forward-solve launch");
            return SMC_OK;
        }
        int T = tuned_block(L.N, precision);
        if (T == 0) T = fem_default_block(L.N, precision);
        if (flow_cell) T = 0;   // the flow cell has one (one-block) form per level
        if (T < 0) {   // compact form: persistent blocks with their refinement state in device memory
            const int blocks = fem_compact_blocks(L.N, -T);
            if (blocks <= 0) return fail(SMC_EINVAL, "no compact form with %d threads at 1/h = %d", -T, L.N);
            const size_t need = (size_t)blocks * fem_compact_ref_floats(L.N, -T);
            if (need > cp_cap) {
                cudaFree(cp_scratch);
                cp_scratch = nullptr;
                cp_cap = 0;
                cudaError_t ea = cudaMalloc((void**)&cp_scratch, need * sizeof(float));
                if (ea != cudaSuccess) return fail(SMC_ENOMEM, "compact-form scratch: %s", cudaGetErrorString(ea));
                cp_cap = need;
            }
            if (!big_counter && cudaMalloc((void**)&big_counter, sizeof(int)) != cudaSuccess)
                return fail(SMC_ENOMEM, "work counter");
            TimedLaunch t{level, nullptr, nullptr};
            if (timing) {
                t.start = take_event();
                t.stop = take_event();
                cudaEventRecord(t.start, st);
            }
            e = fem_eval_compact_launch(a, -T, cp_scratch, blocks, big_counter, st);
            if (timing) {
                cudaEventRecord(t.stop, st);
                timed.push_back(t);
            }
        } else if (timing) {
            TimedLaunch t{level, take_event(), take_event()};
            cudaEventRecord(t.start, st);
            e = fem_eval_launch(a, st, T);
            cudaEventRecord(t.stop, st);
            timed.push_back(t);
        } else {
            e = fem_eval_launch(a, st, T);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "forward-solve launch");
    return SMC_OK;
}

}  // namespace mls2mc

extern "C" {

int smc_init(const smc_problem_desc* P, const smc_sampler_opts* O, smc_handle** out) {
    if (!out) return SMC_EINVAL;
    *out = nullptr;
    if (!P || !O) return SMC_EINVAL;
    Handle* h = new (std::nothrow) Handle();
    if (!h) return SMC_ENOMEM;
    auto bail = [&](int code) {
        // keep the handle so the caller can read the reason, unless nothing was built
        *out = reinterpret_cast<smc_handle*>(h);
        return code;
    };
    if (P->n_levels < 1 || P->n_levels > 8 || !P->inv_h) return bail(h->fail(SMC_EINVAL, "n_levels must be in [1, 8]"));
    // the FP64 solve forms u = theta . Psi itself with theta staged in a 256-entry shared array;
    // the mixed path takes kappa from the synthesis GEMM, which has no limit of its own
    const int k_max = P->forward_kind == SMC_FWD_FEM && O->precision == SMC_MIXED ? 512 : 256;
    if (P->K < 1 || P->K > k_max) return bail(h->fail(SMC_EINVAL, "K must be in [1, %d] here", k_max));
    if (P->n_obs < 1 || P->n_obs > 1024 || !P->obs_xy || !P->y)
        return bail(h->fail(SMC_EINVAL, "n_obs must be in [1, 1024] with obs_xy and y given"));
    if (!(P->sigma > 0.0)) return bail(h->fail(SMC_EINVAL, "sigma must be positive"));
    if (P->forward_kind != SMC_FWD_FEM && P->forward_kind != SMC_FWD_LINEAR)
        return bail(h->fail(SMC_EINVAL, "unknown forward_kind"));
    if (P->forward_kind == SMC_FWD_LINEAR && !P->linear_A)
        return bail(h->fail(SMC_EINVAL, "linear_A required for SMC_FWD_LINEAR"));
    if (O->precision != SMC_FP64 && O->precision != SMC_MIXED) return bail(h->fail(SMC_EINVAL, "unknown precision"));
    if (O->J < 0) return bail(h->fail(SMC_EINVAL, "J must be >= 0"));
    if (O->proposal != SMC_PROP_PCN && O->proposal != SMC_PROP_RWM && O->proposal != SMC_PROP_RWM_COV)
        return bail(h->fail(SMC_EINVAL, "unknown proposal"));
    if (!(O->accept_target >= 0.0 && O->accept_target < 1.0))
        return bail(h->fail(SMC_EINVAL, "accept_target must be in [0, 1)"));
    if (P->forward_kind == SMC_FWD_FEM) {
        if (!(P->corr_len > 0.0) || !(P->variance > 0.0))
            return bail(h->fail(SMC_EINVAL, "corr_len and variance must be positive"));
        if (P->cov_kind != SMC_COV_SEP_EXP && P->cov_kind != SMC_COV_MATERN)
            return bail(h->fail(SMC_EINVAL, "unknown cov_kind"));
        if (P->cov_kind == SMC_COV_MATERN && P->K > matern_max_terms())
            return bail(h->fail(SMC_EINVAL, "the Matern KL keeps at most %d terms", matern_max_terms()));
        if (P->source_kind != SMC_SRC_ONE && P->source_kind != SMC_SRC_NINE)
            return bail(h->fail(SMC_EINVAL, "unknown source_kind"));
        if (P->bc_kind != SMC_BC_DIRICHLET && P->bc_kind != SMC_BC_FLOW_CELL)
            return bail(h->fail(SMC_EINVAL, "unknown bc_kind"));
        if (P->bc_kind == SMC_BC_FLOW_CELL) {
            if (P->source_kind != SMC_SRC_ONE) return bail(h->fail(SMC_EINVAL, "the flow cell has f = 0"));
            const int top = O->precision == SMC_MIXED ? 256 : 32;
            for (int l = 0; l < P->n_levels; ++l)
                if (P->inv_h[l] < 8 || P->inv_h[l] > top)
                    return bail(h->fail(SMC_EINVAL, "flow cell: 1/h must be in [8, %d] at this precision", top));
        }
        for (int l = 0; l < P->n_levels; ++l) {
            if (!fem_level_supported(P->inv_h[l], O->precision))
                return bail(h->fail(SMC_EINVAL, "level %d: 1/h = %d not supported at this precision", l, P->inv_h[l]));
            if (l > 0 && P->inv_h[l] <= P->inv_h[l - 1])
                return bail(h->fail(SMC_EINVAL, "levels must be strictly refining"));
        }
        for (int r = 0; r < P->n_obs; ++r)
            for (int c = 0; c < 2; ++c)
                if (!(P->obs_xy[2 * r + c] >= 0.0 && P->obs_xy[2 * r + c] <= 1.0))
                    return bail(h->fail(SMC_EINVAL, "observation %d outside the unit square", r));
    }
    h->K = P->K;
    h->n_obs = P->n_obs;
    h->sigma = P->sigma;
    h->forward_kind = P->forward_kind;
    h->flow_cell = P->forward_kind == SMC_FWD_FEM && P->bc_kind == SMC_BC_FLOW_CELL ? 1 : 0;
    h->precision = O->precision;
    h->opts = *O;
    h->stream = (cudaStream_t)O->stream;
    h->rtol = O->rtol > 0 ? O->rtol : (O->precision == SMC_MIXED ? 2e-7 : 1e-13);
    h->max_iter = O->max_iter > 0 ? O->max_iter : 100;
    h->y_host.assign(P->y, P->y + P->n_obs);
    cudaError_t e = upload(&h->d_y, P->y, (size_t)P->n_obs);
    if (e != cudaSuccess) return bail(h->cuda_fail(e, "upload y"));
    for (int l = 0; l < P->n_levels; ++l) {
        Level L;
        if (P->forward_kind == SMC_FWD_FEM) {
            L.N = P->inv_h[l];
            std::vector<double> psi, lam;
            if (P->cov_kind == SMC_COV_MATERN) {
                if (!matern_kl_table(L.N, P->corr_len, P->variance, P->K, psi, lam))
                    return bail(h->fail(SMC_EINVAL, "Matern KL: the eigen-solve did not converge"));
            } else {
                kl_table(L.N, P->corr_len, P->variance, P->K, psi, lam);
            }
            std::vector<float> psi32(psi.begin(), psi.end());
            std::vector<int> idx;
            std::vector<double> wts;
            obs_table(L.N, P->n_obs, P->obs_xy, idx, wts);
            e = upload(&L.psi64, psi.data(), psi.size());
            if (e == cudaSuccess) e = upload(&L.psi32, psi32.data(), psi32.size());
            if (e == cudaSuccess && O->precision == SMC_MIXED) {
                std::vector<uint16_t> sp = kl_split_table(psi, P->K, 2 * L.N * L.N);
                e = upload(&L.psi_split, sp.data(), sp.size());
            }
            if (e == cudaSuccess) e = upload(&L.obs_idx, idx.data(), idx.size());
            if (e == cudaSuccess) e = upload(&L.obs_w, wts.data(), wts.size());
            if (e == cudaSuccess && P->source_kind == SMC_SRC_NINE) {
                std::vector<double> b;
                nine_source_load(L.N, b, L.bnorm2);
                if (O->precision == SMC_MIXED) {   // (hi, lo) float pairs: hi + lo = b to ~2^-48
                    std::vector<float> b2(2 * b.size());
                    for (size_t i = 0; i < b.size(); ++i) {
                        b2[2 * i] = (float)b[i];
                        b2[2 * i + 1] = (float)(b[i] - (double)b2[2 * i]);
                    }
                    float* d = nullptr;
                    e = upload(&d, b2.data(), b2.size());
                    L.rhs = d;
                } else {
                    double* d = nullptr;
                    e = upload(&d, b.data(), b.size());
                    L.rhs = d;
                }
            }
            L.lambda = lam;
            L.psi_host = std::move(psi);
        } else {
            L.N = P->inv_h ? P->inv_h[l] : 0;
            e = upload(&L.linA, P->linear_A + (size_t)l * P->n_obs * P->K, (size_t)P->n_obs * P->K);
        }
        h->levels.push_back(L);
        if (e != cudaSuccess) return bail(h->cuda_fail(e, "upload level tables"));
    }
    int rc = h->alloc_sampler();
    if (rc != SMC_OK) return bail(rc);
    *out = reinterpret_cast<smc_handle*>(h);
    return SMC_OK;
}

void smc_destroy(smc_handle* hh) { delete reinterpret_cast<Handle*>(hh); }

const char* smc_last_error(const smc_handle* hh) {
    if (!hh) return "null handle";
    return reinterpret_cast<const Handle*>(hh)->last_error.c_str();
}

int smc_sizes(const smc_handle* hh, int* K, int* n_obs, int* n_levels, int* J) {
    if (!hh) return SMC_EINVAL;
    const Handle* h = reinterpret_cast<const Handle*>(hh);
    if (K) *K = h->K;
    if (n_obs) *n_obs = h->n_obs;
    if (n_levels) *n_levels = (int)h->levels.size();
    if (J) *J = h->opts.J;
    return SMC_OK;
}

int smc_kl_table_host(int cov_kind, int N, double corr_len, double variance, int K, double* psi, double* lambda) {
    if (N < 1 || N > 256 || K < 1 || K > 512 || !(corr_len > 0.0) || !(variance > 0.0)) return SMC_EINVAL;
    if (cov_kind != SMC_COV_SEP_EXP && cov_kind != SMC_COV_MATERN) return SMC_EINVAL;
    if (cov_kind == SMC_COV_MATERN && K > matern_max_terms()) return SMC_EINVAL;
    std::vector<double> p, lam;
    try {
        if (cov_kind == SMC_COV_MATERN) {
            if (!matern_kl_table(N, corr_len, variance, K, p, lam)) return SMC_EINVAL;
        } else {
            kl_table(N, corr_len, variance, K, p, lam);
        }
    } catch (const std::bad_alloc&) {
        return SMC_ENOMEM;
    }
    if (psi) std::copy(p.begin(), p.end(), psi);
    if (lambda) std::copy(lam.begin(), lam.end(), lambda);
    return SMC_OK;
}

int smc_kl_table(const smc_handle* hh, int level, double* psi, double* lambda) {
    if (!hh) return SMC_EINVAL;
    Handle* h = const_cast<Handle*>(reinterpret_cast<const Handle*>(hh));
    if (level < 0 || level >= (int)h->levels.size()) return h->fail(SMC_EINVAL, "level %d out of range", level);
    const Level& L = h->levels[level];
    if (h->forward_kind != SMC_FWD_FEM) return h->fail(SMC_EINVAL, "no KL table for a linear forward model");
    if (psi) std::memcpy(psi, L.psi_host.data(), L.psi_host.size() * sizeof(double));
    if (lambda) std::memcpy(lambda, L.lambda.data(), L.lambda.size() * sizeof(double));
    return SMC_OK;
}

int smc_set_block_size(smc_handle* hh, int level, int T) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (level < 0 || level >= (int)h->levels.size() || h->forward_kind != SMC_FWD_FEM)
        return h->fail(SMC_EINVAL, "level out of range");
    const int N = h->levels[level].N;
    if (T != 0) {
        auto v = fem_block_sizes(N, h->precision);
        if (std::find(v.begin(), v.end(), T) == v.end()) return h->fail(SMC_EINVAL, "block size %d not compiled for 1/h = %d", T, N);
    }
    set_block(N, h->precision, T);
    return SMC_OK;
}

int smc_block_size(smc_handle* hh, int level, int* T) {
    if (!hh || !T) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (level < 0 || level >= (int)h->levels.size() || h->forward_kind != SMC_FWD_FEM)
        return h->fail(SMC_EINVAL, "level out of range");
    const int N = h->levels[level].N;
    const int t = tuned_block(N, h->precision);
    *T = t != 0 ? t : fem_default_block(N, h->precision);
    return SMC_OK;
}

int smc_autotune(smc_handle* hh, int n_tune, int* chosen, float* best_ms) {
    if (!hh || n_tune < 1) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (h->forward_kind != SMC_FWD_FEM) return SMC_OK;
    if (h->flow_cell) {   // one form per level: nothing to choose, and nothing to impose on other handles
        for (int l = 0; l < (int)h->levels.size(); ++l) {
            if (chosen) chosen[l] = 0;
            if (best_ms) best_ms[l] = 0.f;
        }
        return SMC_OK;
    }
    int rc = h->ensure_scratch(n_tune);
    if (rc != SMC_OK) return rc;
    cudaStream_t st = h->stream;
    cudaError_t e = normals_launch(h->scratch_theta, n_tune, h->K, 0x7fffffffu, 9u, h->opts.seed, nullptr, 0.0, 0.0, st);
    if (e != cudaSuccess) return h->cuda_fail(e, "autotune draws");
    cudaEvent_t e0 = h->take_event(), e1 = h->take_event();
    for (int l = 0; l < (int)h->levels.size(); ++l) {
        const int N = h->levels[l].N;
        int bestT = 0;
        float best = 0.f;
        for (int T : fem_block_sizes(N, h->precision)) {
            set_block(N, h->precision, T);
            for (int rep = 0; rep < 4; ++rep) {
                if (rep == 1) cudaEventRecord(e0, st);
                rc = h->eval_device(l, n_tune, h->scratch_theta, nullptr, h->scratch_phi, h->scratch_iters, st);
                if (rc != SMC_OK) return rc;
            }
            cudaEventRecord(e1, st);
            e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) return h->cuda_fail(e, "autotune timing");
            if (bestT == 0 || ms < best) {
                best = ms;
                bestT = T;
            }
        }
        set_block(N, h->precision, bestT);
        if (chosen) chosen[l] = bestT;
        if (best_ms) best_ms[l] = best / 3.0f;
    }
    h->event_pool.push_back(e0);
    h->event_pool.push_back(e1);
    return SMC_OK;
}

long long smc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int smc_set_timing(smc_handle* hh, int enable) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    h->timing = enable != 0;
    return SMC_OK;
}

int smc_get_timing(smc_handle* hh, double* ms_per_level, long long* launches_per_level) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    std::vector<double> ms(8, 0.0);
    std::vector<long long> cnt(8, 0);
    for (auto& t : h->timed) {
        cudaError_t e = cudaEventSynchronize(t.stop);
        float v = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&v, t.start, t.stop);
        if (e != cudaSuccess) return h->cuda_fail(e, "read launch timing");
        if (t.level >= 0 && t.level < 8) {
            ms[t.level] += v;
            cnt[t.level] += 1;
        }
        h->event_pool.push_back(t.start);
        h->event_pool.push_back(t.stop);
    }
    h->timed.clear();
    for (int l = 0; l < 8; ++l) {
        if (ms_per_level) ms_per_level[l] = ms[l];
        if (launches_per_level) launches_per_level[l] = cnt[l];
    }
    return SMC_OK;
}

int smc_get_phase_timing(smc_handle* hh, double* ms8) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    std::vector<double> ms(8, 0.0);
    for (auto& t : h->timed_phase) {
        cudaError_t e = cudaEventSynchronize(t.stop);
        float v = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&v, t.start, t.stop);
        if (e != cudaSuccess) return h->cuda_fail(e, "read phase timing");
        if (t.level >= 0 && t.level < 8) ms[t.level] += v;
        h->event_pool.push_back(t.start);
        h->event_pool.push_back(t.stop);
    }
    h->timed_phase.clear();
    if (ms8)
        for (int i = 0; i < 8; ++i) ms8[i] = ms[i];
    return SMC_OK;
}

int smc_eval_likelihood_device(smc_handle* hh, int level, int n, const double* theta, double* G, double* Phi,
                               int* iters, void* stream) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    return h->eval_device(level, n, theta, G, Phi, iters, stream ? (cudaStream_t)stream : h->stream);
}

int smc_eval_likelihood(smc_handle* hh, int level, int n, const double* theta, double* G, double* Phi) {
    if (!hh) return SMC_EINVAL;
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (n < 0) return h->fail(SMC_EINVAL, "negative particle count");
    if (n == 0) return SMC_OK;
    if (!theta || !Phi) return h->fail(SMC_EINVAL, "theta and Phi must not be NULL");
    int rc = h->ensure_scratch(n);
    if (rc != SMC_OK) return rc;
    cudaStream_t st = h->stream;
    cudaError_t e = cudaMemcpyAsync(h->scratch_theta, theta, sizeof(double) * (size_t)n * h->K,
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return h->cuda_fail(e, "copy theta to device");
    rc = h->eval_device(level, n, h->scratch_theta, G ? h->scratch_G : nullptr, h->scratch_phi, h->scratch_iters, st);
    if (rc != SMC_OK) return rc;
    if (G) {
        e = cudaMemcpyAsync(G, h->scratch_G, sizeof(double) * (size_t)n * h->n_obs, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return h->cuda_fail(e, "copy G to host");
    }
    e = cudaMemcpyAsync(Phi, h->scratch_phi, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return h->cuda_fail(e, "copy Phi to host");
    std::vector<int> its((size_t)n);
    e = cudaMemcpyAsync(its.data(), h->scratch_iters, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return h->cuda_fail(e, "forward solve");
    for (int i = 0; i < n; ++i)
        if (its[i] < 0) return h->fail(SMC_ENOCONV, "particle %d: solve did not reach rtol", i);
    return SMC_OK;
}

}  // extern "C"
