// Many independent inverse problems advanced together (C ABI smc_batch_*).
//
// Each problem is its own handle (own hierarchy, K, data, particles). A batch evaluation takes,
// per problem, a level and a device array of particles, and runs: the tensor-core KL synthesis of
// every mixed-precision problem, then ONE persistent solve launch per level size, whose blocks pull
// (problem, particle) items across all problems of that size from a device counter. The whole
// sequence is captured once into a CUDA graph and replayed while the problems, levels, counts and
// pointers stay the same (the signature); a new signature rebuilds the argument tables and the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <cstdlib>
#include <map>
#include <string>
#include <vector>

#include "batch.h"
#include "handle.h"

namespace mls2mc {

long long launch_count();

namespace {

// enqueue the whole batch evaluation on st (syntheses, counter resets, persistent launches)
int enqueue(Batch* b, const int* level, const int* n, const double* const* theta, cudaStream_t st) {
    for (size_t p = 0; p < b->h.size(); ++p) {
        Handle* h = b->h[p];
        if (n[p] > 0 && h->precision == SMC_MIXED) {
            int rc = h->synth_kappa(level[p], n[p], theta[p], st);
            if (rc != SMC_OK) return rc;
        }
    }
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->groups.size(), st);
    for (size_t g = 0; g < b->groups.size() && e == cudaSuccess; ++g) {
        const auto& G = b->groups[g];
        if (G.N >= 128)   // the form single solves default to (two-CTA on 1/128)
            e = fem_eval_large_multi_launch(G.N, G.d_args, G.d_offsets, G.d_item_group, G.total, b->big_scratch,
                                            b->d_counters + g, st);
        else
            e = fem_eval_persistent_launch(G.N, G.precision, G.T, G.d_args, G.d_offsets, G.d_item_group, G.total,
                                           b->d_counters + g, st);
    }
    return e == cudaSuccess ? SMC_OK : SMC_ECUDA;
}

}  // namespace

}  // namespace mls2mc

using namespace mls2mc;

extern "C" {

int smc_batch_create(int n, smc_handle* const* handles, smc_batch** out) {
    if (!out || n < 1 || !handles) return SMC_EINVAL;
    *out = nullptr;
    Batch* b = new Batch();
    for (int i = 0; i < n; ++i) {
        Handle* h = reinterpret_cast<Handle*>(handles[i]);
        // the persistent multi-problem forms solve the Dirichlet problem only
        if (!h || h->forward_kind != SMC_FWD_FEM || h->flow_cell ||
            std::find(b->h.begin(), b->h.end(), h) != b->h.end()) {
            delete b;
            return SMC_EINVAL;
        }
        b->h.push_back(h);
    }
    *out = reinterpret_cast<smc_batch*>(b);
    return SMC_OK;
}

void smc_batch_destroy(smc_batch* bb) { delete reinterpret_cast<Batch*>(bb); }

const char* smc_batch_last_error(const smc_batch* bb) {
    return bb ? reinterpret_cast<const Batch*>(bb)->last_error.c_str() : "null batch";
}

int smc_batch_eval(smc_batch* bb, const int* level, const int* n, const double* const* theta, double* const* phi,
                   int* const* iters, void* stream, int use_graph) {
    if (!bb || !level || !n || !theta || !phi) return SMC_EINVAL;
    Batch* b = reinterpret_cast<Batch*>(bb);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (use_graph && !st) {
        b->last_error = "graph capture needs a non-default stream";
        return SMC_EINVAL;
    }
    const size_t P = b->h.size();
    std::vector<long long> sig;
    for (size_t p = 0; p < P; ++p) {
        Handle* h = b->h[p];
        if (level[p] < 0 || level[p] >= (int)h->levels.size() || n[p] < 0 || (n[p] > 0 && (!theta[p] || !phi[p]))) {
            b->last_error = "bad level, count or pointer for problem " + std::to_string(p);
            return SMC_EINVAL;
        }
        sig.insert(sig.end(), {(long long)level[p], (long long)n[p], (long long)(uintptr_t)theta[p],
                               (long long)(uintptr_t)phi[p], (long long)(uintptr_t)(iters ? iters[p] : nullptr)});
    }
    if (sig != b->signature) {
        b->free_groups();
        // one eager pass per problem first, so every buffer the syntheses need exists before capture
        for (size_t p = 0; p < P; ++p) {
            Handle* h = b->h[p];
            if (n[p] <= 0) continue;
            int rc = h->ensure_scratch(n[p]);
            if (rc == SMC_OK && h->precision == SMC_MIXED) rc = h->synth_kappa(level[p], n[p], theta[p], st);
            if (rc != SMC_OK) {
                b->last_error = h->last_error;
                return rc;
            }
        }
        std::map<std::pair<int, int>, size_t> gidx;
        for (size_t p = 0; p < P; ++p) {
            Handle* h = b->h[p];
            if (n[p] <= 0) continue;
            const Level& L = h->levels[level[p]];
            auto key = std::make_pair(L.N, h->precision);
            if (!gidx.count(key)) {
                gidx[key] = b->groups.size();
                Batch::Group G;
                G.N = L.N;
                G.precision = h->precision;
                // the persistent form has no compact variant: a compact size -T runs with T threads,
                // the same arithmetic
                G.T = std::abs(h->block_size(L.N));
                b->groups.push_back(G);
            }
            Batch::Group& G = b->groups[gidx[key]];
            FemArgs a = h->fem_args(level[p], n[p], theta[p], nullptr, phi[p], iters ? iters[p] : h->scratch_iters);
            a.kappa = h->precision == SMC_MIXED ? h->synth_kappa_buf : nullptr;
            G.offsets.push_back(G.total);
            G.args.push_back(a);
            G.total += n[p];
        }
        cudaError_t e = cudaMalloc((void**)&b->d_counters, sizeof(int) * std::max<size_t>(1, b->groups.size()));
        size_t big_need = 0;   // one scratch for all large groups: they run one after another
        for (auto& G : b->groups)
            if (G.N >= 128) big_need = std::max(big_need, fem_large_multi_scratch(G.N));
        if (e == cudaSuccess && big_need) e = cudaMalloc((void**)&b->big_scratch, big_need * sizeof(float));
        for (auto& G : b->groups) {
            if (e == cudaSuccess) e = cudaMalloc((void**)&G.d_args, sizeof(FemArgs) * G.args.size());
            if (e == cudaSuccess) e = cudaMalloc((void**)&G.d_offsets, sizeof(int) * G.offsets.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(G.d_args, G.args.data(), sizeof(FemArgs) * G.args.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(G.d_offsets, G.offsets.data(), sizeof(int) * G.offsets.size(), cudaMemcpyHostToDevice);
            std::vector<int> ig((size_t)std::max(G.total, 1), 0);
            for (size_t q = 0; q < G.offsets.size(); ++q) {
                const int end = q + 1 < G.offsets.size() ? G.offsets[q + 1] : G.total;
                for (int i = G.offsets[q]; i < end; ++i) ig[(size_t)i] = (int)q;
            }
            if (e == cudaSuccess) e = cudaMalloc((void**)&G.d_item_group, sizeof(int) * ig.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(G.d_item_group, ig.data(), sizeof(int) * ig.size(), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) {
            b->last_error = cudaGetErrorString(e);
            b->free_groups();
            return SMC_ENOMEM;
        }
        b->signature = sig;
    }
    if (!use_graph) return enqueue(b, level, n, theta, st);
    if (!b->exec) {
        const long long k0 = launch_count();
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            b->last_error = cudaGetErrorString(e);
            return SMC_ECUDA;
        }
        const int rc = enqueue(b, level, n, theta, st);
        e = cudaStreamEndCapture(st, &b->graph);
        if (rc != SMC_OK || e != cudaSuccess) {
            b->last_error = "graph capture failed";
            if (b->graph) cudaGraphDestroy(b->graph);
            b->graph = nullptr;
            return rc != SMC_OK ? rc : SMC_ECUDA;
        }
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            b->last_error = cudaGetErrorString(e);
            return SMC_ECUDA;
        }
        b->graph_kernels = launch_count() - k0;
        count_launches(-b->graph_kernels);   // counted when the graph runs, not when it is captured
    }
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) {
        b->last_error = cudaGetErrorString(e);
        return SMC_ECUDA;
    }
    count_launches(b->graph_kernels);
    return SMC_OK;
}

}  // extern "C"
