// A batch of independent inverse problems (internal; C ABI smc_batch_*): the handles, the tables and
// CUDA graph of the multi-problem evaluation (batch.cpp), and the batched sampler's state
// (batch_sampler.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "handle.h"

namespace mls2mc {

struct BatchSampler;
void batch_sampler_free(BatchSampler* s);

struct Batch {
    std::vector<Handle*> h;
    struct Group {
        int N = 0, precision = 0, T = 0, total = 0;
        std::vector<FemArgs> args;
        std::vector<int> offsets;
        FemArgs* d_args = nullptr;
        int* d_offsets = nullptr;
        int* d_item_group = nullptr;   // group of each work item
    };
    std::vector<Group> groups;
    int* d_counters = nullptr;
    float* big_scratch = nullptr;    // per-block (per-CTA) scratch of the groups of large levels (1/h >= 128)
    std::vector<long long> signature;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long graph_kernels = 0;
    std::string last_error;
    BatchSampler* smp = nullptr;   // state of the batched sampler, made on its first step
    bool owns_handles = false;     // made by smc_init_batch: the handles are destroyed with the batch

    void free_groups() {
        for (auto& g : groups) {
            cudaFree(g.d_args);
            cudaFree(g.d_offsets);
            cudaFree(g.d_item_group);
        }
        groups.clear();
        cudaFree(d_counters);
        d_counters = nullptr;
        cudaFree(big_scratch);
        big_scratch = nullptr;
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~Batch() {
        free_groups();
        batch_sampler_free(smp);
        if (owns_handles)
            for (Handle* x : h) smc_destroy(reinterpret_cast<smc_handle*>(x));
    }
};

}  // namespace mls2mc
