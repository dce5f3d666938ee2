// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mls2mc.h"

namespace mls2mc {

// ---- host set-up (kl_host.cpp) ---------------------------------------------------------
void kl_eig_1d(double corr_len, int n_modes, std::vector<double>& lam, std::vector<double>& omega);
void kl_table(int N, double corr_len, double variance, int K, std::vector<double>& psi,
              std::vector<double>& lambda);
// eigen-decomposition of a symmetric n x n matrix a (row-major, destroyed) (sym_eigen.cpp):
// eigenvalues to w (unordered), eigenvector i to row i of vt; false if the QR iteration stalls
bool symmetric_eigen(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>& vt);
// Matern (smoothness 3/2) KL table by the Nystrom method (matern_host.cpp); K <= matern_max_terms()
// (false if the eigen-solve failed)
int matern_max_terms();
bool matern_kl_table(int N, double corr_len, double variance, int K, std::vector<double>& psi,
                     std::vector<double>& lambda);
// load vector of the nine-source term of Example 5.1 at the nodes of level N (padded row layout
// below, zero at Dirichlet nodes and padding); bnorm2 = sum of squares over the interior nodes
void nine_source_load(int N, std::vector<double>& b, double& bnorm2);
// Nodes of a level with NL cells per side are stored row by row with row stride NL + 2 (one
// padding word per row, never read): with an even stride, nodes of one red-black colour in two
// adjacent rows fall on shared-memory banks of opposite parity.
__host__ __device__ constexpr int fem_row_stride(int NL) { return NL + 2; }
// node indices j * fem_row_stride(N) + i of the three P1 vertices of each observation
void obs_table(int N, int n_obs, const double* xy, std::vector<int>& idx, std::vector<double>& wts);

// ---- kernel launch counter (api.cpp): every kernel the library launches is counted ------
void count_launches(long long n);
long long launch_count();

// ---- forward solve (fem_solve.cu) -------------------------------------------------------
struct FemArgs {
    int N;                  // cells per side of this level (power of two, 4..64)
    int precision;          // SMC_FP64 or SMC_MIXED
    int n;                  // particles
    int K;                  // KL terms
    const double* theta;    // [n][K] device
    const void* psi;        // [K][2N^2] device, double (FP64) or float (MIXED)
    const float* kappa;     // [n][2N^2] kappa = exp(u) per triangle (MIXED: from the tensor-core synthesis), or null
    const int* obs_idx;     // [n_obs][3] node indices j * fem_row_stride(N) + i
    const double* obs_w;    // [n_obs][3] P1 weights
    int n_obs;
    const double* y;        // [n_obs]
    double inv_sigma2;      // 1 / sigma^2
    double* G;              // [n][n_obs] or null
    double* Phi;            // [n]
    int* iters;             // [n] or null
    double rtol;            // FP64 relative residual target
    double rtol_in;         // relative reduction of each inner CG pass
    int max_outer;          // refinement passes
    int max_inner;          // inner CG iterations per pass
    const void* rhs;        // load vector at the nodes (padded row layout): double (FP64) or float2
                            // (MIXED: hi, lo with hi + lo = the FP64 value); null: f = 1 (b = h^2)
    double bnorm2;          // sum of squares of the load vector over the interior nodes (with rhs)
    int flow_cell;          // 1: the flow cell of Example 5.3 (p = 0 / 1 on x = 0 / 1, no flow on
                            // y = 0, 1, f = 0; levels 1/8 .. 1/256, FP64 to 1/32; no compact or
                            // batched form)
};
// Returns cudaSuccess or the launch error.
// T = threads per particle (one of fem_block_sizes; <= 0: the first, the default)
cudaError_t fem_eval_launch(const FemArgs& a, cudaStream_t stream, int T = 0);
std::vector<int> fem_block_sizes(int N, int precision);
// the size used when none is set (negative: a compact form)
int fem_default_block(int N, int precision);
// large levels (1/h = 128, 256; mixed precision, kappa from the synthesis): hierarchy in global
// scratch, blocks x fem_global_slice(N) floats; *counter (device) is reset by the launch
size_t fem_global_slice(int N, bool FC = false);   // FC: the flow cell's layout
int fem_global_blocks(int N);
cudaError_t fem_eval_global_launch(const FemArgs& a, float* scratch, int blocks, int* counter, cudaStream_t st);
// large levels of many problems (groups, offsets, item_group as for fem_eval_persistent_launch;
// *counter zero before the launch), blocks x fem_global_slice(N) floats of scratch
cudaError_t fem_eval_global_multi_launch(int N, const FemArgs* groups, const int* offsets, const int* item_group,
                                         int total, float* scratch, int blocks, int* counter, cudaStream_t st);
// persistent multi-problem launch: groups[g] (device array) are the launch arguments of one
// problem at level size N; offsets[g] (device) the first work item of group g; item_group[i]
// (device) the group of item i; *counter (device, zero before the launch) hands out the total
// items to the blocks
cudaError_t fem_eval_persistent_launch(int N, int precision, int T, const FemArgs* groups, const int* offsets,
                                       const int* item_group, int total, int* counter, cudaStream_t st);
// compact form of the mixed solve (negative block sizes of fem_block_sizes: -512 at 1/h = 64,
// -256 at 1/h = 32): two or four blocks per SM, fem_compact_blocks(N, T) persistent blocks
// (0 for a configuration that is not compiled) with fem_compact_ref_floats(N, T) floats of device
// scratch each for the refinement state; *counter (device) is reset by the launch
int fem_compact_blocks(int N, int T);
size_t fem_compact_ref_floats(int N, int T);
cudaError_t fem_eval_compact_launch(const FemArgs& a, int T, float* ref_scratch, int blocks, int* counter,
                                    cudaStream_t st);
// two-CTA cluster form of the mixed 1/128 solve (block size -1024 of fem_block_sizes): the fine
// level split in row strips over the two CTAs of a cluster, each on its own SM;
// fem_cluster_blocks() CTAs (0 where no cluster fits) with fem_cluster_ref_floats() floats of
// device scratch each for the refinement state; *counter (device) is reset by the launch
int fem_cluster_blocks();
size_t fem_cluster_ref_floats();
cudaError_t fem_eval_cluster_launch(const FemArgs& a, float* ref_scratch, int blocks, int* counter, cudaStream_t st);
// large levels of many problems in the form single solves default to: the two-CTA form on 1/128
// (mixed, not the flow cell) where a cluster fits, else the device-memory form; scratch floats it
// needs (sized before any graph capture) and the launch (*counter zero before it)
bool fem_cluster_form(int N, int precision, bool flow_cell);
size_t fem_large_multi_scratch(int N);
cudaError_t fem_eval_large_multi_launch(int N, const FemArgs* groups, const int* offsets, const int* item_group,
                                        int total, float* scratch, int* counter, cudaStream_t st);
bool fem_level_supported(int N, int precision);

}  // namespace mls2mc
