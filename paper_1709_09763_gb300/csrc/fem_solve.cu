// Batched likelihood evaluation G_l(theta), Phi_l(theta) on one mesh level.
//
// Path (Sec. 2.1, Sec. 5): theta -> u = theta . Psi on every triangle (Eq. truncKL)
// -> kappa = exp(u) -> P1 FEM solve of -div(kappa grad p) = f, p = 0 on the
// boundary -> observations p(d_n) -> Phi = 1/2 sum ((y - G)/sigma)^2 (Eq. phi).
//
// Design: one thread block owns one particle and keeps its whole problem on chip.
// For P1 elements on the uniform mesh whose cells are split by the (i,j)-(i+1,j+1)
// diagonal the stiffness matrix is a 5-point stencil: edge (i,j)-(i+1,j) has
// weight (kappa_lower(i,j) + kappa_upper(i,j-1))/2, edge (i,j)-(i,j+1) has weight
// (kappa_lower(i-1,j) + kappa_upper(i,j))/2, and diagonal-edge couplings vanish. The
// load of f = 1 is h^2 at every interior node; any other f comes as a load-vector table
// (the nine sources of Example 5.1). The linear system is solved matrix-free by
// multigrid-preconditioned CG:
//  * hierarchy N, N/2, ..., 2 cells per side; the coarse mesh is nested, the
//    prolongation is P1 interpolation and restriction its transpose, and the
//    coarse operator is the same stencil built from the mean kappa of the four
//    fine triangles inside each coarse triangle -- for piecewise-constant kappa
//    this equals the Galerkin product P^T A P exactly;
//  * symmetric V(1,1) cycle with red-black Gauss-Seidel (red-black before the
//    coarse correction, black-red after), fused so that each level needs five barriers;
//    the coarsest level is solved exactly (the 9 x 9 inverse at 1/4 on the FP32 path,
//    the single node at 1/2 otherwise);
//  * SMC_MIXED: the field, stencil, multigrid and CG run in FP32; each pass ends
//    with the update of the residual r <- r - A d in double-float arithmetic, in edge
//    form sum_e a_e (d_i - d_j) from the FP32 edge weights (so its diagonal is their
//    exact sum), and x <- x + d, until the relative residual reaches rtol
//    (mixed-precision iterative refinement, no FP64 instruction in the solve);
//    SMC_FP64: the same algorithm in FP64 throughout.
// Shared memory holds, per level, the edge weights aE, aN, the inverse diagonal and the
// vectors e (multigrid correction), res (residual) and rhs (fine level: the CG
// direction p). The fine-level CG vectors r, d, z, p of a thread's nodes live in
// registers (every fine node belongs to one thread for the whole solve); the
// refinement state x, r (double-float pairs) lives in shared memory, or in a per-block
// slice of device memory in the compact forms (two or four blocks per SM, coarse levels
// without residual and inverse-diagonal arrays). Level 1/128 is solved by a cluster of two CTAs
// on two SMs, each keeping half of the fine rows on chip (fem_eval_cluster); levels 1/128 (block
// size 1024, the flow cell) and 1/256 can keep their two finest levels in device memory
// (fem_eval_global).
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace mls2mc {

namespace {

__host__ __device__ constexpr int padded(int n) { return (n + 3) & ~3; }
// FC (the flow cell of Example 5.3): the rows j = 0 and j = NL are unknowns, so every array of a
// level gets a zero ghost row below and above (NL + 3 rows, the array pointer on row 0)
__host__ __device__ constexpr int lvl_size(int NL, bool FC = false) {
    return padded((NL + (FC ? 3 : 1)) * fem_row_stride(NL));
}
// element offset of level NL inside the shared arena of a hierarchy with top level N
__host__ __device__ constexpr int lvl_offset(int N, int NL, bool FC = false) {
    return N == NL ? 0 : 6 * lvl_size(N, FC) + lvl_offset(N / 2, NL, FC);
}
__host__ __device__ constexpr int arena_size(int N, bool FC = false) {
    return N < 2 ? 0 : 6 * lvl_size(N, FC) + arena_size(N / 2, FC);
}

template <typename Real>
struct Lv {
    Real *aE, *aN, *iD, *e, *res, *rhs;   // iD: inverse of the stencil diagonal
};

// Compact hierarchy (two blocks per SM at 1/64): the top level keeps five arrays (res shares
// the storage of rhs, which holds the CG direction p: p is dead while the V-cycle runs, its
// values live in registers), the coarse levels four (aE, aN, e, rhs: no res, and the inverse
// diagonal is formed from the edge weights where a sweep needs it).
__host__ __device__ constexpr int coarse_size_cp(int NL) { return NL < 2 ? 0 : 4 * lvl_size(NL) + coarse_size_cp(NL / 2); }
__host__ __device__ constexpr int coarse_offset_cp(int NL, int NC) {
    return NL == NC ? 0 : 4 * lvl_size(NL) + coarse_offset_cp(NL / 2, NC);
}
__host__ __device__ constexpr int arena_size_cp(int N) { return 5 * lvl_size(N) + coarse_size_cp(N / 2); }

template <typename Real, int N, int NL, int CP = 0, bool FC = false>
__device__ __forceinline__ Lv<Real> level_ptrs(Real* arena) {
    if constexpr (FC) {   // ghost row -1 first: each pointer is one row stride into its array
        constexpr int z = lvl_size(NL, true);
        Real* b = arena + lvl_offset(N, NL, true) + fem_row_stride(NL);
        return Lv<Real>{b, b + z, b + 2 * z, b + 3 * z, b + 4 * z, b + 5 * z};
    }
    constexpr int z = lvl_size(NL);
    if constexpr (!CP) {
        Real* b = arena + lvl_offset(N, NL);
        return Lv<Real>{b, b + z, b + 2 * z, b + 3 * z, b + 4 * z, b + 5 * z};
    } else if constexpr (CP == 2) {   // coarse levels N/2 .. 2 alone, from the arena's start
        static_assert(NL < N, "the two-CTA form keeps its top level apart");
        Real* b = arena + coarse_offset_cp(N / 2, NL);
        return Lv<Real>{b, b + z, nullptr, b + 2 * z, nullptr, b + 3 * z};
    } else if constexpr (NL == N) {
        Real* b = arena;
        return Lv<Real>{b, b + z, b + 2 * z, b + 3 * z, b + 4 * z, b + 4 * z};
    } else {
        Real* b = arena + 5 * lvl_size(N) + coarse_offset_cp(N / 2, NL);
        return Lv<Real>{b, b + z, nullptr, b + 2 * z, nullptr, b + 3 * z};
    }
}

// load vector at node n from a table: FP64 values, or (hi, lo) float pairs with hi + lo = b
__device__ __forceinline__ void load_rhs(const void* t, int n, double& hi, double& lo) {
    hi = static_cast<const double*>(t)[n];
    lo = 0.0;
}
__device__ __forceinline__ void load_rhs(const void* t, int n, float& hi, float& lo) {
    const float2 v = static_cast<const float2*>(t)[n];
    hi = v.x;
    lo = v.y;
}

// 1 / x rounded to nearest (the same value as the IEEE division 1 / x)
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
// The smoother's inverse diagonals on the coarse levels: the approximate reciprocal of the special
// function unit (one instruction, relative error below 2^-22) on the FP32 path. They only shape the
// multigrid preconditioner -- the CG operator and the refinement residual use the edge weights --
// and the preconditioner stays symmetric because every sweep uses the same value at a node.
__device__ __forceinline__ float recip_coarse(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double recip_coarse(double x) { return __drcp_rn(x); }

// inverse stencil diagonal at interior node n: stored, or formed from the four edge weights
// (the same expression and order as where it is stored)
template <typename Real, int S>
__device__ __forceinline__ Real inv_diag(const Lv<Real>& L, int n) {
    if (L.iD) return L.iD[n];
    return recip_coarse(L.aE[n] + L.aE[n - 1] + L.aN[n] + L.aN[n - S]);
}

// sum of a_nb * v_nb over the four stencil neighbours of padded node n (row stride S)
template <typename Real, int S>
__device__ __forceinline__ Real offsum(const Real* aE, const Real* aN, const Real* v, int n) {
    return aE[n] * v[n + 1] + aE[n - 1] * v[n - 1] + aN[n] * v[n + S] + aN[n - S] * v[n - S];
}

// (A v)_n in edge form: sum over the four edges at n of a_e (v_n - v_nb); the diagonal is
// the sum of the edge weights by construction
template <typename Real, int S>
__device__ __forceinline__ Real stencil_apply(const Real* aE, const Real* aN, const Real* v, int n) {
    const Real vn = v[n];
    return aE[n] * (vn - v[n + 1]) + aE[n - 1] * (vn - v[n - 1]) + aN[n] * (vn - v[n + S]) +
           aN[n - S] * (vn - v[n - S]);
}

// the same with the value at n supplied by the caller (held in a register)
template <typename Real, int S>
__device__ __forceinline__ Real stencil_apply_at(const Real* aE, const Real* aN, const Real* v, int n, Real vn) {
    return aE[n] * (vn - v[n + 1]) + aE[n - 1] * (vn - v[n - 1]) + aN[n] * (vn - v[n + S]) +
           aN[n - S] * (vn - v[n - S]);
}

// ---- block reductions (every thread gets the same result, summed in a fixed order) ----
template <int T, typename Acc>
__device__ __forceinline__ void block_sum(Acc& a, double* buf_raw) {
    Acc* buf = reinterpret_cast<Acc*>(buf_raw);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if ((threadIdx.x & 31) == 0) buf[threadIdx.x >> 5] = a;
    __syncthreads();
    Acc s = 0;
#pragma unroll
    for (int i = 0; i < T / 32; ++i) s += buf[i];
    a = s;
}

// ---- error-free transformations (Knuth TwoSum, Dekker), double-float accumulation ----
template <typename Real>
__device__ __forceinline__ void two_sum(Real a, Real b, Real& s, Real& e) {
    s = a + b;
    const Real bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (ah, al) += (bh, bl), result renormalised so that |al| <= ulp(ah)/2
template <typename Real>
__device__ __forceinline__ void df_add(Real& ah, Real& al, Real bh, Real bl) {
    Real s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    ah = s + e;
    al = e - (ah - s);
}

// ---- red/black enumeration -----------------------------------------------------------------
// Position k of colour col (0 red: i + j even, 1 black) on a level with NL cells per side. A
// colour has NL/2 positions per row (the last one idle in rows with NL/2 - 1 nodes of that
// colour); 2G consecutive positions (G = min(16, NL/2)) take G positions of row 2R + 1 and the
// same positions of row 2R + 2. With the even row stride the two rows' nodes of one colour lie on
// banks of opposite parity, so for NL >= 32 a warp's 32 accesses hit 32 distinct banks. All
// divisions are by powers of two. Returns false for idle positions.
// FC: rows 0 .. NL are unknowns (pairs 2R, 2R + 1), colour_positions<NL, true> positions.
template <int NL, bool FC = false>
__host__ __device__ constexpr int colour_positions() { return FC ? (NL / 2 + 1) * NL : NL * NL / 2; }
template <int NL, bool FC = false>
__device__ __forceinline__ bool colour_node(int k, int col, int& i, int& j) {
    constexpr int G = NL / 2 < 16 ? NL / 2 : 16;
    const int blk = k / (2 * G), l = k - blk * 2 * G;
    const int R = blk / (NL / 2 / G), sg = blk - R * (NL / 2 / G);
    j = 2 * R + (FC ? 0 : 1) + l / G;
    i = (((j & 1) ^ col) ? 1 : 2) + 2 * (sg * G + l % G);
    return k < colour_positions<NL, FC>() && j <= (FC ? NL : NL - 1) && i <= NL - 1;
}

// ---- coarse-level multigrid pieces (rhs in shared memory) --------------------------------
// V(1,1) with red-black Gauss-Seidel: pre-smoothing red then black from e = 0, post-smoothing
// black then red (a symmetric preconditioner). Two identities of the red-black ordering remove
// passes from the textbook cycle:
//  - after the black pre-sweep every black node satisfies its equation (zero residual) and the
//    residual of a red node is the off-diagonal sum of the new black values (the red node held
//    its equation before), so the restriction needs residuals at red nodes only;
//  - Gauss-Seidel overwrites a node from its neighbours alone, so the coarse correction added to
//    the black nodes and the red nodes' pre-sweep values are never read: the black post-sweep
//    reads its red neighbours as e + P e_c directly.
template <typename Real, int NL, int T, bool FC = false>
__device__ __forceinline__ void smooth_color(const Lv<Real>& L, int color) {
    constexpr int S = fem_row_stride(NL);
    for (int k = threadIdx.x; k < colour_positions<NL, FC>(); k += T) {
        int i, j;
        if (!colour_node<NL, FC>(k, color, i, j)) continue;
        const int n = j * S + i;
        L.e[n] = (L.rhs[n] + offsum<Real, S>(L.aE, L.aN, L.e, n)) * inv_diag<Real, S>(L, n);
    }
}

// coarse rhs = P^T (fine residual) after the red and black pre-sweeps. P^T takes weight 1 from
// the coincident fine node and 1/2 from its six neighbours along the mesh directions (+-x, +-y
// and the (1,1) diagonal); of these only the coincident node and the two diagonal neighbours are
// red, and their residuals are the off-diagonal sums of the black values.
//
// The coarse level's red pre-sweep from zero (e = rhs / D at red nodes) is folded in: it needs
// nothing but the node's own rhs.
template <typename Real, int NC, int T, bool FC = false>
__device__ __forceinline__ void restrict_red(const Lv<Real>& F, const Lv<Real>& C) {
    constexpr int MC = NC - 1, SC = fem_row_stride(NC), SF = fem_row_stride(2 * NC);
    constexpr int ROWS = FC ? NC + 1 : MC, ROW0 = FC ? 0 : 1;   // coarse rows with unknowns
    for (int idx = threadIdx.x; idx < MC * ROWS; idx += T) {
        const int J = idx / MC + ROW0, I = idx - (J - ROW0) * MC + 1;
        const int f = (2 * J) * SF + 2 * I, c = J * SC + I;
        const Real v = offsum<Real, SF>(F.aE, F.aN, F.e, f) +
                       Real(0.5) * (offsum<Real, SF>(F.aE, F.aN, F.e, f + SF + 1) +
                                    offsum<Real, SF>(F.aE, F.aN, F.e, f - SF - 1));
        C.rhs[c] = v;
        if (((I + J) & 1) == 0) C.e[c] = v * inv_diag<Real, SC>(C, c);
    }
}

// the same restriction from red residuals stored in res (fine level of the on-chip solve, where
// each thread computes the residuals of its own red nodes first)
template <typename Real, int NC, int T, bool FC = false>
__device__ __forceinline__ void restrict_gather(const Real* res, const Lv<Real>& C) {
    constexpr int MC = NC - 1, SC = fem_row_stride(NC), SF = fem_row_stride(2 * NC);
    constexpr int ROWS = FC ? NC + 1 : MC, ROW0 = FC ? 0 : 1;
    for (int idx = threadIdx.x; idx < MC * ROWS; idx += T) {
        const int J = idx / MC + ROW0, I = idx - (J - ROW0) * MC + 1;
        const int f = (2 * J) * SF + 2 * I, c = J * SC + I;
        const Real v = res[f] + Real(0.5) * (res[f + SF + 1] + res[f - SF - 1]);
        C.rhs[c] = v;
        if (((I + J) & 1) == 0) C.e[c] = v * inv_diag<Real, SC>(C, c);
    }
}

// zero the boundary rings of e, res, rhs on every level from NL down (interior values are always
// written before they are read; the rings must read as zero)
template <typename Real, int N, int NL, int T, int CP = 0, bool FC = false>
__device__ __forceinline__ void zero_rings(Real* arena) {
    constexpr int S = fem_row_stride(NL);
    const Lv<Real> L = level_ptrs<Real, N, NL, CP, FC>(arena);
    if constexpr (FC) {
        // ghost rows -1 and NL + 1 (whole rows), and the Dirichlet columns 0 and NL and the padding
        // column NL + 1 of rows 0 .. NL; rows 0 and NL are unknowns here
        for (int k = threadIdx.x; k < 2 * S + 3 * (NL + 1); k += T) {
            const int n = k < S ? k - S : k < 2 * S ? (NL + 1) * S + (k - S)
                        : ((k - 2 * S) / 3) * S + ((k - 2 * S) % 3 == 0 ? 0 : (k - 2 * S) % 3 == 1 ? NL : NL + 1);
            L.e[n] = L.rhs[n] = L.res[n] = Real(0);
        }
        if constexpr (NL > 4) zero_rings<Real, N, NL / 2, T, false, true>(arena);
        return;
    }
    for (int k = threadIdx.x; k < 4 * NL; k += T) {   // rows 0 and NL, then columns 0 and NL
        const int n = k <= NL ? k : k <= 2 * NL + 1 ? NL * S + (k - NL - 1)
                                                     : (1 + ((k - 2 * NL - 2) >> 1)) * S + (((k - 2 * NL - 2) & 1) ? NL : 0);
        L.e[n] = L.rhs[n] = Real(0);
        if (L.res) L.res[n] = Real(0);
    }
    if constexpr (NL > 2) zero_rings<Real, N, NL / 2, T, CP>(arena);
}

// off-diagonal sum at black node n = (i, j) with its red neighbours read as e + P e_c (P1
// interpolation of the coarse correction ec). c0 = (j/2) SC + i/2 (integer halves) is the
// coarse node at or below-left of n; jeven selects which neighbours coincide with coarse nodes.
template <typename Real, int S, int SC>
__device__ __forceinline__ Real offsum_prolong(const Real* aE, const Real* aN, const Real* e, const Real* ec, int n,
                                               int c0, bool jeven) {
    // both cases read ec at c0 and c0 + SC + 1 (the diagonal pair) and at two more nodes
    const Real e0 = ec[c0], e1 = ec[c0 + SC + 1];
    const Real eu = ec[jeven ? c0 + 1 : c0 + SC], ev = ec[jeven ? c0 - SC : c0 - 1];
    const Real dg = Real(0.5) * (e0 + e1), hf = Real(0.5) * (ev + eu);
    // i odd (j even): E, W coincide with coarse nodes, N, S lie on coarse diagonals; i even: the reverse
    const Real pE = jeven ? eu : dg, pW = jeven ? e0 : hf, pN = jeven ? dg : eu, pS = jeven ? hf : e0;
    return aE[n] * (e[n + 1] + pE) + aE[n - 1] * (e[n - 1] + pW) + aN[n] * (e[n + S] + pN) +
           aN[n - S] * (e[n - S] + pS);
}

// black post-sweep with the coarse correction of level NL / 2 folded in
template <typename Real, int NL, int T, bool FC = false>
__device__ __forceinline__ void black_prolong(const Lv<Real>& L, const Real* ec) {
    constexpr int S = fem_row_stride(NL), SC = fem_row_stride(NL / 2);
    for (int k = threadIdx.x; k < colour_positions<NL, FC>(); k += T) {
        int i, j;
        if (!colour_node<NL, FC>(k, 1, i, j)) continue;
        const int n = j * S + i;
        const int c0 = (j >> 1) * SC + (i >> 1);
        L.e[n] = (L.rhs[n] + offsum_prolong<Real, S, SC>(L.aE, L.aN, L.e, ec, n, c0, (j & 1) == 0)) *
                 inv_diag<Real, S>(L, n);
    }
}

// ---- exact solve on the coarsest level kept ------------------------------------------------
// The multigrid recursion stops at level direct_level(N) (1/4 for N >= 16; below that the
// setup costs more than the cycles it saves): there the Galerkin operator (the same 5-point stencil,
// m = (NL - 1)^2 = 9 unknowns) is inverted once per particle and applied as a dense
// matrix-vector product, replacing the cycles of the levels below it. (An exact solve one level
// higher, m = 49, lowers the iteration count by about 8 % but its m^3 setup costs more than that.)
// The FP64 path keeps the full cycle: its Gauss-Jordan setup would run on the FP64 pipe, which
// on this part costs more than the cycles it saves.
// The flow cell (FC) always stops at 1/4 (15 unknowns: rows 0 .. 4 of columns 1 .. 3), on both
// paths: its coarsest levels would need the boundary rows in the single-node solve.
template <typename Real, bool FC = false>
__host__ __device__ constexpr int direct_level(int N) {
    return FC ? (N >= 8 ? 4 : 0) : sizeof(Real) == 8 ? 0 : (N >= 16 ? 4 : 0);
}
// unknowns of the dense level NL: (NL - 1)^2, or (NL - 1)(NL + 1) for the flow cell
__host__ __device__ constexpr int dense_unknowns(int NL, bool FC) { return (NL - 1) * (FC ? NL + 1 : NL - 1); }
template <typename Real, bool FC = false>
__host__ __device__ constexpr int dense_reals(int N) {
    return direct_level<Real, FC>(N) ? padded(dense_unknowns(direct_level<Real, FC>(N), FC) *
                                              (dense_unknowns(direct_level<Real, FC>(N), FC) + 4))
                                     : 0;
}

// Ainv [m][m] := A^{-1} by in-place Gauss-Jordan elimination without pivoting (A is symmetric
// positive definite). Step k turns row k into row k / a_kk, column k into -column k / a_kk, the
// pivot into 1 / a_kk and every other entry into a_uv - a_uk a_kv / a_kk; the old row and column
// k are read from a buffer that step k - 1 filled, so one barrier per step suffices (a warp
// barrier when one warp runs it, T = 32).
// Ainv is followed by that buffer: [2][row | column], 4m Reals.
template <typename Real, int NL, int T, bool FC = false>
__device__ void dense_setup(const Lv<Real>& L, Real* Ainv) {
    constexpr int MM = NL - 1, m = dense_unknowns(NL, FC), S = fem_row_stride(NL), ROW0 = FC ? 0 : 1;
    Real* buf = Ainv + m * m;
    for (int idx = threadIdx.x; idx < m * m; idx += T) {
        const int u = idx / m, v = idx - u * m;
        const int ui = u % MM, uj = u / MM, vi = v % MM, vj = v / MM;
        const int n = (uj + ROW0) * S + ui + 1;
        Real val = 0;
        if (u == v) val = L.aE[n] + L.aE[n - 1] + L.aN[n] + L.aN[n - S];
        else if (uj == vj && vi == ui + 1) val = -L.aE[n];
        else if (uj == vj && vi == ui - 1) val = -L.aE[n - 1];
        else if (ui == vi && vj == uj + 1) val = -L.aN[n];
        else if (ui == vi && vj == uj - 1) val = -L.aN[n - S];
        Ainv[idx] = val;
        if (u == 0) buf[v] = val;
        if (v == 0) buf[m + u] = val;
    }
    if constexpr (T == 32) __syncwarp(); else __syncthreads();
    for (int k = 0; k < m; ++k) {
        const Real* rowk = buf + (k & 1) * 2 * m;
        const Real* colk = rowk + m;
        Real* rown = buf + ((k + 1) & 1) * 2 * m;
        Real* coln = rown + m;
        const Real ip = Real(1) / rowk[k];
        for (int idx = threadIdx.x; idx < m * m; idx += T) {
            const int u = idx / m, v = idx - u * m;
            Real val;
            if (u == k) val = (v == k) ? ip : rowk[v] * ip;
            else if (v == k) val = -colk[u] * ip;
            else val = Ainv[idx] - colk[u] * rowk[v] * ip;
            Ainv[idx] = val;
            if (u == k + 1) rown[v] = val;
            if (v == k + 1) coln[u] = val;
        }
        if constexpr (T == 32) __syncwarp(); else __syncthreads();
    }
}

// L.e = Ainv L.rhs on the interior nodes: 8 lanes per row, reduced by warp shuffles
template <typename Real, int NL, int T, bool FC = false>
__device__ __forceinline__ void dense_solve(const Lv<Real>& L, const Real* Ainv) {
    constexpr int MM = NL - 1, m = dense_unknowns(NL, FC), S = fem_row_stride(NL), ROW0 = FC ? 0 : 1;
    constexpr int W = (m * 8 + 31) / 32 * 32;   // whole warps: every lane takes part in the shuffles
    for (int w = threadIdx.x; w < W; w += T) {
        const int u = w >> 3, part = w & 7;
        Real acc = 0;
        if (u < m)
            for (int v = part; v < m; v += 8) acc = fma(Ainv[u * m + v], L.rhs[(v / MM + ROW0) * S + v % MM + 1], acc);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (part == 0 && u < m) L.e[(u / MM + ROW0) * S + u % MM + 1] = acc;
    }
}

// barrier between the phases of a V-cycle: the whole block, or only warp 0 on the small levels
template <bool WARP>
__device__ __forceinline__ void phase_sync() {
    if constexpr (WARP) __syncwarp();
    else __syncthreads();
}

// V(1,1) cycle on a coarse level: reads L.rhs, writes L.e. Levels with at most 4 cells per side
// (<= 9 unknowns) run inside warp 0 only (T = 32, warp barriers); the caller's next block
// barrier publishes the result.
template <typename Real, int N, int NL, int T, bool WARP = false, int CP = 0, bool FC = false>
__device__ void vcycle_coarse(Real* arena, const Real* dinv) {
    if constexpr (NL == direct_level<Real, FC>(N)) {
        dense_solve<Real, NL, T, FC>(level_ptrs<Real, N, NL, CP, FC>(arena), dinv);
        phase_sync<WARP>();
    } else if constexpr (!WARP && NL <= 4) {
        if (threadIdx.x < 32) vcycle_coarse<Real, N, NL, 32, true, CP, FC>(arena, dinv);
        __syncthreads();
        return;
    } else {
        Lv<Real> L = level_ptrs<Real, N, NL, CP, FC>(arena);
        if constexpr (NL == 2) {
            constexpr int n11 = fem_row_stride(2) + 1;           // single interior node (1,1)
            if (threadIdx.x == 0) L.e[n11] = L.rhs[n11] * inv_diag<Real, fem_row_stride(2)>(L, n11);
            phase_sync<WARP>();
        } else {
            Lv<Real> C = level_ptrs<Real, N, NL / 2, CP, FC>(arena);
            smooth_color<Real, NL, T, FC>(L, 1);   // red pre-sweep done by the restriction above
            phase_sync<WARP>();
            restrict_red<Real, NL / 2, T, FC>(L, C);
            phase_sync<WARP>();
            vcycle_coarse<Real, N, NL / 2, T, WARP, CP, FC>(arena, dinv);
            black_prolong<Real, NL, T, FC>(L, C.e);
            phase_sync<WARP>();
            smooth_color<Real, NL, T, FC>(L, 0);
            phase_sync<WARP>();
        }
    }
}

// ---- stencil coefficients from per-triangle kappa ----------------------------------------
// kappa in element order e = 2*(j*NL+i) + t (t = 0 lower, 1 upper half of cell (i, j))
template <typename Real, int NL, int T>
__device__ __forceinline__ void build_coeffs(const Lv<Real>& L, const Real* kap) {
    constexpr int S = fem_row_stride(NL);
    for (int n = threadIdx.x; n < (NL + 1) * S; n += T) {
        const int j = n / S, i = n - j * S;
        Real ae = 0, an = 0;
        if (i > NL) {   // padding column
            L.aE[n] = L.aN[n] = Real(0);
            continue;
        }
        if (i < NL) {   // horizontal edge (i,j)-(i+1,j): lower of cell (i,j), upper of cell (i,j-1)
            if (j < NL) ae += kap[2 * (j * NL + i)];
            if (j > 0) ae += kap[2 * ((j - 1) * NL + i) + 1];
        }
        if (j < NL) {   // vertical edge (i,j)-(i,j+1): lower of cell (i-1,j), upper of cell (i,j)
            if (i > 0) an += kap[2 * (j * NL + i - 1)];
            if (i < NL) an += kap[2 * (j * NL + i) + 1];
        }
        L.aE[n] = Real(0.5) * ae;
        L.aN[n] = Real(0.5) * an;
    }
}

template <typename Real, int NL, int T, bool FC = false, bool COARSE = false>
__device__ __forceinline__ void build_diag(const Lv<Real>& L) {
    constexpr int S = fem_row_stride(NL);
    for (int n = threadIdx.x; n < (NL + 1) * S; n += T) {
        const int j = n / S, i = n - j * S;
        Real d = 0;   // the flow cell's boundary rows read the zero ghost rows for their missing edges
        if (i > 0 && i < NL && (FC || (j > 0 && j < NL))) d = L.aE[n] + L.aE[n - 1] + L.aN[n] + L.aN[n - S];
        L.iD[n] = (d == Real(0)) ? Real(1) : COARSE ? recip_coarse(d) : recip(d);   // boundary entries are never used
    }
}

// mean kappa of the four fine triangles inside each coarse triangle
template <typename Real, int NC, int T>
__device__ __forceinline__ void coarsen_kappa(const Real* kf, Real* kc) {
    constexpr int NF = 2 * NC;
    for (int c = threadIdx.x; c < NC * NC; c += T) {
        const int J = c / NC, I = c - J * NC;
        const int i = 2 * I, j = 2 * J;
        auto lo = [&](int a, int b) { return kf[2 * (b * NF + a)]; };
        auto up = [&](int a, int b) { return kf[2 * (b * NF + a) + 1]; };
        kc[2 * c] = Real(0.25) * (lo(i, j) + lo(i + 1, j) + up(i + 1, j) + lo(i + 1, j + 1));
        kc[2 * c + 1] = Real(0.25) * (up(i, j) + up(i, j + 1) + lo(i, j + 1) + up(i + 1, j + 1));
    }
}

// builds coefficients of level NL from kappa at kin, coarser kappa into the other half
// of the staging area, then recurses
template <typename Real, int N, int NL, int T, bool FC = false>
__device__ void setup_levels(Real* arena, Real* stage, bool ping) {
    Lv<Real> L = level_ptrs<Real, N, NL, false, FC>(arena);
    Real* kin = ping ? stage : stage + 2 * N * N;
    build_coeffs<Real, NL, T>(L, kin);
    if constexpr (NL > 2) {
        Real* kout = ping ? stage + 2 * N * N : stage;
        coarsen_kappa<Real, NL / 2, T>(kin, kout);
        __syncthreads();
        build_diag<Real, NL, T, FC, (NL < N)>(L);
        setup_levels<Real, N, NL / 2, T, FC>(arena, stage, !ping);
    } else {
        __syncthreads();
        build_diag<Real, NL, T, FC, (NL < N)>(L);
        __syncthreads();
    }
}

// compact hierarchy: coefficients of coarse level NL from kappa in kin, coarser kappa into kout,
// then recurse with the buffers swapped (no stored inverse diagonal)
template <typename Real, int N, int NL, int T, int CP = 1>
__device__ void setup_levels_cp(Real* arena, Real* kin, Real* kout) {
    Lv<Real> L = level_ptrs<Real, N, NL, CP>(arena);
    build_coeffs<Real, NL, T>(L, kin);
    if constexpr (NL > 2) {
        coarsen_kappa<Real, NL / 2, T>(kin, kout);
        __syncthreads();
        setup_levels_cp<Real, N, NL / 2, T, CP>(arena, kout, kin);
    } else {
        __syncthreads();
    }
}

// flow cell: the ghost rows -1 and NL + 1 of the coefficient arrays on every level down to 1/4
// (the boundary rows' stencils read aN there); set before the coefficients are built
template <typename Real, int N, int NL, int T>
__device__ __forceinline__ void zero_ghost_weights(Real* arena) {
    constexpr int S = fem_row_stride(NL);
    const Lv<Real> L = level_ptrs<Real, N, NL, false, true>(arena);
    for (int k = threadIdx.x; k < 2 * S; k += T) {
        const int n = k < S ? k - S : (NL + 1) * S + (k - S);
        L.aE[n] = L.aN[n] = L.iD[n] = Real(0);
    }
    if constexpr (NL > 4) zero_ghost_weights<Real, N, NL / 2, T>(arena);
}

template <typename Real, int N>
struct Fine {
    static constexpr int M = N - 1, S = fem_row_stride(N), NI = M * M;
};

// fine-level slots per thread (half red, half black) of the on-chip solve
__host__ __device__ constexpr int fine_slots(int N, int T, bool FC = false) {
    return 2 * (((FC ? (N / 2 + 1) * N : N * N / 2) + T - 1) / T);
}
// dynamic shared memory of the on-chip solve, in Reals: the level arena, then the refinement
// state (x and r, each a hi/lo pair) of every thread's slots, then the dense inverse of the
// coarsest level kept
template <typename Real, bool FC = false>
__host__ __device__ constexpr int solve_smem_reals(int N, int T) {
    return arena_size(N, FC) + 4 * fine_slots(N, T, FC) * T + dense_reals<Real, FC>(N);
}

// ---- the kernel ----------------------------------------------------------------------
// the whole solve of particle p of a.n, by one thread block (all threads call it)
// CP: compact hierarchy (mixed path, kappa from the synthesis) with the refinement state at
// ref_ext (device memory) instead of shared memory. RHS: the load vector may come from a table
// (a.rhs); false compiles the f = 1 path alone (the compact kernels are instantiated both ways:
// at 64 registers a thread the table read's code costs them 20 % of their speed)
template <typename Real, int N, int T, int CP = 0, bool RHS = true, bool FC = false>
__device__ __forceinline__ void solve_particle(const FemArgs& a, const int p, Real* arena, double (*red_buf)[64],
                                               Real* theta_s, Real* ref_ext = nullptr) {
    constexpr int S = Fine<Real, N>::S, NI = Fine<Real, N>::NI;
    constexpr int NPT = fine_slots(N, T, FC);          // slots per thread (colour_node positions)
    constexpr int NPH = NPT / 2;                       // per colour
    constexpr int E = 2 * N * N;
    const int tid = threadIdx.x;

    Lv<Real> F = level_ptrs<Real, N, N, CP, FC>(arena);
    Real* stage = F.e;     // e, res, p of the fine level are contiguous: 3*lvl_size(N) >= 2.5 N^2
                           // (compact: e and p, 2*lvl_size(N) >= 2 N^2)
    if constexpr (FC) zero_ghost_weights<Real, N, N, T>(arena);   // read by the boundary rows

    // 1) kappa = exp(u) on every fine triangle: read from the tensor-core synthesis, or
    //    u = theta . Psi computed here (FP64 path)
    if (CP || a.kappa) {
        const float* kp = a.kappa + (size_t)p * E;
        for (int e = tid; e < E; e += T) stage[e] = (Real)kp[e];
    } else {
        for (int k = tid; k < a.K; k += T) theta_s[k] = (Real)a.theta[(size_t)p * a.K + k];
        __syncthreads();
        const Real* psi = static_cast<const Real*>(a.psi);
        for (int e = tid; e < E; e += T) {
            Real u = 0;
            for (int k = 0; k < a.K; ++k) u = fma(theta_s[k], psi[(size_t)k * E + e], u);
            stage[e] = exp(u);
        }
    }
    __syncthreads();

    // 2) stencil hierarchy
    if constexpr (CP) {
        // kappa ping-pongs between the fine level's e/p storage and its inverse-diagonal storage,
        // which is filled last
        build_coeffs<Real, N, T>(F, stage);
        coarsen_kappa<Real, N / 2, T>(stage, F.iD);
        __syncthreads();
        setup_levels_cp<Real, N, N / 2, T>(arena, F.iD, stage);
        build_diag<Real, N, T>(F);
    } else {
        setup_levels<Real, N, N, T, FC>(arena, stage, true);
    }
    zero_rings<Real, N, N, T, CP, FC>(arena);
    __syncthreads();
    Real* dinv = CP ? arena + arena_size_cp(N) : arena + arena_size(N, FC) + 4 * NPT * T;
    if constexpr (direct_level<Real, FC>(N) != 0) {
        if constexpr (CP) {
            // compact forms: one warp runs the pivot steps while the SM's other blocks keep it busy
            // (with one block per SM the block-wide form is faster)
            if (tid < 32)
                dense_setup<Real, direct_level<Real, FC>(N), 32, FC>(
                    level_ptrs<Real, N, direct_level<Real, FC>(N), CP, FC>(arena), dinv);
            __syncthreads();
        } else {
            dense_setup<Real, direct_level<Real, FC>(N), T, FC>(
                level_ptrs<Real, N, direct_level<Real, FC>(N), CP, FC>(arena), dinv);
        }
    }

    // fine nodes owned by this thread, one packed int each: bits 0-12 node index n, 13-23 the
    // coarse node c under it ((j/2) SC + i/2), 24-25 (i & 1) + 2 (j & 1), 26 red, 27 valid.
    // Slots 0..NPH-1 hold red nodes (i + j even), NPH..NPT-1 black ones (colour_node
    // enumeration), so that every lane has a node in each colour sweep, without bank conflicts.
    constexpr int SC = fem_row_stride(N / 2);
    int slot[NPT];
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
        const bool red = q < NPH;
        const int k = tid + T * (red ? q : q - NPH);
        int ii, jj;
        const int v = colour_node<N, FC>(k, red ? 0 : 1, ii, jj);
        if (!v) ii = jj = 1;
        const int n0 = jj * S + ii;
        const int c = (jj >> 1) * SC + (ii >> 1);
        const int code = (ii & 1) + 2 * (jj & 1);
        slot[q] = n0 | (c << 13) | (code << 24) | ((red ? 1 : 0) << 26) | (v << 27);
    }
    // right-hand side h^2 (f = 1), exact in FP32 for N a power of two
    const Real h2 = Real(1) / (Real(N) * Real(N));
    // solution x and residual r of the refinement: FP64, or double-float pairs (hi + lo) of FP32
    // numbers on the mixed path so that no FP64 instruction runs in the solve. They are touched
    // once per refinement pass, so they live in shared memory after the arena ([4][NPT][T]:
    // x hi, x lo, r hi, r lo), conflict-free per slot.
    Real* ref = CP ? ref_ext : arena + arena_size(N, FC);
    auto XH = [&](int q) -> Real& { return ref[(0 * NPT + q) * T + tid]; };
    auto XL = [&](int q) -> Real& { return ref[(1 * NPT + q) * T + tid]; };
    auto RH = [&](int q) -> Real& { return ref[(2 * NPT + q) * T + tid]; };
    auto RL = [&](int q) -> Real& { return ref[(3 * NPT + q) * T + tid]; };
#pragma unroll
    for (int q = 0; q < NPT; ++q) {   // r = b - A 0: the load vector (h^2 at every node for f = 1)
        XH(q) = XL(q) = RL(q) = Real(0);
        RH(q) = ((slot[q] >> 27) & 1) ? h2 : Real(0);
    }
    Real bflow = 0;   // flow cell: sum of b^2
    if constexpr (FC) {
        // f = 0 and p = 1 on x = 1: b = -A_UD p_D is the edge weight to the Dirichlet node (N, j)
        // at the nodes of column N - 1, zero elsewhere
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            const int n = slot[q] & 0x1fff;
            const bool last = ((slot[q] >> 27) & 1) && n % S == N - 1;
            RH(q) = last ? F.aE[n] : Real(0);
            bflow += RH(q) * RH(q);
        }
        block_sum<T>(bflow, red_buf[1]);
    } else if (RHS && a.rhs) {
        // the load vector, read in a rolled loop of its own (node indices recomputed, no register
        // array touched), which leaves the register allocation of the solve as it is for f = 1
#pragma unroll 1
        for (int q = 0; q < NPT; ++q) {
            const bool red = q < NPH;
            int ii, jj;
            if (colour_node<N>(tid + T * (red ? q : q - NPH), red ? 0 : 1, ii, jj)) {
                Real hi, lo;
                load_rhs(a.rhs, jj * S + ii, hi, lo);
                RH(q) = hi;
                RL(q) = lo;
            }
        }
    }
    // inner CG state of this thread's nodes: residual r, correction d, preconditioned residual z
    // and search direction p (p is also published in shared memory for the stencil)
    Real r[NPT], d[NPT], z[NPT], pv[NPT];
    const Real bnorm2 = FC ? bflow : (RHS && a.rhs) ? Real(a.bnorm2) : Real(NI) * h2 * h2;
    const Real stop_outer = Real(a.rtol * a.rtol) * bnorm2;
    // an inner pass ends at its relative reduction or once its residual is below half the outer
    // target, whichever comes first (the last pass then stops where the solve is done)
    const Real stop_last = Real(0.25 * a.rtol * a.rtol) * bnorm2;
    const Real rtol_in2 = Real(a.rtol_in * a.rtol_in);
    int parity = 0;
    int total_it = 0;
    bool converged = false;
    Lv<Real> C1 = level_ptrs<Real, N, N / 2, CP, FC>(arena);
    Real* P = F.rhs;   // fine-level CG direction (the fine rhs is r, held in registers)

    for (int pass = 0; pass < a.max_outer && !converged; ++pass) {
        // ---- inner multigrid-preconditioned CG on A d = r (working precision) ----
        Real rr0 = 0;
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            r[q] = RH(q);
            d[q] = Real(0);
            pv[q] = Real(0);
            rr0 += r[q] * r[q];
        }
#pragma unroll
        for (int q = 0; q < NPH; ++q)   // red pre-sweep of the first cycle (see the r update below)
            if (((slot[q] >> 27) & 1)) F.e[(slot[q] & 0x1fff)] = r[q] * F.iD[(slot[q] & 0x1fff)];
        block_sum<T>(rr0, red_buf[parity]);
        parity ^= 1;
        if (!(rr0 > Real(0))) break;
        const Real stop2 = fmax(rtol_in2 * rr0, stop_last);
        Real rz = 0;
        for (int it = 0; it < a.max_inner; ++it) {
            // z = M^{-1} r: V(1,1) cycle with the fine rhs held in registers (red pre-sweep
            // from zero, written where r was last updated; black pre-sweep, restriction of the
            // red residuals, coarse cycle, black post-sweep with the prolongation folded in, red
            // post-sweep). The red post-sweep values are read by nothing but this thread, so they
            // stay in registers.
#pragma unroll
            for (int q = NPH; q < NPT; ++q)
                if (((slot[q] >> 27) & 1)) {
                    const int n = (slot[q] & 0x1fff);
                    F.e[n] = (r[q] + offsum<Real, S>(F.aE, F.aN, F.e, n)) * F.iD[n];
                }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NPH; ++q)   // red residuals: off-diagonal sums of the new black values
                if (((slot[q] >> 27) & 1)) {
                    const int n = (slot[q] & 0x1fff);
                    F.res[n] = offsum<Real, S>(F.aE, F.aN, F.e, n);
                }
            __syncthreads();
            restrict_gather<Real, N / 2, T, FC>(F.res, C1);
            __syncthreads();
            vcycle_coarse<Real, N, N / 2, T, false, CP, FC>(arena, dinv);
#pragma unroll
            for (int q = NPH; q < NPT; ++q) {
                z[q] = Real(0);
                if (((slot[q] >> 27) & 1)) {
                    const int n = (slot[q] & 0x1fff);
                    const int c = (slot[q] >> 13) & 0x7ff, code = (slot[q] >> 24) & 3;
                    z[q] = (r[q] + offsum_prolong<Real, S, SC>(F.aE, F.aN, F.e, C1.e, n, c, code == 1)) * F.iD[n];
                    F.e[n] = z[q];
                }
            }
            __syncthreads();
            Real rz_new = 0;
#pragma unroll
            for (int q = 0; q < NPH; ++q) {
                z[q] = Real(0);
                if (((slot[q] >> 27) & 1)) {
                    const int n = (slot[q] & 0x1fff);
                    z[q] = (r[q] + offsum<Real, S>(F.aE, F.aN, F.e, n)) * F.iD[n];
                }
            }
#pragma unroll
            for (int q = 0; q < NPT; ++q) rz_new += r[q] * z[q];   // idle slots hold r = z = 0
            block_sum<T>(rz_new, red_buf[parity]);
            parity ^= 1;
            // p = z + beta p
            const Real beta = (it == 0) ? Real(0) : rz_new / rz;
            rz = rz_new;
#pragma unroll
            for (int q = 0; q < NPT; ++q) {
                pv[q] = (it == 0) ? z[q] : z[q] + beta * pv[q];
                if (((slot[q] >> 27) & 1)) P[(slot[q] & 0x1fff)] = pv[q];
            }
            __syncthreads();
            // q = A p, alpha = rz / p.q
            Real qv[NPT];
            Real pq = 0;
#pragma unroll
            for (int q = 0; q < NPT; ++q) {
                qv[q] = Real(0);
                if (((slot[q] >> 27) & 1)) {
                    const int n = (slot[q] & 0x1fff);
                    qv[q] = stencil_apply_at<Real, S>(F.aE, F.aN, P, n, pv[q]);
                    pq += pv[q] * qv[q];
                }
            }
            block_sum<T>(pq, red_buf[parity]);
            parity ^= 1;
            const Real alpha = rz / pq;
            Real rr = 0;
#pragma unroll
            for (int q = 0; q < NPT; ++q) {
                d[q] = fma(alpha, pv[q], d[q]);
                r[q] = fma(-alpha, qv[q], r[q]);
                rr += r[q] * r[q];
            }
#pragma unroll
            for (int q = 0; q < NPH; ++q)   // red pre-sweep of the next cycle (nothing reads F.e now)
                if (((slot[q] >> 27) & 1)) F.e[(slot[q] & 0x1fff)] = r[q] * F.iD[(slot[q] & 0x1fff)];
            block_sum<T>(rr, red_buf[parity]);
            parity ^= 1;
            ++total_it;
            if (!(rr > stop2)) break;   // also leaves on NaN
        }
        // ---- refinement: x += d, r -= A d in extended precision ----
        // A d in edge form sum_e a_e (d_i - d_j): its diagonal is the exact sum of the four
        // edge weights, so the refined system is the FEM stencil of the stored edge weights
        // (the rounded working-precision diagonal would act as a spurious reaction term).
#pragma unroll
        for (int q = 0; q < NPT; ++q)
            if (((slot[q] >> 27) & 1)) P[(slot[q] & 0x1fff)] = d[q];
        __syncthreads();
        Real rr_out = 0;
#pragma unroll
        for (int q = 0; q < NPT; ++q)
            if (((slot[q] >> 27) & 1)) {
                const int n = (slot[q] & 0x1fff);
                const Real di = P[n];
                const Real w[4] = {F.aE[n], F.aE[n - 1], F.aN[n], F.aN[n - S]};
                const Real dj[4] = {P[n + 1], P[n - 1], P[n + S], P[n - S]};
                if constexpr (sizeof(Real) == 8) {
                    Real Ad = 0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) Ad = fma(w[t], di - dj[t], Ad);
                    RH(q) -= Ad;
                    XH(q) += d[q];
                } else {
                    Real ah = 0, al = 0;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        Real sh, sl;
                        two_sum(di, -dj[t], sh, sl);        // d_i - d_j exactly
                        const Real ph = __fmul_rn(w[t], sh);   // kept out of FMA contraction
                        Real pl = fma(w[t], sh, -ph);          // exact product error
                        pl = fma(w[t], sl, pl);
                        df_add(ah, al, ph, pl);
                    }
                    Real rh = RH(q), rl = RL(q), xh = XH(q), xl = XL(q);
                    df_add(rh, rl, -ah, -al);
                    df_add(xh, xl, d[q], Real(0));
                    RH(q) = rh;
                    RL(q) = rl;
                    XH(q) = xh;
                    XL(q) = xl;
                }
                rr_out += RH(q) * RH(q);
            }
        block_sum<T>(rr_out, red_buf[parity]);
        parity ^= 1;
        converged = rr_out <= stop_outer;
    }

    // ---- observations and misfit (FP64) ----
    // the solution goes to shared memory as stored (double, or the double-float pair as float2,
    // so that FP64 arithmetic runs only at the observed nodes); the boundary ring reads as zero
    using Node = typename std::conditional<sizeof(Real) == 8, double, float2>::type;
    Node* xs = reinterpret_cast<Node*>(F.e);   // e and res: 2*lvl_size(N) Real >= (N+1) S Nodes
    if constexpr (FC) {   // the Dirichlet columns: p = 0 on x = 0, p = 1 on x = 1
        for (int k = tid; k < 2 * (N + 1); k += T) {
            const int n = (k >> 1) * S + ((k & 1) ? N : 0);
            const Real v = (k & 1) ? Real(1) : Real(0);
            if constexpr (sizeof(Real) == 8) xs[n] = v;
            else xs[n] = make_float2(v, 0.f);
        }
    } else {
        for (int k = tid; k < 4 * N; k += T) {   // rows 0 and N (N + 1 nodes each), then columns 0 and N
            const int n = k <= N ? k : k <= 2 * N + 1 ? N * S + (k - N - 1)
                                                     : (1 + ((k - 2 * N - 2) >> 1)) * S + (((k - 2 * N - 2) & 1) ? N : 0);
            if constexpr (sizeof(Real) == 8) xs[n] = 0.0;
            else xs[n] = make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int q = 0; q < NPT; ++q)
        if (((slot[q] >> 27) & 1)) {
            if constexpr (sizeof(Real) == 8) xs[(slot[q] & 0x1fff)] = (double)XH(q);
            else xs[(slot[q] & 0x1fff)] = make_float2((float)XH(q), (float)XL(q));
        }
    __syncthreads();
    if (tid < 32) {   // one warp gathers and reduces the misfit (no block-wide FP64 work)
        auto val = [&](int n) -> double {
            if constexpr (sizeof(Real) == 8) return xs[n];
            else return (double)xs[n].x + (double)xs[n].y;
        };
        double misfit = 0.0;
        for (int o = tid; o < a.n_obs; o += 32) {
            const double g = a.obs_w[3 * o] * val(a.obs_idx[3 * o]) + a.obs_w[3 * o + 1] * val(a.obs_idx[3 * o + 1]) +
                             a.obs_w[3 * o + 2] * val(a.obs_idx[3 * o + 2]);
            if (a.G) a.G[(size_t)p * a.n_obs + o] = g;
            const double rdf = a.y[o] - g;
            misfit += rdf * rdf;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) misfit += __shfl_xor_sync(0xffffffffu, misfit, off);
        if (tid == 0) {
            a.Phi[p] = 0.5 * misfit * a.inv_sigma2;
            if (a.iters) a.iters[p] = converged ? total_it : -(total_it + 1);
        }
    }
}

// Two-arena hierarchy of the large levels: levels with 1/h >= 128 live in device memory (the
// arena of a top level N), levels 1/h <= 64 in shared memory (the arena of a top level 64).
template <typename Real, int N, int NL, bool FC = false>
__device__ __forceinline__ Lv<Real> ptrs2(Real* garena, Real* sarena) {
    if constexpr (NL > 64) return level_ptrs<Real, N, NL, false, FC>(garena);
    else return level_ptrs<Real, 64, NL, false, FC>(sarena);
}

template <typename Real, int N, int NL, int T, bool FC = false>
__device__ void vcycle2(Real* garena, Real* sarena, const Real* dinv) {
    if constexpr (NL <= 64) {
        vcycle_coarse<Real, 64, NL, T, false, false, FC>(sarena, dinv);
    } else {
        Lv<Real> L = ptrs2<Real, N, NL, FC>(garena, sarena);
        Lv<Real> C = ptrs2<Real, N, NL / 2, FC>(garena, sarena);
        smooth_color<Real, NL, T, FC>(L, 1);   // red pre-sweep done by the restriction above
        __syncthreads();
        restrict_red<Real, NL / 2, T, FC>(L, C);
        __syncthreads();
        vcycle2<Real, N, NL / 2, T, FC>(garena, sarena, dinv);
        black_prolong<Real, NL, T, FC>(L, C.e);
        __syncthreads();
        smooth_color<Real, NL, T, FC>(L, 0);
        __syncthreads();
    }
}

// Large levels (1/h >= 128): the same solve with the levels 1/h >= 128 in a per-block slice of
// device memory (L2-resident for 1/128), the levels 1/h <= 64 in shared memory, and the fine-level
// CG and refinement vectors as arrays indexed by interior node (too many nodes per thread for
// registers). vec: 6 arrays of NI entries after the level arena: r, d, x_hi, x_lo, r_hi, r_lo.
// FC: the flow cell (rows 0 .. N unknowns, ghost rows, the lifted Dirichlet data).
template <typename Real, int N, int T, bool FC = false>
__device__ __forceinline__ void solve_particle_mem(const FemArgs& a, const int p, Real* arena, Real* sarena,
                                                   double (*red_buf)[64]) {
    constexpr int M = Fine<Real, N>::M, S = Fine<Real, N>::S;
    constexpr int ROW0 = FC ? 0 : 1, NI = M * (FC ? N + 1 : M);   // first unknown row, unknowns
    constexpr int E = 2 * N * N;
    constexpr int SC = fem_row_stride(N / 2);
    const int tid = threadIdx.x;
    Lv<Real> F = level_ptrs<Real, N, N, false, FC>(arena);
    Real* vec = arena + arena_size(N, FC);
    Real *R = vec, *Dv = vec + NI, *XH = vec + 2 * NI, *XL = vec + 3 * NI, *RH = vec + 4 * NI, *RL = vec + 5 * NI;
    // A p is kept in the fine level's residual array (dead outside the restriction): one array
    // fewer in the working set that must stay in L2
    Real* stage = F.e;

    if constexpr (FC) {   // ghost rows of the coefficient arrays, read by the boundary rows
        zero_ghost_weights<Real, N, N, T>(arena);
        zero_ghost_weights<Real, 64, 64, T>(sarena);
    }
    const float* kp = a.kappa + (size_t)p * E;
    for (int e = tid; e < E; e += T) stage[e] = (Real)kp[e];
    __syncthreads();
    // device-memory levels (N, and 128 when N = 256), then the shared-memory hierarchy from 64 down;
    // kappa is staged in the fine level's e/res/rhs region
    {
        Real* k1 = stage + 2 * N * N;
        build_coeffs<Real, N, T>(F, stage);
        coarsen_kappa<Real, N / 2, T>(stage, k1);
        __syncthreads();
        build_diag<Real, N, T, FC>(F);
        Real* k64 = k1;
        if constexpr (N == 256) {
            Lv<Real> L1 = level_ptrs<Real, N, 128, false, FC>(arena);
            build_coeffs<Real, 128, T>(L1, k1);
            coarsen_kappa<Real, 64, T>(k1, stage);
            __syncthreads();
            build_diag<Real, 128, T, FC>(L1);
            k64 = stage;
        }
        setup_levels<Real, 64, 64, T, FC>(sarena, k64, true);
    }
    {
        int off = 0;
#pragma unroll
        for (int NL = N; NL >= 128; NL >>= 1) {
            const int z = lvl_size(NL, FC);
            for (int q = tid; q < 3 * z; q += T) arena[off + 3 * z + q] = Real(0);
            off += 6 * z;
        }
        off = 0;
#pragma unroll
        for (int NL = 64; NL >= 2; NL >>= 1) {
            const int z = lvl_size(NL, FC);
            for (int q = tid; q < 3 * z; q += T) sarena[off + 3 * z + q] = Real(0);
            off += 6 * z;
        }
    }
    __syncthreads();
    Real* dinv = sarena + arena_size(64, FC);
    dense_setup<Real, direct_level<Real, FC>(64), T, FC>(
        level_ptrs<Real, 64, direct_level<Real, FC>(64), false, FC>(sarena), dinv);
    const Real h2 = Real(1) / (Real(N) * Real(N));
    Real bflow = 0;   // flow cell: sum of b^2
    for (int i = tid; i < NI; i += T) {   // r = b: the load vector (h^2 at every node for f = 1)
        XH[i] = XL[i] = RL[i] = Real(0);
        RH[i] = h2;
        if constexpr (FC) {   // b = the edge weight to the Dirichlet node (N, j) in column N - 1
            const int jj = i / M, ii = i - jj * M + 1;
            RH[i] = ii == N - 1 ? F.aE[jj * S + ii] : Real(0);
            bflow += RH[i] * RH[i];
        } else if (a.rhs) {
            const int jj = i / M + ROW0, ii = i - (jj - ROW0) * M + 1;
            Real hi, lo;
            load_rhs(a.rhs, jj * S + ii, hi, lo);
            RH[i] = hi;
            RL[i] = lo;
        }
    }
    if constexpr (FC) block_sum<T>(bflow, red_buf[1]);
    __syncthreads();
    const Real bnorm2 = FC ? bflow : a.rhs ? Real(a.bnorm2) : Real(NI) * h2 * h2;
    const Real stop_outer = Real(a.rtol * a.rtol) * bnorm2;
    const Real stop_last = Real(0.25 * a.rtol * a.rtol) * bnorm2;   // as in solve_particle
    const Real rtol_in2 = Real(a.rtol_in * a.rtol_in);
    int parity = 0, total_it = 0;
    bool converged = false;
    Lv<Real> C1 = ptrs2<Real, N, N / 2, FC>(arena, sarena);
    Real* P = F.rhs;
#define NODE_OF(i) const int jj = (i) / M + ROW0, ii = (i) - (jj - ROW0) * M + 1, n = jj * S + ii
    // colour sweeps run over colour_node positions (every lane busy), the vector updates over the
    // interior index (coalesced); the red pre-sweep from zero is written where R is updated.
    // The fine level lives in device memory, so its loops are latency-bound: each takes two
    // positions per thread at a time and reads the operands of both before it stores either
    // result (the compiler cannot move a load above a store to an array it cannot tell apart).
    // Within a colour sweep or a vector update no position reads what another one writes, so the
    // results are those of the one-at-a-time loops.
    constexpr int CPOS = colour_positions<N, FC>();
    auto sweep2 = [&](int col, auto&& compute, auto&& commit) {
        for (int k0 = tid; k0 < CPOS; k0 += 2 * T) {
            int ia, ja, ib, jb;
            const bool va = colour_node<N, FC>(k0, col, ia, ja);
            const bool vb = colour_node<N, FC>(k0 + T, col, ib, jb);
            Real xa = 0, xb = 0;
            if (va) xa = compute(ia, ja);
            if (vb) xb = compute(ib, jb);
            if (va) commit(ia, ja, xa);
            if (vb) commit(ib, jb, xb);
        }
    };
    auto vec2 = [&](auto&& compute, auto&& commit) {
        for (int i0 = tid; i0 < NI; i0 += 2 * T) {
            const int i1 = i0 + T;
            const bool vb = i1 < NI;
            Real xa = compute(i0), xb = 0;
            if (vb) xb = compute(i1);
            commit(i0, xa);
            if (vb) commit(i1, xb);
        }
    };
    for (int pass = 0; pass < a.max_outer && !converged; ++pass) {
        Real rr0 = 0;
        for (int i = tid; i < NI; i += T) {
            NODE_OF(i);
            R[i] = RH[i];
            Dv[i] = Real(0);
            rr0 += RH[i] * RH[i];
            if (((ii + jj) & 1) == 0) F.e[n] = RH[i] * F.iD[n];
        }
        block_sum<T>(rr0, red_buf[parity]);
        parity ^= 1;
        if (!(rr0 > Real(0))) break;
        const Real stop2 = fmax(rtol_in2 * rr0, stop_last);
        Real rz = 0;
        for (int it = 0; it < a.max_inner; ++it) {
            sweep2(1, [&](int ii, int jj) {   // black pre-sweep
                const int n = jj * S + ii, i = (jj - ROW0) * M + ii - 1;
                return (R[i] + offsum<Real, S>(F.aE, F.aN, F.e, n)) * F.iD[n];
            }, [&](int ii, int jj, Real v) { F.e[jj * S + ii] = v; });
            __syncthreads();
            sweep2(0, [&](int ii, int jj) {   // red residuals
                return offsum<Real, S>(F.aE, F.aN, F.e, jj * S + ii);
            }, [&](int ii, int jj, Real v) { F.res[jj * S + ii] = v; });
            __syncthreads();
            restrict_gather<Real, N / 2, T, FC>(F.res, C1);
            __syncthreads();
            vcycle2<Real, N, N / 2, T, FC>(arena, sarena, dinv);
            Real rz_new = 0;
            sweep2(1, [&](int ii, int jj) {   // black post-sweep with the prolongation
                const int n = jj * S + ii, i = (jj - ROW0) * M + ii - 1;
                const int c = (jj >> 1) * SC + (ii >> 1);
                return (R[i] + offsum_prolong<Real, S, SC>(F.aE, F.aN, F.e, C1.e, n, c, (jj & 1) == 0)) * F.iD[n];
            }, [&](int ii, int jj, Real z) {
                F.e[jj * S + ii] = z;
                rz_new += R[(jj - ROW0) * M + ii - 1] * z;
            });
            __syncthreads();
            sweep2(0, [&](int ii, int jj) {   // red post-sweep
                const int n = jj * S + ii, i = (jj - ROW0) * M + ii - 1;
                return (R[i] + offsum<Real, S>(F.aE, F.aN, F.e, n)) * F.iD[n];
            }, [&](int ii, int jj, Real z) {
                F.e[jj * S + ii] = z;
                rz_new += R[(jj - ROW0) * M + ii - 1] * z;
            });
            block_sum<T>(rz_new, red_buf[parity]);
            parity ^= 1;
            const Real beta = (it == 0) ? Real(0) : rz_new / rz;
            rz = rz_new;
            vec2([&](int i) {
                NODE_OF(i);
                return (it == 0) ? F.e[n] : F.e[n] + beta * P[n];
            }, [&](int i, Real v) { NODE_OF(i); P[n] = v; });
            __syncthreads();
            Real pq = 0;
            vec2([&](int i) {
                NODE_OF(i);
                return stencil_apply<Real, S>(F.aE, F.aN, P, n);
            }, [&](int i, Real q) {
                NODE_OF(i);
                F.res[n] = q;
                pq += P[n] * q;
            });
            block_sum<T>(pq, red_buf[parity]);
            parity ^= 1;
            const Real alpha = rz / pq;
            Real rr = 0;
            for (int i0 = tid; i0 < NI; i0 += 2 * T) {   // two positions: all loads before the stores
                const int i1 = i0 + T;
                const bool vb = i1 < NI;
                const int ja = i0 / M + ROW0, ia = i0 - (ja - ROW0) * M + 1, na = ja * S + ia;
                const int jb = vb ? i1 / M + ROW0 : ja, ib = vb ? i1 - (jb - ROW0) * M + 1 : ia, nb = jb * S + ib;
                const bool ra = ((ia + ja) & 1) == 0, rb = vb && ((ib + jb) & 1) == 0;
                const Real pa = P[na], da = Dv[i0], qa = F.res[na], sa = R[i0], ga = ra ? F.iD[na] : Real(0);
                Real pb = 0, db = 0, qb = 0, sb = 0, gb = 0;
                if (vb) {
                    pb = P[nb];
                    db = Dv[i1];
                    qb = F.res[nb];
                    sb = R[i1];
                    gb = rb ? F.iD[nb] : Real(0);
                }
                const Real rna = fma(-alpha, qa, sa), rnb = fma(-alpha, qb, sb);
                Dv[i0] = fma(alpha, pa, da);
                R[i0] = rna;
                rr += rna * rna;
                if (ra) F.e[na] = rna * ga;   // red pre-sweep of the next cycle
                if (vb) {
                    Dv[i1] = fma(alpha, pb, db);
                    R[i1] = rnb;
                    rr += rnb * rnb;
                    if (rb) F.e[nb] = rnb * gb;
                }
            }
            block_sum<T>(rr, red_buf[parity]);
            parity ^= 1;
            ++total_it;
            if (!(rr > stop2)) break;
        }
        for (int i = tid; i < NI; i += T) {
            NODE_OF(i);
            P[n] = Dv[i];
        }
        __syncthreads();
        Real rr_out = 0;
        for (int i = tid; i < NI; i += T) {
            NODE_OF(i);
            const Real di = P[n];
            const Real w[4] = {F.aE[n], F.aE[n - 1], F.aN[n], F.aN[n - S]};
            const Real dj[4] = {P[n + 1], P[n - 1], P[n + S], P[n - S]};
            Real ah = 0, al = 0;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                Real sh, sl;
                two_sum(di, -dj[t], sh, sl);
                const Real ph = __fmul_rn(w[t], sh);
                Real pl = fma(w[t], sh, -ph);
                pl = fma(w[t], sl, pl);
                df_add(ah, al, ph, pl);
            }
            Real rh = RH[i], rl = RL[i], xh = XH[i], xl = XL[i];
            df_add(rh, rl, -ah, -al);
            df_add(xh, xl, Dv[i], Real(0));
            RH[i] = rh;
            RL[i] = rl;
            XH[i] = xh;
            XL[i] = xl;
            rr_out += rh * rh;
        }
        block_sum<T>(rr_out, red_buf[parity]);
        parity ^= 1;
        converged = rr_out <= stop_outer;
    }
#undef NODE_OF
    __syncthreads();
    if (tid < 32) {   // the observed nodes straight from the interior arrays; one warp reduces
        auto val = [&](int n) -> double {
            const int j = n / S, i = n - j * S;
            if (FC && i == N) return 1.0;   // the flow cell's Dirichlet datum on x = 1
            if (i < 1 || i > M || j < ROW0 || j > (FC ? N : M)) return 0.0;
            const int k = (j - ROW0) * M + (i - 1);
            return (double)XH[k] + (double)XL[k];
        };
        double misfit = 0.0;
        for (int o = tid; o < a.n_obs; o += 32) {
            const double g = a.obs_w[3 * o] * val(a.obs_idx[3 * o]) + a.obs_w[3 * o + 1] * val(a.obs_idx[3 * o + 1]) +
                             a.obs_w[3 * o + 2] * val(a.obs_idx[3 * o + 2]);
            if (a.G) a.G[(size_t)p * a.n_obs + o] = g;
            const double rdf = a.y[o] - g;
            misfit += rdf * rdf;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) misfit += __shfl_xor_sync(0xffffffffu, misfit, off);
        if (tid == 0) {
            a.Phi[p] = 0.5 * misfit * a.inv_sigma2;
            if (a.iters) a.iters[p] = converged ? total_it : -(total_it + 1);
        }
    }
}

// large levels: persistent blocks, each with its own arena slice of `scratch`
template <int N, int T, bool FC = false>
__global__ void __launch_bounds__(T, 1) fem_eval_global(FemArgs a, float* scratch, size_t slice, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_buf[2][64];
    __shared__ int item_s;
    float* arena = scratch + slice * blockIdx.x;
    float* sarena = reinterpret_cast<float*>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= a.n) break;
        solve_particle_mem<float, N, T, FC>(a, item, arena, sarena, red_buf);
        __syncthreads();
    }
}

// large levels of many problems: the same persistent loop over (problem, particle) items, the
// item's problem found in a per-item table and its launch arguments copied to shared memory
template <int N, int T>
__global__ void __launch_bounds__(T, 1)
fem_eval_global_multi(const FemArgs* groups, const int* offsets, const int* item_group, int total, float* scratch,
                      size_t slice, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_buf[2][64];
    __shared__ int item_s, p_s;
    __shared__ FemArgs args_s;
    float* arena = scratch + slice * blockIdx.x;
    float* sarena = reinterpret_cast<float*>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = atomicAdd(counter, 1);
            item_s = item;
            if (item < total) {
                const int g = item_group[item];
                args_s = groups[g];
                p_s = item - offsets[g];
            }
        }
        __syncthreads();
        if (item_s >= total) break;
        solve_particle_mem<float, N, T>(args_s, p_s, arena, sarena, red_buf);
        __syncthreads();
    }
}

// blocks per SM the register file can hold at 128 registers a thread (the per-problem kernels
// compile below that; without the bound the persistent form took 143 at N = 32, T = 256, which
// halved its occupancy)
__host__ __device__ constexpr int min_blocks_128(int T) { return T >= 512 ? 1 : 65536 / (T * 128); }

// blocks per SM the register bound aims for, the same for the per-problem and the persistent
// forms: FP32 blocks are compiled for at most 85 registers a thread (three 256-thread blocks at
// 1/32, whose 64 KB of shared memory allow three; twelve 64-thread blocks at 1/16), FP64 blocks
// for 128
template <typename Real, int N, int T>
__host__ __device__ constexpr int solve_min_blocks() {
    return sizeof(Real) == 4 ? (65536 / (T * 85) > 1 ? (65536 / (T * 85) < 32 ? 65536 / (T * 85) : 32) : 1)
                             : min_blocks_128(T);
}

template <typename Real, int N, int T>
__global__ void __launch_bounds__(T, (solve_min_blocks<Real, N, T>()))
fem_eval_kernel(FemArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_buf[2][64];
    __shared__ Real theta_s[256];
    if ((int)blockIdx.x >= a.n) return;
    solve_particle<Real, N, T>(a, blockIdx.x, reinterpret_cast<Real*>(smem_raw), red_buf, theta_s);
}

// flow cell of Example 5.3 (FemArgs::flow_cell): the same solve with Neumann rows and the lifted
// Dirichlet data
template <typename Real, int N, int T>
__global__ void __launch_bounds__(T, (solve_min_blocks<Real, N, T>()))
fem_eval_kernel_fc(FemArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_buf[2][64];
    __shared__ Real theta_s[256];
    if ((int)blockIdx.x >= a.n) return;
    solve_particle<Real, N, T, false, false, true>(a, blockIdx.x, reinterpret_cast<Real*>(smem_raw), red_buf,
                                                   theta_s);
}

// compact form (mixed, kappa from the synthesis): MINB blocks per SM, persistent over the
// particles; each block keeps its refinement state in its own slice of ref_scratch (L2-resident)
template <int N, int T, int MINB, bool RHS>
__global__ void __launch_bounds__(T, MINB) fem_eval_compact(FemArgs a, float* ref_scratch, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_buf[2][64];
    __shared__ int item_s;
    float* ref = ref_scratch + (size_t)blockIdx.x * (4 * fine_slots(N, T) * T);
    for (;;) {
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_s;
        __syncthreads();
        if (item >= a.n) break;
        solve_particle<float, N, T, true, RHS>(a, item, reinterpret_cast<float*>(smem_raw), red_buf, nullptr, ref);
        __syncthreads();
    }
}

// ---- two-CTA cluster form of the 1/128 solve (mixed path) ------------------------------------
// One particle per cluster of two CTAs, one CTA per SM. CTA r keeps the fine rows 64 r + 1 ..
// 64 r + 64 of the 1/128 level on chip (rank 1's last row, 128, is the boundary) with one halo row
// on either side; the coarse levels 1/64 .. 1/2 are replicated, and both CTAs run the coarse
// V-cycle on identical data. A value the partner reads (the boundary row of a sweep, the red
// residuals of row 65, the coarse rows a CTA restricts) is also stored into the partner's shared
// memory (distributed shared memory), and every fine-level phase ends at a cluster barrier
// (release / acquire at cluster scope). A reduction sums the 64 warp partials of both CTAs in one
// fixed order, so both CTAs hold bit-identical scalars and take the same branches: no barrier is
// left waiting. Fine-level arrays (local index (j - 64 r) S + i, local rows 0 .. 65): edge
// weights aE, aN; e, which also holds the CG direction p (p is dead while the V-cycle runs and e
// is dead between the red post-sweep and the next pre-sweep); the red residuals in an array of
// their own indexed by n / 2. The inverse diagonals are formed from the edge weights where a
// sweep needs them (approximate reciprocal: they only shape the preconditioner).
namespace cl {
constexpr int N = 128, T = 1024, S = fem_row_stride(N), SC = fem_row_stride(N / 2);
constexpr int FS = 66 * S;                    // floats per strip array (local rows 0 .. 65)
constexpr int RS = padded(FS / 2);            // red-only residual array
constexpr int NPT = 8, NPH = 4;               // fine slots per thread (4 red, 4 black)
constexpr int OFF_AE = 0, OFF_AN = FS, OFF_E = 2 * FS, OFF_RES = 3 * FS, OFF_C = 3 * FS + RS;
constexpr int OFF_DINV = OFF_C + coarse_size_cp(N / 2);
constexpr int SMEM_FLOATS = OFF_DINV + dense_reals<float>(N);
constexpr int REF_FLOATS = 4 * NPT * T;       // refinement state of one CTA (device memory)
static_assert(fine_slots(N, T) == 2 * NPT, "two CTAs share the fine slots");
static_assert(OFF_C % 4 == 0 && FS % 4 == 0, "16-byte aligned arrays");
static_assert(SMEM_FLOATS * 4 <= 227 * 1024, "shared memory of one CTA");
// packed slot: bits 0-13 local node, 14-26 coarse node under it, 27-28 (i & 1) + 2 (j & 1),
// 29 red, 30 valid, 31 on the row the partner keeps as its halo
__device__ __forceinline__ int sn(unsigned s) { return (int)(s & 0x3fffu); }
__device__ __forceinline__ int sc(unsigned s) { return (int)((s >> 14) & 0x1fffu); }
__device__ __forceinline__ int scode(unsigned s) { return (int)((s >> 27) & 3u); }
__device__ __forceinline__ bool sv(unsigned s) { return (s >> 30) & 1u; }
__device__ __forceinline__ bool ssend(unsigned s) { return (s >> 31) != 0u; }
}  // namespace cl

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ int cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, int rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_peer(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void st_peer(uint32_t a, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ float2 ld_peer2(uint32_t a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
// all threads of both CTAs; orders shared (local and distributed) and global memory at cluster scope
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// sum over the cluster: warp sums written to [rank][warp] of both CTAs' buffers, one cluster
// barrier, then the 64 partials summed in index order (the same value in both CTAs)
__device__ __forceinline__ float cluster_sum(float a, float* buf, uint32_t peer_buf, int rank) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    if ((threadIdx.x & 31) == 0) {
        const int k = rank * 32 + (threadIdx.x >> 5);
        buf[k] = a;
        st_peer(peer_buf + 4u * k, a);
    }
    cluster_sync();
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const float4 v = reinterpret_cast<const float4*>(buf)[i];
        s += v.x;
        s += v.y;
        s += v.z;
        s += v.w;
    }
    return s;
}

// inverse stencil diagonal at a fine node of the strip, from its four edge weights
__device__ __forceinline__ float cl_idiag(const float* aE, const float* aN, int n) {
    return recip_coarse(aE[n] + aE[n - 1] + aN[n] + aN[n - cl::S]);
}

// the solve of particle p by the calling cluster (all threads of both CTAs call it); sm: this
// CTA's dynamic shared memory (cl::SMEM_FLOATS), cbuf: [2][64] reduction buffers, ref: this CTA's
// refinement state in device memory
template <bool RHS>
__device__ void solve_particle_cl(const FemArgs& a, const int p, float* sm, float (*cbuf)[64], float* ref,
                                  const int rank) {
    using namespace cl;
    constexpr int E = 2 * N * N, NI = (N - 1) * (N - 1);
    const int tid = threadIdx.x, partner = rank ^ 1;
    float* aE = sm + OFF_AE;
    float* aN = sm + OFF_AN;
    float* e = sm + OFF_E;   // also the CG direction p and the refinement's correction d
    float* res = sm + OFF_RES;
    float* coarse = sm + OFF_C;
    float* dinv = sm + OFF_DINV;
    // partner addresses: this CTA's row j sits at local index (j - 64 r) S + i here and at
    // (j - 64 (1 - r)) S + i in the partner
    const int shift = rank ? 64 * S : -64 * S;
    const uint32_t pe = peer_addr(smem_addr(e), partner) + 4u * (uint32_t)shift;
    const uint32_t pres = peer_addr(smem_addr(res), partner) + 4u * (uint32_t)(shift / 2);
    const uint32_t pcb[2] = {peer_addr(smem_addr(cbuf[0]), partner), peer_addr(smem_addr(cbuf[1]), partner)};
    const Lv<float> C1 = level_ptrs<float, N, N / 2, 2>(coarse);
    const uint32_t pc_rhs = peer_addr(smem_addr(C1.rhs), partner), pc_e = peer_addr(smem_addr(C1.e), partner);

    // 1) stencil of the strip (local rows 0 .. 65 = rows 64 r .. 64 r + 65) straight from kappa,
    //    kappa of 1/64 staged in e, the replicated hierarchy 1/64 .. 1/2, the 1/4 inverse
    const float* kp = a.kappa + (size_t)p * E;
    coarsen_kappa<float, N / 2, T>(kp, e);
    for (int n = tid; n < FS; n += T) {
        const int lr = n / S, i = n - lr * S, j = 64 * rank + lr;
        float ae = 0.f, an = 0.f;
        if (i <= N && j <= N) {
            if (i < N) {
                if (j < N) ae += kp[2 * (j * N + i)];
                if (j > 0) ae += kp[2 * ((j - 1) * N + i) + 1];
            }
            if (j < N) {
                if (i > 0) an += kp[2 * (j * N + i - 1)];
                if (i < N) an += kp[2 * (j * N + i) + 1];
            }
        }
        aE[n] = 0.5f * ae;
        aN[n] = 0.5f * an;
    }
    __syncthreads();
    setup_levels_cp<float, N, N / 2, T, 2>(coarse, e, res);
    for (int n = tid; n < FS + RS; n += T) e[n] = 0.f;   // e and res (contiguous): zero halos and rings
    zero_rings<float, N, N / 2, T, 2>(coarse);
    if (tid < 32) dense_setup<float, 4, 32>(level_ptrs<float, N, 4, 2>(coarse), dinv);
    cluster_sync();   // also: the partner writes into this CTA's arrays only after they are zeroed

    unsigned slot[NPT];
    const int send_row = rank ? 65 : 64;
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
        const bool red = q < NPH;
        int ii, jj;
        const bool v = colour_node<N>(4096 * rank + tid + T * (red ? q : q - NPH), red ? 0 : 1, ii, jj);
        if (!v) {
            ii = 1;
            jj = 64 * rank + 1;
        }
        const unsigned nl = (unsigned)((jj - 64 * rank) * S + ii);
        const unsigned c = (unsigned)((jj >> 1) * SC + (ii >> 1));
        const unsigned code = (unsigned)((ii & 1) + 2 * (jj & 1));
        slot[q] = nl | (c << 14) | (code << 27) | ((red ? 1u : 0u) << 29) | ((v ? 1u : 0u) << 30) |
                  ((v && jj == send_row) ? 1u : 0u) << 31;
    }
    const float h2 = 1.f / (float(N) * float(N));
    auto XH = [&](int q) -> float& { return ref[(0 * NPT + q) * T + tid]; };
    auto XL = [&](int q) -> float& { return ref[(1 * NPT + q) * T + tid]; };
    auto RH = [&](int q) -> float& { return ref[(2 * NPT + q) * T + tid]; };
    auto RL = [&](int q) -> float& { return ref[(3 * NPT + q) * T + tid]; };
#pragma unroll
    for (int q = 0; q < NPT; ++q) {
        XH(q) = XL(q) = RL(q) = 0.f;
        RH(q) = sv(slot[q]) ? h2 : 0.f;
    }
    if (RHS && a.rhs) {
#pragma unroll 1
        for (int q = 0; q < NPT; ++q) {
            const bool red = q < NPH;
            int ii, jj;
            if (colour_node<N>(4096 * rank + tid + T * (red ? q : q - NPH), red ? 0 : 1, ii, jj)) {
                float hi, lo;
                load_rhs(a.rhs, jj * S + ii, hi, lo);
                RH(q) = hi;
                RL(q) = lo;
            }
        }
    }
    float r[NPT], d[NPT], z[NPT], pv[NPT];
    const float bnorm2 = (RHS && a.rhs) ? float(a.bnorm2) : float(NI) * h2 * h2;
    const float stop_outer = float(a.rtol * a.rtol) * bnorm2;
    const float stop_last = float(0.25 * a.rtol * a.rtol) * bnorm2;
    const float rtol_in2 = float(a.rtol_in * a.rtol_in);
    int parity = 0, total_it = 0;
    bool converged = false;
    // coarse rows this CTA restricts: 1 .. 32 (rank 0; row 32 reads the red residuals of row 65
    // from the halo) or 33 .. 63 (rank 1)
    const int J0 = rank ? 33 : 1, NJ = rank ? 31 : 32;

    for (int pass = 0; pass < a.max_outer && !converged; ++pass) {
        float rr0 = 0.f;
#pragma unroll
        for (int q = 0; q < NPT; ++q) {
            r[q] = RH(q);
            d[q] = 0.f;
            pv[q] = 0.f;
            rr0 += r[q] * r[q];
        }
#pragma unroll
        for (int q = 0; q < NPH; ++q)   // red pre-sweep of the first cycle
            if (sv(slot[q])) {
                const int n = sn(slot[q]);
                const float v = r[q] * cl_idiag(aE, aN, n);
                e[n] = v;
                if (ssend(slot[q])) st_peer(pe + 4u * n, v);
            }
        rr0 = cluster_sum(rr0, cbuf[parity], pcb[parity], rank);
        parity ^= 1;
        if (!(rr0 > 0.f)) break;
        const float stop2 = fmaxf(rtol_in2 * rr0, stop_last);
        float rz = 0.f;
        for (int it = 0; it < a.max_inner; ++it) {
            // black pre-sweep
#pragma unroll
            for (int q = NPH; q < NPT; ++q)
                if (sv(slot[q])) {
                    const int n = sn(slot[q]);
                    const float v = (r[q] + offsum<float, S>(aE, aN, e, n)) * cl_idiag(aE, aN, n);
                    e[n] = v;
                    if (ssend(slot[q])) st_peer(pe + 4u * n, v);
                }
            cluster_sync();
            // red residuals (rank 1 also sends row 65, which rank 0 restricts into coarse row 32)
#pragma unroll
            for (int q = 0; q < NPH; ++q)
                if (sv(slot[q])) {
                    const int n = sn(slot[q]);
                    const float v = offsum<float, S>(aE, aN, e, n);
                    res[n >> 1] = v;
                    if (rank == 1 && ssend(slot[q])) st_peer(pres + 4u * (n >> 1), v);
                }
            cluster_sync();
            // restriction of this CTA's coarse rows into both CTAs (with the coarse red pre-sweep)
            for (int idx = tid; idx < NJ * (N / 2 - 1); idx += T) {
                const int Jr = idx / (N / 2 - 1), J = J0 + Jr, I = idx - Jr * (N / 2 - 1) + 1;
                const int f = (2 * J - 64 * rank) * S + 2 * I, c = J * SC + I;
                const float v = res[f >> 1] + 0.5f * (res[(f + S + 1) >> 1] + res[(f - S - 1) >> 1]);
                C1.rhs[c] = v;
                st_peer(pc_rhs + 4u * c, v);
                if (((I + J) & 1) == 0) {
                    const float ev = v * inv_diag<float, SC>(C1, c);
                    C1.e[c] = ev;
                    st_peer(pc_e + 4u * c, ev);
                }
            }
            cluster_sync();
            vcycle_coarse<float, N, N / 2, T, false, 2>(coarse, dinv);
            // black post-sweep with the prolongation folded in
#pragma unroll
            for (int q = NPH; q < NPT; ++q) {
                z[q] = 0.f;
                if (sv(slot[q])) {
                    const int n = sn(slot[q]);
                    const float v = (r[q] + offsum_prolong<float, S, SC>(aE, aN, e, C1.e, n, sc(slot[q]),
                                                                          scode(slot[q]) == 1)) *
                                    cl_idiag(aE, aN, n);
                    z[q] = v;
                    e[n] = v;
                    if (ssend(slot[q])) st_peer(pe + 4u * n, v);
                }
            }
            cluster_sync();
            float rz_new = 0.f;
#pragma unroll
            for (int q = 0; q < NPH; ++q) {   // red post-sweep
                z[q] = 0.f;
                if (sv(slot[q])) {
                    const int n = sn(slot[q]);
                    z[q] = (r[q] + offsum<float, S>(aE, aN, e, n)) * cl_idiag(aE, aN, n);
                }
            }
#pragma unroll
            for (int q = 0; q < NPT; ++q) rz_new += r[q] * z[q];
            rz_new = cluster_sum(rz_new, cbuf[parity], pcb[parity], rank);
            parity ^= 1;
            const float beta = (it == 0) ? 0.f : rz_new / rz;
            rz = rz_new;
#pragma unroll
            for (int q = 0; q < NPT; ++q) {
                pv[q] = (it == 0) ? z[q] : z[q] + beta * pv[q];
                if (sv(slot[q])) {
                    e[sn(slot[q])] = pv[q];
                    if (ssend(slot[q])) st_peer(pe + 4u * sn(slot[q]), pv[q]);
                }
            }
            cluster_sync();
            float qv[NPT];
            float pq = 0.f;
#pragma unroll
            for (int q = 0; q < NPT; ++q) {
                qv[q] = 0.f;
                if (sv(slot[q])) {
                    qv[q] = stencil_apply_at<float, S>(aE, aN, e, sn(slot[q]), pv[q]);
                    pq += pv[q] * qv[q];
                }
            }
            pq = cluster_sum(pq, cbuf[parity], pcb[parity], rank);
            parity ^= 1;
            const float alpha = rz / pq;
            float rr = 0.f;
#pragma unroll
            for (int q = 0; q < NPT; ++q) {
                d[q] = fmaf(alpha, pv[q], d[q]);
                r[q] = fmaf(-alpha, qv[q], r[q]);
                rr += r[q] * r[q];
            }
#pragma unroll
            for (int q = 0; q < NPH; ++q)   // red pre-sweep of the next cycle
                if (sv(slot[q])) {
                    const int n = sn(slot[q]);
                    const float v = r[q] * cl_idiag(aE, aN, n);
                    e[n] = v;
                    if (ssend(slot[q])) st_peer(pe + 4u * n, v);
                }
            rr = cluster_sum(rr, cbuf[parity], pcb[parity], rank);
            parity ^= 1;
            ++total_it;
            if (!(rr > stop2)) break;
        }
        // refinement: x += d, r -= A d in double-float arithmetic (edge form, as in the one-CTA forms)
#pragma unroll
        for (int q = 0; q < NPT; ++q)
            if (sv(slot[q])) {
                e[sn(slot[q])] = d[q];
                if (ssend(slot[q])) st_peer(pe + 4u * sn(slot[q]), d[q]);
            }
        cluster_sync();
        float rr_out = 0.f;
#pragma unroll
        for (int q = 0; q < NPT; ++q)
            if (sv(slot[q])) {
                const int n = sn(slot[q]);
                const float di = e[n];
                const float w[4] = {aE[n], aE[n - 1], aN[n], aN[n - S]};
                const float dj[4] = {e[n + 1], e[n - 1], e[n + S], e[n - S]};
                float ah = 0.f, al = 0.f;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    float sh, sl;
                    two_sum(di, -dj[t], sh, sl);
                    const float ph = __fmul_rn(w[t], sh);
                    float pl = fmaf(w[t], sh, -ph);
                    pl = fmaf(w[t], sl, pl);
                    df_add(ah, al, ph, pl);
                }
                float rh = RH(q), rl = RL(q), xh = XH(q), xl = XL(q);
                df_add(rh, rl, -ah, -al);
                df_add(xh, xl, d[q], 0.f);
                RH(q) = rh;
                RL(q) = rl;
                XH(q) = xh;
                XL(q) = xl;
                rr_out += rh * rh;
            }
        rr_out = cluster_sum(rr_out, cbuf[parity], pcb[parity], rank);
        parity ^= 1;
        converged = rr_out <= stop_outer;
    }

    // ---- observations and misfit (FP64): each CTA writes its strip's solution (double-float pair
    // as float2, boundary nodes zero) over the edge weights; warp 0 of rank 0 gathers from both
    float2* xs = reinterpret_cast<float2*>(aE);   // FS float2 = the aE and aN arrays
    for (int n = tid; n < FS; n += T) xs[n] = make_float2(0.f, 0.f);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NPT; ++q)
        if (sv(slot[q])) xs[sn(slot[q])] = make_float2(XH(q), XL(q));
    cluster_sync();
    if (rank == 0 && tid < 32) {
        const uint32_t pxs = peer_addr(smem_addr(xs), 1);
        auto val = [&](int n) -> double {   // n = j S + i on the whole level
            const int j = n / S, i = n - j * S;
            float2 v;
            if (j <= 64) v = xs[j * S + i];
            else v = ld_peer2(pxs + 8u * (uint32_t)((j - 64) * S + i));
            return (double)v.x + (double)v.y;
        };
        double misfit = 0.0;
        for (int o = tid; o < a.n_obs; o += 32) {
            const double g = a.obs_w[3 * o] * val(a.obs_idx[3 * o]) + a.obs_w[3 * o + 1] * val(a.obs_idx[3 * o + 1]) +
                             a.obs_w[3 * o + 2] * val(a.obs_idx[3 * o + 2]);
            if (a.G) a.G[(size_t)p * a.n_obs + o] = g;
            const double rdf = a.y[o] - g;
            misfit += rdf * rdf;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) misfit += __shfl_xor_sync(0xffffffffu, misfit, off);
        if (tid == 0) {
            a.Phi[p] = 0.5 * misfit * a.inv_sigma2;
            if (a.iters) a.iters[p] = converged ? total_it : -(total_it + 1);
        }
    }
}

// persistent clusters: rank 0 takes the next particle from the counter and hands it to rank 1;
// the cluster barrier at the end of each particle keeps either CTA from overwriting memory the
// other still reads (halo rows, coarse rows, the solution gathered by rank 0, the ticket)
template <bool RHS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(cl::T, 1)
    fem_eval_cluster(FemArgs a, float* ref_scratch, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) float cbuf[2][64];
    __shared__ int item_s;
    const int rank = cluster_rank();
    float* ref = ref_scratch + (size_t)blockIdx.x * cl::REF_FLOATS;
    const uint32_t p_item = peer_addr(smem_addr(&item_s), rank ^ 1);
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int item = atomicAdd(counter, 1);
            item_s = item;
            st_peer(p_item, item);
        }
        cluster_sync();
        const int item = item_s;
        if (item >= a.n) break;   // the same item in both CTAs
        solve_particle_cl<RHS>(a, item, reinterpret_cast<float*>(smem_raw), cbuf, ref, rank);
        cluster_sync();
    }
}

// many problems at 1/128: the same persistent clusters take (problem, particle) items; the item's
// problem is found in a per-item table and each CTA copies its launch arguments to shared memory
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(cl::T, 1)
    fem_eval_cluster_multi(const FemArgs* groups, const int* offsets, const int* item_group, int total,
                           float* ref_scratch, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) float cbuf[2][64];
    __shared__ int item_s, p_s;
    __shared__ FemArgs args_s;
    const int rank = cluster_rank();
    float* ref = ref_scratch + (size_t)blockIdx.x * cl::REF_FLOATS;
    const uint32_t p_item = peer_addr(smem_addr(&item_s), rank ^ 1);
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int item = atomicAdd(counter, 1);
            item_s = item;
            st_peer(p_item, item);
        }
        cluster_sync();
        const int item = item_s;
        if (item >= total) break;   // the same item in both CTAs
        if (threadIdx.x == 0) {
            const int g = item_group[item];
            args_s = groups[g];
            p_s = item - offsets[g];
        }
        __syncthreads();
        solve_particle_cl<true>(args_s, p_s, reinterpret_cast<float*>(smem_raw), cbuf, ref, rank);
        cluster_sync();
    }
}

// persistent form: grid-sized blocks pull (group, particle) items from a device counter; every
// group is one problem's launch arguments at this level size (many independent inverse problems
// in one launch)

template <typename Real, int N, int T>
__global__ void __launch_bounds__(T, (solve_min_blocks<Real, N, T>()))
fem_eval_persistent(const FemArgs* groups, const int* offsets, const int* item_group, int total, int* counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red_buf[2][64];
    __shared__ Real theta_s[256];
    __shared__ int item_s, p_s;
    __shared__ FemArgs args_s;                  // this item's launch arguments, read once per particle
    // thread 0 takes the ticket of the next item before each solve: the atomic's latency overlaps
    // the solve, and item_group maps an item to its group in one load
    int next = 0;
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = next;
            item_s = item;
            if (item < total) {
                const int g = item_group[item];
                args_s = groups[g];
                p_s = item - offsets[g];
                next = atomicAdd(counter, 1);
            }
        }
        __syncthreads();
        if (item_s >= total) break;
        solve_particle<Real, N, T>(args_s, p_s, reinterpret_cast<Real*>(smem_raw), red_buf, theta_s);
        __syncthreads();
    }
}

template <typename Real, int N, int T>
cudaError_t launch_one(const FemArgs& a, cudaStream_t st) {
    const size_t smem = sizeof(Real) * (size_t)solve_smem_reals<Real>(N, T);
    auto kern = fem_eval_kernel<Real, N, T>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<a.n, T, smem, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <typename Real, int N, int T>
cudaError_t launch_one_fc(const FemArgs& a, cudaStream_t st) {
    const size_t smem = sizeof(Real) * (size_t)solve_smem_reals<Real, true>(N, T);
    auto kern = fem_eval_kernel_fc<Real, N, T>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    kern<<<a.n, T, smem, st>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <typename Real, int N, int T>
cudaError_t launch_persistent(const FemArgs* groups, const int* offsets, const int* item_group, int total, int* counter,
                              cudaStream_t st) {
    const size_t smem = sizeof(Real) * (size_t)solve_smem_reals<Real>(N, T);
    auto kern = fem_eval_persistent<Real, N, T>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem);
    if (err != cudaSuccess) return err;
    const int grid = std::max(1, std::min(total, sms * std::max(per_sm, 1)));
    kern<<<grid, T, smem, st>>>(groups, offsets, item_group, total, counter);
    count_launches(1);
    return cudaGetLastError();
}

template <int N, int T, bool FC = false>
cudaError_t launch_global(const FemArgs& a, float* scratch, size_t slice, int blocks, int* counter, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)(arena_size(64, FC) + dense_reals<float, FC>(64));
    cudaError_t e =
        cudaFuncSetAttribute(fem_eval_global<N, T, FC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fem_eval_global<N, T, FC><<<blocks, T, smem, st>>>(a, scratch, slice, counter);
    count_launches(1);
    return cudaGetLastError();
}

template <int N, int T>
cudaError_t launch_global_multi(const FemArgs* groups, const int* offsets, const int* item_group, int total,
                                float* scratch, size_t slice, int blocks, int* counter, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)(arena_size(64) + dense_reals<float>(64));
    cudaError_t e =
        cudaFuncSetAttribute(fem_eval_global_multi<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fem_eval_global_multi<N, T><<<blocks, T, smem, st>>>(groups, offsets, item_group, total, scratch, slice, counter);
    count_launches(1);
    return cudaGetLastError();
}

// compiled compact configurations: blocks per SM that the registers are sized for (0: none)
constexpr int compact_min_blocks(int N, int T) {
    return (N == 64 && T == 512) ? 2 : (N == 32 && T == 256) ? 4 : 0;
}

template <int N>
constexpr size_t compact_smem() {
    return sizeof(float) * (size_t)(arena_size_cp(N) + dense_reals<float>(N));
}

template <int N, int T, bool RHS>
cudaError_t launch_compact_t(const FemArgs& a, float* ref_scratch, int blocks, int* counter, cudaStream_t st) {
    constexpr int MINB = compact_min_blocks(N, T);
    cudaError_t e = cudaFuncSetAttribute(fem_eval_compact<N, T, MINB, RHS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)compact_smem<N>());
    if (e != cudaSuccess) return e;
    fem_eval_compact<N, T, MINB, RHS><<<blocks, T, compact_smem<N>(), st>>>(a, ref_scratch, counter);
    count_launches(1);
    return cudaGetLastError();
}

template <int N, int T>
cudaError_t launch_compact(const FemArgs& a, float* ref_scratch, int blocks, int* counter, cudaStream_t st) {
    return a.rhs ? launch_compact_t<N, T, true>(a, ref_scratch, blocks, counter, st)
                 : launch_compact_t<N, T, false>(a, ref_scratch, blocks, counter, st);
}

template <int N, int T>
int compact_resident_blocks() {
    constexpr int MINB = compact_min_blocks(N, T);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the two instantiations share the launch bounds and the shared-memory size
    cudaFuncSetAttribute(fem_eval_compact<N, T, MINB, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)compact_smem<N>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fem_eval_compact<N, T, MINB, false>, T,
                                                  compact_smem<N>());
    return sms * std::max(1, per_sm);
}

// ---- two-CTA cluster form of 1/128 ----
template <bool RHS>
int cluster_resident_clusters() {
    const size_t smem = sizeof(float) * (size_t)cl::SMEM_FLOATS;
    cudaFuncSetAttribute(fem_eval_cluster<RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(cl::T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)fem_eval_cluster<RHS>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

template <bool RHS>
cudaError_t launch_cluster_t(const FemArgs& a, float* ref_scratch, int blocks, int* counter, cudaStream_t st) {
    const size_t smem = sizeof(float) * (size_t)cl::SMEM_FLOATS;
    cudaError_t e = cudaFuncSetAttribute(fem_eval_cluster<RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fem_eval_cluster<RHS><<<blocks, cl::T, smem, st>>>(a, ref_scratch, counter);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace

int fem_compact_blocks(int N, int T) {
    // resident blocks of a compact kernel, queried once per device and configuration
    static int cached[64][2] = {};
    const int c = (N == 64 && T == 512) ? 0 : (N == 32 && T == 256) ? 1 : -1;
    if (c < 0) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cached[dev][c] > 0) return cached[dev][c];
    const int blocks = c == 0 ? compact_resident_blocks<64, 512>() : compact_resident_blocks<32, 256>();
    if (dev >= 0 && dev < 64) cached[dev][c] = blocks;
    return blocks;
}
size_t fem_compact_ref_floats(int N, int T) { return (size_t)4 * fine_slots(N, T) * T; }

int fem_cluster_blocks() {
    // CTAs of the two-CTA form that are resident at once, queried once per device
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
    const int blocks = 2 * cluster_resident_clusters<false>();
    if (dev >= 0 && dev < 64 && blocks > 0) cached[dev] = blocks;
    return blocks;
}
size_t fem_cluster_ref_floats() { return (size_t)cl::REF_FLOATS; }

cudaError_t fem_eval_cluster_launch(const FemArgs& a, float* ref_scratch, int blocks, int* counter, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    if (a.N != 128 || a.precision != SMC_MIXED || !a.kappa || a.flow_cell || blocks < 2) return cudaErrorInvalidValue;
    const int grid = 2 * std::max(1, std::min(a.n, blocks / 2));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    return a.rhs ? launch_cluster_t<true>(a, ref_scratch, grid, counter, st)
                 : launch_cluster_t<false>(a, ref_scratch, grid, counter, st);
}

cudaError_t fem_eval_compact_launch(const FemArgs& a, int T, float* ref_scratch, int blocks, int* counter,
                                    cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    if (a.precision != SMC_MIXED || !a.kappa || compact_min_blocks(a.N, T) == 0) return cudaErrorInvalidValue;
    const int grid = std::max(1, std::min(a.n, blocks));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (a.N == 64 && T == 512) return launch_compact<64, 512>(a, ref_scratch, grid, counter, st);
    if (a.N == 32 && T == 256) return launch_compact<32, 256>(a, ref_scratch, grid, counter, st);
    return cudaErrorInvalidValue;
}

size_t fem_global_slice(int N, bool FC) {
    const int NI = (N - 1) * (FC ? N + 1 : N - 1);
    const size_t floats = (size_t)arena_size(N, FC) + 6 * (size_t)NI;
    return (floats + 63) / 64 * 64;   // floats per block, 256-byte aligned slices
}

int fem_global_blocks(int N) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = sizeof(float) * (size_t)(arena_size(64) + dense_reals<float>(64));
    if (N == 128) {
        cudaFuncSetAttribute(fem_eval_global<128, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fem_eval_global<128, 1024>, 1024, smem);
    } else {
        cudaFuncSetAttribute(fem_eval_global<256, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fem_eval_global<256, 1024>, 1024, smem);
    }
    return sms * std::max(1, per_sm);
}

cudaError_t fem_eval_global_launch(const FemArgs& a, float* scratch, int blocks, int* counter, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    const size_t slice = fem_global_slice(a.N, a.flow_cell != 0);
    const int grid = std::max(1, std::min(a.n, blocks));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (a.flow_cell) {
        if (a.N == 128) return launch_global<128, 1024, true>(a, scratch, slice, grid, counter, st);
        if (a.N == 256) return launch_global<256, 1024, true>(a, scratch, slice, grid, counter, st);
        return cudaErrorInvalidValue;
    }
    if (a.N == 128) return launch_global<128, 1024>(a, scratch, slice, grid, counter, st);
    if (a.N == 256) return launch_global<256, 1024>(a, scratch, slice, grid, counter, st);
    return cudaErrorInvalidValue;
}

bool fem_cluster_form(int N, int precision, bool flow_cell) {
    return N == 128 && precision == SMC_MIXED && !flow_cell && fem_cluster_blocks() >= 2;
}

size_t fem_large_multi_scratch(int N) {
    if (fem_cluster_form(N, SMC_MIXED, false)) return (size_t)fem_cluster_blocks() * cl::REF_FLOATS;
    return (size_t)fem_global_blocks(N) * fem_global_slice(N);
}

cudaError_t fem_eval_large_multi_launch(int N, const FemArgs* groups, const int* offsets, const int* item_group,
                                        int total, float* scratch, int* counter, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    if (!fem_cluster_form(N, SMC_MIXED, false))
        return fem_eval_global_multi_launch(N, groups, offsets, item_group, total, scratch, fem_global_blocks(N),
                                            counter, st);
    const size_t smem = sizeof(float) * (size_t)cl::SMEM_FLOATS;
    cudaError_t e = cudaFuncSetAttribute(fem_eval_cluster_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = 2 * std::max(1, std::min(total, fem_cluster_blocks() / 2));
    fem_eval_cluster_multi<<<grid, cl::T, smem, st>>>(groups, offsets, item_group, total, scratch, counter);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t fem_eval_global_multi_launch(int N, const FemArgs* groups, const int* offsets, const int* item_group,
                                         int total, float* scratch, int blocks, int* counter, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    const size_t slice = fem_global_slice(N);
    const int grid = std::max(1, std::min(total, blocks));
    if (N == 128) return launch_global_multi<128, 1024>(groups, offsets, item_group, total, scratch, slice, grid, counter, st);
    if (N == 256) return launch_global_multi<256, 1024>(groups, offsets, item_group, total, scratch, slice, grid, counter, st);
    return cudaErrorInvalidValue;
}

cudaError_t fem_eval_persistent_launch(int N, int precision, int T, const FemArgs* groups, const int* offsets,
                                       const int* item_group, int total, int* counter, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    if (T <= 0) T = fem_block_sizes(N, precision).at(0);
    if (precision == SMC_MIXED) {
        switch (N * 10000 + T) {
            case 4 * 10000 + 32: return launch_persistent<float, 4, 32>(groups, offsets, item_group, total, counter, st);
            case 8 * 10000 + 64: return launch_persistent<float, 8, 64>(groups, offsets, item_group, total, counter, st);
            case 8 * 10000 + 32: return launch_persistent<float, 8, 32>(groups, offsets, item_group, total, counter, st);
            case 16 * 10000 + 128: return launch_persistent<float, 16, 128>(groups, offsets, item_group, total, counter, st);
            case 16 * 10000 + 64: return launch_persistent<float, 16, 64>(groups, offsets, item_group, total, counter, st);
            case 32 * 10000 + 256: return launch_persistent<float, 32, 256>(groups, offsets, item_group, total, counter, st);
            case 32 * 10000 + 512: return launch_persistent<float, 32, 512>(groups, offsets, item_group, total, counter, st);
            case 64 * 10000 + 512: return launch_persistent<float, 64, 512>(groups, offsets, item_group, total, counter, st);
            case 64 * 10000 + 1024: return launch_persistent<float, 64, 1024>(groups, offsets, item_group, total, counter, st);
        }
    } else {
        switch (N * 10000 + T) {
            case 4 * 10000 + 32: return launch_persistent<double, 4, 32>(groups, offsets, item_group, total, counter, st);
            case 8 * 10000 + 64: return launch_persistent<double, 8, 64>(groups, offsets, item_group, total, counter, st);
            case 16 * 10000 + 128: return launch_persistent<double, 16, 128>(groups, offsets, item_group, total, counter, st);
            case 16 * 10000 + 256: return launch_persistent<double, 16, 256>(groups, offsets, item_group, total, counter, st);
            case 32 * 10000 + 256: return launch_persistent<double, 32, 256>(groups, offsets, item_group, total, counter, st);
            case 32 * 10000 + 512: return launch_persistent<double, 32, 512>(groups, offsets, item_group, total, counter, st);
        }
    }
    return cudaErrorInvalidValue;
}

bool fem_level_supported(int N, int precision) {
    if (precision == SMC_MIXED) return N == 4 || N == 8 || N == 16 || N == 32 || N == 64 || N == 128 || N == 256;
    return N == 4 || N == 8 || N == 16 || N == 32;
}

// the block size used when none was chosen: the compact form where it is compiled (it is
// faster at J = 4000 on 1/32 and 1/64, and bit-identical to the size -T), the two-CTA form on
// 1/128, else the first size
int fem_default_block(int N, int precision) {
    if (precision == SMC_MIXED && (N == 32 || N == 64)) return N == 64 ? -512 : -256;
    // 1/128: the two-CTA cluster form where a cluster fits (1.2x the device-memory form at J = 4000
    // and 8000), else the device-memory form
    if (precision == SMC_MIXED && N == 128) return fem_cluster_blocks() >= 2 ? -1024 : 1024;
    const std::vector<int> s = fem_block_sizes(N, precision);
    return s.empty() ? 0 : s[0];
}

// block sizes compiled for each level (threads per particle); the autotuner picks one
std::vector<int> fem_block_sizes(int N, int precision) {
    if (precision == SMC_MIXED) {
        switch (N) {
            case 4: return {32};
            case 8: return {32, 64};
            case 16: return {128, 64};
            case 32: return {256, 512, -256};   // -256: compact form, four blocks per SM
            case 64: return {512, 1024, -512};  // -512: compact form, two blocks per SM
            case 128: return {1024, -1024};     // -1024: two-CTA cluster form (fine level on chip)
            case 256: return {1024};
        }
    } else {
        switch (N) {
            case 4: return {32};
            case 8: return {64};
            case 16: return {128, 256};
            case 32: return {256, 512};
        }
    }
    return {};
}

cudaError_t fem_eval_launch(const FemArgs& a, cudaStream_t st, int T) {
    if (a.n <= 0) return cudaSuccess;
    if (a.flow_cell) {   // one block size per level (1/64: 448 threads keep it within shared memory)
        if (a.precision == SMC_MIXED) {
            switch (a.N) {
                case 8: return launch_one_fc<float, 8, 32>(a, st);
                case 16: return launch_one_fc<float, 16, 128>(a, st);
                case 32: return launch_one_fc<float, 32, 256>(a, st);
                case 64: return launch_one_fc<float, 64, 448>(a, st);
            }
        } else {
            switch (a.N) {
                case 8: return launch_one_fc<double, 8, 64>(a, st);
                case 16: return launch_one_fc<double, 16, 128>(a, st);
                case 32: return launch_one_fc<double, 32, 256>(a, st);
            }
        }
        return cudaErrorInvalidValue;
    }
    if (T <= 0) T = fem_block_sizes(a.N, a.precision).at(0);
    if (a.precision == SMC_MIXED) {
        switch (a.N * 10000 + T) {
            case 4 * 10000 + 32: return launch_one<float, 4, 32>(a, st);
            case 8 * 10000 + 64: return launch_one<float, 8, 64>(a, st);
            case 8 * 10000 + 32: return launch_one<float, 8, 32>(a, st);
            case 16 * 10000 + 128: return launch_one<float, 16, 128>(a, st);
            case 16 * 10000 + 64: return launch_one<float, 16, 64>(a, st);
            case 32 * 10000 + 256: return launch_one<float, 32, 256>(a, st);
            case 32 * 10000 + 512: return launch_one<float, 32, 512>(a, st);
            case 64 * 10000 + 512: return launch_one<float, 64, 512>(a, st);
            case 64 * 10000 + 1024: return launch_one<float, 64, 1024>(a, st);
        }
    } else {
        switch (a.N * 10000 + T) {
            case 4 * 10000 + 32: return launch_one<double, 4, 32>(a, st);
            case 8 * 10000 + 64: return launch_one<double, 8, 64>(a, st);
            case 16 * 10000 + 128: return launch_one<double, 16, 128>(a, st);
            case 16 * 10000 + 256: return launch_one<double, 16, 256>(a, st);
            case 32 * 10000 + 256: return launch_one<double, 32, 256>(a, st);
            case 32 * 10000 + 512: return launch_one<double, 32, 512>(a, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace mls2mc
