// Internal declarations shared by the C-ABI layer (vp_api.cu) and the FMM
// kernels (vp_fmm.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "vp.h"
#include "vp_tree.h"

namespace vp {

// Device view of the tree, the points in tree order and the operator tables.
// Roles: "charge" points carry the charges of a pass, "eval" points receive the
// potential. The forward pass has charges at sources and evaluates at targets;
// the transposed pass swaps them. The interaction lists serve both directions
// (U and V are symmetric; W of one direction is X of the other).
struct DevTree {
    int32_t nbox = 0;
    int32_t nlevels = 0;
    int32_t nleaf = 0;
    const double2* center = nullptr;    // [nbox]
    const double* radius = nullptr;     // [nbox] half side R
    const double* log_radius = nullptr; // [nbox] log R
    const int32_t* ixy = nullptr;       // [nbox][2]
    const int32_t* level = nullptr;     // [nbox]
    const int32_t* parent = nullptr;    // [nbox]
    const int32_t* child = nullptr;     // [nbox][4]
    const int32_t* is_leaf = nullptr;   // [nbox]
    const int32_t* src_rng = nullptr;   // [nbox][2]
    const int32_t* tgt_rng = nullptr;   // [nbox][2]
    const int32_t* leaves = nullptr;    // [nleaf]
    const int32_t *u_ptr = nullptr, *u_idx = nullptr;
    const int32_t *v_ptr = nullptr, *v_idx = nullptr;
    const int32_t *w_ptr = nullptr, *w_idx = nullptr;
    const int32_t *x_ptr = nullptr, *x_idx = nullptr;
    std::vector<int32_t> level_start;   // host copy, [nlevels + 1]
};

// Translation-operator tables for one expansion order P (P1 = P + 1 entries).
struct DevTables {
    const double* H = nullptr;      // [P1][P1] H[l][k] = C(l+k-1, k-1)            (M2L)
    const double* Bm = nullptr;     // [P1][P1] Bm[l][k] = C(l-1, k-1) 2^-k        (M2M)
    const double* Bl = nullptr;     // [P1][P1] Bl[l][k] = C(k, l) 2^-l            (L2L)
    const double2* tpow = nullptr;  // [49][P1] t_o^l, t_o = 1/(2 (ox + i oy))     (M2L)
    const double2* mtpow = nullptr; // [49][P1] (-t_o)^k                           (M2L)
    const double* log2o = nullptr;  // [49] log(2 |o|)                             (M2L)
    const double2* zpow = nullptr;  // [4][P1] zeta_c^m, zeta_c = child offset / R_parent
    const float4* logtab = nullptr; // [128] {1/c_k, T_hi, T_lo, 0}, T = -log(1/c_k)  (P2P log)
};

// One direction of the FMM: where charges sit and where the potential is taken.
struct PassGeom {
    const double2* cxy = nullptr;   // charge points, tree order
    const int32_t* crng = nullptr;  // per box [begin, end) into cxy
    const float4* crho = nullptr;   // charge points relative to their leaf: (x - c)/side as hi/lo floats
    int32_t n_charge = 0;
    const double2* exy = nullptr;   // evaluation points, tree order
    const int32_t* erng = nullptr;
    const float4* erho = nullptr;
    int32_t n_eval = 0;
};

struct Workspace {
    double* q = nullptr;      // [max(n_src, n_tgt)][ND] charges, tree order
    float2* qf = nullptr;     // [max(n_src, n_tgt)][ND] the same charges as hi/lo float pairs
    double2* M = nullptr;     // [nbox][P1][ND] multipole coefficients (scaled)
    double2* L = nullptr;     // [nbox][P1][ND] local coefficients (scaled)
    double* psi = nullptr;    // [max(n_src, n_tgt)][2][ND] potential (or gradient) in tree order
    int32_t nd_cap = 0;
};

struct PhaseTimer {
    bool on = false;
    cudaStream_t stream = nullptr;
    std::vector<cudaEvent_t> pool;
    std::vector<int> phase_of;      // per recorded interval: phase index
    int used = 0;
    std::vector<std::string> names; // phase names
    int begin(const char* name);    // records a start event, returns interval id (-1 if off)
    void end(int id);
};

// Launchers (vp_fmm.cu). All enqueue on `s`; nd is the density chunk (1, 2, 4 or 8).
cudaError_t launch_charges(int nd, int32_t n, const int32_t* perm, const double* w_sorted,
                           const double* f, int64_t ld_f, double* q, float2* qf, cudaStream_t s);
// p2p_fp64: evaluate the near field with FP64 log instead of the float-float path
cudaError_t launch_fmm_potential(int P, int nd, const DevTree& t, const DevTables& tab,
                                 const PassGeom& g, Workspace& ws, bool gradient, bool p2p_fp64,
                                 PhaseTimer* timer, cudaStream_t s);
cudaError_t launch_out_forward(int nd, int32_t n_tgt, const int32_t* tgt_inv, const double* psi,
                               const int64_t* rowptr, const int32_t* col, const double* val,
                               const double* f, int64_t ld_f, double* out, int64_t ld_out,
                               cudaStream_t s);
cudaError_t launch_out_adjoint(int nd, int32_t n_src, const int32_t* src_inv, const double* w_caller,
                               const double* psi, const int64_t* cptr, const int32_t* crow,
                               const double* cval, const double* g, int64_t ld_g, double* out,
                               int64_t ld_out, cudaStream_t s);
cudaError_t launch_grad_out(int nd, bool accumulate, int32_t n_tgt, const int32_t* tgt_perm,
                            const double* gpsi, const double* g, int64_t ld_g, double* grad,
                            cudaStream_t s);

bool p_supported(int P);

}  // namespace vp
