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
    const float4* u_off = nullptr;      // per U entry (b, A): ((c_A - c_b)/side_b as x, y, side_A/side_b, 0)
    const int32_t *v_ptr = nullptr, *v_idx = nullptr;
    const int32_t *w_ptr = nullptr, *w_idx = nullptr;
    const int32_t *x_ptr = nullptr, *x_idx = nullptr;
    const float4* x_off = nullptr;      // per X entry (b, C): the same offsets as u_off
    std::vector<int32_t> level_start;   // host copy, [nlevels + 1]
    // Symmetric near field (charge points identical to evaluation points, same
    // tree order): each pair of distinct adjacent leaves (b, A), A > b, is summed
    // once by the block of b, which also produces q_b-weighted sums for A's
    // points in "slots" (one run of |A| float-float values per group of 32 of
    // b's points), added to A's potentials afterwards in a fixed order.
    bool sym = false;
    const int32_t* sym_leaves = nullptr;  // [nleaf] leaf order for the symmetric kernel (costliest first)
    const int64_t* sym_off = nullptr;     // per U entry (b, A): first slot when A > b, else -1
    const int32_t* sym_in_ptr = nullptr;  // per box: range of sym_in_slot (groups received)
    const int64_t* sym_in_slot = nullptr; // slot bases received by a leaf
    const int32_t* sym_in_pptr = nullptr; // per box: range of sym_in_pbox
    const int32_t* sym_in_pbox = nullptr; // leaves b that sent slots to a leaf
    const int32_t* sym_pt_leaf = nullptr; // [points] the leaf of each point (tree order)
    // Within a leaf (at most kOwnGroups groups of 32 points, no two points at the
    // same coordinates) each pair of its points is also evaluated once: in-warp for
    // pairs inside a group of 32, and between groups with the partial sums handed
    // over through shared memory.
    const int32_t* sym_own = nullptr;     // [nbox] 1: the leaf's own pairs are symmetric
    int64_t sym_slots = 0;
};

constexpr int kOwnGroups = 4;  // leaves of at most 128 points take the symmetric own-leaf sum

// Table of the FP64 near-field logarithm (vp_fmm64.cu): 2^kLog64Bits entries.
constexpr int kLog64Bits = 12;

// Arithmetic of a plan's evaluation (fixed at plan creation).
enum class Arith {
    kF64,    // default: every step in float64 on the FP64 pipes (vp_fmm64.cu, k_out_grouped64)
    kFF,     // VP_FLAG_FF: heavy steps in float-float on the FP32 pipes
    kPlain   // VP_FLAG_FP64: the plain float64 reference kernels
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
    const double2* log64 = nullptr; // [1 << kLog64Bits] {s_k, -log s_k}               (FP64 log)
    const double* elog64 = nullptr; // [128] (i - 64) log 2                            (FP64 log)
    const double2* m2m64 = nullptr; // [4][P1][P1] M2M coefficients per child quadrant   (float64 M2M)
    const double2* l2l64 = nullptr; // [4][P1][P1] L2L coefficients per child quadrant   (float64 L2L)
    const uint32_t* m2lh = nullptr; // [8][32][40] bf16 digits of the scaled M2L matrix, as 32-bit words
    const int32_t* m2le = nullptr;  // [32] row exponents of those digits
    const double2* mtpow_s = nullptr; // [49][P1] (-t_o / tau)^k, tau = 2^-1.5            (float64 M2L)
    const double* tau_pow = nullptr;  // [P1] tau^k
    const longlong2* logint = nullptr; // [1 << kLog64Bits] (S_k, T_k) of the fixed-point logarithm
    // float-float copies for the FP32-pipe M2L
    const float2* Hf = nullptr;     // [P1][P1]
    const float4* tpowf = nullptr;  // [49][P1] complex (re_h, re_l, im_h, im_l)
    const float4* mtpowf = nullptr; // [49][P1]
    const float2* log2of = nullptr; // [49]
    const float2* invlf = nullptr;  // [P1] 1/l (0 for l = 0)
    const float2* Bmf = nullptr;    // [P1][P1] C(l-1, k-1) 2^-k as hi/lo
    const float2* Blf = nullptr;    // [P1][P1] C(k, l) 2^-l as hi/lo
    const float2* zpowf = nullptr;  // [4][P1] zeta_c^m (exact in float)
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
    // the same points as integers on the grid 2^-sigma (x 2^sigma exactly, rounded
    // only where |x| < 2^(61 - sigma - 53)), |value| < 2^61
    const longlong2* cfix = nullptr;
    const longlong2* efix = nullptr;
    int32_t fix_sigma = 60;
    // powers u^k (k = 1..P) of each point relative to its leaf, [n][P] (float64 plans)
    const double2* cpow = nullptr;
    const double2* epow = nullptr;
};

// Correction matrix with consecutive rows that share one column list grouped
// together (the rows of one cell couple to the same near cells), and values
// as hi/lo float pairs. Rows are in caller order.
struct DevGroupedCSR {
    int32_t nrows = 0;
    int32_t ngroups = 0;
    int32_t max_m = 0;                 // longest column list
    const int32_t* g_r0 = nullptr;     // [ngroups + 1] first row of each group
    const int64_t* g_c0 = nullptr;     // [ngroups + 1] offsets into cols
    const int32_t* cols = nullptr;     // column list of each group
    const int64_t* rowptr = nullptr;   // [nrows + 1] offsets into vf / vi
    const float2* vf = nullptr;        // [nnz] values as hi/lo floats (float-float plans)
    // float64 plans: the values of row r in fixed point, v = V 2^vexp[r] with
    // |V| <= 2^52, stored as {V mod 2^26, V >> 26} (both int32)
    const int2* vi = nullptr;          // [nnz]
    const int32_t* vexp = nullptr;     // [nrows]
    // transposed product: the positions p (into cols) where column c appears,
    // ascending, for c < adj_ncols
    int64_t adj_ncols = 0;
    const int64_t* inc_ptr = nullptr;  // [adj_ncols + 1]
    const int64_t* inc_pos = nullptr;  // [g_c0[ngroups]]
};

// Per-cell interpolation from the density's p-nodes to the FMM's q-nodes
// (oversampled smooth quadrature). Type t: tinfo[8 t ..] = kind, n_q, n_p, qa,
// pa, qb, pb, 0; its matrices start at mats + toff[2 t] (dense O, or A) and
// mats + toff[2 t + 1] (B).
struct DevUpsample {
    int32_t n_cells = 0;
    int32_t n_types = 0;
    int32_t max_q = 0, max_p = 0, max_tmp = 0;  // largest n_q, n_p, pa * qb over the types
    const int32_t* cell_type = nullptr;
    const int64_t* f_start = nullptr;
    const int64_t* src_start = nullptr;
    const int32_t* tinfo = nullptr;
    const int64_t* toff = nullptr;
    const double* mats = nullptr;
};

// Modified-Helmholtz kernel (vp_mhelm.cu): per-level operator tables and the
// near-field series. sigma_l = lambda R_l, R_l the half side of level-l boxes.
struct DevMH {
    double lambda = 0.0;
    double lam2_4 = 0.0;             // lambda^2 / 4
    double c0 = 0.0;                 // log(lambda / 2) + Euler's gamma
    double psi_scale = 0.0;          // -lambda^2 (psi = -lambda^2 sum q K0)
    double inv_fact_P = 0.0;         // 1 / P!
    int near_deg = 0;                // near-field series terms k = 0..near_deg (largest over the leaves)
    const int32_t* leaf_deg = nullptr;  // [nbox] per leaf: series degree (bits 0-7, <= near_deg) and the
                                        // first term summed in FP32 by the float-float near field (bits 8+)
    const double* near_a = nullptr;  // [near_deg + 1] 1/(k!)^2
    const double* near_b = nullptr;  // [near_deg + 1] H_k/(k!)^2
    const double* spow = nullptr;    // [nlevels][P1] sigma_l^k
    const double2* Tm = nullptr;     // [nlevels][4][P1][2][P1] M2M into a parent of level l (terms j, -j folded)
    const double2* Tl = nullptr;     // [nlevels][4][P1][2][P1] L2L into a child of level l (terms m, -m folded)
    const double2* Tv = nullptr;     // [nlevels][49][P1][2][P1] M2L on scaled coefficients (k, -k folded)
    const float4* Tvf = nullptr;     // the same divided by m! |k|!, float-float (re_h, re_l, im_h, im_l)
};

struct MhTables {
    std::vector<double> spow, near_a, near_b;
    std::vector<int32_t> leaf_deg;
    std::vector<double2> Tm, Tl, Tv;
    std::vector<float4> Tvf;
    double inv_fact_P = 0.0;
    int near_deg = 0;
};

struct Workspace {
    double* q = nullptr;      // [max(n_src, n_tgt)][ND] charges, tree order
    float2* qf = nullptr;     // [max(n_src, n_tgt)][ND] the same charges as hi/lo float pairs
    double2* M = nullptr;     // [nbox][P1][ND] multipole coefficients (scaled)
    float4* Mf = nullptr;     // [nbox][P1][ND] multipoles as float-float complex (re_h, re_l, im_h, im_l)
    float4* Lf = nullptr;     // [nbox][P1][ND] locals as float-float complex
    double2* L = nullptr;     // [nbox][P1][ND] local coefficients (scaled)
    double* psi = nullptr;    // [max(n_src, n_tgt)][2][ND] potential (or gradient) in tree order
    float2* xf = nullptr;     // [ND][max(n_src, n_tgt)] correction input (f or g) as hi/lo floats
    int* work = nullptr;      // work-queue counter of the persistent near-field kernel
    float2* slots = nullptr;  // [sym_slots][ND] symmetric near-field partial sums
    int* m2m_count = nullptr; // [nbox] arrivals of finished children (zero between launches)
    double* adj_partial = nullptr;  // [positions of the grouped correction][ND] transposed partial sums
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

// The float64 FMM (vp_fmm64.cu): upward pass, M2L, L2L and the leaf kernel with the
// symmetric near field when t.sym. Enqueues on `s`; nd is 1, 2, 4 or 8.
// gradient: the leaf kernel writes grad Re phi (psi[(e * 2 + c) * ND + d]) instead of the potential.
cudaError_t launch_point_powers(int P, const DevTree& t, const int32_t* rng, const double2* xy, double2* out,
                                cudaStream_t s);
cudaError_t launch_fmm64(int P, int nd, const DevTree& t, const DevTables& tab, const PassGeom& g, Workspace& ws,
                         bool gradient, PhaseTimer* timer, cudaStream_t s);
void make_log64_tables(std::vector<double2>& tab, std::vector<double>& etab);
std::vector<longlong2> make_logint_table();
std::vector<double2> make_m2m64_table(int P);
std::vector<double2> make_l2l64_table(int P);
void make_m2l_tensor_tables(int P, std::vector<uint16_t>& hd, std::vector<int32_t>& eh, std::vector<double2>& mts,
                            std::vector<double>& taup);
// Device-side construction of the grouped correction (vp_csr.cu). err: device int,
// bit 1 = column out of range, bit 2 = non-finite value. same[i] = row i repeats row i - 1.
cudaError_t launch_csr_check(int64_t nnz, const int32_t* col, const double* val, int64_t ncols, int* err,
                             cudaStream_t s);
cudaError_t launch_row_same(int64_t nrows, const int64_t* rowptr, const int32_t* col, uint8_t* same, cudaStream_t s);
cudaError_t launch_group_cols(int32_t ngroups, const int32_t* g_r0, const int64_t* g_c0, const int64_t* rowptr,
                              const int32_t* col, int32_t* cols, cudaStream_t s);
// the values into the padded layout as hi/lo floats (float-float plans)
cudaError_t launch_pad_values(int64_t nrows, const int64_t* rowptr, const int64_t* prow, const double* val,
                              float2* vf, cudaStream_t s);
// the values into the padded layout in per-row fixed point (float64 plans: vi, vexp
// of DevGroupedCSR)
cudaError_t launch_fix_values(int64_t nrows, const int64_t* rowptr, const int64_t* prow, const double* val, int2* vi,
                              int32_t* vexp, cudaStream_t s);
// out (columns, caller order) = Pi^T x in the modes of launch_out_grouped (inv, w_sorted,
// psi index the columns' tree positions); partial: [g_c0[ngroups]][nd] scratch.
cudaError_t launch_adj_grouped(int nd, const DevGroupedCSR& A, bool f64, const double* x, int64_t ld_x,
                               double* partial, const int32_t* inv, const double* w_sorted, const double* psi,
                               double* out, int64_t ld_out, int mode, int max_blocks, cudaStream_t s);

// Correction apply in float64 (vp_spmv.cu): the same modes as launch_out_grouped, values
// A.vd, x read in caller order (x[d * ld_x + col]).
cudaError_t launch_out_grouped64(int nd, const DevGroupedCSR& A, const int32_t* inv, const double* w_sorted,
                                 const double* psi, const double* x, int64_t ld_x, double* out, int64_t ld_out,
                                 int mode, int max_blocks, cudaStream_t s);

// Launchers (vp_fmm.cu). All enqueue on `s`; nd is the density chunk (1, 2, 4 or 8).
cudaError_t launch_charges(int nd, int32_t n, const int32_t* perm, const double* w_sorted,
                           const double* f, int64_t ld_f, double* q, float2* qf, cudaStream_t s);
// fp64: run the near field and M2L in FP64 instead of on the float-float paths
cudaError_t launch_fmm_potential(int P, int nd, const DevTree& t, const DevTables& tab,
                                 const PassGeom& g, Workspace& ws, bool gradient, bool fp64,
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

// Correction apply on the FP32 pipes (vp_spmv.cu): out[d][r] = -(1/2pi) w psi[inv[r]][d] + (A x)[d][r]
// for every row r of A, w = w_sorted[inv[r]] or 1 when w_sorted is NULL (see mode below;
// launch_out_adjoint accumulates when psi is NULL).
cudaError_t launch_to_ff_rows(int nd, int32_t n, const double* x, int64_t ld_x, float2* xf, cudaStream_t s);
// mode: kOutWithPsi (out = -(1/2pi) w psi + A x), kOutAccumulate (out += A x),
// kOutOverwrite (out = A x). max_blocks > 0 caps the grid (a product run beside other
// kernels takes a share of each SM only).
constexpr int kOutWithPsi = 0, kOutAccumulate = 1, kOutOverwrite = 2;
cudaError_t launch_out_grouped(int nd, const DevGroupedCSR& A, const int32_t* inv, const double* w_sorted,
                               const double* psi, const float2* xf, int64_t ld_xf, double* out, int64_t ld_out,
                               int mode, int max_blocks, cudaStream_t s);
// out[d][r] += -(1/2pi) w psi[inv[r]][d] for r < n (w = w_sorted[inv[r]] or 1)
cudaError_t launch_add_psi(int nd, int32_t n, const int32_t* inv, const double* w_sorted, const double* psi,
                           double* out, int64_t ld_out, cudaStream_t s);

// Oversampling (vp_upsample.cu). Charges q[pos][d] = w_pos (O f)[d][j], pos = inv[j]
// the tree position of q-node j, fused with the interpolation; and the transposed
// interpolation out[d][i] = sum_j O_ji (-(1/2pi) w_pos psi[pos][d]) over each cell.
cudaError_t launch_ups_charges(int nd, const DevUpsample& u, const int32_t* inv, const double* w_sorted,
                               const double* f, int64_t ld_f, double* q, float2* qf, cudaStream_t s);
cudaError_t launch_ups_adjoint(int nd, const DevUpsample& u, const int32_t* inv, const double* w_sorted,
                               const double* psi, double* out, int64_t ld_out, cudaStream_t s);

// Modified-Helmholtz FMM (vp_mhelm.cu): one density per pass; psi = -lambda^2 sum q K0.
// fp64: the near field in FP64 instead of float-float on the FP32 pipes.
cudaError_t launch_fmm_mhelm(int P, const DevTree& t, const DevMH& mh, const float4* logtab, const PassGeom& g,
                             Workspace& ws, bool fp64, PhaseTimer* timer, cudaStream_t s);
int64_t mhelm_launches(int nlevels, bool sym_reduce);
// Host tables for half sides R_level[l]; leaf_dmax[b] bounds the near-field
// distances of leaf b (0 for other boxes). Returns an error message, or "".
std::string make_mh_tables(int P, double lambda, const std::vector<double>& R_level,
                           const std::vector<double>& leaf_dmax, bool ff, MhTables& T);
double green_mhelm_host(double lambda, double r);

bool p_supported(int P);

// The adaptive tree and its lists built on the device from device coordinates
// (vp_tree_gpu.cu): the same Tree, bit for bit, as build_tree on the host.
// Returns "" or a message ("CUDA: ..." for runtime failures). Synchronizes s.
std::string build_tree_gpu(int64_t n_src, const double* src_xy, int64_t n_tgt, const double* tgt_xy,
                           const TreeOptions& opt, Tree& t, cudaStream_t s);

}  // namespace vp
