/*
 * vp.h — C ABI of libvp, the GB300 (sm_103a) evaluator of the FMM-accelerated
 * volume potential with sparse singular/near-singular corrections of
 * Anderson, Zhu and Veerapaneni, "A fast, high-order scheme for evaluating
 * volume potentials on complex 2D geometries via area-to-line integral
 * conversion and domain mappings" (arXiv 2203.05933).
 *
 * What one evaluation computes, for every target t_i and density d:
 *
 *   out[d][i] = sum_{j : r_j != t_i} w_j f[d][j] G(r_j, t_i)  +  sum_k Pi_ik f[d][k]
 *
 *   G(r, r0) = -(1/2pi) log|r - r0|                       (Sec. 2.1), or the
 *              modified-Helmholtz kernel (VP_KERNEL_MHELMHOLTZ, below)
 *   first sum: the target-independent smooth quadrature rule over all cells,
 *              Jacobians folded into the weights w_j       (Eq. Tk_smooth_quad
 *              and the remark after it; Eq. vio_rokh_quad_rule; Sec. 4.2)
 *   second sum: the sparse correction matrix Pi that collects the per-cell
 *              maps Pi_k(r0), "accurate minus smooth"      (Sec. 4, paragraph
 *              after Eq. nsrcs)
 *
 * The first sum is evaluated by a fast multipole method (the paper's "point
 * FMM", Sec. 1 synopsis and Sec. 4); the second by a CSR sparse product. A
 * source/target pair with bitwise equal coordinates contributes no smooth term.
 *
 * Conventions shared by every entry point
 *   - Points are interleaved float64 pairs: xy[2*i] = x_i, xy[2*i+1] = y_i.
 *   - Densities are row-major float64 [ndens][ld] with ld >= n (leading
 *     dimension in elements); results likewise.
 *   - The correction matrix is CSR with rows = targets, columns = sources:
 *     rowptr int64 [n_tgt+1] (rowptr[0] = 0, non-decreasing), col int32 [nnz]
 *     in [0, n_src), val float64 [nnz]. Column order inside a row is free.
 *   - "device" pointers are CUDA device (or managed) memory on the current
 *     device; "host" pointers are ordinary or pinned host memory.
 *   - The caller keeps ownership of every pointer it passes. A plan copies what
 *     it needs (in tree order) into memory it owns and frees in
 *     vp_plan_destroy.
 *   - stream is a cudaStream_t cast to void* (NULL = legacy default stream).
 *     vp_eval and vp_eval_adjoint only enqueue work on it and never synchronize
 *     the device; vp_plan_create and the *_host entry points synchronize it.
 *   - Every entry point returns a vp_status. No exception crosses the ABI. On
 *     error the output buffers hold unspecified values and the plan stays
 *     usable unless the status is VP_ERR_CUDA (sticky CUDA errors).
 *   - Arithmetic: by default inputs, expansions and results are IEEE float64;
 *     where exact integer arithmetic can replace float64 operations it does
 *     (details at the flags below), rounding no worse than float64. VP_FLAG_FF moves
 *     the heavy steps to the FP32 pipes in float-float arithmetic (an
 *     unevaluated sum of two floats, about 48 significant bits, narrower than
 *     float64 in significand and exponent range) with float64 inputs and
 *     outputs; VP_FLAG_FP64 selects the plain float64 reference kernels.
 */
#ifndef VP_H
#define VP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VP_OK = 0,
    VP_ERR_ARG = 1,         /* null pointer, negative size, malformed CSR, non-finite input,
                               point outside a caller-given root box, ld < n            */
    VP_ERR_CUDA = 2,        /* a CUDA runtime call failed (message: vp_last_error)        */
    VP_ERR_OOM = 3,         /* device or host allocation failed                           */
    VP_ERR_TIMEOUT = 4,     /* reserved: no kernel of this library waits on the device, so
                               no entry point returns it                                  */
    VP_ERR_UNSUPPORTED = 5, /* option outside the compiled set (e.g. p_fmm not built)     */
    VP_ERR_STATE = 6        /* plan used after destroy, or on another device              */
} vp_status;

typedef struct vp_plan_s* vp_plan;

/* Plan options. Zero-initialise and set what you need; zeros pick defaults. */
typedef struct {
    int32_t p_fmm;      /* expansion order P: coefficients 0..P; one of 16, 24, 30 (0 -> 30) */
    int32_t leaf;       /* split a box while it holds more than `leaf` sources or targets
                           (0 -> 64; 1..4096)                                                */
    int32_t max_level;  /* deepest tree level (0 -> 24; at most 27)                          */
    int32_t max_dens;   /* densities processed per pass; workspace is sized for it (0 -> 1)  */
    int32_t flags;      /* VP_FLAG_* bits                                                    */
    int32_t kernel;     /* VP_KERNEL_LAPLACE (0, default) or VP_KERNEL_MHELMHOLTZ           */
    double root[3];     /* enclosing square (x0, y0, side); side <= 0 -> smallest square
                           around all points. Every point must satisfy
                           x0 <= x < x0 + side and y0 <= y < y0 + side.                      */
    double lambda;      /* modified-Helmholtz parameter (> 0; VP_KERNEL_MHELMHOLTZ only)     */
} vp_options;

/* Green functions (arXiv 2203.05933, Sec. 2):
 *   VP_KERNEL_LAPLACE      G(r, r0) = -(1/2pi) log|r - r0|                (L = -Delta)
 *   VP_KERNEL_MHELMHOLTZ   G(r, r0) = (lambda^2/2pi) K0(lambda |r - r0|)  (L = -Delta + lambda^2)
 * The prefactor lambda^2/2pi is the one the paper states; V then solves
 * (-Delta + lambda^2) V = lambda^2 f. Modified-Helmholtz plans come from
 * vp_plan_create only and evaluate one density per pass: P2M, M2L, L2P and the
 * near field (symmetric when the targets are the nodes) in float-float on the
 * FP32 pipes, M2M, L2L, P2L and M2P in FP64; VP_FLAG_FP64 runs every step in
 * FP64. They support vp_eval, vp_eval_host, vp_eval_batch and
 * the grad_f part of vp_eval_adjoint (the kernel is symmetric), and reject
 * grad_tgt with VP_ERR_UNSUPPORTED. Plan creation fails with VP_ERR_ARG if
 * lambda * (box half side) puts the expansion tables out of FP64 range (roughly
 * below 1e-4 for p_fmm = 30, or above a few hundred). */
#define VP_KERNEL_LAPLACE 0
#define VP_KERNEL_MHELMHOLTZ 1

/* Record CUDA events around every phase of vp_eval (read with vp_plan_phase_times). */
#define VP_FLAG_TIMING 1u
/* Arithmetic of a plan (fixed at creation; the two flags exclude each other).
 * Default (neither flag): float64 results, shaped for GB300's narrow FP64 unit. The
 * directed near field forms r^2 exactly from integer coordinates and its logarithm in
 * fixed point (error about 2^-59), summing with float64 FMAs; when the targets are
 * the nodes each distance between two adjacent leaves is evaluated once for both
 * directions with the library's own table-driven float64 logarithm (within about 1.5
 * ulp). M2L: the contraction as exact integer digit products on the tensor cores (62-bit
 * operands), the rest in float64. M2M and L2L: exact in 128-bit fixed point, each
 * coefficient correctly rounded. P2M, L2P: float64. Correction product: the values are
 * stored per row in 52-bit fixed point (rounded to at most 2^-52 of the row's largest
 * value) and the densities staged per row group the same way, summed exactly in 128
 * bits and rounded once per row; the adjoint converts the stored values back exactly
 * and sums in float64.
 * VP_FLAG_FP64: the plain float64 reference kernels (directed near field with CUDA's
 * log, one warp per box and coefficient lane for the expansions); the target gradient
 * of vp_eval_adjoint always runs these.
 * VP_FLAG_FF: the near field, M2L, P2M/M2M/L2L/L2P and the correction product on the
 * FP32 pipes in float-float arithmetic (about 48 significant bits, narrower than
 * float64; float64 inputs and outputs), several times faster on GB300; the results
 * agree with the float64 ones to about 1e-12 of the total charge. */
#define VP_FLAG_FP64 2u
#define VP_FLAG_FF 8u
/* Capture each distinct vp_eval call (same f, out, leading dimensions and ndens) once
 * into a CUDA graph and replay it afterwards. The first call with new arguments
 * synchronizes `stream` and captures on a plan-owned stream; later calls only launch
 * the graph on `stream`. Ignored while VP_FLAG_TIMING is set. */
#define VP_FLAG_GRAPH 4u

/*
 * vp_plan_create — "vp_plan(nodes, weights, targets, corr_csr)".
 * Builds the adaptive quadtree over sources and targets (Morton order, leaves of
 * at most opt->leaf points, interaction lists U/V/W/X of the adaptive FMM) and
 * copies geometry, weights and the correction matrix, permuted into tree
 * order, into plan-owned device memory. Geometry is static after this call
 * (the paper's setting: static geometry, Sec. 1 "Limitations").
 *   src_xy [n_src][2], w [n_src]     device; quadrature nodes and weights (w includes J)
 *   tgt_xy [n_tgt][2]                device; evaluation points (may coincide with nodes)
 *   corr_rowptr/col/val, nnz         device; Pi in CSR (all NULL with nnz = 0: no correction)
 *   opt                              host; may be NULL (all defaults)
 * n_src >= 0, n_tgt >= 0. Synchronizes `stream`. Errors: VP_ERR_ARG, VP_ERR_OOM,
 * VP_ERR_CUDA, VP_ERR_UNSUPPORTED. *out is NULL on error.
 */
vp_status vp_plan_create(vp_plan* out,
                         int64_t n_src, const double* src_xy, const double* w,
                         int64_t n_tgt, const double* tgt_xy,
                         const int64_t* corr_rowptr, const int32_t* corr_col,
                         const double* corr_val, int64_t nnz,
                         const vp_options* opt, void* stream);

/*
 * vp_plan_create_many — one plan for nprob independent problems (many uneven
 * problems evaluated together). Problem k has n_src[k] sources src_xy[k] with
 * weights w[k], n_tgt[k] targets tgt_xy[k] and an optional correction
 * (corr_rowptr[k], corr_col[k], corr_val[k], nnz[k]; corr_rowptr itself may be
 * NULL for no corrections anywhere). roots: NULL, or [nprob][3] root squares
 * (side <= 0 -> derived). The arrays of pointers are host arrays; the pointed-to
 * data follow vp_plan_create's conventions. opt (shared by all problems) as in
 * vp_plan_create; opt->root is ignored.
 * The plan behaves as one problem whose sources, targets and densities are the
 * problems' concatenated in order (caller index of problem k's j-th point =
 * sum_{m<k} n[m] + j) and whose correction is block diagonal: vp_eval,
 * vp_eval_adjoint and vp_eval_host take [ndens][sum n_src] densities and give
 * [ndens][sum n_tgt] results. Interactions never cross problems. The boxes of
 * all problems are stored level by level, so each FMM phase is one launch per
 * level for the whole batch.
 */
vp_status vp_plan_create_many(vp_plan* out, int32_t nprob,
                              const int64_t* n_src, const double* const* src_xy,
                              const double* const* w,
                              const int64_t* n_tgt, const double* const* tgt_xy,
                              const int64_t* const* corr_rowptr, const int32_t* const* corr_col,
                              const double* const* corr_val, const int64_t* nnz,
                              const double* roots, const vp_options* opt, void* stream);

/*
 * vp_plan_create_upsampled — plan of the oversampled smooth quadrature
 * (Sec. 2, "Oversampled smooth quadratures", Eq. Tk_smooth_quad; Sec. 4.2 for
 * boxes; the twofold q = 2p of the Remark after Eq. nsrcs). The density is
 * given at the p-nodes of each cell; the FMM sources are the cells' q-nodes,
 * whose values are interpolated per cell by a fixed matrix of the cell's type,
 *     f_q^k = O_{p,q} f_p^k,
 * fused into the charge load. One evaluation computes
 *     out[d][i] = sum_{j: r_j != t_i} w_j (O f[d])_j G(r_j, t_i) + sum_k Pi_ik f[d][k]
 * where j runs over the q-nodes (src_xy, w: their positions and weights with
 * Jacobians, device, as in vp_plan_create) and the correction's columns index
 * the p-nodes (0 <= col < n_f, n_f = ups->f_start[ups->n_cells]).
 *   ups: host description. Cell k owns q-nodes [src_start[k], src_start[k+1])
 *   and p-nodes [f_start[k], f_start[k+1]) (both starting at 0, non-decreasing,
 *   src_start[n_cells] = n_src; the counts equal the type's n_q and n_p).
 *   A VP_UPS_DENSE type gives O [n_q][n_p] row-major in `mat`; a VP_UPS_TENSOR
 *   type gives O = A (x) B (Kronecker product: row ra*qb + rb, column
 *   ia*pb + ib) with A [qa][pa] in `a` and B [qb][pb] in `b`, row-major, as for
 *   tensor-product nodes of boxes. 1 <= n_q, n_p <= 1024.
 * On such a plan vp_eval, vp_eval_host and the f of vp_eval_adjoint take
 * densities [ndens][ld_f] with ld_f >= n_f, and vp_eval_adjoint's grad_f is
 * [ndens][ld_gf] with ld_gf >= n_f: grad_f = O^T (w * transposed sum) + Pi^T g.
 * Other conventions and errors as in vp_plan_create.
 */
#define VP_UPS_DENSE 0
#define VP_UPS_TENSOR 1
typedef struct {
    int32_t kind;               /* VP_UPS_DENSE or VP_UPS_TENSOR                         */
    int32_t n_q, n_p;           /* rows (q-nodes) and columns (p-nodes) of O             */
    int32_t qa, pa, qb, pb;     /* VP_UPS_TENSOR: n_q = qa * qb, n_p = pa * pb            */
    int32_t reserved;
    const double* mat;          /* VP_UPS_DENSE: [n_q][n_p], host                         */
    const double* a;            /* VP_UPS_TENSOR: [qa][pa], host                          */
    const double* b;            /* VP_UPS_TENSOR: [qb][pb], host                          */
} vp_upsample_type;
typedef struct {
    int32_t n_types;
    int32_t reserved;
    const vp_upsample_type* types;  /* host [n_types]                                     */
    int64_t n_cells;
    const int32_t* cell_type;       /* host [n_cells], each in [0, n_types)               */
    const int64_t* f_start;         /* host [n_cells + 1]                                 */
    const int64_t* src_start;       /* host [n_cells + 1]                                 */
} vp_upsample;
vp_status vp_plan_create_upsampled(vp_plan* out,
                                   int64_t n_src, const double* src_xy, const double* w,
                                   int64_t n_tgt, const double* tgt_xy,
                                   const int64_t* corr_rowptr, const int32_t* corr_col,
                                   const double* corr_val, int64_t nnz,
                                   const vp_upsample* ups, const vp_options* opt, void* stream);
/*
 * vp_eval — "vp_eval(plan, f, out)": out[d][i] for d < ndens (formula above).
 *   f   [ndens][ld_f]   device, ld_f >= n_src, caller (input) order
 *   out [ndens][ld_out] device, ld_out >= n_tgt, caller (input) order; overwritten
 * ndens >= 0; densities beyond max_dens are processed in successive passes.
 * Enqueues on `stream` only; f and out must stay valid until the work completes.
 * Not reentrant on one plan: calls on different streams with the same plan race
 * on the plan's workspace.
 */
vp_status vp_eval(vp_plan plan, int32_t ndens, const double* f, int64_t ld_f,
                  double* out, int64_t ld_out, void* stream);

/*
 * vp_eval_adjoint — transpose of vp_eval and target-position gradient.
 * For upstream gradients g[d][i] = dL/dout[d][i]:
 *   grad_f[d][j]  = w_j sum_{i: t_i != r_j} G(r_j, t_i) g[d][i] + sum_i Pi_ij g[d][i]
 *                   (transposed FMM, charges at the targets, plus Pi^T g)
 *   grad_tgt[i]   = sum_d g[d][i] sum_{j: r_j != t_i} w_j f[d][j] grad_{t_i} G(r_j, t_i)
 *                   (Pi held fixed: correction weights are set-up data)
 *   g        [ndens][ld_g]    device, ld_g >= n_tgt
 *   grad_f   [ndens][ld_gf]   device or NULL (skip), ld_gf >= n_src; overwritten
 *   f        [ndens][ld_f]    device; required when grad_tgt != NULL, else may be NULL
 *   grad_tgt [n_tgt][2]       device or NULL (skip); overwritten
 * Expansions are recomputed from g (and f) on every call, never stored per
 * right-hand side. Enqueues on `stream` only.
 */
vp_status vp_eval_adjoint(vp_plan plan, int32_t ndens,
                          const double* g, int64_t ld_g,
                          double* grad_f, int64_t ld_gf,
                          const double* f, int64_t ld_f,
                          double* grad_tgt, void* stream);

/*
 * vp_eval_host — vp_eval on host buffers: copies f (host, [ndens][n_src] dense)
 * to plan-owned device staging, evaluates, copies out back (host,
 * [ndens][n_tgt] dense), and synchronizes `stream` before returning. Pinned host
 * memory gives asynchronous copies; pageable memory works but is staged by the
 * driver. The staging buffers grow on demand (VP_ERR_OOM if that fails).
 */
vp_status vp_eval_host(vp_plan plan, int32_t ndens, const double* f_host,
                       double* out_host, void* stream);

/*
 * vp_eval_batch — several independent plans evaluated on one stream, in order:
 * plan k takes ndens[k] densities f[k] (leading dimension ld_f[k]) into out[k]
 * (ld_out[k]), with the conventions of vp_eval (each plan replays its own graph
 * with VP_FLAG_GRAPH). For many small problems the single-launch form is one
 * forest plan (vp_plan_create_many): one launch per phase for all problems and
 * one graph per evaluation. Stops at the first error (earlier plans' results
 * stand). Host arrays of length nplans; device buffers as in vp_eval.
 */
vp_status vp_eval_batch(int32_t nplans, const vp_plan* plans, const int32_t* ndens, const double* const* f,
                        const int64_t* ld_f, double* const* out, const int64_t* ld_out, void* stream);

/* Plan summary (host struct filled by vp_plan_info). */
typedef struct {
    int64_t n_src, n_tgt, nnz;
    int32_t p_fmm, leaf, max_dens, n_levels;
    int64_t n_boxes, n_leaves;
    int64_t n_u_pairs;      /* sum over target leaves of |U| (leaf-leaf P2P blocks)     */
    int64_t n_v_pairs;      /* sum over boxes of |V| (M2L translations)                 */
    int64_t n_w_pairs;      /* sum over leaves of |W| (multipole-to-target blocks)      */
    int64_t n_x_pairs;      /* sum over boxes of |X| (source-to-local blocks)           */
    int64_t p2p_pairs;      /* source-target pairs summed directly (one density)        */
    int64_t last_launches;  /* kernel launches made by the last vp_eval on this plan      */
    int64_t n_problems;     /* independent problems in the plan (vp_plan_create_many)     */
    double root[3];         /* root square of the (first) problem                         */
    int64_t n_f;            /* length of a density: n_src, or the p-nodes of an upsampled plan */
    int64_t n_cells;        /* cells of an upsampled plan (0 otherwise)                    */
    int64_t sym_slots;      /* > 0: passes of one or two densities sum the near field once per
                               pair of adjacent leaves (evaluation points = quadrature nodes)
                               and hand the partial sums between leaves through this many
                               slots; more densities per pass sum every directed pair        */
    int64_t p2p_evals;      /* source-target distances such a symmetric pass evaluates (one
                               density): the pairs inside leaves plus one per pair of points
                               in distinct adjacent leaves; p2p_pairs without symmetry       */
    int32_t kernel;         /* VP_KERNEL_*                                                 */
    int32_t near_terms;     /* modified Helmholtz: terms of the near-field series (0 otherwise) */
    double lambda;          /* modified-Helmholtz parameter (0 for Laplace)                */
    int64_t near_ops;       /* modified Helmholtz: modelled FP32 operations of the float-float
                               near field per density (about 92 + 2 (deg - m + 1) + 24 m per
                               evaluated distance, deg and m the leaf's series degree and
                               split, +14 where one evaluation serves both directions) */
} vp_plan_stats;

vp_status vp_plan_info(vp_plan plan, vp_plan_stats* out);
/*
 * Per-phase device times of the last vp_eval on this plan, in milliseconds,
 * measured with CUDA events recorded on the evaluation stream (only with
 * VP_FLAG_TIMING). Synchronizes on the last recorded event. names/ms are host
 * arrays of capacity `cap`; *n receives the number of phases.
 */
vp_status vp_plan_phase_times(vp_plan plan, int32_t cap, const char** names,
                              double* ms, int32_t* n);

/* Change the run-time flags of a plan (VP_FLAG_TIMING, VP_FLAG_GRAPH); the other
 * bits must equal those given at creation (VP_ERR_ARG otherwise). */
vp_status vp_plan_set_flags(vp_plan plan, uint32_t flags);
/* With a correction matrix and blocks_per_sm > 0, vp_eval and vp_eval_adjoint run
 * the correction product beside the FMM on a plan-owned low-priority stream
 * (captured graphs: the FMM stream has the highest priority), with a grid of
 * blocks_per_sm blocks on every SM, then add the smooth part. 0 (the default) runs
 * the product after the FMM in one kernel. The best share depends on the balance
 * of the two (autotune.tune_overlap measures it). Drops captured graphs. Phase
 * timing always runs the product after the FMM. */
vp_status vp_plan_set_overlap(vp_plan plan, int32_t blocks_per_sm);

vp_status vp_plan_destroy(vp_plan plan);

/* G(r) of `kernel` (lambda as in vp_options) at n distances r[i] > 0, on the
 * host, with the Bessel routines the plans use for their operator tables
 * (K0 by its ascending series for lambda r <= 2, by the trapezoidal rule on its
 * integral representation above; relative error about 1e-15). r, g: host,
 * [n]. Errors: VP_ERR_ARG (NULL pointer, n < 0, r[i] <= 0, bad kernel or
 * lambda). */
vp_status vp_green_eval_host(int32_t kernel, double lambda, int64_t n, const double* r, double* g);

/* Roofline denominators measured on the current device at its present clocks:
 * sustained FP64 and FP32 fused multiply-add throughput in TFLOP/s (2 flops per FMA),
 * from chains of independent FMAs in every lane of a full grid (best of two timed
 * launches after a warm-up launch, CUDA events on `stream`); if `dmma_tflops`,
 * `bf16_mma_tflops` / `s8_mma_tops` are not NULL, also the FP64 tensor
 * instruction (mma.sync m8n8k4 f64), the bf16 warp-level tensor instruction
 * (mma.sync m16n8k16, f32 accumulation) and the int8 one (mma.sync m16n8k32,
 * s32 accumulation, in T operations/s) measured the same way. The paper has no counterpart: this
 * supports the measurement of the kernels against their roofline. Allocates and
 * frees a small device buffer and synchronizes `stream`. Takes about 0.2 s.
 * Errors: VP_ERR_ARG (NULL fp64/fp32 output), VP_ERR_OOM, VP_ERR_CUDA. */
vp_status vp_measure_peaks(double* fp64_tflops, double* fp32_tflops, double* dmma_tflops, double* bf16_mma_tflops,
                           double* s8_mma_tops, void* stream);

/* Static description of a status code; never NULL. */
const char* vp_status_string(int32_t status);

/* Text of the last error raised on the calling thread ("" if none). */
const char* vp_last_error(void);

/* Library version string, e.g. "libvp 0.1 sm_103a". */
const char* vp_version(void);

/*
 * Host-side inspection of the tree and interaction lists (no GPU needed).
 * vp_tree_build builds exactly the tree vp_plan_create builds (on the GPU) for
 * the same points and options, on the host, from host arrays.
 * vp_tree_get copies one array out (which = VP_TREE_*); pass dst = NULL to get
 * the element count in *count first. Arrays:
 *   VP_TREE_BOX_LEVEL   int32 [n_boxes]
 *   VP_TREE_BOX_IXY     int32 [n_boxes][2]   integer box coordinates at its level
 *   VP_TREE_BOX_PARENT  int32 [n_boxes]      -1 for the root
 *   VP_TREE_BOX_LEAF    int32 [n_boxes]      1 if leaf
 *   VP_TREE_BOX_SRC     int32 [n_boxes][2]   [begin, end) in sorted source order
 *   VP_TREE_BOX_TGT     int32 [n_boxes][2]   [begin, end) in sorted target order
 *   VP_TREE_SRC_PERM    int32 [n_src]        sorted position -> caller index
 *   VP_TREE_TGT_PERM    int32 [n_tgt]
 *   VP_TREE_{U,V,W,X}_PTR int32 [n_boxes+1]  CSR offsets of each list
 *   VP_TREE_{U,V,W,X}_IDX int32 [...]        box indices
 */
typedef struct vp_tree_s* vp_tree;
enum {
    VP_TREE_BOX_LEVEL = 0, VP_TREE_BOX_IXY, VP_TREE_BOX_PARENT, VP_TREE_BOX_LEAF,
    VP_TREE_BOX_SRC, VP_TREE_BOX_TGT, VP_TREE_SRC_PERM, VP_TREE_TGT_PERM,
    VP_TREE_U_PTR, VP_TREE_U_IDX, VP_TREE_V_PTR, VP_TREE_V_IDX,
    VP_TREE_W_PTR, VP_TREE_W_IDX, VP_TREE_X_PTR, VP_TREE_X_IDX
};
vp_status vp_tree_build(vp_tree* out, int64_t n_src, const double* src_xy_host,
                        int64_t n_tgt, const double* tgt_xy_host, const vp_options* opt);
/*
 * vp_tree_build_device — the same tree and lists, bit for bit, built on the GPU
 * from device point arrays (what vp_plan_create uses): Morton keys on the 28-bit
 * grid of the root square, an LSD radix sort that keeps equal keys in caller
 * order, splitting level by level and the U/V/W/X lists, as kernels; the result
 * is copied into a host-side vp_tree for vp_tree_get. src_xy, tgt_xy: device.
 * Synchronizes `stream`. Errors: VP_ERR_ARG (as vp_tree_build), VP_ERR_CUDA.
 */
vp_status vp_tree_build_device(vp_tree* out, int64_t n_src, const double* src_xy, int64_t n_tgt,
                               const double* tgt_xy, const vp_options* opt, void* stream);
vp_status vp_tree_get(vp_tree tree, int32_t which, int32_t* dst, int64_t* count);
vp_status vp_tree_destroy(vp_tree tree);

/*
 * Interpolation of nodal values to arbitrary points (Sec. 3.2.1, Eq.
 * vals_to_coeffs and the Koornwinder expansion above it; Sec. 4.2 for boxes):
 * inside each cell the values at the cell's nodes determine a polynomial
 * expansion, coefficients a = C v (C the values-to-coefficients map of the
 * cell's type), which is then summed at the reference coordinates of every
 * point located in that cell:
 *     out[d][k] = sum_b a_b phi_b(xi_k, eta_k).
 * Typical use: V at off-node points from V at the nodes (vp_eval's output).
 * Bases (n_basis = n_nodes of the type):
 *   VP_BASIS_LEGENDRE2: P_i(xi) P_j(eta) on [-1, 1]^2, 0 <= i, j < order,
 *     index b = j * order + i (eta-major, xi fastest, like the box nodes).
 *   VP_BASIS_SIMPLEX: on {xi, eta >= 0, xi + eta <= 1}, total degree < order,
 *     phi_(m,k) = P_m(s / t) t^m P_k^(2m+1,0)(2 eta - 1), s = 2 xi - 1 + eta,
 *     t = 1 - eta, index running over m = 0..order-1 and k = 0..order-1-m
 *     (m-major); P_k^(a,b) the Jacobi polynomials.
 * Point location and the inverse cell maps are set-up work (static geometry):
 * the caller gives each point's cell and reference coordinates.
 */
#define VP_BASIS_LEGENDRE2 0
#define VP_BASIS_SIMPLEX 1
typedef struct vp_interp_s* vp_interp;
typedef struct {
    int32_t basis;        /* VP_BASIS_*                                                  */
    int32_t order;        /* 1..32                                                       */
    int32_t n_nodes;      /* order^2 (LEGENDRE2) or order (order + 1) / 2 (SIMPLEX)       */
    int32_t reserved;
    const double* coef;   /* C [n_nodes][n_nodes] row-major, a_b = sum_i C[b][i] v_i, host */
} vp_interp_type;
/*
 * vp_interp_create — copies the description into device memory.
 *   types [n_types], cell_type [n_cells], node_start [n_cells + 1] (node range
 *   of each cell in the value vector, starting at 0, counts = the type's
 *   n_nodes): host. pt_cell [n_pts] int32 in [0, n_cells) and pt_ref
 *   [n_pts][2] (xi, eta): device. Synchronizes `stream`.
 */
vp_status vp_interp_create(vp_interp* out, int32_t n_types, const vp_interp_type* types,
                           int64_t n_cells, const int32_t* cell_type, const int64_t* node_start,
                           int64_t n_pts, const int32_t* pt_cell, const double* pt_ref, void* stream);
/*
 * vp_interp_eval — v [ndens][ld_v] (device, ld_v >= node_start[n_cells]) to
 * out [ndens][ld_out] (device, ld_out >= n_pts). Enqueues on `stream` only.
 */
vp_status vp_interp_eval(vp_interp ip, int32_t ndens, const double* v, int64_t ld_v,
                         double* out, int64_t ld_out, void* stream);
vp_status vp_interp_destroy(vp_interp ip);

/*
 * Singular (self) corrections of mapped triangles, generated on the GPU
 * (Sec. 3.3; efficient pre-computation of Sec. 3.4, Eq. singcorr_inner_prod).
 * For the target at reference node a of a cell with map R and Jacobian J:
 *   Vhat_b = sum_i g_i B[a][b][i],
 *   g_i = J(chi_i) / (2 pi)                                   if tau[a][i] < 0,
 *   g_i = -(log|R(chi_i) - R(zeta_a)| - log tau[a][i]) J(chi_i) / (2 pi)   otherwise,
 *   corr[c][a][j] = sum_b Vhat_b coef[b][j] - w_j J(zeta_j) G(R(zeta_j), R(zeta_a))
 *                   (the smooth term only for j != a),
 * the "accurate minus smooth" self block of cell c (Sec. 4). chi, tau and B are
 * the same for every cell (the kind of node, tau < 0, marks the nodes whose
 * -log t factor is folded into B; |tau| is the node's ray parameter t). The
 * set-up (host) builds them once; the GPU evaluates the mapped Green function
 * and Jacobian and the contraction for all cells.
 * vp_tricorr_create: host tables node_ref [n_nodes][2] (reference nodes
 * zeta_j), node_w [n_nodes] (reference weights w_j), coef [n_basis][n_nodes]
 * (values-to-coefficients map), chi [n_nodes][n_rule][2], tau
 * [n_nodes][n_rule] (0 < |tau| <= 1), B [n_nodes][n_basis][n_rule];
 * n_basis <= 36. Synchronizes `stream`.
 * vp_tricorr_eval: geom [n_cells][12] device: v0, v1, v2 (x, y), kind (0
 * straight, 1 circle arc cx, cy, r, th0, th1; 2 polar arc r = 1 + a cos(k th)
 * with a, k, th0, th1), the curved edge running from v0 (th0) to v1 (th1);
 * out [n_cells][n_nodes][n_nodes] device. Enqueues on `stream` only.
 */
typedef struct vp_tricorr_s* vp_tricorr;
vp_status vp_tricorr_create(vp_tricorr* out, int32_t n_nodes, int32_t n_basis, int32_t n_rule,
                            const double* node_ref, const double* node_w, const double* coef,
                            const double* chi, const double* tau, const double* B, void* stream);

/*
 * Near-singular corrections of mapped triangles (Sec. 3.3.3, Eq.
 * vp_near_singular, and the inner product of Eq. singcorr_inner_prod): for
 * pair p, a cell (geom[p], as in vp_tricorr_eval) and a target r0 = tgt[p]
 * strictly outside it (in its near zone, Sec. 3.1),
 *   out[p][j] = sum_b Vhat_b coef[b][j] - w_j J(zeta_j) G(R(zeta_j), r0),
 *   Vhat_b = int_T0 G(R(zeta), r0) K_b(zeta) J(zeta) dzeta,
 * the "accurate minus smooth" block row of the pair (Sec. 4). Vhat is taken by
 * the area-to-line conversion (Lemma 1) with the star point at the cell point
 * nearest r0 (Eq. rstar_def): rays to the edges not through it, Gauss-Legendre
 * in t (8 points) on panels graded dyadically towards both ends of the rays
 * and in s (10 points) on panels graded towards the star point's foot and
 * towards the point nearest r0 on each edge; K_b is the collapsed-coordinate
 * Legendre x Jacobi basis (total degree <= 7, the order of coef's rows).
 * Measured against adaptive quadrature: about 1e-13 of the accurate part for
 * targets down to 1e-3 cell sizes on cells whose smallest angle is 20 degrees
 * or more (on slivers of a few degrees the fixed rules lose accuracy, as the
 * self blocks do). geom [n_pairs][12],
 * tgt [n_pairs][2], out [n_pairs][n_nodes]: device. A target on or inside the
 * cell is outside the contract (its result is not finite or not accurate).
 * Errors: VP_ERR_STATE (invalid plan, other device), VP_ERR_ARG (n_pairs < 0,
 * NULL pointers), VP_ERR_UNSUPPORTED (n_basis not a complete basis of degree
 * <= 7), VP_ERR_CUDA. Enqueues on `stream` only.
 */
vp_status vp_tricorr_near_eval(vp_tricorr tc, int64_t n_pairs, const double* geom, const double* tgt, double* out,
                               void* stream);
vp_status vp_tricorr_eval(vp_tricorr tc, int64_t n_cells, const double* geom, double* out,
                          void* stream);
vp_status vp_tricorr_destroy(vp_tricorr tc);

/*
 * vp_eval_direct_static — evaluation that allocates nothing.
 *
 * For callers that cannot allocate device memory when they need the volume
 * potential: a host application that owns every device allocation and hands
 * out only buffers it made itself, a plug-in running inside someone else's
 * stream capture where an allocation would break the capture, or an embedded
 * user whose device footprint must not grow after start-up. vp_plan_create
 * allocates (tree, workspace), so such callers use this entry point instead.
 * The paper has no counterpart: this is a convenience variant of the direct
 * (P2P) kernel without a tree, summing over every source, so its cost is
 * O(n_src * n_tgt) and it suits small problems.
 *
 * It computes the same quantity as vp_eval:
 *   out[d][i] = sum_{j: r_j != t_i} w_j f[d][j] G(r_j, t_i) + sum_k Pi_ik f[d][k]
 * with the same argument conventions (device pointers, caller order, CSR
 * optional: corr_rowptr = NULL means no correction). It calls no cudaMalloc,
 * cudaFree or other allocating routine. Its intermediate charges and partial
 * sums live in one file-scope device array of VP_STATIC_SCRATCH_DOUBLES
 * doubles (16 MiB) that every GPU which loads libvp holds until the process
 * exits. Limits: n_src + n_tgt <= VP_STATIC_SCRATCH_DOUBLES, else VP_ERR_ARG
 * ("problem too large for the static scratch"; see vp_last_error).
 *
 * Argument checks: src_xy and tgt_xy must be 16-byte aligned (they are read
 * as pairs of doubles), else VP_ERR_ARG; a correction matrix with n_src == 0
 * is rejected with VP_ERR_ARG. The CSR itself is trusted, not validated:
 * rowptr must be non-decreasing with rowptr[0] = 0 and every column index in
 * [0, n_src). Validating it would need a pass with scratch of its own; a
 * malformed CSR makes the kernel read outside f (undefined results or a device
 * fault), so pass one built or validated by vp_plan_create's rules.
 *
 * Each call made outside a stream capture looks up the array's device address
 * (cudaGetSymbolAddress, with the device current); a call made while `stream`
 * is being captured reuses the address of the last uncaptured call on that
 * device, so make one call before any stream capture that should contain
 * later calls (else VP_ERR_STATE). All calls share
 * the one array and it keeps the last call's contents; every element a call
 * reads is written earlier in the same call, so nothing needs clearing. Calls
 * whose work overlaps on the GPU (different streams, or different host threads
 * on one device) race on the array: serialize them.
 */
#define VP_STATIC_SCRATCH_DOUBLES (1 << 21)
vp_status vp_eval_direct_static(int64_t n_src, const double* src_xy, const double* w,
                                int32_t ndens, const double* f, int64_t ld_f,
                                int64_t n_tgt, const double* tgt_xy,
                                const int64_t* corr_rowptr, const int32_t* corr_col,
                                const double* corr_val, double* out, int64_t ld_out,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* VP_H */
