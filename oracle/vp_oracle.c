/*
 * Plain CPU FP64 oracle for the volume-potential hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library path may link, load or
 * call this file: it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA path against a slow,
 * obviously correct evaluation of the same discrete sums. It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes (Anderson, Zhu, Veerapaneni, arXiv 2203.05933):
 *
 *   V_i^d = sum_{j : r_j != t_i} w_j f_j^d G(r_j, t_i)  +  sum_k Pi_ik f_k^d
 *
 *   - G(r, r0) = -(1/2pi) log|r - r0|, the Laplace Green's function (Sec. 2.1).
 *   - The first sum is the target-independent smooth quadrature rule applied
 *     to G f over every cell, with the Jacobian already folded into w_j, so
 *     that it is a plain point sum over all quadrature nodes (Eq. Tk_smooth_quad
 *     in Sec. 3.2 and the remark after it; Eq. vio_rokh_quad_rule).
 *   - The second sum is the sparse correction map Pi ("accurate minus smooth")
 *     assembled from the per-cell maps Pi_k(r0) into one sparse matrix whose
 *     rows are targets and columns are source nodes (Sec. 4, paragraph after
 *     Eq. nsrcs).
 *   - A pair whose source and target coordinates are bitwise equal contributes
 *     nothing: the smooth rule is undefined there and the paper folds that cell
 *     into the correction.
 *
 * Adjoint and target gradient, written from the same definition:
 *   (A^T g)_j^d = w_j sum_{i : t_i != r_j} G(r_j, t_i) g_i^d + sum_i Pi_ij g_i^d
 *   dL/dt_i     = sum_d g_i^d sum_{j : r_j != t_i} w_j f_j^d (-1/2pi)(t_i - r_j)/|t_i - r_j|^2
 *   (Pi held fixed: correction weights are set-up data, not differentiated.)
 *
 * Every sum is accumulated with Neumaier's compensated summation in FP64.
 * Points are interleaved (x, y) pairs; densities are row-major [ndens][ld].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double VPO_INV_2PI = 0.159154943091895335768883763372514362;

/* Neumaier (improved Kahan-Babuska) compensated sum. */
typedef struct {
    double s;
    double c;
} vpo_sum;

static inline void vpo_add(vpo_sum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static inline double vpo_val(const vpo_sum* a) { return a->s + a->c; }

/* G(r, r0) = -(1/2pi) log|r - r0|  (Sec. 2.1). */
static inline double vpo_green(double x, double y, double x0, double y0)
{
    return -VPO_INV_2PI * log(hypot(x - x0, y - y0));
}

static void vpo_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int vpo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * out[d][i] = sum_{j: r_j != t_i} w_j f[d][j] G(r_j, t_i)
 *           + (rowptr ? sum_{k in row i} val[k] f[d][col[k]] : 0)
 * One compensated accumulator per (i, d) covers both sums.
 */
int vpo_eval(int64_t n_src, const double* src_xy, const double* w,
             int32_t ndens, const double* f, int64_t ld_f,
             int64_t n_tgt, const double* tgt_xy,
             const int64_t* rowptr, const int32_t* col, const double* val,
             double* out, int64_t ld_out, int nthreads)
{
    if (n_src < 0 || n_tgt < 0 || ndens < 0) return 1;
    vpo_threads(nthreads);
    int bad = 0;
#pragma omp parallel
    {
        vpo_sum* acc = (vpo_sum*)malloc(sizeof(vpo_sum) * (size_t)(ndens > 0 ? ndens : 1));
        if (!acc) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < n_tgt; ++i) {
            if (!acc) continue;
            const double x0 = tgt_xy[2 * i], y0 = tgt_xy[2 * i + 1];
            for (int32_t d = 0; d < ndens; ++d) acc[d].s = acc[d].c = 0.0;
            for (int64_t j = 0; j < n_src; ++j) {
                const double x = src_xy[2 * j], y = src_xy[2 * j + 1];
                if (x == x0 && y == y0) continue; /* coincident pair: no smooth term */
                const double g = vpo_green(x, y, x0, y0);
                for (int32_t d = 0; d < ndens; ++d)
                    vpo_add(&acc[d], w[j] * f[d * ld_f + j] * g);
            }
            if (rowptr) {
                for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
                    for (int32_t d = 0; d < ndens; ++d)
                        vpo_add(&acc[d], val[k] * f[d * ld_f + col[k]]);
            }
            for (int32_t d = 0; d < ndens; ++d) out[d * ld_out + i] = vpo_val(&acc[d]);
        }
        free(acc);
    }
    return bad ? 2 : 0;
}

/*
 * Adjoint of vpo_eval with respect to f:
 * out[d][j] = w_j sum_{i: t_i != r_j} G(r_j, t_i) g[d][i] + sum_i Pi_ij g[d][i].
 * The transposed correction is gathered column by column through a CSC copy
 * built here by counting sort (a plain transpose of the CSR pattern).
 */
int vpo_adjoint(int64_t n_src, const double* src_xy, const double* w,
                int32_t ndens, const double* g, int64_t ld_g,
                int64_t n_tgt, const double* tgt_xy,
                const int64_t* rowptr, const int32_t* col, const double* val,
                double* out, int64_t ld_out, int nthreads)
{
    if (n_src < 0 || n_tgt < 0 || ndens < 0) return 1;
    vpo_threads(nthreads);
    int64_t* cptr = NULL;
    int64_t* crow = NULL;
    double* cval = NULL;
    if (rowptr) {
        const int64_t nnz = rowptr[n_tgt];
        cptr = (int64_t*)calloc((size_t)n_src + 1, sizeof(int64_t));
        crow = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
        cval = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_src + 1));
        if (!cptr || !crow || !cval || !fill) {
            free(cptr); free(crow); free(cval); free(fill);
            return 2;
        }
        for (int64_t k = 0; k < nnz; ++k) cptr[col[k] + 1]++;
        for (int64_t j = 0; j < n_src; ++j) cptr[j + 1] += cptr[j];
        memcpy(fill, cptr, sizeof(int64_t) * (size_t)(n_src + 1));
        for (int64_t i = 0; i < n_tgt; ++i)
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
                const int64_t p = fill[col[k]]++;
                crow[p] = i;
                cval[p] = val[k];
            }
        free(fill);
    }
    int bad = 0;
#pragma omp parallel
    {
        vpo_sum* acc = (vpo_sum*)malloc(sizeof(vpo_sum) * (size_t)(ndens > 0 ? ndens : 1));
        vpo_sum* cor = (vpo_sum*)malloc(sizeof(vpo_sum) * (size_t)(ndens > 0 ? ndens : 1));
        if (!acc || !cor) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 8)
        for (int64_t j = 0; j < n_src; ++j) {
            if (!acc || !cor) continue;
            const double x = src_xy[2 * j], y = src_xy[2 * j + 1];
            for (int32_t d = 0; d < ndens; ++d) acc[d].s = acc[d].c = cor[d].s = cor[d].c = 0.0;
            for (int64_t i = 0; i < n_tgt; ++i) {
                const double x0 = tgt_xy[2 * i], y0 = tgt_xy[2 * i + 1];
                if (x == x0 && y == y0) continue;
                const double gr = vpo_green(x, y, x0, y0);
                for (int32_t d = 0; d < ndens; ++d) vpo_add(&acc[d], gr * g[d * ld_g + i]);
            }
            if (cptr) {
                for (int64_t k = cptr[j]; k < cptr[j + 1]; ++k)
                    for (int32_t d = 0; d < ndens; ++d) vpo_add(&cor[d], cval[k] * g[d * ld_g + crow[k]]);
            }
            for (int32_t d = 0; d < ndens; ++d) {
                vpo_sum t = {0.0, 0.0};
                vpo_add(&t, w[j] * acc[d].s);
                vpo_add(&t, w[j] * acc[d].c);
                vpo_add(&t, cor[d].s);
                vpo_add(&t, cor[d].c);
                out[d * ld_out + j] = vpo_val(&t);
            }
        }
        free(acc);
        free(cor);
    }
    free(cptr); free(crow); free(cval);
    return bad ? 2 : 0;
}

/*
 * Target-position gradient of L with upstream gradient g = dL/dV, Pi fixed:
 * out[i][0..1] = sum_d g[d][i] sum_{j: r_j != t_i} w_j f[d][j] (-1/2pi)(t_i - r_j)/|t_i - r_j|^2.
 */
int vpo_grad_targets(int64_t n_src, const double* src_xy, const double* w,
                     int32_t ndens, const double* f, int64_t ld_f,
                     const double* g, int64_t ld_g,
                     int64_t n_tgt, const double* tgt_xy,
                     double* out, int nthreads)
{
    if (n_src < 0 || n_tgt < 0 || ndens < 0) return 1;
    vpo_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n_tgt; ++i) {
        const double x0 = tgt_xy[2 * i], y0 = tgt_xy[2 * i + 1];
        vpo_sum gx = {0.0, 0.0}, gy = {0.0, 0.0};
        for (int64_t j = 0; j < n_src; ++j) {
            const double x = src_xy[2 * j], y = src_xy[2 * j + 1];
            if (x == x0 && y == y0) continue;
            const double dx = x0 - x, dy = y0 - y;
            const double r2 = dx * dx + dy * dy;
            double q = 0.0;
            for (int32_t d = 0; d < ndens; ++d) q += g[d * ld_g + i] * f[d * ld_f + j];
            const double s = -VPO_INV_2PI * w[j] * q / r2;
            vpo_add(&gx, s * dx);
            vpo_add(&gy, s * dy);
        }
        out[2 * i] = vpo_val(&gx);
        out[2 * i + 1] = vpo_val(&gy);
    }
    return 0;
}

/*
 * Normaliser of the target gradient's error, the analogue of sum_j |w_j f_j| for
 * the potential: the sum of the absolute values of the terms of dL/dt_i,
 * out[i] = sum_d |g[d][i]| sum_{j: r_j != t_i} |w_j f[d][j]| / (2 pi |t_i - r_j|).
 * It bounds |dL/dt_i| (triangle inequality) and equals it when every term points
 * the same way.
 */
int vpo_grad_scale(int64_t n_src, const double* src_xy, const double* w,
                   int32_t ndens, const double* f, int64_t ld_f,
                   const double* g, int64_t ld_g,
                   int64_t n_tgt, const double* tgt_xy,
                   double* out, int nthreads)
{
    if (n_src < 0 || n_tgt < 0 || ndens < 0) return 1;
    vpo_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < n_tgt; ++i) {
        const double x0 = tgt_xy[2 * i], y0 = tgt_xy[2 * i + 1];
        vpo_sum acc = {0.0, 0.0};
        for (int64_t j = 0; j < n_src; ++j) {
            const double x = src_xy[2 * j], y = src_xy[2 * j + 1];
            if (x == x0 && y == y0) continue;
            const double dx = x0 - x, dy = y0 - y;
            double q = 0.0;
            for (int32_t d = 0; d < ndens; ++d) q += fabs(g[d * ld_g + i] * f[d * ld_f + j]);
            vpo_add(&acc, VPO_INV_2PI * fabs(w[j]) * q / sqrt(dx * dx + dy * dy));
        }
        out[i] = vpo_val(&acc);
    }
    return 0;
}
