// Interpolation of nodal values to arbitrary points inside cells (Sec. 3.2.1:
// values-to-coefficients map of Eq. vals_to_coeffs and the orthogonal
// expansion on the simplex; Sec. 4.2: tensor expansions on boxes).
//
// Two passes per density chunk:
//   k_interp_coef: one block per cell, a = C v_cell (C of the cell's type), in FP64;
//   k_interp_eval: one thread per point (points sorted by cell at create time),
//                  sum_b a_b phi_b(xi, eta) with the basis generated by its
//                  three-term recurrences (Legendre; scaled Legendre
//                  Q_m = P_m(s/t) t^m; Jacobi P_k^(2m+1,0)), written back in
//                  caller order. The recurrence coefficients come from a
//                  table built once on the host, so the kernel only multiplies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "vp.h"

namespace vp {
void set_last_error(const std::string& msg);  // defined with the rest of the ABI (vp_api.cu)
}

struct vp_interp_s {
    int device = 0;
    int64_t n_pts = 0, n_vals = 0, n_cells = 0;
    int32_t max_nodes = 1;
    int32_t* tinfo = nullptr;      // [n_types][4]: basis, order, n_nodes, 0
    int64_t* toff = nullptr;       // [n_types] offset of C in cmat
    double* cmat = nullptr;
    int32_t* cell_type = nullptr;
    int64_t* node_start = nullptr;
    int32_t* pcell = nullptr;      // sorted by cell
    double2* pref = nullptr;       // reference coordinates, sorted
    int32_t* pperm = nullptr;      // sorted position -> caller index
    double* coef = nullptr;        // [8][n_vals]
    double* rec = nullptr;         // recurrence coefficients (kRecLeg + kRecJac doubles)
    std::vector<void*> allocs;
    bool alive = true;

    template <typename T>
    cudaError_t alloc(T** p, size_t n)
    {
        *p = nullptr;
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, (n ? n : 1) * sizeof(T));
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        *p = (T*)q;
        return cudaSuccess;
    }
    ~vp_interp_s()
    {
        for (void* p : allocs) cudaFree(p);
    }
};

namespace {

constexpr int kInterpThreads = 128;
constexpr int kMaxChunk = 8;
constexpr int kMaxOrder = 32;
// rec[2 n], rec[2 n + 1]: Legendre P_n = rec[2n] x P_{n-1} - rec[2n+1] P_{n-2} (n >= 2)
// rec[kRecLeg + 3 (m kMaxOrder + n) + {0,1,2}]: Jacobi P_n^(2m+1,0)(b) = (c0 + c1 b) P_{n-1} - c2 P_{n-2}
constexpr int kRecLeg = 2 * kMaxOrder;
constexpr int kRecJac = 3 * kMaxOrder * kMaxOrder;

std::vector<double> recurrence_table()
{
    std::vector<double> r((size_t)(kRecLeg + kRecJac), 0.0);
    for (int n = 2; n < kMaxOrder; ++n) {
        r[2 * (size_t)n] = (2.0 * n - 1.0) / n;
        r[2 * (size_t)n + 1] = (n - 1.0) / n;
    }
    for (int m = 0; m < kMaxOrder; ++m) {
        const double al = 2.0 * m + 1.0;
        for (int n = 2; n < kMaxOrder; ++n) {
            const double a1 = 2.0 * n * (n + al) * (2.0 * n + al - 2.0);
            const double a2 = (2.0 * n + al - 1.0) * al * al;
            const double a3 = (2.0 * n + al - 2.0) * (2.0 * n + al - 1.0) * (2.0 * n + al);
            const double a4 = 2.0 * (n + al - 1.0) * (n - 1.0) * (2.0 * n + al);
            double* c = r.data() + kRecLeg + 3 * ((size_t)m * kMaxOrder + n);
            c[0] = a2 / a1;
            c[1] = a3 / a1;
            c[2] = a4 / a1;
        }
    }
    return r;
}

vp_status ifail(vp_status st, const std::string& m)
{
    vp::set_last_error(m);
    return st;
}

template <int ND>
__global__ void __launch_bounds__(kInterpThreads)
    k_interp_coef(int64_t n_cells, const int32_t* __restrict__ cell_type, const int64_t* __restrict__ node_start,
                  const int32_t* __restrict__ tinfo, const int64_t* __restrict__ toff, const double* __restrict__ cmat,
                  int32_t max_nodes, const double* __restrict__ v, int64_t ld_v, double* __restrict__ coef,
                  int64_t ld_c)
{
    extern __shared__ double vs[];  // [ND][max_nodes]
    for (int64_t c = blockIdx.x; c < n_cells; c += gridDim.x) {
        const int t = cell_type[c];
        const int n = tinfo[4 * t + 2];
        const double* C = cmat + toff[t];
        const int64_t s0 = node_start[c];
        __syncthreads();
        for (int i = threadIdx.x; i < n * ND; i += blockDim.x) {
            const int d = i / n, k = i - d * n;
            vs[d * max_nodes + k] = v[d * ld_v + s0 + k];
        }
        __syncthreads();
        for (int b = threadIdx.x; b < n; b += blockDim.x) {
            double acc[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[d] = 0.0;
            for (int i = 0; i < n; ++i) {
                const double cv = C[(int64_t)b * n + i];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = fma(cv, vs[d * max_nodes + i], acc[d]);
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) coef[d * ld_c + s0 + b] = acc[d];
        }
    }
}

template <int ND>
__global__ void __launch_bounds__(kInterpThreads)
    k_interp_eval(int64_t n_pts, const int32_t* __restrict__ pcell, const double2* __restrict__ pref,
                  const int32_t* __restrict__ pperm, const int32_t* __restrict__ cell_type,
                  const int64_t* __restrict__ node_start, const int32_t* __restrict__ tinfo,
                  const double* __restrict__ rec, const double* __restrict__ coef, int64_t ld_c,
                  double* __restrict__ out, int64_t ld_out)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_pts;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = pcell[k];
        const int t = cell_type[c];
        const int basis = tinfo[4 * t], order = tinfo[4 * t + 1];
        const double* a = coef + node_start[c];
        const double2 r = pref[k];
        double acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = 0.0;
        if (basis == VP_BASIS_LEGENDRE2) {
            // sum_j P_j(eta) sum_i a[j order + i] P_i(xi), the P_i(xi) generated once
            double px[kMaxOrder];
            px[0] = 1.0;
            if (order > 1) px[1] = r.x;
            for (int i = 2; i < order; ++i) px[i] = fma(rec[2 * i] * r.x, px[i - 1], -rec[2 * i + 1] * px[i - 2]);
            double py = 1.0, pym = 0.0;
            for (int j = 0; j < order; ++j) {
                if (j == 1) {
                    pym = 1.0;
                    py = r.y;
                } else if (j > 1) {
                    const double nx = fma(rec[2 * j] * r.y, py, -rec[2 * j + 1] * pym);
                    pym = py;
                    py = nx;
                }
                double inner[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) inner[d] = 0.0;
                for (int i = 0; i < order; ++i) {
#pragma unroll
                    for (int d = 0; d < ND; ++d) inner[d] = fma(a[d * ld_c + j * order + i], px[i], inner[d]);
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = fma(inner[d], py, acc[d]);
            }
        } else {
            const double s = 2.0 * r.x - 1.0 + r.y, tt = 1.0 - r.y, b = 2.0 * r.y - 1.0, t2 = tt * tt;
            double q = 1.0, qm = 0.0;
            int idx = 0;
            for (int m = 0; m < order; ++m) {
                if (m == 1) {
                    qm = 1.0;
                    q = s;
                } else if (m > 1) {
                    const double nq = fma(rec[2 * m] * s, q, -rec[2 * m + 1] * t2 * qm);
                    qm = q;
                    q = nq;
                }
                const double al = 2.0 * m + 1.0;  // Jacobi alpha of this m
                const double* jc = rec + kRecLeg + 3 * m * kMaxOrder;
                double pj = 1.0, pjm = 0.0;
                for (int kk = 0; kk < order - m; ++kk) {
                    if (kk == 1) {
                        pjm = 1.0;
                        pj = (al + 1.0) + (al + 2.0) * (b - 1.0) * 0.5;
                    } else if (kk > 1) {
                        const double* c = jc + 3 * kk;
                        const double nj = fma(fma(c[1], b, c[0]), pj, -c[2] * pjm);
                        pjm = pj;
                        pj = nj;
                    }
                    const double phi = q * pj;
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = fma(a[d * ld_c + idx], phi, acc[d]);
                    ++idx;
                }
            }
        }
        const int32_t o = pperm[k];
#pragma unroll
        for (int d = 0; d < ND; ++d) out[d * ld_out + o] = acc[d];
    }
}

template <int ND>
cudaError_t interp_chunk(vp_interp ip, const double* v, int64_t ld_v, double* out, int64_t ld_out, cudaStream_t s)
{
    const size_t bytes = sizeof(double) * ND * (size_t)ip->max_nodes;
    cudaError_t e = cudaFuncSetAttribute(k_interp_coef<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (ip->n_cells > 0) {
        const int blocks = (int)std::min<int64_t>(ip->n_cells, 152 * 16);
        k_interp_coef<ND><<<blocks, kInterpThreads, bytes, s>>>(ip->n_cells, ip->cell_type, ip->node_start,
                                                               ip->tinfo, ip->toff, ip->cmat, ip->max_nodes, v, ld_v,
                                                               ip->coef, ip->n_vals);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (ip->n_pts > 0) {
        const int blocks = (int)std::min<int64_t>((ip->n_pts + kInterpThreads - 1) / kInterpThreads, 152 * 32);
        k_interp_eval<ND><<<blocks, kInterpThreads, 0, s>>>(ip->n_pts, ip->pcell, ip->pref, ip->pperm,
                                                           ip->cell_type, ip->node_start, ip->tinfo, ip->rec,
                                                           ip->coef, ip->n_vals, out, ld_out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

extern "C" {

vp_status vp_interp_create(vp_interp* out, int32_t n_types, const vp_interp_type* types, int64_t n_cells,
                           const int32_t* cell_type, const int64_t* node_start, int64_t n_pts,
                           const int32_t* pt_cell, const double* pt_ref, void* stream)
{
    vp::set_last_error("");
    if (!out) return ifail(VP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_types < 1 || !types || n_cells < 0 || n_pts < 0 || !node_start || (n_cells > 0 && !cell_type) ||
        (n_pts > 0 && (!pt_cell || !pt_ref)))
        return ifail(VP_ERR_ARG, "incomplete interpolation description");
    if (n_cells > (1LL << 30) || n_pts > (1LL << 30)) return ifail(VP_ERR_ARG, "more than 2^30 cells or points");
    std::vector<int32_t> tinfo((size_t)n_types * 4, 0);
    std::vector<int64_t> toff((size_t)n_types, 0);
    std::vector<double> cmat;
    int32_t max_nodes = 1;
    for (int32_t t = 0; t < n_types; ++t) {
        const vp_interp_type& ty = types[t];
        const int o = ty.order;
        if (o < 1 || o > kMaxOrder || !ty.coef) return ifail(VP_ERR_ARG, "interpolation type: order outside 1..32 or NULL C");
        const int n = ty.basis == VP_BASIS_LEGENDRE2 ? o * o : ty.basis == VP_BASIS_SIMPLEX ? o * (o + 1) / 2 : -1;
        if (n < 0) return ifail(VP_ERR_ARG, "interpolation type: unknown basis");
        if (ty.n_nodes != n) return ifail(VP_ERR_ARG, "interpolation type: n_nodes does not match the basis");
        tinfo[4 * (size_t)t] = ty.basis;
        tinfo[4 * (size_t)t + 1] = o;
        tinfo[4 * (size_t)t + 2] = n;
        toff[(size_t)t] = (int64_t)cmat.size();
        cmat.insert(cmat.end(), ty.coef, ty.coef + (size_t)n * n);
        max_nodes = std::max(max_nodes, n);
    }
    for (double x : cmat)
        if (!std::isfinite(x)) return ifail(VP_ERR_ARG, "non-finite coefficient map");
    if (node_start[0] != 0) return ifail(VP_ERR_ARG, "node ranges must start at 0");
    for (int64_t c = 0; c < n_cells; ++c) {
        const int32_t t = cell_type[c];
        if (t < 0 || t >= n_types) return ifail(VP_ERR_ARG, "cell type out of range");
        if (node_start[c + 1] - node_start[c] != tinfo[4 * (size_t)t + 2])
            return ifail(VP_ERR_ARG, "cell " + std::to_string(c) + ": node count differs from its type");
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> hcell((size_t)n_pts);
    std::vector<double> href((size_t)n_pts * 2);
    cudaError_t e = cudaSuccess;
    if (n_pts) {
        e = cudaMemcpyAsync(hcell.data(), pt_cell, hcell.size() * sizeof(int32_t), cudaMemcpyDefault, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(href.data(), pt_ref, href.size() * sizeof(double), cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ifail(VP_ERR_CUDA, std::string("vp_interp_create copy: ") + cudaGetErrorString(e));
    }
    for (int64_t k = 0; k < n_pts; ++k) {
        if (hcell[(size_t)k] < 0 || hcell[(size_t)k] >= n_cells) return ifail(VP_ERR_ARG, "point cell out of range");
        if (!std::isfinite(href[2 * (size_t)k]) || !std::isfinite(href[2 * (size_t)k + 1]))
            return ifail(VP_ERR_ARG, "non-finite reference coordinate");
    }
    // points sorted by cell, so neighbouring threads share a cell's coefficients
    std::vector<int32_t> perm((size_t)n_pts);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return hcell[(size_t)a] < hcell[(size_t)b]; });
    std::vector<int32_t> scell((size_t)n_pts);
    std::vector<double> sref((size_t)n_pts * 2);
    for (int64_t k = 0; k < n_pts; ++k) {
        const int32_t o = perm[(size_t)k];
        scell[(size_t)k] = hcell[(size_t)o];
        sref[2 * (size_t)k] = href[2 * (size_t)o];
        sref[2 * (size_t)k + 1] = href[2 * (size_t)o + 1];
    }
    vp_interp ip = new (std::nothrow) vp_interp_s;
    if (!ip) return ifail(VP_ERR_OOM, "host allocation");
    cudaGetDevice(&ip->device);
    ip->n_pts = n_pts;
    ip->n_cells = n_cells;
    ip->n_vals = node_start[n_cells];
    ip->max_nodes = max_nodes;
    std::vector<int32_t> hct(cell_type, cell_type + n_cells);
    std::vector<int64_t> hns(node_start, node_start + n_cells + 1);
    auto up = [&](auto** dst, const auto& h) {
        if (e != cudaSuccess) return;
        e = ip->alloc(dst, h.size());
        if (e == cudaSuccess && !h.empty())
            e = cudaMemcpyAsync(*dst, h.data(), h.size() * sizeof(h[0]), cudaMemcpyHostToDevice, s);
    };
    up(&ip->tinfo, tinfo);
    up(&ip->toff, toff);
    up(&ip->cmat, cmat);
    up(&ip->cell_type, hct);
    up(&ip->node_start, hns);
    up(&ip->pcell, scell);
    double* dref = nullptr;
    up(&dref, sref);
    ip->pref = (double2*)dref;
    up(&ip->pperm, perm);
    up(&ip->rec, recurrence_table());
    if (e == cudaSuccess) e = ip->alloc(&ip->coef, (size_t)kMaxChunk * std::max<int64_t>(ip->n_vals, 1));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete ip;
        return ifail(e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA,
                     std::string("vp_interp_create upload: ") + cudaGetErrorString(e));
    }
    *out = ip;
    return VP_OK;
}

vp_status vp_interp_eval(vp_interp ip, int32_t ndens, const double* v, int64_t ld_v, double* out, int64_t ld_out,
                         void* stream)
{
    if (!ip || !ip->alive) return ifail(VP_ERR_STATE, "invalid interpolation plan");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != ip->device)
        return ifail(VP_ERR_STATE, "interpolation plan used on another device");
    if (ndens < 0) return ifail(VP_ERR_ARG, "ndens < 0");
    if (ndens == 0 || ip->n_pts == 0) return VP_OK;
    if (!out || (ip->n_vals > 0 && !v)) return ifail(VP_ERR_ARG, "NULL values or output");
    if (ld_v < ip->n_vals || ld_out < ip->n_pts) return ifail(VP_ERR_ARG, "leading dimension too small");
    cudaStream_t s = (cudaStream_t)stream;
    for (int d0 = 0; d0 < ndens;) {
        int nd = 1;
        while (nd * 2 <= ndens - d0 && nd * 2 <= kMaxChunk) nd *= 2;
        const double* vc = v + (int64_t)d0 * ld_v;
        double* oc = out + (int64_t)d0 * ld_out;
        cudaError_t e = nd == 1 ? interp_chunk<1>(ip, vc, ld_v, oc, ld_out, s)
                        : nd == 2 ? interp_chunk<2>(ip, vc, ld_v, oc, ld_out, s)
                        : nd == 4 ? interp_chunk<4>(ip, vc, ld_v, oc, ld_out, s)
                                  : interp_chunk<8>(ip, vc, ld_v, oc, ld_out, s);
        if (e != cudaSuccess) return ifail(VP_ERR_CUDA, std::string("vp_interp_eval: ") + cudaGetErrorString(e));
        d0 += nd;
    }
    return VP_OK;
}

vp_status vp_interp_destroy(vp_interp ip)
{
    if (!ip || !ip->alive) return ifail(VP_ERR_STATE, "invalid interpolation plan");
    ip->alive = false;
    delete ip;
    return VP_OK;
}

}  // extern "C"
