// Singular (self) corrections of mapped triangles on the GPU (Sec. 3.3, and the
// efficient pre-computation of Sec. 3.4, Eq. singcorr_inner_prod): for the
// target at reference node a of a cell with map R and Jacobian J,
//
//   Vhat[K_b](zeta_a) = sum_i g_i B_a[b][i],   g_i = mapped Green function x J at chi_i,
//
// with the nodes chi_i, the kind of each node (tau) and B_a = K(chi) omega fixed
// for every cell; the correction of source node j is
//   corr[a][j] = sum_b Vhat[b] C[b][j] - w_j J(zeta_j) G(R(zeta_j), R(zeta_a))   (j != a),
// "accurate minus smooth" (Sec. 4). One block per (target node, cell); blocks
// of the same target node run together so that B_a stays in L2.
//
// Cell maps: affine, or the blending map of Eq. deformed_triangle_maps whose
// curved edge (from v0 to v1) is a circle arc or an arc of the polar curve
// r(theta) = 1 + a cos(k theta).
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "vp.h"
#include "vp_ff.cuh"

namespace vp {
void set_last_error(const std::string& msg);  // defined with the rest of the ABI (vp_api.cu)
std::vector<float> log_table();               // the table of the float-float log (vp_api.cu)
}

struct vp_tricorr_s {
    int device = 0;
    int32_t n_nodes = 0, n_basis = 0, n_rule = 0;
    double* node_ref = nullptr;  // [n_nodes][2]
    double* node_w = nullptr;    // [n_nodes]
    double* coef = nullptr;      // [n_basis][n_nodes]
    double* chi = nullptr;       // [n_nodes][n_rule][2]
    double* tau = nullptr;       // [n_nodes][n_rule]
    double* B = nullptr;         // [n_nodes][n_basis][n_rule] (device copy unused; the kernel reads Bf)
    float2* Bf = nullptr;        // B as hi/lo floats
    double* logt2 = nullptr;     // [n_nodes][n_rule] 2 log|tau| (tau > 0 nodes)
    float4* logtab = nullptr;    // [128] table of the float-float log
    std::vector<void*> allocs;
    bool alive = true;
    ~vp_tricorr_s()
    {
        for (void* p : allocs) cudaFree(p);
    }
};

namespace {

namespace ff = vp::ff;

constexpr int kTcThreads = 128;
constexpr int kTcMaxBasis = 36;
constexpr double kInv2PiT = 0.159154943091895335768883763372514362;

vp_status tfail(vp_status st, const std::string& m)
{
    vp::set_last_error(m);
    return st;
}

struct TriGeom {
    double v0x, v0y, v1x, v1y, v2x, v2y;
    int kind;
    double c0, c1, c2, c3, c4;
};

// Point and Jacobian of the cell map at (xi, eta)
__device__ __forceinline__ void tri_map(const TriGeom& g, double xi, double eta, double& x, double& y, double& J)
{
    const double l0 = 1.0 - xi - eta;
    x = l0 * g.v0x + xi * g.v1x + eta * g.v2x;
    y = l0 * g.v0y + xi * g.v1y + eta * g.v2y;
    double x_xi = g.v1x - g.v0x, y_xi = g.v1y - g.v0y, x_eta = g.v2x - g.v0x, y_eta = g.v2y - g.v0y;
    if (g.kind != 0) {
        double lam, mu, dlam, dmu;
        if (g.kind == 1) {  // circle arc (cx, cy, r, th0, th1)
            const double dth = g.c4 - g.c3;
            double sn, cs;
            sincos(g.c3 + xi * dth, &sn, &cs);
            lam = g.c0 + g.c2 * cs;
            mu = g.c1 + g.c2 * sn;
            dlam = -g.c2 * dth * sn;
            dmu = g.c2 * dth * cs;
        } else {  // polar arc r = 1 + a cos(k th) (a, k, th0, th1)
            const double dth = g.c3 - g.c2;
            const double th = g.c2 + xi * dth;
            double sn, cs, skt, ckt;
            sincos(th, &sn, &cs);
            sincos(g.c1 * th, &skt, &ckt);
            const double r = 1.0 + g.c0 * ckt, dr = -g.c0 * g.c1 * skt;
            lam = r * cs;
            mu = r * sn;
            dlam = dth * (dr * cs - r * sn);
            dmu = dth * (dr * sn + r * cs);
        }
        const double om = 1.0 - xi;
        const double gg = l0 / om;
        const double phx = lam - om * g.v0x - xi * g.v1x;
        const double phy = mu - om * g.v0y - xi * g.v1y;
        x += gg * phx;
        y += gg * phy;
        const double dg = -eta / (om * om);
        x_xi += dg * phx + gg * (dlam + g.v0x - g.v1x);
        y_xi += dg * phy + gg * (dmu + g.v0y - g.v1y);
        x_eta -= phx / om;
        y_eta -= phy / om;
    }
    J = fabs(x_xi * y_eta - x_eta * y_xi);
}

// One block per (target node a, cell). The mapped Green function at each rule
// node is assembled in float-float on the FP32 pipes from FP64 map values
// (log r^2 by the float-float table log, in units of the cell's bounding size,
// log tau^2 precomputed), and the contraction with B_a runs in float-float; the
// cell map itself (blending map, trigonometry) stays FP64.
__global__ void __launch_bounds__(kTcThreads)
    k_tricorr(int64_t n_cells, int32_t n_nodes, int32_t n_basis, int32_t n_rule, const double* __restrict__ geom,
              const double* __restrict__ node_ref, const double* __restrict__ node_w, const double* __restrict__ coef,
              const double* __restrict__ chi, const double* __restrict__ tau, const float2* __restrict__ Bf,
              const double* __restrict__ logt2, const float4* __restrict__ logtab, double* __restrict__ out)
{
    __shared__ double red[kTcThreads / 32][kTcMaxBasis];
    __shared__ double vhat[kTcMaxBasis];
    __shared__ float4 s_tab[128];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 128; i += kTcThreads) s_tab[i] = logtab[i];
    __syncthreads();
    for (int64_t blk = blockIdx.x; blk < n_cells * n_nodes; blk += gridDim.x) {
        const int a = (int)(blk / n_cells);  // target node major: blocks of one node share B_a
        const int64_t c = blk - (int64_t)a * n_cells;
        const double* gp = geom + c * 12;
        TriGeom g;
        g.v0x = gp[0];
        g.v0y = gp[1];
        g.v1x = gp[2];
        g.v1y = gp[3];
        g.v2x = gp[4];
        g.v2y = gp[5];
        g.kind = (int)gp[6];
        g.c0 = gp[7];
        g.c1 = gp[8];
        g.c2 = gp[9];
        g.c3 = gp[10];
        g.c4 = gp[11];
        double x0, y0, J0;
        tri_map(g, node_ref[2 * a], node_ref[2 * a + 1], x0, y0, J0);
        // length unit of the cell: its longest vertex-to-vertex distance squared
        const double h2 = fmax(fmax((g.v1x - g.v0x) * (g.v1x - g.v0x) + (g.v1y - g.v0y) * (g.v1y - g.v0y),
                                    (g.v2x - g.v0x) * (g.v2x - g.v0x) + (g.v2y - g.v0y) * (g.v2y - g.v0y)),
                               (g.v2x - g.v1x) * (g.v2x - g.v1x) + (g.v2y - g.v1y) * (g.v2y - g.v1y));
        const double inv_h2 = 1.0 / h2, log_h2 = log(h2);
        ff::F acc[kTcMaxBasis];
#pragma unroll
        for (int b = 0; b < kTcMaxBasis; ++b) acc[b] = ff::F{0.f, 0.f};
        const double* ch = chi + (int64_t)a * n_rule * 2;
        const double* ta = tau + (int64_t)a * n_rule;
        const double* lt = logt2 + (int64_t)a * n_rule;
        const float2* Ba = Bf + (int64_t)a * n_basis * n_rule;
        for (int i = tid; i < n_rule; i += kTcThreads) {
            double x, y, J;
            tri_map(g, ch[2 * i], ch[2 * i + 1], x, y, J);
            ff::F gi;
            if (ta[i] < 0.0) {
                gi = ff::from_double(kInv2PiT * J);  // the -log t part sits in the weights
            } else {
                // -(1/2pi) J log(r / t) = -(1/4pi) J (log(r^2/h^2) + log h^2 - log t^2)
                const double dx = x - x0, dy = y - y0;
                const double rs = (dx * dx + dy * dy) * inv_h2;
                const ff::F r2 = ff::from_double(rs);
                float S, lo;
                ff::log_pair(r2.h, r2.l, s_tab, S, lo);
                const ff::F L = ff::add(ff::F{S, lo}, ff::from_double(log_h2 - lt[i]));
                gi = ff::mul(L, ff::from_double(-0.5 * kInv2PiT * J));
            }
#pragma unroll
            for (int b = 0; b < kTcMaxBasis; ++b)
                if (b < n_basis) {
                    const float2 bv = Ba[(int64_t)b * n_rule + i];
                    acc[b] = ff::add(acc[b], ff::mul(ff::F{bv.x, bv.y}, gi));
                }
        }
#pragma unroll
        for (int b = 0; b < kTcMaxBasis; ++b) {
            ff::F v = acc[b];
            for (int o = 16; o > 0; o >>= 1) {
                const float h = __shfl_xor_sync(0xffffffffu, v.h, o), l = __shfl_xor_sync(0xffffffffu, v.l, o);
                v = ff::add(v, ff::F{h, l});
            }
            if (lane == 0) red[warp][b] = ff::to_double(v);
        }
        __syncthreads();
        if (tid < n_basis) {
            double v = 0.0;
            for (int w = 0; w < kTcThreads / 32; ++w) v += red[w][tid];
            vhat[tid] = v;
        }
        __syncthreads();
        for (int j = tid; j < n_nodes; j += kTcThreads) {
            double s = 0.0;
            for (int b = 0; b < n_basis; ++b) s = fma(vhat[b], coef[(int64_t)b * n_nodes + j], s);
            if (j != a) {
                double xj, yj, Jj;
                tri_map(g, node_ref[2 * j], node_ref[2 * j + 1], xj, yj, Jj);
                s -= node_w[j] * Jj * (-kInv2PiT) * log(hypot(xj - x0, yj - y0));
            }
            out[(c * n_nodes + a) * n_nodes + j] = s;
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" {

vp_status vp_tricorr_create(vp_tricorr* out, int32_t n_nodes, int32_t n_basis, int32_t n_rule, const double* node_ref,
                            const double* node_w, const double* coef, const double* chi, const double* tau,
                            const double* B, void* stream)
{
    vp::set_last_error("");
    if (!out) return tfail(VP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_nodes < 1 || n_basis < 1 || n_basis > kTcMaxBasis || n_rule < 1 || !node_ref || !node_w || !coef || !chi ||
        !tau || !B)
        return tfail(VP_ERR_ARG, "vp_tricorr_create: sizes out of range (n_basis <= 36) or NULL table");
    const size_t sizes[6] = {2 * (size_t)n_nodes, (size_t)n_nodes, (size_t)n_basis * n_nodes,
                             (size_t)n_nodes * n_rule * 2, (size_t)n_nodes * n_rule,
                             (size_t)n_nodes * n_basis * n_rule};
    const double* src[6] = {node_ref, node_w, coef, chi, tau, B};
    for (int k = 0; k < 6; ++k)
        for (size_t i = 0; i < sizes[k]; ++i)
            if (!std::isfinite(src[k][i])) return tfail(VP_ERR_ARG, "vp_tricorr_create: non-finite table entry");
    for (size_t i = 0; i < sizes[4]; ++i)
        if (tau[i] == 0.0 || std::fabs(tau[i]) > 1.0) return tfail(VP_ERR_ARG, "vp_tricorr_create: |tau| not in (0, 1]");
    vp_tricorr tc = new (std::nothrow) vp_tricorr_s;
    if (!tc) return tfail(VP_ERR_OOM, "host allocation");
    cudaGetDevice(&tc->device);
    tc->n_nodes = n_nodes;
    tc->n_basis = n_basis;
    tc->n_rule = n_rule;
    double** dst[6] = {&tc->node_ref, &tc->node_w, &tc->coef, &tc->chi, &tc->tau, &tc->B};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
        void* q = nullptr;
        e = cudaMalloc(&q, sizes[k] * sizeof(double));
        if (e != cudaSuccess) break;
        tc->allocs.push_back(q);
        *dst[k] = (double*)q;
        e = cudaMemcpyAsync(q, src[k], sizes[k] * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    // B as hi/lo floats, 2 log|tau| per rule node, and the table of the float-float log
    std::vector<float> hbf(2 * sizes[5]);
    for (size_t i = 0; i < sizes[5]; ++i) {
        const float h = (float)B[i];
        hbf[2 * i] = h;
        hbf[2 * i + 1] = (float)(B[i] - (double)h);
    }
    std::vector<double> hlt(sizes[4]);
    for (size_t i = 0; i < sizes[4]; ++i) hlt[i] = tau[i] > 0.0 ? 2.0 * std::log(tau[i]) : 0.0;
    const std::vector<float> hlog = vp::log_table();
    auto up = [&](void** dstp, const void* srcp, size_t bytes) {
        if (e != cudaSuccess) return;
        void* q = nullptr;
        e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return;
        tc->allocs.push_back(q);
        *dstp = q;
        e = cudaMemcpyAsync(q, srcp, bytes, cudaMemcpyHostToDevice, s);
    };
    up((void**)&tc->Bf, hbf.data(), hbf.size() * sizeof(float));
    up((void**)&tc->logt2, hlt.data(), hlt.size() * sizeof(double));
    up((void**)&tc->logtab, hlog.data(), hlog.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete tc;
        return tfail(e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA,
                     std::string("vp_tricorr_create: ") + cudaGetErrorString(e));
    }
    *out = tc;
    return VP_OK;
}

vp_status vp_tricorr_eval(vp_tricorr tc, int64_t n_cells, const double* geom, double* out, void* stream)
{
    if (!tc || !tc->alive) return tfail(VP_ERR_STATE, "invalid triangle-correction plan");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != tc->device)
        return tfail(VP_ERR_STATE, "triangle-correction plan used on another device");
    if (n_cells < 0) return tfail(VP_ERR_ARG, "n_cells < 0");
    if (n_cells == 0) return VP_OK;
    if (!geom || !out) return tfail(VP_ERR_ARG, "NULL geometry or output");
    if (n_cells > (1LL << 40) / tc->n_nodes) return tfail(VP_ERR_ARG, "too many cells");
    const int64_t work = n_cells * tc->n_nodes;
    const int blocks = (int)(work < 152 * 16 ? work : 152 * 16);
    k_tricorr<<<blocks, kTcThreads, 0, (cudaStream_t)stream>>>(n_cells, tc->n_nodes, tc->n_basis, tc->n_rule, geom,
                                                                tc->node_ref, tc->node_w, tc->coef, tc->chi, tc->tau,
                                                                tc->Bf, tc->logt2, tc->logtab, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tfail(VP_ERR_CUDA, std::string("vp_tricorr_eval: ") + cudaGetErrorString(e));
    return VP_OK;
}

vp_status vp_tricorr_destroy(vp_tricorr tc)
{
    if (!tc || !tc->alive) return tfail(VP_ERR_STATE, "invalid triangle-correction plan");
    tc->alive = false;
    delete tc;
    return VP_OK;
}

}  // extern "C"
