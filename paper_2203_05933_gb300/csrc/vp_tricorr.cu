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
    float2* Bf = nullptr;        // B node-major [n_nodes][n_rule][n_basis] as hi/lo floats
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
    // curved edge: sin and cos of the start angle (and of k times it for the polar
    // arc), for the angle-addition form of the edge parametrisation
    bool small;  // every angle increment along the edge below 0.3 in magnitude
    double s0, cs0, sk0, ck0;
};

// sin and cos of a small angle d (|d| <= 0.3) by their Taylor series to d^13 and
// d^14 (relative error below 1e-16)
__device__ __forceinline__ void sincos_small(double d, double& sn, double& cs)
{
    // nested Horner form with the reciprocals as constants (no divisions)
    constexpr double r6 = 1.0 / 6.0, r20 = 1.0 / 20.0, r42 = 1.0 / 42.0, r72 = 1.0 / 72.0, r110 = 1.0 / 110.0,
                     r156 = 1.0 / 156.0;
    constexpr double r2 = 0.5, r12 = 1.0 / 12.0, r30 = 1.0 / 30.0, r56 = 1.0 / 56.0, r90 = 1.0 / 90.0,
                     r132 = 1.0 / 132.0, r182 = 1.0 / 182.0;
    const double d2 = d * d;
    double t = fma(-d2 * r156, 1.0, 1.0);
    t = fma(-d2 * r110, t, 1.0);
    t = fma(-d2 * r72, t, 1.0);
    t = fma(-d2 * r42, t, 1.0);
    t = fma(-d2 * r20, t, 1.0);
    t = fma(-d2 * r6, t, 1.0);
    sn = d * t;
    double u = fma(-d2 * r182, 1.0, 1.0);
    u = fma(-d2 * r132, u, 1.0);
    u = fma(-d2 * r90, u, 1.0);
    u = fma(-d2 * r56, u, 1.0);
    u = fma(-d2 * r30, u, 1.0);
    u = fma(-d2 * r12, u, 1.0);
    cs = fma(-d2 * r2, u, 1.0);
}

// the per-cell part of the curved-edge parametrisation
__device__ __forceinline__ void tri_prepare(TriGeom& g)
{
    g.small = false;
    g.s0 = g.cs0 = g.sk0 = g.ck0 = 0.0;
    if (g.kind == 1) {
        g.small = fabs(g.c4 - g.c3) <= 0.3;
        sincos(g.c3, &g.s0, &g.cs0);
    } else if (g.kind == 2) {
        const double dth = g.c3 - g.c2;
        g.small = fabs(dth) <= 0.3 && fabs(g.c1 * dth) <= 0.3;
        sincos(g.c2, &g.s0, &g.cs0);
        sincos(g.c1 * g.c2, &g.sk0, &g.ck0);
    }
}

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
            if (g.small) {  // sin and cos of th0 + xi dth by angle addition
                double sd, cd;
                sincos_small(xi * dth, sd, cd);
                sn = fma(g.s0, cd, g.cs0 * sd);
                cs = fma(g.cs0, cd, -g.s0 * sd);
            } else {
                sincos(g.c3 + xi * dth, &sn, &cs);
            }
            lam = g.c0 + g.c2 * cs;
            mu = g.c1 + g.c2 * sn;
            dlam = -g.c2 * dth * sn;
            dmu = g.c2 * dth * cs;
        } else {  // polar arc r = 1 + a cos(k th) (a, k, th0, th1)
            const double dth = g.c3 - g.c2;
            const double th = g.c2 + xi * dth;
            double sn, cs, skt, ckt;
            if (g.small) {
                double sd, cd, skd, ckd;
                sincos_small(xi * dth, sd, cd);
                sincos_small(g.c1 * xi * dth, skd, ckd);
                sn = fma(g.s0, cd, g.cs0 * sd);
                cs = fma(g.cs0, cd, -g.s0 * sd);
                skt = fma(g.sk0, ckd, g.ck0 * skd);
                ckt = fma(g.ck0, ckd, -g.sk0 * skd);
            } else {
                sincos(th, &sn, &cs);
                sincos(g.c1 * th, &skt, &ckt);
            }
            const double r = 1.0 + g.c0 * ckt, dr = -g.c0 * g.c1 * skt;
            lam = r * cs;
            mu = r * sn;
            dlam = dth * (dr * cs - r * sn);
            dmu = dth * (dr * sn + r * cs);
        }
        const double om = 1.0 - xi;
        const double iom = 1.0 / om;  // one division per node
        const double gg = l0 * iom;
        const double phx = lam - om * g.v0x - xi * g.v1x;
        const double phy = mu - om * g.v0y - xi * g.v1y;
        x += gg * phx;
        y += gg * phy;
        const double dg = -eta * iom * iom;
        x_xi += dg * phx + gg * (dlam + g.v0x - g.v1x);
        y_xi += dg * phy + gg * (dmu + g.v0y - g.v1y);
        x_eta -= phx * iom;
        y_eta -= phy * iom;
    }
    J = fabs(x_xi * y_eta - x_eta * y_xi);
}

// One block per (target node a, cell). Each warp takes 32 rule nodes at a time:
// lane l assembles the mapped Green function at node l of the chunk (FP64 cell
// map; log r^2 by the float-float table log in units of the cell's bounding
// size, log tau^2 precomputed; the rest in float-float) and parks it in shared
// memory; then lane b accumulates basis function b (and b + 32) over the chunk
// from B_a stored node-major (coalesced). Few registers per thread, so that
// enough warps hide the latency of the FP64 map.
__global__ void __launch_bounds__(kTcThreads)
    k_tricorr(int64_t n_cells, int32_t n_nodes, int32_t n_basis, int32_t n_rule, const double* __restrict__ geom,
              const double* __restrict__ node_ref, const double* __restrict__ node_w, const double* __restrict__ coef,
              const double* __restrict__ chi, const double* __restrict__ tau, const float2* __restrict__ Bt,
              const double* __restrict__ logt2, const float4* __restrict__ logtab, double* __restrict__ out)
{
    __shared__ double red[kTcThreads / 32][kTcMaxBasis];
    __shared__ double vhat[kTcMaxBasis];
    __shared__ float4 s_tab[128];
    __shared__ float2 gs[kTcThreads / 32][32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nwarp = kTcThreads / 32;
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
        tri_prepare(g);
        double x0, y0, J0;
        tri_map(g, node_ref[2 * a], node_ref[2 * a + 1], x0, y0, J0);
        // length unit of the cell: its longest vertex-to-vertex distance squared
        const double h2 = fmax(fmax((g.v1x - g.v0x) * (g.v1x - g.v0x) + (g.v1y - g.v0y) * (g.v1y - g.v0y),
                                    (g.v2x - g.v0x) * (g.v2x - g.v0x) + (g.v2y - g.v0y) * (g.v2y - g.v0y)),
                               (g.v2x - g.v1x) * (g.v2x - g.v1x) + (g.v2y - g.v1y) * (g.v2y - g.v1y));
        const double inv_h2 = 1.0 / h2, log_h2 = log(h2);
        ff::F acc0{0.f, 0.f}, acc1{0.f, 0.f};  // basis functions lane and lane + 32
        const double* ch = chi + (int64_t)a * n_rule * 2;
        const double* ta = tau + (int64_t)a * n_rule;
        const double* lt = logt2 + (int64_t)a * n_rule;
        const float2* Ba = Bt + (int64_t)a * n_rule * n_basis;
        for (int base = warp * 32; base < n_rule; base += nwarp * 32) {
            const int i = base + lane;
            ff::F gi{0.f, 0.f};
            if (i < n_rule) {
                double x, y, J;
                tri_map(g, ch[2 * i], ch[2 * i + 1], x, y, J);
                if (ta[i] < 0.0) {
                    gi = ff::from_double(kInv2PiT * J);  // the -log t part sits in the weights
                } else {
                    // -(1/2pi) J log(r / t) = -(1/4pi) J (log(r^2/h^2) + log h^2 - log t^2)
                    const double dx = x - x0, dy = y - y0;
                    const ff::F r2 = ff::from_double((dx * dx + dy * dy) * inv_h2);
                    float S, lo;
                    ff::log_pair(r2.h, r2.l, s_tab, S, lo);
                    const ff::F L = ff::add(ff::F{S, lo}, ff::from_double(log_h2 - lt[i]));
                    gi = ff::mul(L, ff::from_double(-0.5 * kInv2PiT * J));
                }
            }
            gs[warp][lane] = make_float2(gi.h, gi.l);
            __syncwarp();
            const int n = min(32, n_rule - base);
            const float2* Bc = Ba + (int64_t)base * n_basis;
            // the chunk's sum first, then into the running total: the terms cancel
            // strongly, and short sequential sums keep the float-float rounding small
            ff::F c0{0.f, 0.f}, c1{0.f, 0.f};
            for (int j = 0; j < n; ++j) {
                const ff::F gj{gs[warp][j].x, gs[warp][j].y};
                if (lane < n_basis) {
                    const float2 bv = Bc[(int64_t)j * n_basis + lane];
                    c0 = ff::add(c0, ff::mul(ff::F{bv.x, bv.y}, gj));
                }
                if (lane + 32 < n_basis) {
                    const float2 bv = Bc[(int64_t)j * n_basis + lane + 32];
                    c1 = ff::add(c1, ff::mul(ff::F{bv.x, bv.y}, gj));
                }
            }
            acc0 = ff::add(acc0, c0);
            acc1 = ff::add(acc1, c1);
            __syncwarp();
        }
        if (lane < n_basis) red[warp][lane] = ff::to_double(acc0);
        if (lane + 32 < n_basis) red[warp][lane + 32] = ff::to_double(acc1);
        __syncthreads();
        if (tid < n_basis) {
            double v = 0.0;
            for (int w = 0; w < nwarp; ++w) v += red[w][tid];
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
    // B node-major ([n_nodes][n_rule][n_basis]) as hi/lo floats, 2 log|tau| per rule
    // node, and the table of the float-float log
    std::vector<float> hbf(2 * sizes[5]);
    for (size_t a = 0; a < (size_t)n_nodes; ++a)
        for (size_t bb = 0; bb < (size_t)n_basis; ++bb)
            for (size_t i = 0; i < (size_t)n_rule; ++i) {
                const double v = B[(a * n_basis + bb) * n_rule + i];
                const size_t o = (a * n_rule + i) * n_basis + bb;
                const float h = (float)v;
                hbf[2 * o] = h;
                hbf[2 * o + 1] = (float)(v - (double)h);
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
