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


// ---------------------------------------------------------------------------
// Near-singular corrections (Sec. 3.3.3, Eq. vp_near_singular; the inner
// product of Eq. singcorr_inner_prod): a target r0 outside the cell, within
// its near zone. The star point is the point of the cell nearest r0 (Eq.
// rstar_def), zeta* on the boundary of T0 (straight edges by projection; the
// curved edge by a search in its parameter, which the reference coordinate xi
// follows linearly). The area-to-line conversion with star point zeta* gives
//   Vhat_b = sum_e D_e int_0^1 ds int_0^1 t G(R(zeta* + t v_e(s)), r0) K_b J dt,
// D_e = (P_e0 - zeta*) x (P_e1 - P_e0), edges through zeta* dropping out. The
// integrand is smooth but steep at t = 0 (the distance there is |r0 - r*|) and,
// on a thin cell, at the far end of the rays that end near another boundary
// point close to r0. So the t rule is Gauss-Legendre (8 points) on panels
// graded dyadically towards both ends ([0, 2^-10], [2^-(k+1), 2^-k], and
// [1 - 2^-k, 1 - 2^-(k+1)] up to 1 - 2^-8), and the s rule Gauss-Legendre (10
// points) on panels graded geometrically (ratio 1/4, no panel wider than 1/2)
// towards the foot of zeta* on the edge and towards the edge point nearest r0
// (down to panels of about |r0 - r_e| over the edge's length). The rule is formed
// for the exact zeta* of each pair rather than taken from a table of star points
// (a table's spacing limits the accuracy for targets closer than it), and the
// basis values K_b (collapsed-coordinate Legendre x Jacobi, by their
// recurrences) are evaluated at its nodes. Then
//   corr[j] = sum_b Vhat_b C[b][j] - w_j J(zeta_j) G(R(zeta_j), r0).
constexpr int kNearThreads = 128;
constexpr int kNearL0 = 10;        // dyadic t panels towards 0: [0, 2^-10] .. [1/4, 1/2]
constexpr int kNearL1 = 8;         // and towards 1: [1/2, 3/4] .. [1 - 2^-8, 1]
constexpr int kNearTPanels = kNearL0 + kNearL1;
constexpr int kNearPtsT = 8;       // Gauss-Legendre points per t panel
constexpr int kNearPtsS = 10;      // and per s panel
constexpr int kNearMaxBreaks = 96;

// Gauss-Legendre nodes and weights of order n on [0, 1]: Newton on the
// Legendre recurrence from the Tricomi initial guesses
__device__ void gl_nodes(int n, double* x, double* w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(3.141592653589793 * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        const double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = 0.5 * (1.0 - z);
        x[n - 1 - i] = 0.5 * (1.0 + z);
        w[i] = w[n - 1 - i] = 0.5 * wi;
    }
}

// Breakpoints of [0, 1] graded geometrically (ratio 1/4) towards p down to
// panels of about `scale`, then no panel wider than 1/2; returns their count
__device__ int graded_breaks(double p, double scale, double* br, int cap)
{
    p = fmin(fmax(p, 0.0), 1.0);
    double tmp[2 * 48 + 3];
    int n = 0;
    tmp[n++] = 0.0;
    tmp[n++] = 1.0;
    tmp[n++] = p;
    for (int side = -1; side <= 1; side += 2) {
        const double span = side < 0 ? p : 1.0 - p;
        double width = span;
        for (int level = 0; level < 40 && width > fmax(scale, 1e-14); ++level) {
            width *= 0.25;
            tmp[n++] = p + side * width;
        }
    }
    // sort (insertion), drop duplicates and out-of-range points
    for (int i = 1; i < n; ++i) {
        const double v = tmp[i];
        int j = i - 1;
        while (j >= 0 && tmp[j] > v) {
            tmp[j + 1] = tmp[j];
            --j;
        }
        tmp[j + 1] = v;
    }
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const double v = tmp[i];
        if (v < 0.0 || v > 1.0) continue;
        if (m > 0 && v == br[m - 1]) continue;
        if (m > 0 && v - br[m - 1] > 0.5) {  // split a wide panel
            const double a = br[m - 1];
            const int k = (int)ceil((v - a) / 0.5 - 1e-12);
            for (int q = 1; q < k && m < cap - 1; ++q) br[m++] = a + (v - a) * q / k;
        }
        if (m < cap) br[m++] = v;
    }
    return m;
}

// union of two increasing break lists (equal points once) into out; returns its length
__device__ int merge_breaks(const double* a, int na, const double* b, int nb, double* out, int cap)
{
    int i = 0, j = 0, m = 0;
    while ((i < na || j < nb) && m < cap) {
        double v;
        if (j >= nb || (i < na && a[i] <= b[j]))
            v = a[i++];
        else
            v = b[j++];
        if (m == 0 || v > out[m - 1] + 1e-15) out[m++] = v;
    }
    return m;
}

// the collapsed-coordinate basis of total degree <= deg at (xi, eta), in the
// order m = 0..deg, k = 0..deg-m: P_m(s/t) t^m P_k^(2m+1,0)(2 eta - 1), s = 2 xi
// - 1 + eta, t = 1 - eta (homogeneous Legendre recurrence, no division by t);
// jc[(m * 8 + k) * 3 + .] = the Jacobi recurrence's coefficients for step k -> k + 1
template <int DEG>
__device__ __forceinline__ void simplex_basis(double xi, double eta, const double* __restrict__ jc, double* K)
{
    const double s = 2.0 * xi - 1.0 + eta, t = 1.0 - eta, b = 2.0 * eta - 1.0, t2 = t * t;
    double Qm1 = 0.0, Qm = 1.0;
    int idx = 0;
#pragma unroll
    for (int m = 0; m <= DEG; ++m) {
        if (m == 1) {
            Qm1 = 1.0;
            Qm = s;
        } else if (m >= 2) {
            const double Qn = ((2.0 * m - 1.0) * s * Qm - (m - 1.0) * t2 * Qm1) * (1.0 / m);
            Qm1 = Qm;
            Qm = Qn;
        }
        const double al = 2.0 * m + 1.0;
        double p0 = 1.0;
        K[idx++] = Qm;
        if (DEG - m >= 1) {
            double p1 = 0.5 * ((al + 2.0) * b + al);
            K[idx++] = Qm * p1;
#pragma unroll
            for (int k = 1; k < DEG - m; ++k) {
                const double* c = jc + (m * 8 + k) * 3;
                const double p2 = fma(fma(c[0], b, c[1]), p1, -c[2] * p0);
                p0 = p1;
                p1 = p2;
                K[idx++] = Qm * p1;
            }
        }
    }
}

__device__ __forceinline__ void dist2_to(const TriGeom& g, double xi, double eta, double x0, double y0, double& d2)
{
    double x, y, J;
    tri_map(g, xi, eta, x, y, J);
    d2 = (x - x0) * (x - x0) + (y - y0) * (y - y0);
}

template <int DEG>
__global__ void __launch_bounds__(kNearThreads)
    k_tricorr_near(int64_t n_pairs, int32_t n_nodes, const double* __restrict__ geom,
                   const double* __restrict__ tgt, const double* __restrict__ node_ref,
                   const double* __restrict__ node_w, const double* __restrict__ coef, double* __restrict__ out)
{
    constexpr int n_basis = (DEG + 1) * (DEG + 2) / 2;
    __shared__ double s_gsx[kNearPtsS], s_gsw[kNearPtsS], s_gtx[kNearPtsT], s_gtw[kNearPtsT];
    __shared__ double s_tb[kNearTPanels + 1];
    __shared__ double s_jc[8 * 8 * 3];
    __shared__ double s_br[3][kNearMaxBreaks];
    __shared__ int s_nbr[3];
    __shared__ double s_D[3], s_zs[2];
    __shared__ double red[kNearThreads / 32][n_basis];
    __shared__ double vhat[n_basis];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        gl_nodes(kNearPtsS, s_gsx, s_gsw);
        gl_nodes(kNearPtsT, s_gtx, s_gtw);
        // t breaks: 0, 2^-L0 .. 2^-1, then 1 - 2^-2 .. 1 - 2^-L1, 1
        int m = 0;
        s_tb[m++] = 0.0;
        for (int k = kNearL0; k >= 1; --k) s_tb[m++] = ldexp(1.0, -k);
        for (int k = 2; k <= kNearL1; ++k) s_tb[m++] = 1.0 - ldexp(1.0, -k);
        s_tb[m++] = 1.0;
        for (int mm = 0; mm < 8; ++mm)
            for (int k = 0; k < 8; ++k) {  // Jacobi (alpha = 2mm + 1, beta = 0), step k -> k + 1
                const double al = 2.0 * mm + 1.0, n2 = 2.0 * k + al;
                const double a1 = 2.0 * (k + 1.0) * (k + al + 1.0) * n2;
                s_jc[(mm * 8 + k) * 3 + 0] = n2 * (n2 + 1.0) * (n2 + 2.0) / a1;
                s_jc[(mm * 8 + k) * 3 + 1] = (n2 + 1.0) * al * al / a1;
                s_jc[(mm * 8 + k) * 3 + 2] = 2.0 * k * (k + al) * (n2 + 2.0) / a1;
            }
    }
    // edge e of T0 runs from vertex e to vertex (e + 1) mod 3: (0, 0), (1, 0), (0, 1)
    auto vx = [](int i) { return i == 1 ? 1.0 : 0.0; };
    auto vy = [](int i) { return i == 2 ? 1.0 : 0.0; };
    for (int64_t pr = blockIdx.x; pr < n_pairs; pr += gridDim.x) {
        __syncthreads();
        const double* gp = geom + pr * 12;
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
        const double x0 = tgt[2 * pr], y0 = tgt[2 * pr + 1];
        if (tid == 0) {
            // per edge e (parameter s from vertex e to vertex e + 1): the point
            // nearest r0, its distance and the edge's length
            double es[3], ed[3], el[3];
            // straight edges v1 -> v2 and v2 -> v0 by projection
            for (int e = 1; e <= 2; ++e) {
                const double ax = e == 1 ? g.v1x : g.v2x, ay = e == 1 ? g.v1y : g.v2y;
                const double bx = e == 1 ? g.v2x : g.v0x, by = e == 1 ? g.v2y : g.v0y;
                const double ex = bx - ax, ey = by - ay;
                const double l2 = ex * ex + ey * ey;
                const double u = fmin(fmax(((x0 - ax) * ex + (y0 - ay) * ey) / l2, 0.0), 1.0);
                const double px = ax + u * ex - x0, py = ay + u * ey - y0;
                es[e] = u;
                ed[e] = sqrt(px * px + py * py);
                el[e] = sqrt(l2);
            }
            // edge v0 -> v1 (eta = 0), straight or curved: samples, then golden section
            {
                const int ns = 64;
                double bd = INFINITY;
                int bi = 0;
                for (int i = 0; i <= ns; ++i) {
                    double d2;
                    dist2_to(g, fmin((double)i / ns, 1.0 - 1e-12), 0.0, x0, y0, d2);
                    if (d2 < bd) {
                        bd = d2;
                        bi = i;
                    }
                }
                double lo = fmax((bi - 1.0) / ns, 0.0), hi = fmin((bi + 1.0) / ns, 1.0 - 1e-12);
                const double gr = 0.6180339887498949;
                double a1 = hi - gr * (hi - lo), b1 = lo + gr * (hi - lo), fa, fb;
                dist2_to(g, a1, 0.0, x0, y0, fa);
                dist2_to(g, b1, 0.0, x0, y0, fb);
                for (int it = 0; it < 60; ++it) {
                    if (fa < fb) {
                        hi = b1;
                        b1 = a1;
                        fb = fa;
                        a1 = hi - gr * (hi - lo);
                        dist2_to(g, a1, 0.0, x0, y0, fa);
                    } else {
                        lo = a1;
                        a1 = b1;
                        fa = fb;
                        b1 = lo + gr * (hi - lo);
                        dist2_to(g, b1, 0.0, x0, y0, fb);
                    }
                }
                double xi = 0.5 * (lo + hi), d2;
                dist2_to(g, xi, 0.0, x0, y0, d2);
                if (bd < d2) {  // a sample beat the search (an end of the edge)
                    d2 = bd;
                    xi = fmin((double)bi / ns, 1.0);
                }
                es[0] = xi;
                ed[0] = sqrt(d2);
                el[0] = sqrt((g.v1x - g.v0x) * (g.v1x - g.v0x) + (g.v1y - g.v0y) * (g.v1y - g.v0y));  // chord
            }
            // the star point: the nearest of the three
            int eb = 0;
            for (int e = 1; e < 3; ++e)
                if (ed[e] < ed[eb]) eb = e;
            const double zx = vx(eb) + es[eb] * (vx((eb + 1) % 3) - vx(eb));
            const double zy = vy(eb) + es[eb] * (vy((eb + 1) % 3) - vy(eb));
            s_zs[0] = zx;
            s_zs[1] = zy;
            // the rule's edges: D_e and the s panels
            for (int e = 0; e < 3; ++e) {
                const double ax = vx(e), ay = vy(e), ex = vx((e + 1) % 3) - ax, ey = vy((e + 1) % 3) - ay;
                const double D = (ax - zx) * ey - (ay - zy) * ex;
                s_D[e] = D;
                if (fabs(D) < 1e-14) {
                    s_nbr[e] = 0;
                    continue;
                }
                const double L2 = ex * ex + ey * ey;
                const double sf = ((zx - ax) * ex + (zy - ay) * ey) / L2;
                const double sc = fmin(fmax(sf, 0.0), 1.0);
                const double fx = ax + sc * ex - zx, fy = ay + sc * ey - zy;
                const double dline = sqrt(fx * fx + fy * fy);
                double b1[kNearMaxBreaks / 2], b2[kNearMaxBreaks / 2];
                const int n1 = graded_breaks(sf, fmax(dline, 1e-4) / sqrt(L2) * 0.5, b1, kNearMaxBreaks / 2);
                const int n2 = graded_breaks(es[e], fmax(ed[e] / el[e], 1e-6) * 0.5, b2, kNearMaxBreaks / 2);
                s_nbr[e] = merge_breaks(b1, n1, b2, n2, s_br[e], kNearMaxBreaks);
            }
        }
        __syncthreads();
        const double zx = s_zs[0], zy = s_zs[1];
        constexpr int perPanel = kNearPtsS * kNearTPanels * kNearPtsT;  // nodes per s panel
        int cnt0 = s_nbr[0] > 1 ? (s_nbr[0] - 1) * perPanel : 0;
        int cnt1 = s_nbr[1] > 1 ? (s_nbr[1] - 1) * perPanel : 0;
        int cnt2 = s_nbr[2] > 1 ? (s_nbr[2] - 1) * perPanel : 0;
        const int total = cnt0 + cnt1 + cnt2;
        double acc[n_basis];
#pragma unroll
        for (int bb = 0; bb < n_basis; ++bb) acc[bb] = 0.0;
        double K[n_basis];
        for (int idx = tid; idx < total; idx += kNearThreads) {
            int e = 0, r = idx;
            if (r >= cnt0) {
                r -= cnt0;
                e = 1;
                if (r >= cnt1) {
                    r -= cnt1;
                    e = 2;
                }
            }
            const int panel = r / perPanel;
            int q = r % perPanel;
            const int si = q / (kNearTPanels * kNearPtsT);
            q %= kNearTPanels * kNearPtsT;
            const int tp = q / kNearPtsT, ti = q % kNearPtsT;
            const double sa = s_br[e][panel], sb = s_br[e][panel + 1];
            const double sv = sa + (sb - sa) * s_gsx[si], ws = (sb - sa) * s_gsw[si];
            const double ta = s_tb[tp], tb = s_tb[tp + 1];
            const double tv = ta + (tb - ta) * s_gtx[ti], wt = (tb - ta) * s_gtw[ti] * tv;
            const double ex = vx((e + 1) % 3) - vx(e), ey = vy((e + 1) % 3) - vy(e);
            const double px = vx(e) + sv * ex, py = vy(e) + sv * ey;
            const double xi = zx + tv * (px - zx), eta = zy + tv * (py - zy);
            double x, y, J;
            tri_map(g, xi, eta, x, y, J);
            const double gv = -kInv2PiT * log(hypot(x - x0, y - y0)) * J * (s_D[e] * ws * wt);
            simplex_basis<DEG>(xi, eta, s_jc, K);
#pragma unroll
            for (int bb = 0; bb < n_basis; ++bb) acc[bb] = fma(gv, K[bb], acc[bb]);
        }
#pragma unroll
        for (int bb = 0; bb < n_basis; ++bb) {
            double v = acc[bb];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) red[warp][bb] = v;
        }
        __syncthreads();
        if (tid < n_basis) {
            double v = 0.0;
            for (int w = 0; w < kNearThreads / 32; ++w) v += red[w][tid];
            vhat[tid] = v;
        }
        __syncthreads();
        for (int j = tid; j < n_nodes; j += kNearThreads) {
            double sacc = 0.0;
            for (int bb = 0; bb < n_basis; ++bb) sacc = fma(vhat[bb], coef[(int64_t)bb * n_nodes + j], sacc);
            double xj, yj, Jj;
            tri_map(g, node_ref[2 * j], node_ref[2 * j + 1], xj, yj, Jj);
            sacc -= node_w[j] * Jj * (-kInv2PiT) * log(hypot(xj - x0, yj - y0));
            out[pr * n_nodes + j] = sacc;
        }
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

vp_status vp_tricorr_near_eval(vp_tricorr tc, int64_t n_pairs, const double* geom, const double* tgt, double* out,
                               void* stream)
{
    if (!tc || !tc->alive) return tfail(VP_ERR_STATE, "invalid triangle-correction plan");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != tc->device)
        return tfail(VP_ERR_STATE, "triangle-correction plan used on another device");
    if (n_pairs < 0) return tfail(VP_ERR_ARG, "n_pairs < 0");
    if (n_pairs == 0) return VP_OK;
    if (!geom || !tgt || !out) return tfail(VP_ERR_ARG, "NULL geometry, target or output");
    int deg = 0;
    while ((deg + 1) * (deg + 2) / 2 < tc->n_basis) ++deg;
    if ((deg + 1) * (deg + 2) / 2 != tc->n_basis || deg > 7)
        return tfail(VP_ERR_UNSUPPORTED, "near corrections need a complete basis of total degree <= 7");
    const int blocks = (int)(n_pairs < 152 * 16 ? n_pairs : 152 * 16);
    cudaStream_t s = (cudaStream_t)stream;
    const int nn = tc->n_nodes;
    switch (deg) {
        case 0: k_tricorr_near<0><<<blocks, kNearThreads, 0, s>>>(n_pairs, nn, geom, tgt, tc->node_ref, tc->node_w, tc->coef, out); break;
        case 1: k_tricorr_near<1><<<blocks, kNearThreads, 0, s>>>(n_pairs, nn, geom, tgt, tc->node_ref, tc->node_w, tc->coef, out); break;
        case 2: k_tricorr_near<2><<<blocks, kNearThreads, 0, s>>>(n_pairs, nn, geom, tgt, tc->node_ref, tc->node_w, tc->coef, out); break;
        case 3: k_tricorr_near<3><<<blocks, kNearThreads, 0, s>>>(n_pairs, nn, geom, tgt, tc->node_ref, tc->node_w, tc->coef, out); break;
        case 4: k_tricorr_near<4><<<blocks, kNearThreads, 0, s>>>(n_pairs, nn, geom, tgt, tc->node_ref, tc->node_w, tc->coef, out); break;
        case 5: k_tricorr_near<5><<<blocks, kNearThreads, 0, s>>>(n_pairs, nn, geom, tgt, tc->node_ref, tc->node_w, tc->coef, out); break;
        case 6: k_tricorr_near<6><<<blocks, kNearThreads, 0, s>>>(n_pairs, nn, geom, tgt, tc->node_ref, tc->node_w, tc->coef, out); break;
        default: k_tricorr_near<7><<<blocks, kNearThreads, 0, s>>>(n_pairs, nn, geom, tgt, tc->node_ref, tc->node_w, tc->coef, out); break;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tfail(VP_ERR_CUDA, std::string("vp_tricorr_near_eval: ") + cudaGetErrorString(e));
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
