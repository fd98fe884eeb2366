// FMM for the modified-Helmholtz kernel G(r, r0) = (lambda^2/2pi) K0(lambda |r - r0|)
// (arXiv 2203.05933, Sec. 2: the Green function of L = -Delta + lambda^2; the
// experiment of Sec. 5 with lambda^2 = 100 on the unit disk), in FP64 on sm_103a.
//
// Complex notation: for w = rho e^{i theta}, I_n(w) = I_n(lambda rho) e^{i n theta}
// and K_n(w) = K_n(lambda rho) e^{i n theta} (n of either sign; I_{-n}(w) and
// K_{-n}(w) are the conjugates). Graf's addition theorem gives
//   K0(lambda |z - z'|) = sum_n K_n(z - c) conj(I_n(z' - c))   |z - c| > |z' - c|
//                       = sum_n I_n(z - c) conj(K_n(z' - c))   |z - c| < |z' - c|
//   I_n(u + v) = sum_k I_{n-k}(u) I_k(v)
//   K_n(u + v) = sum_k (-1)^k K_{n-k}(v) I_k(u)                |u| < |v|
// so that, with real charges (coefficients of -n are the conjugates of those of n),
//   multipole  M'_n = sum_j q_j conj(I_n(z_j - c))           phi = sum_n K_n(z - c) M'_n
//   local      L'_m (P2L: sum_j q_j conj(K_m(z_j - c)))      phi = sum_m I_m(z - c) L'_m
//   M2M        M'_p,n = sum_j M'_c,j conj(I_{n-j}(d))         d = c_child - c_parent
//   M2L        L'_m = (-1)^m sum_k K_{k-m}(v) M'_k            v = c_target - c_source
//   L2L        L'_c,k = sum_m L'_p,m I_{m-k}(d)
// Stored coefficients are scaled by sigma = lambda R (R the box half side):
// M_n = M'_n / sigma^n, L_m = L'_m sigma^m, n, m = 0..P, which keeps them O(1)
// for every box size. Per level the operators are fixed (four child quadrants,
// 49 source-box offsets), so M2M, L2L and M2L read plan-time tables, with the
// orders n and -n folded into one real 2x2 product per n (real charges).
//
// Near field (direct sum over the U list): with y = lambda^2 r^2 / 4,
//   K0 = I0(y) (-log(r^2)/2 - log(lambda/2) - gamma) + sum_{k>=1} H_k y^k / (k!)^2,
//   I0(y) = sum_k y^k / (k!)^2 (Abramowitz & Stegun 9.6.13), H_k the harmonic numbers,
// both series summed to the degree the target leaf's largest near-field distance
// needs (y <= 1); log r^2 comes from the float-float table log of the Laplace kernels
// (about 1e-12 absolute), everything else is FP64. Pairs with y > 1 take the
// integral representation of K0 (vp_bessel.cuh).
//
// psi convention: psi = -lambda^2 sum_j q_j K0(lambda |z - z_j|), so that the
// output kernels' V = -(1/2pi) psi (+ Pi f) give the modified-Helmholtz potential.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "vp_bessel.cuh"
#include "vp_ff.cuh"
#include "vp_internal.h"

namespace vp {
namespace {

constexpr int kWarps = 4;
constexpr int kMhChunk = 16;        // charges staged per step in P2M / P2L
constexpr int kMhLeafThreads = 64;  // one target per thread in the leaf kernel (two warps: a leaf of 64 keeps all lanes busy)
constexpr int kMaxNearTerms = 16;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// a * b + c
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

__device__ __forceinline__ int gwarp() { return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int nwarps() { return (int)((gridDim.x * blockDim.x) >> 5); }

int wblocks(int64_t nwork)
{
    int64_t b = (nwork + kWarps - 1) / kWarps;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// ----------------------------------------------------------------------------
// P2M, one warp per leaf: M_n = sum_j q_j conj(u_j)^n h_n(y_j), u = (z - c)/(2R),
// y = sigma^2 |u|^2 (= lambda^2 rho^2 / 4); h_P, h_{P+1} by their series, the
// others by the downward recurrence.
// Two warps per block and 32 charges per step, so that every lane prepares one
// charge's terms.
constexpr int kP2mWarps = 2;

template <int P, bool FF>
__global__ void __launch_bounds__(kP2mWarps * 32)
    k_p2m_mh(DevTree t, DevMH mh, PassGeom g, const double* __restrict__ q, const float2* __restrict__ qf,
             double2* __restrict__ M)
{
    constexpr int P1 = P + 1;
    constexpr int kMhChunk = 32;
    // FF: the powers, the recurrence and the sums in float-float on the FP32 pipes
    __shared__ double2 pw[kP2mWarps][FF ? 1 : kMhChunk][FF ? 1 : P1];
    __shared__ double qs[kP2mWarps][FF ? 1 : kMhChunk];
    __shared__ float4 pwf[kP2mWarps][FF ? kMhChunk : 1][FF ? P1 : 1];
    __shared__ float2 qsf[kP2mWarps][FF ? kMhChunk : 1];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    for (int li = gwarp(); li < t.nleaf; li += nwarps()) {
        const int b = t.leaves[li];
        const int s0 = g.crng[2 * b], s1 = g.crng[2 * b + 1];
        const double2 c = t.center[b];
        const double inv2R = 0.5 / t.radius[b];
        const double sig = mh.spow[t.level[b] * P1 + 1];
        double2 acc = make_double2(0.0, 0.0);
        ff::C accf{{0.f, 0.f}, {0.f, 0.f}};
        for (int base = s0; base < s1; base += kMhChunk) {
            const int n = min(kMhChunk, s1 - base);
            if (lane < n) {
                const double2 z = g.cxy[base + lane];
                const double2 u = make_double2((z.x - c.x) * inv2R, -(z.y - c.y) * inv2R);  // conj(u)
                const double y = sig * sig * (u.x * u.x + u.y * u.y);
                double hm, hm1;
                bessel::h_series2(P, y, mh.inv_fact_P, hm, hm1);
                if (FF) {
                    const ff::F yf = ff::from_double(y);
                    ff::F h = ff::from_double(hm), h1 = ff::from_double(hm1);
                    pwf[wb][lane][P] = make_float4(h.h, h.l, 0.f, 0.f);
                    for (int m = P; m >= 1; --m) {
                        const ff::F hp = ff::add(ff::mul(h, ff::F{(float)m, 0.f}), ff::mul(yf, h1));
                        h1 = h;
                        h = hp;
                        pwf[wb][lane][m - 1] = make_float4(hp.h, hp.l, 0.f, 0.f);
                    }
                    const ff::C uf = ff::from_double2(u);
                    ff::C pp{{1.f, 0.f}, {0.f, 0.f}};
                    for (int m = 0; m <= P; ++m) {
                        const float4 hv = pwf[wb][lane][m];
                        const ff::F hh{hv.x, hv.y};
                        pwf[wb][lane][m] = ff::to_float4(ff::C{ff::mul(pp.re, hh), ff::mul(pp.im, hh)});
                        pp = ff::cnorm(ff::cmul(pp, uf));
                    }
                    qsf[wb][lane] = qf[base + lane];
                } else {
                    pw[wb][lane][P].x = hm;
                    for (int m = P; m >= 1; --m) {
                        const double hp = fma((double)m, hm, y * hm1);
                        hm1 = hm;
                        hm = hp;
                        pw[wb][lane][m - 1].x = hp;
                    }
                    double2 p = make_double2(1.0, 0.0);
                    for (int m = 0; m <= P; ++m) {
                        const double h = pw[wb][lane][m].x;
                        pw[wb][lane][m] = make_double2(p.x * h, p.y * h);
                        p = cmul(p, u);
                    }
                    qs[wb][lane] = q[base + lane];
                }
            }
            __syncwarp();
            if (lane <= P) {
                if (FF) {
                    for (int j = 0; j < n; ++j) {
                        const ff::C v = ff::from_float4(pwf[wb][j][lane]);
                        const ff::F qq{qsf[wb][j].x, qsf[wb][j].y};
                        accf.re = ff::add(accf.re, ff::mul(qq, v.re));
                        accf.im = ff::add(accf.im, ff::mul(qq, v.im));
                    }
                } else {
                    for (int j = 0; j < n; ++j) {
                        const double2 v = pw[wb][j][lane];
                        acc.x = fma(qs[wb][j], v.x, acc.x);
                        acc.y = fma(qs[wb][j], v.y, acc.y);
                    }
                }
            }
            __syncwarp();
        }
        if (lane <= P) M[(int64_t)b * P1 + lane] = FF ? ff::to_double2(accf) : acc;
    }
}

// ----------------------------------------------------------------------------
// M2M into the non-leaf boxes of level l, one warp per parent; lane n owns M_n.
template <int P>
__global__ void __launch_bounds__(kWarps * 32)
    k_m2m_mh(DevTree t, DevMH mh, int l, int b0, int b1, double2* __restrict__ M)
{
    constexpr int P1 = P + 1;
    __shared__ double2 Ms[kWarps][P1];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    for (int b = b0 + gwarp(); b < b1; b += nwarps()) {
        if (t.is_leaf[b]) continue;
        double2 acc = make_double2(0.0, 0.0);
        for (int c = 0; c < 4; ++c) {
            const int ch = t.child[4 * b + c];
            if (ch < 0) continue;
            if (lane <= P) Ms[wb][lane] = M[(int64_t)ch * P1 + lane];
            __syncwarp();
            const int cq = (t.ixy[2 * ch] & 1) | ((t.ixy[2 * ch + 1] & 1) << 1);
            if (lane <= P) {
                const double2* T = mh.Tm + ((int64_t)(l * 4 + cq) * 2 * P1) * P1 + lane;
                for (int j = 0; j <= P; ++j) {
                    const double2 m = Ms[wb][j], u = T[2 * j * P1], v = T[(2 * j + 1) * P1];
                    acc.x = fma(m.x, u.x, fma(m.y, u.y, acc.x));
                    acc.y = fma(m.x, v.x, fma(m.y, v.y, acc.y));
                }
            }
            __syncwarp();
        }
        if (lane <= P) M[(int64_t)b * P1 + lane] = acc;
    }
}

// ----------------------------------------------------------------------------
// L2L from the parents into the boxes of level l, one warp per child; lane k owns L_k.
template <int P>
__global__ void __launch_bounds__(kWarps * 32)
    k_l2l_mh(DevTree t, DevMH mh, int l, int b0, int b1, double2* __restrict__ L)
{
    constexpr int P1 = P + 1;
    __shared__ double2 Ls[kWarps][P1];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    for (int b = b0 + gwarp(); b < b1; b += nwarps()) {
        const int p = t.parent[b];
        if (lane <= P) Ls[wb][lane] = L[(int64_t)p * P1 + lane];
        __syncwarp();
        const int cq = (t.ixy[2 * b] & 1) | ((t.ixy[2 * b + 1] & 1) << 1);
        if (lane <= P) {
            const double2* T = mh.Tl + ((int64_t)(l * 4 + cq) * 2 * P1) * P1 + lane;
            double2 acc = make_double2(0.0, 0.0);
            for (int m = 0; m <= P; ++m) {
                const double2 c = Ls[wb][m], u = T[2 * m * P1], v = T[(2 * m + 1) * P1];
                acc.x = fma(c.x, u.x, fma(c.y, u.y, acc.x));
                acc.y = fma(c.x, v.x, fma(c.y, v.y, acc.y));
            }
            const int64_t i = (int64_t)b * P1 + lane;
            const double2 o = L[i];
            L[i] = make_double2(o.x + acc.x, o.y + acc.y);
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------------------
// M2L over the V list plus P2L over the X list, one warp per box; lane m owns
// L_m. Every box's L is written (zeros when both lists are empty).
// FF: the V-list products in float-float on the FP32 pipes, on coefficients
// normalised by factorials (M~_k = k! M_k, L~_m = L_m / m!, operator entries
// divided by m! |k|!), which keeps every operand O(1) and inside the float range;
// else in FP64 on the scaled coefficients.
template <int P, bool FF>
__global__ void __launch_bounds__(kWarps * 32)
    k_m2l_mh(DevTree t, DevMH mh, PassGeom g, const double2* __restrict__ M, double2* __restrict__ L,
             const double* __restrict__ q)
{
    constexpr int P1 = P + 1;
    __shared__ double2 Ms[kWarps][FF ? 1 : P1];
    __shared__ float4 Mf[kWarps][FF ? P1 : 1];
    __shared__ double2 pw[kWarps][kMhChunk][P1];
    __shared__ double qs[kWarps][kMhChunk];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    double fact = 1.0;  // lane!
    for (int i = 2; i <= lane; ++i) fact *= (double)i;
    for (int b = gwarp(); b < t.nbox; b += nwarps()) {
        const int lev = t.level[b];
        const double* sp = mh.spow + lev * P1;
        const int bx = t.ixy[2 * b], by = t.ixy[2 * b + 1];
        double2 lacc = make_double2(0.0, 0.0);
        const int v0 = t.v_ptr[b], v1 = t.v_ptr[b + 1];
        if (FF) {
            ff::F re{0.f, 0.f}, im{0.f, 0.f};
            for (int e = v0; e < v1; ++e) {
                const int C = t.v_idx[e];
                const int o = (t.ixy[2 * C + 1] - by + 3) * 7 + (t.ixy[2 * C] - bx + 3);
                if (lane <= P) {
                    const double2 m = M[(int64_t)C * P1 + lane];
                    const ff::F a = ff::from_double(m.x * fact), c = ff::from_double(m.y * fact);
                    Mf[wb][lane] = make_float4(a.h, a.l, c.h, c.l);
                }
                __syncwarp();
                if (lane <= P) {
                    const float4* T = mh.Tvf + ((int64_t)(lev * 49 + o) * P1) * 2 * P1 + lane;
#pragma unroll 5
                    for (int k = 0; k <= P; ++k) {
                        const float4 mk = Mf[wb][k], u = T[2 * k * P1], v = T[(2 * k + 1) * P1];
                        const ff::F a{mk.x, mk.y}, c{mk.z, mk.w};
                        re = ff::add(re, ff::add(ff::mul(a, ff::F{u.x, u.y}), ff::mul(c, ff::F{u.z, u.w})));
                        im = ff::add(im, ff::add(ff::mul(a, ff::F{v.x, v.y}), ff::mul(c, ff::F{v.z, v.w})));
                    }
                }
                __syncwarp();
            }
            if (lane <= P) lacc = make_double2(ff::to_double(re) * fact, ff::to_double(im) * fact);
        }
        if (!FF) {
            for (int e = v0; e < v1; ++e) {
                const int C = t.v_idx[e];
                const int o = (t.ixy[2 * C + 1] - by + 3) * 7 + (t.ixy[2 * C] - bx + 3);
                if (lane <= P) Ms[wb][lane] = M[(int64_t)C * P1 + lane];
                __syncwarp();
                if (lane <= P) {
                    // the level's operator for this offset, acting on the scaled M and giving
                    // the scaled L, with the orders k and -k folded (real 2x2 per k)
                    const double2* T = mh.Tv + ((int64_t)(lev * 49 + o) * P1) * 2 * P1 + lane;
#pragma unroll 5
                    for (int k = 0; k <= P; ++k) {
                        const double2 m = Ms[wb][k], u = T[2 * k * P1], v = T[(2 * k + 1) * P1];
                        lacc.x = fma(m.x, u.x, fma(m.y, u.y, lacc.x));
                        lacc.y = fma(m.x, v.x, fma(m.y, v.y, lacc.y));
                    }
                }
                __syncwarp();
            }
        }
        const int x0 = t.x_ptr[b], x1 = t.x_ptr[b + 1];
        if (x1 > x0) {
            const double2 c = t.center[b];
            const double sig = sp[1];
            for (int e = x0; e < x1; ++e) {
                const int C = t.x_idx[e];
                const int s0 = g.crng[2 * C], s1 = g.crng[2 * C + 1];
                for (int base = s0; base < s1; base += kMhChunk) {
                    const int n = min(kMhChunk, s1 - base);
                    if (lane < n) {
                        // sigma^n K_n(lambda rho) e^{-i n theta} of this charge about c
                        const double2 z = g.cxy[base + lane];
                        const double dx = z.x - c.x, dy = z.y - c.y;
                        const double rho = sqrt(dx * dx + dy * dy);
                        const double x = mh.lambda * rho;
                        double k0, k1;
                        bessel::k01(x, k0, k1);
                        const double2 ph = make_double2(dx / rho, -dy / rho);
                        double ka = k0, kb = sig * k1;
                        const double s2 = sig * sig, r = 2.0 * sig / x;
                        pw[wb][lane][0] = make_double2(ka, 0.0);
                        double2 p = ph;
                        pw[wb][lane][1] = make_double2(kb * p.x, kb * p.y);
                        for (int m = 1; m < P; ++m) {
                            const double kc = fma(s2, ka, (double)m * r * kb);
                            ka = kb;
                            kb = kc;
                            p = cmul(p, ph);
                            pw[wb][lane][m + 1] = make_double2(kb * p.x, kb * p.y);
                        }
                        qs[wb][lane] = q[base + lane];
                    }
                    __syncwarp();
                    if (lane <= P) {
                        for (int j = 0; j < n; ++j) {
                            const double2 v = pw[wb][j][lane];
                            lacc.x = fma(qs[wb][j], v.x, lacc.x);
                            lacc.y = fma(qs[wb][j], v.y, lacc.y);
                        }
                    }
                    __syncwarp();
                }
            }
        }
        if (lane <= P) L[(int64_t)b * P1 + lane] = lacc;
    }
}

// ----------------------------------------------------------------------------
// Near field of one target over a staged tile of charges, float-float on the
// FP32 pipes. Per pair (units of the target leaf's side): r'^2 from exact
// leaf-centre offsets, log r'^2 by the table log, y = (lambda^2 side^2/4) r'^2,
// T = -log(r'^2)/2 - (log side + log(lambda/2) + gamma), and
// K0 = T I0(y) + S(y) with both series by Horner: the terms k >= m in FP32 (their
// share of K0 is below the leaf's bound, see near_split), the terms k < m in
// float-float. Pairs with y > 1 take the integral representation in FP64.
// EXACT: the hi parts of target and source differ exactly in float.
// K0(lambda r) of one pair in float-float (see mh_tile); false for a coincident pair.
template <bool EXACT>
__device__ __forceinline__ bool mh_pair(const float4 rt, const float4 sr, const float4* __restrict__ s_tab,
                                        const float2* __restrict__ a2, const float2* __restrict__ b2, int deg, int m,
                                        ff::F cy, ff::F Tc, double lam_side, ff::F& K)
{
    float dxs, dxe, dys, dye;
    if (EXACT) {
        dxs = __fsub_rn(rt.x, sr.x);
        dxe = __fsub_rn(rt.y, sr.y);
        dys = __fsub_rn(rt.z, sr.z);
        dye = __fsub_rn(rt.w, sr.w);
    } else {
        ff::two_sum(rt.x, -sr.x, dxs, dxe);
        dxe = __fadd_rn(dxe, __fsub_rn(rt.y, sr.y));
        ff::two_sum(rt.z, -sr.z, dys, dye);
        dye = __fadd_rn(dye, __fsub_rn(rt.w, sr.w));
    }
    const float px = __fmul_rn(dxs, dxs);
    float pxe = fmaf(dxs, dxs, -px);
    pxe = fmaf(__fadd_rn(dxs, dxs), dxe, pxe);
    pxe = fmaf(dxe, dxe, pxe);
    const float py = __fmul_rn(dys, dys);
    float pye = fmaf(dys, dys, -py);
    pye = fmaf(__fadd_rn(dys, dys), dye, pye);
    pye = fmaf(dye, dye, pye);
    const float rs = __fadd_rn(px, py);
    float re = __fsub_rn(fminf(px, py), __fsub_rn(rs, fmaxf(px, py)));
    re = __fadd_rn(re, __fadd_rn(pxe, pye));
    if (rs == 0.0f && re == 0.0f) return false;  // coincident pair: no smooth term
    const ff::F r2{rs, re};
    const ff::F y = ff::mul(r2, cy);
    if (y.h > 1.0f) {
        K = ff::from_double(bessel::k0_large(lam_side * sqrt((double)rs + (double)re)));
        return true;
    }
    float S, lo;
    ff::log_pair(rs, re, s_tab, S, lo);
    const ff::F T = ff::add(ff::F{-0.5f * S, -0.5f * lo}, Tc);
    float ta = 0.0f, tb = 0.0f;
    for (int j = deg; j >= m; --j) {
        ta = fmaf(ta, y.h, a2[j].x);
        tb = fmaf(tb, y.h, b2[j].x);
    }
    ff::F A{ta, 0.0f}, B{tb, 0.0f};
    for (int j = m - 1; j >= 0; --j) {
        A = ff::add(ff::mul(A, y), ff::F{a2[j].x, a2[j].y});
        B = ff::add(ff::mul(B, y), ff::F{b2[j].x, b2[j].y});
    }
    K = ff::add(ff::mul(A, T), B);
    return true;
}

// (ah, al) += q K in float-float
__device__ __forceinline__ void ff_acc(float2 q, ff::F K, float& ah, float& al)
{
    const float p = __fmul_rn(q.x, K.h);
    float pe = fmaf(q.x, K.h, -p);
    pe = fmaf(q.x, K.l, pe);
    pe = fmaf(q.y, K.h, pe);
    float sh, se;
    ff::two_sum(ah, p, sh, se);
    ah = sh;
    al = __fadd_rn(al, __fadd_rn(se, pe));
}

// Near field of one target over a staged tile of charges, float-float on the
// FP32 pipes. Per pair (units of the target leaf's side): r'^2 from exact
// leaf-centre offsets, log r'^2 by the table log, y = (lambda^2 side^2/4) r'^2,
// T = -log(r'^2)/2 - (log side + log(lambda/2) + gamma), and
// K0 = T I0(y) + S(y) with both series by Horner: the terms k >= m in FP32 (their
// share of K0 is below the leaf's bound, see near_split), the terms k < m in
// float-float. Pairs with y > 1 take the integral representation in FP64.
// EXACT: the hi parts of target and source differ exactly in float.
template <bool EXACT>
__device__ __forceinline__ void mh_tile(const float4 rt, const float4* __restrict__ s_rho,
                                        const float2* __restrict__ s_q, int n, const float4* __restrict__ s_tab,
                                        const float2* __restrict__ a2, const float2* __restrict__ b2, int deg, int m,
                                        ff::F cy, ff::F Tc, double lam_side, float& ah, float& al)
{
#pragma unroll 2
    for (int k = 0; k < n; ++k) {
        ff::F K;
        if (mh_pair<EXACT>(rt, s_rho[k], s_tab, a2, b2, deg, m, cy, Tc, lam_side, K)) ff_acc(s_q[k], K, ah, al);
    }
}

// Symmetric pass over one chunk of at most 32 charges of a leaf A for the 32
// targets of one warp (the targets are the charge points of the warp's own leaf
// b, A != b): as in the Laplace kernel, lane l takes charge (l + t) mod 32 at
// step t, adds q_j K to its target and q_i K to a float-float sum for that
// charge, and the sums move one lane down after each step, so that lane l ends
// with the warp's total for charge l. rh, rl must be zero on entry.
template <bool EXACT>
__device__ __forceinline__ void mh_chunk_sym(const float4 rt, float2 qi, bool valid_i, const float4* __restrict__ s_rho,
                                             const float2* __restrict__ s_q, int n, int lane,
                                             const float4* __restrict__ s_tab, const float2* __restrict__ a2,
                                             const float2* __restrict__ b2, int deg, int m, ff::F cy, ff::F Tc,
                                             double lam_side, float& ah, float& al, float& rh, float& rl)
{
    const int from = (lane + 1) & 31;
    for (int t = 0; t < 32; ++t) {
        const int j = (lane + t) & 31;
        if (valid_i && j < n) {
            ff::F K;
            if (mh_pair<EXACT>(rt, s_rho[j], s_tab, a2, b2, deg, m, cy, Tc, lam_side, K)) {
                ff_acc(s_q[j], K, ah, al);
                ff_acc(qi, K, rh, rl);
            }
        }
        rh = __shfl_sync(0xffffffffu, rh, from);
        rl = __shfl_sync(0xffffffffu, rl, from);
    }
}

// ----------------------------------------------------------------------------
// Per leaf: L2P, M2P over the W list and the direct sum over the U list; one
// block per leaf, one target per thread. FF: the near field in float-float on
// the FP32 pipes (mh_tile); else in FP64.
template <int P, bool FF, bool SYM>
__global__ void __launch_bounds__(kMhLeafThreads, SYM ? 10 : 16)
    k_leaf_mh(DevTree t, DevMH mh, PassGeom g, const double* __restrict__ q, const float2* __restrict__ qf,
              const double2* __restrict__ M, const double2* __restrict__ L, const float4* __restrict__ logtab,
              double* __restrict__ psi, float2* __restrict__ slots)
{
    static_assert(FF || !SYM, "the symmetric near field is float-float");
    constexpr int P1 = P + 1;
    __shared__ double2 Cs[P1];
    __shared__ float4 Csf[FF ? P1 : 1];
    __shared__ double2 sxy[FF ? 1 : kMhLeafThreads];
    __shared__ double sq[FF ? 1 : kMhLeafThreads];
    __shared__ float4 s_rho[FF ? kMhLeafThreads : 1];
    __shared__ float2 s_qf[FF ? kMhLeafThreads : 1];
    __shared__ float4 s_tab[FF ? 128 : 1];
    __shared__ double na[kMaxNearTerms], nb[kMaxNearTerms];
    __shared__ float2 a2[kMaxNearTerms], b2[kMaxNearTerms];
    const int tid = threadIdx.x;
    if (tid <= mh.near_deg) {
        na[tid] = mh.near_a[tid];
        nb[tid] = mh.near_b[tid];
        const ff::F fa = ff::from_double(mh.near_a[tid]), fb = ff::from_double(mh.near_b[tid]);
        a2[tid] = make_float2(fa.h, fa.l);
        b2[tid] = make_float2(fb.h, fb.l);
    }
    if (FF)
        for (int i = tid; i < 128; i += kMhLeafThreads) s_tab[i] = logtab[i];
    for (int li = blockIdx.x; li < t.nleaf; li += gridDim.x) {
        const int b = SYM ? t.sym_leaves[li] : t.leaves[li];
        const int e0 = g.erng[2 * b], e1 = g.erng[2 * b + 1];
        if (e0 == e1) continue;
        const int code = mh.leaf_deg[b];  // series terms this leaf's near field needs, and its split
        const int deg = code & 0xff, msplit = code >> 8;
        const double2 cb = t.center[b];
        const double Rb = t.radius[b];
        const double sig = mh.spow[t.level[b] * P1 + 1];
        const double side = 2.0 * Rb;
        const double inv_side2 = 1.0 / (side * side);
        const double log_side2 = 2.0 * log(side);
        const ff::F cy = ff::from_double(mh.lam2_4 * side * side);
        const ff::F Tc = ff::from_double(-(0.5 * log_side2 + mh.c0));
        const int u0 = t.u_ptr[b], u1 = t.u_ptr[b + 1];
        const int w0 = t.w_ptr[b], w1 = t.w_ptr[b + 1];
        for (int tb = e0; tb < e1; tb += kMhLeafThreads) {
            const int ti = tb + tid;
            const bool valid = ti < e1;
            const double2 z = valid ? g.exy[ti] : cb;
            double acc = 0.0;

            // L2P: phi = 2 Re sum_m u^m h_m L_m - h_0 L_0, by Horner in u while h_m
            // runs down its recurrence (FF: in float-float)
            __syncthreads();
            for (int i = tid; i < P1; i += kMhLeafThreads) {
                Cs[i] = L[(int64_t)b * P1 + i];
                if (FF) Csf[i] = ff::to_float4(ff::from_double2(Cs[i]));
            }
            __syncthreads();
            if (FF && valid) {
                const double2 ud = make_double2((z.x - cb.x) / side, (z.y - cb.y) / side);
                const double y = sig * sig * (ud.x * ud.x + ud.y * ud.y);
                double hm, hm1;
                bessel::h_series2(P, y, mh.inv_fact_P, hm, hm1);
                const ff::C u = ff::from_double2(ud);
                const ff::F yf = ff::from_double(y);
                ff::F h = ff::from_double(hm), h1 = ff::from_double(hm1);
                const ff::C cP = ff::from_float4(Csf[P]);
                ff::C S{ff::mul(cP.re, h), ff::mul(cP.im, h)};
                for (int m = P; m >= 1; --m) {
                    const ff::F hp = ff::add(ff::mul(h, ff::F{(float)m, 0.f}), ff::mul(yf, h1));
                    h1 = h;
                    h = hp;
                    const ff::C cm = ff::from_float4(Csf[m - 1]);
                    S = ff::cnorm(ff::cadd(ff::cmul(S, u), ff::C{ff::mul(cm.re, hp), ff::mul(cm.im, hp)}));
                }
                acc += 2.0 * ff::to_double(S.re) - ff::to_double(h) * Cs[0].x;
            } else if (valid) {
                const double2 u = make_double2((z.x - cb.x) / side, (z.y - cb.y) / side);
                const double y = sig * sig * (u.x * u.x + u.y * u.y);
                double hm, hm1;
                bessel::h_series2(P, y, mh.inv_fact_P, hm, hm1);
                double2 S = make_double2(Cs[P].x * hm, Cs[P].y * hm);
                for (int m = P; m >= 1; --m) {
                    const double hp = fma((double)m, hm, y * hm1);
                    hm1 = hm;
                    hm = hp;
                    const double2 c = Cs[m - 1];
                    S = cfma(S, u, make_double2(c.x * hp, c.y * hp));
                }
                acc += 2.0 * S.x - hm * Cs[0].x;
            }
            // M2P over W: phi = K_0 M_0 + 2 Re sum_{n>=1} sigma_D^n K_n e^{i n theta} M_n
            for (int e = w0; e < w1; ++e) {
                const int D = t.w_idx[e];
                __syncthreads();
                for (int i = tid; i < P1; i += kMhLeafThreads) Cs[i] = M[(int64_t)D * P1 + i];
                __syncthreads();
                if (valid) {
                    const double2 cD = t.center[D];
                    const double sD = mh.spow[t.level[D] * P1 + 1];
                    const double dx = z.x - cD.x, dy = z.y - cD.y;
                    const double rho = sqrt(dx * dx + dy * dy);
                    const double x = mh.lambda * rho;
                    double k0, k1;
                    bessel::k01(x, k0, k1);
                    const double2 ph = make_double2(dx / rho, dy / rho);
                    double ka = k0, kb = sD * k1;
                    const double s2 = sD * sD, r = 2.0 * sD / x;
                    double2 p = ph;
                    double s = kb * (p.x * Cs[1].x - p.y * Cs[1].y);
                    for (int n = 1; n < P; ++n) {
                        const double kc = fma(s2, ka, (double)n * r * kb);
                        ka = kb;
                        kb = kc;
                        p = cmul(p, ph);
                        s = fma(kb, p.x * Cs[n + 1].x - p.y * Cs[n + 1].y, s);
                    }
                    acc += fma(2.0, s, k0 * Cs[0].x);
                }
            }
            // P2P over U
            double near = 0.0;
            if (FF) {
                const float4 rt = valid ? g.erho[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
                float ah = 0.0f, al = 0.0f;
                // SYM: leaves A < b are skipped (A's block hands their part over through
                // the slots), leaves A > b are summed in both directions
                const int warp = tid >> 5, lane = tid & 31;
                const int grp = (tb - e0) / 32 + warp;  // this warp's group of 32 targets of b
                const bool grp_live = tb + 32 * warp < e1;
                const float2 qi = (SYM && valid) ? qf[ti] : make_float2(0.f, 0.f);
                for (int e = u0; e < u1; ++e) {
                    const int A = t.u_idx[e];
                    const int a0 = g.crng[2 * A], a1 = g.crng[2 * A + 1];
                    if (a0 == a1) continue;
                    if (SYM && A < b) continue;
                    const bool rev = SYM && A > b;
                    const int64_t sbase = rev ? t.sym_off[e] + (int64_t)grp * (a1 - a0) : 0;
                    const float4 uo = t.u_off[e];  // leaf A's centre offset and scale in b units
                    const bool exact_hi = uo.z >= 0.5f && uo.z <= 2.0f;
                    for (int sb = a0; sb < a1; sb += kMhLeafThreads) {
                        const int n = min(kMhLeafThreads, a1 - sb);
                        __syncthreads();
                        if (tid < n) {
                            const int j = sb + tid;
                            const float4 r = g.crho[j];
                            ff::F sx, sy;
                            if (exact_hi) {
                                sx = ff::F{__fadd_rn(uo.x, __fmul_rn(uo.z, r.x)), __fmul_rn(uo.z, r.y)};
                                sy = ff::F{__fadd_rn(uo.y, __fmul_rn(uo.z, r.z)), __fmul_rn(uo.z, r.w)};
                            } else {
                                sx = ff::shift_scale(uo.x, uo.z, r.x, r.y);
                                sy = ff::shift_scale(uo.y, uo.z, r.z, r.w);
                            }
                            s_rho[tid] = make_float4(sx.h, sx.l, sy.h, sy.l);
                            s_qf[tid] = qf[j];
                        }
                        __syncthreads();
                        if (rev) {
                            if (grp_live) {  // warp-uniform
                                for (int c = 0; c < n; c += 32) {
                                    const int nc = min(32, n - c);
                                    float rh = 0.0f, rl = 0.0f;
                                    if (exact_hi)
                                        mh_chunk_sym<true>(rt, qi, valid, s_rho + c, s_qf + c, nc, lane, s_tab, a2, b2,
                                                           deg, msplit, cy, Tc, mh.lambda * side, ah, al, rh, rl);
                                    else
                                        mh_chunk_sym<false>(rt, qi, valid, s_rho + c, s_qf + c, nc, lane, s_tab, a2,
                                                            b2, deg, msplit, cy, Tc, mh.lambda * side, ah, al, rh, rl);
                                    if (lane < nc) slots[sbase + (sb - a0) + c + lane] = make_float2(rh, rl);
                                }
                            }
                        } else if (valid) {
                            if (exact_hi)
                                mh_tile<true>(rt, s_rho, s_qf, n, s_tab, a2, b2, deg, msplit, cy, Tc,
                                              mh.lambda * side, ah, al);
                            else
                                mh_tile<false>(rt, s_rho, s_qf, n, s_tab, a2, b2, deg, msplit, cy, Tc,
                                               mh.lambda * side, ah, al);
                        }
                    }
                }
                near = (double)ah + (double)al;
            } else {
                for (int e = u0; e < u1; ++e) {
                    const int A = t.u_idx[e];
                    const int a0 = g.crng[2 * A], a1 = g.crng[2 * A + 1];
                    for (int sb = a0; sb < a1; sb += kMhLeafThreads) {
                        const int n = min(kMhLeafThreads, a1 - sb);
                        __syncthreads();
                        if (tid < n) {
                            sxy[tid] = g.cxy[sb + tid];
                            sq[tid] = q[sb + tid];
                        }
                        __syncthreads();
                        if (valid) {
                            for (int j = 0; j < n; ++j) {
                                const double dx = z.x - sxy[j].x, dy = z.y - sxy[j].y;
                                const double r2 = fma(dx, dx, dy * dy);
                                if (r2 == 0.0) continue;  // coincident pair: no smooth term
                                const double y = mh.lam2_4 * r2;
                                double k0;
                                if (y <= 1.0) {
                                    const double rs = r2 * inv_side2;
                                    const float h = __double2float_rn(rs);
                                    const float l = __double2float_rn(rs - (double)h);
                                    float S, lo;
                                    ff::log_pair(h, l, logtab, S, lo);
                                    const double lg = (double)S + (double)lo + log_side2;  // log r^2
                                    double ia = na[deg], sb2 = nb[deg];
                                    for (int k = deg - 1; k >= 0; --k) {
                                        ia = fma(ia, y, na[k]);
                                        sb2 = fma(sb2, y, nb[k]);
                                    }
                                    k0 = fma(ia, fma(-0.5, lg, -mh.c0), sb2);
                                } else {
                                    k0 = bessel::k0_large(mh.lambda * sqrt(r2));
                                }
                                near = fma(sq[j], k0, near);
                            }
                        }
                    }
                }
            }
            if (valid) psi[ti] = mh.psi_scale * (acc + near);
        }
    }
}

// Symmetric near field: adds the slots handed over to each point by the
// lower adjacent leaves, in a fixed order, times psi_scale.
__global__ void k_sym_reduce_mh(DevTree t, DevMH mh, PassGeom g, const float2* __restrict__ slots,
                                double* __restrict__ psi)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.n_eval; j += gridDim.x * blockDim.x) {
        const int A = t.sym_pt_leaf[j];
        const int s0 = t.sym_in_ptr[A], s1 = t.sym_in_ptr[A + 1];
        if (s0 == s1) continue;
        const int jl = j - g.erng[2 * A];
        ff::F acc{0.f, 0.f};
#pragma unroll 4
        for (int k = s0; k < s1; ++k) {
            const float2 v = slots[t.sym_in_slot[k] + jl];
            acc = ff::add(acc, ff::F{v.x, v.y});
        }
        psi[j] = fma(mh.psi_scale, ff::to_double(acc), psi[j]);
    }
}

template <int P>
cudaError_t fmm_mh(const DevTree& t, const DevMH& mh, const float4* logtab, const PassGeom& g, Workspace& ws,
                   bool fp64, PhaseTimer* tm, cudaStream_t s)
{
    const int threads = kWarps * 32;
    int id = tm ? tm->begin("upward") : -1;
    const int pblocks = std::max(1, std::min((t.nleaf + kP2mWarps - 1) / kP2mWarps, 152 * 64));
    if (fp64)
        k_p2m_mh<P, false><<<pblocks, kP2mWarps * 32, 0, s>>>(t, mh, g, ws.q, ws.qf, ws.M);
    else
        k_p2m_mh<P, true><<<pblocks, kP2mWarps * 32, 0, s>>>(t, mh, g, ws.q, ws.qf, ws.M);
    for (int l = t.nlevels - 2; l >= 2; --l) {  // multipoles of levels 0 and 1 are never read
        const int b0 = t.level_start[l], b1 = t.level_start[l + 1];
        k_m2m_mh<P><<<wblocks(b1 - b0), threads, 0, s>>>(t, mh, l, b0, b1, ws.M);
    }
    if (tm) tm->end(id);
    id = tm ? tm->begin("m2l") : -1;
    if (fp64)
        k_m2l_mh<P, false><<<wblocks(t.nbox), threads, 0, s>>>(t, mh, g, ws.M, ws.L, ws.q);
    else
        k_m2l_mh<P, true><<<wblocks(t.nbox), threads, 0, s>>>(t, mh, g, ws.M, ws.L, ws.q);
    if (tm) tm->end(id);
    id = tm ? tm->begin("l2l") : -1;
    for (int l = 3; l < t.nlevels; ++l) {  // locals of levels 0 to 2 receive nothing from above
        const int b0 = t.level_start[l], b1 = t.level_start[l + 1];
        k_l2l_mh<P><<<wblocks(b1 - b0), threads, 0, s>>>(t, mh, l, b0, b1, ws.L);
    }
    if (tm) tm->end(id);
    id = tm ? tm->begin("leaf") : -1;
    const int blocks = std::max(1, std::min(t.nleaf, 152 * 32));
    if (fp64) {
        k_leaf_mh<P, false, false><<<blocks, kMhLeafThreads, 0, s>>>(t, mh, g, ws.q, ws.qf, ws.M, ws.L, logtab,
                                                                    ws.psi, nullptr);
    } else if (t.sym) {
        k_leaf_mh<P, true, true><<<blocks, kMhLeafThreads, 0, s>>>(t, mh, g, ws.q, ws.qf, ws.M, ws.L, logtab, ws.psi,
                                                                  ws.slots);
        const int rblocks = std::max(1, std::min((g.n_eval + 255) / 256, 152 * 32));
        k_sym_reduce_mh<<<rblocks, 256, 0, s>>>(t, mh, g, ws.slots, ws.psi);
    } else {
        k_leaf_mh<P, true, false><<<blocks, kMhLeafThreads, 0, s>>>(t, mh, g, ws.q, ws.qf, ws.M, ws.L, logtab,
                                                                   ws.psi, nullptr);
    }
    if (tm) tm->end(id);
    return cudaGetLastError();
}

double2 d2(double x, double y)
{
    double2 r;
    r.x = x;
    r.y = y;
    return r;
}

}  // namespace

cudaError_t launch_fmm_mhelm(int P, const DevTree& t, const DevMH& mh, const float4* logtab, const PassGeom& g,
                             Workspace& ws, bool fp64, PhaseTimer* timer, cudaStream_t s)
{
    switch (P) {
        case 16: return fmm_mh<16>(t, mh, logtab, g, ws, fp64, timer, s);
        case 24: return fmm_mh<24>(t, mh, logtab, g, ws, fp64, timer, s);
        case 30: return fmm_mh<30>(t, mh, logtab, g, ws, fp64, timer, s);
        default: return cudaErrorInvalidValue;
    }
}

int64_t mhelm_launches(int nlevels, bool sym_reduce)
{
    return 3 + 2 * (int64_t)std::max(0, nlevels - 3) + (sym_reduce ? 1 : 0);
}

// Series terms k = 0..deg for |y| <= ymax (<= 1): until the first omitted term,
// weighted by the size of its harmonic-number coefficient, is below 1e-18.
int near_degree(double ymax)
{
    int deg = 1;
    double term = ymax;  // y^k / (k!)^2 at k = deg
    while (deg < kMaxNearTerms - 1) {
        const double next = term * ymax / ((double)(deg + 1) * (double)(deg + 1));
        if (next * (4.0 + std::log((double)deg + 2.0)) < 1e-18) break;
        term = next;
        ++deg;
    }
    return deg;
}

// Smallest m in [1, deg + 1] such that the terms k >= m of both series, summed in
// FP32 (relative error below 2^-20 for at most 16 terms), change K0 = T I0 + S by
// less than 2e-15 for every 0 < y <= ymax, with |T| <= |log(4y/lambda^2)|/2 + |c0|.
int near_split(int deg, double ymax, double lambda, double c0, const std::vector<double>& ca,
               const std::vector<double>& cb)
{
    for (int m = 1; m <= deg; ++m) {
        double worst = 0.0;
        for (int i = 0; i < 400; ++i) {
            const double y = ymax * std::ldexp(1.0, -i / 4);
            if (y <= 0.0) break;
            double ta = 0.0, tb = 0.0, ym = std::pow(y, m);
            for (int k = m; k <= deg; ++k) {
                ta += ca[(size_t)k] * std::pow(y, k - m);
                tb += cb[(size_t)k] * std::pow(y, k - m);
            }
            const double Tabs = 0.5 * std::fabs(std::log(4.0 * y / (lambda * lambda))) + std::fabs(c0);
            worst = std::max(worst, ym * (ta * Tabs + tb));
        }
        if (worst * 0x1p-20 < 2e-15) return m;
    }
    return deg + 1;
}

std::string make_mh_tables(int P, double lambda, const std::vector<double>& R_level,
                           const std::vector<double>& leaf_dmax, bool ff, MhTables& T)
{
    const int P1 = P + 1, NJ = 2 * P + 1;
    const int nl = (int)R_level.size();
    T.spow.assign((size_t)nl * P1, 0.0);
    std::vector<double2> fullM((size_t)nl * 4 * NJ * P1, d2(0.0, 0.0)), fullL(fullM);
    T.Tv.assign((size_t)nl * 49 * 2 * P1 * P1, d2(0.0, 0.0));
    // 1/m! and h_m(y_d) for the child offset d (|d| = sqrt(2) R_child, y_d = sigma_child^2 / 2)
    std::vector<double> inv_fact((size_t)3 * P + 2, 1.0);
    for (size_t m = 1; m < inv_fact.size(); ++m) inv_fact[m] = inv_fact[m - 1] / (double)m;
    T.inv_fact_P = inv_fact[(size_t)P];
    for (int l = 0; l < nl; ++l) {
        const double sig = lambda * R_level[(size_t)l];
        double pw = 1.0;
        for (int k = 0; k <= P; ++k) {
            T.spow[(size_t)l * P1 + k] = pw;
            pw *= sig;
        }
    }
    // M2M into a parent of level l (children at level l + 1) and L2L into a child of
    // level l (parent at level l - 1): both shift by d = child centre - parent centre
    for (int l = 0; l < nl; ++l) {
        for (int pass = 0; pass < 2; ++pass) {
            const int lc = pass == 0 ? l + 1 : l;  // level of the child
            if (lc >= nl || lc < 1) continue;
            const double sc = lambda * R_level[(size_t)lc];
            const double yd = 0.5 * sc * sc;
            std::vector<double> h((size_t)NJ + 1);
            for (int a = 0; a <= 2 * P; ++a) h[(size_t)a] = bessel::h_series(a, yd, inv_fact[(size_t)a]);
            for (int cq = 0; cq < 4; ++cq) {
                const double th = std::atan2((cq & 2) ? 1.0 : -1.0, (cq & 1) ? 1.0 : -1.0);
                double2* dst = (pass == 0 ? fullM.data() : fullL.data()) + (size_t)(l * 4 + cq) * NJ * P1;
                for (int j = -P; j <= P; ++j) {
                    for (int n = 0; n <= P; ++n) {
                        double mag, ang;
                        if (pass == 0) {
                            // sigma_c^|j| / sigma_p^n conj(I_{n-j}(d)), sigma_p = 2 sigma_c
                            const int a = std::abs(n - j);
                            mag = std::ldexp(1.0, -n) * std::pow(sc, std::abs(j) - n + a) *
                                  std::pow(std::sqrt(0.5), a) * h[(size_t)a];
                            ang = -(double)(n - j) * th;
                        } else {
                            // sigma_c^k sigma_p^-|m| I_{m-k}(d) with (m, k) = (j, n)
                            const int a = std::abs(j - n);
                            mag = std::ldexp(1.0, -std::abs(j)) * std::pow(sc, n - std::abs(j) + a) *
                                  std::pow(std::sqrt(0.5), a) * h[(size_t)a];
                            ang = (double)(j - n) * th;
                        }
                        dst[(size_t)(j + P) * P1 + n] = d2(mag * std::cos(ang), mag * std::sin(ang));
                    }
                }
            }
        }
    }
    // With real charges the coefficient of index -j is the conjugate of that of j, so
    // the terms j and -j fold into one real 2x2 product per j >= 0: for entries
    // T_j = p + iq, T_-j = r + is and a coefficient a + ib,
    //   T_j (a + ib) + T_-j (a - ib) = a (p + r) + b (s - q) + i (a (q + s) + b (p - r)),
    // stored as (p + r, s - q), (q + s, p - r) per (j, n); j = 0 is the plain product.
    auto fold = [&](const std::vector<double2>& full, std::vector<double2>& out) {
        out.assign((size_t)nl * 4 * 2 * P1 * P1, d2(0.0, 0.0));
        for (size_t lq = 0; lq < (size_t)nl * 4; ++lq)
            for (int j = 0; j <= P; ++j)
                for (int n = 0; n <= P; ++n) {
                    const double2 a = full[(lq * NJ + (size_t)(j + P)) * P1 + n];
                    const double2 b = j > 0 ? full[(lq * NJ + (size_t)(P - j)) * P1 + n] : d2(0.0, 0.0);
                    double2* o = out.data() + (lq * 2 * P1 + 2 * (size_t)j) * P1 + n;
                    if (j == 0) {
                        o[0] = d2(a.x, -a.y);
                        o[P1] = d2(a.y, a.x);
                    } else {
                        o[0] = d2(a.x + b.x, b.y - a.y);
                        o[P1] = d2(a.y + b.y, a.x - b.x);
                    }
                }
    };
    fold(fullM, T.Tm);
    fold(fullL, T.Tl);
    // M2L per level and source-box offset (ox, oy) = ixy_source - ixy_target, on the
    // scaled coefficients: L_m = sum_k (-1)^m sigma^(m + |k|) K_{k-m}(v) M_k (k < 0:
    // conj(M_|k|)), v = c_target - c_source = -2 R_l (ox + i oy), folded as above
    std::vector<double> K((size_t)2 * P + 1);
    std::vector<double2> A((size_t)P1 * NJ);
    for (int l = 2; l < nl; ++l) {
        const double R = R_level[(size_t)l], sig = lambda * R;
        for (int oy = -3; oy <= 3; ++oy)
            for (int ox = -3; ox <= 3; ++ox) {
                if (std::abs(ox) <= 1 && std::abs(oy) <= 1) continue;
                const double vx = -2.0 * R * ox, vy = -2.0 * R * oy;
                const double x = lambda * std::sqrt(vx * vx + vy * vy);
                const double th = std::atan2(vy, vx);
                double k0, k1;
                bessel::k01(x, k0, k1);
                K[0] = k0;
                K[1] = k1;
                for (int n = 1; n < 2 * P; ++n) K[(size_t)n + 1] = K[(size_t)n - 1] + (2.0 * n / x) * K[(size_t)n];
                for (int m = 0; m <= P; ++m)
                    for (int k = -P; k <= P; ++k) {
                        const int n = k - m;
                        const double mag = ((m & 1) ? -1.0 : 1.0) * std::pow(sig, m + std::abs(k)) * K[(size_t)std::abs(n)];
                        A[(size_t)m * NJ + (size_t)(k + P)] = d2(mag * std::cos(n * th), mag * std::sin(n * th));
                    }
                double2* dst = T.Tv.data() + ((size_t)l * 49 + (size_t)((oy + 3) * 7 + ox + 3)) * 2 * P1 * P1;
                for (int k = 0; k <= P; ++k)
                    for (int m = 0; m <= P; ++m) {
                        const double2 a = A[(size_t)m * NJ + (size_t)(k + P)];
                        const double2 b = k > 0 ? A[(size_t)m * NJ + (size_t)(P - k)] : d2(0.0, 0.0);
                        double2* o = dst + 2 * (size_t)k * P1 + m;
                        if (k == 0) {
                            o[0] = d2(a.x, -a.y);
                            o[P1] = d2(a.y, a.x);
                        } else {
                            o[0] = d2(a.x + b.x, b.y - a.y);
                            o[P1] = d2(a.y + b.y, a.x - b.x);
                        }
                    }
            }
    }
    // float-float copy of the M2L tables, entries divided by m! |k|! (the kernel
    // multiplies M_k by k! and L~_m by m!)
    if (ff) {
        T.Tvf.assign(T.Tv.size(), make_float4(0.f, 0.f, 0.f, 0.f));
        auto split = [](double v, float& h, float& l) {
            h = (float)v;
            l = (float)(v - (double)h);
        };
        for (size_t lo = 0; lo < (size_t)nl * 49; ++lo)
            for (int k = 0; k <= P; ++k)
                for (int m = 0; m <= P; ++m)
                    for (int half = 0; half < 2; ++half) {
                        const size_t i = (lo * P1 + (size_t)k) * 2 * P1 + (size_t)half * P1 + (size_t)m;
                        const double sc = inv_fact[(size_t)m] * inv_fact[(size_t)k];
                        float4 o;
                        split(T.Tv[i].x * sc, o.x, o.y);
                        split(T.Tv[i].y * sc, o.z, o.w);
                        T.Tvf[i] = o;
                    }
        T.Tv.clear();
    }
    // near-field series: per leaf, the terms its largest near-field distance needs
    // (pairs beyond y = 1 take the integral representation) and the split between
    // the float-float head and the FP32 tail of the Horner sums
    std::vector<double> ca(kMaxNearTerms), cb(kMaxNearTerms);
    {
        double a = 1.0, H = 0.0;
        for (int k = 0; k < kMaxNearTerms; ++k) {
            if (k > 0) {
                a /= (double)k * (double)k;
                H += 1.0 / (double)k;
            }
            ca[(size_t)k] = a;
            cb[(size_t)k] = H * a;
        }
    }
    const double c0 = std::log(0.5 * lambda) + bessel::kEulerGamma;
    int deg = 1;
    T.leaf_deg.assign(leaf_dmax.size(), 1 | (2 << 8));
    // ymax rounded up to a power of 2^(1/4) (the bounds grow with ymax), one
    // evaluation per distinct value
    std::vector<int> memo(512, -1);
    for (size_t b = 0; b < leaf_dmax.size(); ++b) {
        const double d = leaf_dmax[b];
        const double y = std::min(1.0, 0.25 * lambda * lambda * d * d);
        const int key = y > 0.0 ? std::max(0, std::min(511, (int)std::floor(-4.0 * std::log2(y)))) : 511;
        if (memo[(size_t)key] < 0) {
            const double yq = std::ldexp(1.0, -key / 4) * std::pow(2.0, -(key % 4) / 4.0);
            const int db = near_degree(yq);
            memo[(size_t)key] = db | (near_split(db, yq, lambda, c0, ca, cb) << 8);
        }
        T.leaf_deg[b] = memo[(size_t)key];
        deg = std::max(deg, memo[(size_t)key] & 0xff);
    }
    T.near_deg = deg;
    T.near_a.assign(ca.begin(), ca.begin() + deg + 1);
    T.near_b.assign(cb.begin(), cb.begin() + deg + 1);
    auto finite = [](const std::vector<double2>& v) {
        for (const double2& z : v)
            if (!std::isfinite(z.x) || !std::isfinite(z.y)) return false;
        return true;
    };
    for (double v : T.spow)
        if (!std::isfinite(v)) return "lambda times the box size is outside the range of the expansions";
    if (!finite(T.Tm) || !finite(T.Tl) || !finite(T.Tv))
        return "lambda times the box size is outside the range of the expansions";
    for (const float4& v : T.Tvf)
        if (!std::isfinite(v.x) || !std::isfinite(v.y) || !std::isfinite(v.z) || !std::isfinite(v.w))
            return "lambda times the box size is outside the range of the float-float M2L";
    return "";
}

double green_mhelm_host(double lambda, double r)
{
    double k0, k1;
    bessel::k01(lambda * r, k0, k1);
    return lambda * lambda * 0.159154943091895335768883763372514362 * k0;
}

}  // namespace vp
