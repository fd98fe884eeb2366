// FMM kernels (Laplace kernel) for the smooth-quadrature point sum of the
// volume potential (arXiv 2203.05933, Eq. Tk_smooth_quad): an all-FP64 set
// (VP_FLAG_FP64, and the target gradient) and the default set in float-float
// arithmetic on the FP32 pipes (k_*_ff), on sm_103a; plus the FP64 reference
// forms of the output and correction steps.
//
// Potential convention inside this file: psi(z) = Re sum_j q_j log(z - z_j),
// so that V = -(1/2pi) psi with G = -(1/2pi) log|r - r0| (Sec. 2.1). The
// complex-variable Laplace expansions are the classical ones (multipole
// a_0 log(z - c) + sum_k a_k / (z - c)^k, local sum_l b_l (z - c)^l), stored
// scaled by the box half-side R so that every coefficient stays O(1):
//   M_k = a_k / R^k,  L_l = b_l R^l.
// Translation operators in scaled form (z0 = source centre - target centre):
//   P2M  M_0 = sum q,  M_k = -(1/k) sum q u^k,              u = (z - c)/R
//   M2M  B_l = -M_0 zeta^l / l + sum_{k<=l} C(l-1,k-1) 2^-k M_k zeta^(l-k)
//   M2L  A_k = M_k (-t)^k, t = R/z0;  L_0 = M_0 log|z0| + sum_k A_k,
//        L_l = t^l (-M_0/l + sum_k C(l+k-1,k-1) A_k)
//   L2L  L'_l = 2^-l sum_{k>=l} C(k,l) zeta^(k-l) L_k
//   P2L  L_0 = q log|z - c|, L_l = -(q/l) v^l,               v = R/(z - c)
//   M2P  M_0 log|z - c| + Re sum_k M_k v^k
//   L2P  Re sum_l L_l u^l
// zeta is the child-centre offset over the parent half-side, (+-1 +- i)/2.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "vp_ff.cuh"
#include "vp_internal.h"

namespace vp {
namespace {

constexpr double kInv2Pi = 0.159154943091895335768883763372514362;
constexpr int kWarpsPerBlock = 4;
constexpr int kLeafThreads = 64;
constexpr int kChunk = 16;  // charges staged per step in P2M / P2L

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// a * b + c
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ int global_warp() { return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int num_warps() { return (int)((gridDim.x * blockDim.x) >> 5); }

int warp_blocks(int64_t nwork)
{
    int64_t b = (nwork + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

// ----------------------------------------------------------------------------
// a1: charges q_j = w_j f_j gathered into tree order, density-fastest layout.
// Also writes each charge as an unevaluated sum of two floats (hi + lo) for the
// float-float near-field kernel.
template <int ND>
__global__ void k_charges(int32_t n, const int32_t* __restrict__ perm, const double* __restrict__ w,
                          const double* __restrict__ f, int64_t ld_f, double* __restrict__ q,
                          float2* __restrict__ qf)
{
    const int64_t total = (int64_t)n * ND;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = (int32_t)(i / ND);
        const int d = (int)(i % ND);
        const double wv = w ? w[s] : 1.0;
        const double v = wv * f[d * ld_f + perm[s]];
        q[i] = v;
        const float hi = __double2float_rn(v);
        qf[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

// ----------------------------------------------------------------------------
// a3: P2M, one warp per leaf; lane k accumulates coefficient k.
template <int P, int ND>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_p2m(DevTree t, PassGeom g, const double* __restrict__ q, double2* __restrict__ M)
{
    constexpr int P1 = P + 1;
    __shared__ double2 pw[kWarpsPerBlock][kChunk][P1];
    __shared__ double qs[kWarpsPerBlock][kChunk][ND];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    for (int li = global_warp(); li < t.nleaf; li += num_warps()) {
        const int b = t.leaves[li];
        const int s0 = g.crng[2 * b], s1 = g.crng[2 * b + 1];
        double2 acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = make_double2(0.0, 0.0);
        const double2 c = t.center[b];
        const double invR = 1.0 / t.radius[b];
        for (int base = s0; base < s1; base += kChunk) {
            const int n = min(kChunk, s1 - base);
            if (lane < n) {
                const double2 z = g.cxy[base + lane];
                const double2 u = make_double2((z.x - c.x) * invR, (z.y - c.y) * invR);
                double2 p = make_double2(1.0, 0.0);
                pw[wb][lane][0] = p;
#pragma unroll 4
                for (int k = 1; k <= P; ++k) {
                    p = cmul(p, u);
                    pw[wb][lane][k] = p;
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) qs[wb][lane][d] = q[(int64_t)(base + lane) * ND + d];
            }
            __syncwarp();
            if (lane <= P) {
                for (int j = 0; j < n; ++j) {
                    const double2 pv = pw[wb][j][lane];
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        acc[d].x = fma(qs[wb][j][d], pv.x, acc[d].x);
                        acc[d].y = fma(qs[wb][j][d], pv.y, acc[d].y);
                    }
                }
            }
            __syncwarp();
        }
        if (lane <= P) {
            const double s = lane == 0 ? 1.0 : -1.0 / (double)lane;
#pragma unroll
            for (int d = 0; d < ND; ++d)
                M[((int64_t)b * P1 + lane) * ND + d] = make_double2(acc[d].x * s, acc[d].y * s);
        }
    }
}

// ----------------------------------------------------------------------------
// a3: M2M for the non-leaf boxes of one level, one warp per parent.
template <int P, int ND>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_m2m(DevTree t, DevTables tab, int b0, int b1, double2* __restrict__ M)
{
    constexpr int P1 = P + 1;
    __shared__ double2 Ms[kWarpsPerBlock][P1][ND];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const double inv_l = lane == 0 ? 0.0 : -1.0 / (double)lane;
    for (int b = b0 + global_warp(); b < b1; b += num_warps()) {
        if (t.is_leaf[b]) continue;
        double2 acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = make_double2(0.0, 0.0);
        for (int c = 0; c < 4; ++c) {
            const int ch = t.child[4 * b + c];
            if (ch < 0) continue;
            if (lane <= P) {
#pragma unroll
                for (int d = 0; d < ND; ++d) Ms[wb][lane][d] = M[((int64_t)ch * P1 + lane) * ND + d];
            }
            __syncwarp();
            if (lane <= P) {
                const double2* zp = tab.zpow + c * P1;
                if (lane == 0) {
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = cadd(acc[d], Ms[wb][0][d]);
                } else {
                    const double2 zl = zp[lane];
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const double m0 = Ms[wb][0][d].x * inv_l;
                        acc[d].x = fma(m0, zl.x, acc[d].x);
                        acc[d].y = fma(m0, zl.y, acc[d].y);
                    }
                    for (int k = 1; k <= lane; ++k) {
                        const double bm = tab.Bm[lane * P1 + k];
                        const double2 z = zp[lane - k];
                        const double2 zb = make_double2(z.x * bm, z.y * bm);
#pragma unroll
                        for (int d = 0; d < ND; ++d) acc[d] = cfma(zb, Ms[wb][k][d], acc[d]);
                    }
                }
            }
            __syncwarp();
        }
        if (lane <= P) {
#pragma unroll
            for (int d = 0; d < ND; ++d) M[((int64_t)b * P1 + lane) * ND + d] = acc[d];
        }
    }
}

// ----------------------------------------------------------------------------
// a4: M2L over the V list plus P2L over the X list, one warp per target box;
// lane l owns local coefficient l. Writes every box's L (zeros if no lists).
template <int P, int ND>
struct M2LSmem {
    static constexpr int P1 = P + 1;
    static constexpr int kA = P1 * ND;                    // double2 per warp, M2L staging
    static constexpr int kPw = kChunk * P1;               // double2 per warp, P2L powers
    static constexpr int kUnion = (kA > kPw + (kChunk * (ND + 1) + 1) / 2) ? kA
                                                                           : kPw + (kChunk * (ND + 1) + 1) / 2;
};

template <int P, int ND>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_m2l(DevTree t, DevTables tab, PassGeom g, const double2* __restrict__ M, double2* __restrict__ L,
          const double* __restrict__ q)
{
    constexpr int P1 = P + 1;
    using S = M2LSmem<P, ND>;
    __shared__ double Hs[P1 * P1];
    __shared__ double2 buf[kWarpsPerBlock][S::kUnion];
    for (int i = threadIdx.x; i < P1 * P1; i += blockDim.x) Hs[i] = tab.H[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    double2(*As)[ND] = reinterpret_cast<double2(*)[ND]>(&buf[wb][0]);
    double2(*pw)[P1] = reinterpret_cast<double2(*)[P1]>(&buf[wb][0]);
    double* qs = reinterpret_cast<double*>(&buf[wb][S::kPw]);  // [kChunk][ND]
    double* lgs = qs + kChunk * ND;                            // [kChunk]
    const double inv_l = lane == 0 ? 0.0 : 1.0 / (double)lane;

    for (int b = global_warp(); b < t.nbox; b += num_warps()) {
        double2 lacc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) lacc[d] = make_double2(0.0, 0.0);
        const int v0 = t.v_ptr[b], v1 = t.v_ptr[b + 1];
        const int x0 = t.x_ptr[b], x1 = t.x_ptr[b + 1];
        const int bx = t.ixy[2 * b], by = t.ixy[2 * b + 1];
        const double logR = t.log_radius[b];
        for (int e = v0; e < v1; ++e) {
            const int C = t.v_idx[e];
            const int o = (t.ixy[2 * C + 1] - by + 3) * 7 + (t.ixy[2 * C] - bx + 3);
            if (lane <= P) {
                const double2 mt = tab.mtpow[o * P1 + lane];
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double2 m = M[((int64_t)C * P1 + lane) * ND + d];
                    As[lane][d] = lane == 0 ? m : cmul(m, mt);
                }
            }
            __syncwarp();
            if (lane <= P) {
                double2 acc[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = make_double2(0.0, 0.0);
                for (int k = 1; k <= P; ++k) {
                    const double h = Hs[lane * P1 + k];
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        acc[d].x = fma(h, As[k][d].x, acc[d].x);
                        acc[d].y = fma(h, As[k][d].y, acc[d].y);
                    }
                }
                if (lane == 0) {
                    const double lz = logR + tab.log2o[o];
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        lacc[d].x += fma(As[0][d].x, lz, acc[d].x);
                        lacc[d].y += acc[d].y;
                    }
                } else {
                    const double2 tl = tab.tpow[o * P1 + lane];
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const double2 a = make_double2(fma(-As[0][d].x, inv_l, acc[d].x),
                                                       fma(-As[0][d].y, inv_l, acc[d].y));
                        lacc[d] = cfma(tl, a, lacc[d]);
                    }
                }
            }
            __syncwarp();
        }
        if (x1 > x0) {
            const double2 c = t.center[b];
            const double R = t.radius[b];
            for (int e = x0; e < x1; ++e) {
                const int C = t.x_idx[e];
                const int s0 = g.crng[2 * C], s1 = g.crng[2 * C + 1];
                for (int base = s0; base < s1; base += kChunk) {
                    const int n = min(kChunk, s1 - base);
                    if (lane < n) {
                        const double2 z = g.cxy[base + lane];
                        const double dx = z.x - c.x, dy = z.y - c.y;
                        const double r2 = dx * dx + dy * dy;
                        const double s = R / r2;
                        const double2 v = make_double2(dx * s, -dy * s);
                        double2 p = make_double2(1.0, 0.0);
                        pw[lane][0] = p;
#pragma unroll 4
                        for (int k = 1; k <= P; ++k) {
                            p = cmul(p, v);
                            pw[lane][k] = p;
                        }
#pragma unroll
                        for (int d = 0; d < ND; ++d) qs[lane * ND + d] = q[(int64_t)(base + lane) * ND + d];
                        lgs[lane] = 0.5 * log(r2);
                    }
                    __syncwarp();
                    if (lane <= P) {
                        for (int j = 0; j < n; ++j) {
                            if (lane == 0) {
#pragma unroll
                                for (int d = 0; d < ND; ++d) lacc[d].x = fma(qs[j * ND + d], lgs[j], lacc[d].x);
                            } else {
                                const double2 pv = pw[j][lane];
#pragma unroll
                                for (int d = 0; d < ND; ++d) {
                                    const double cq = -qs[j * ND + d] * inv_l;
                                    lacc[d].x = fma(cq, pv.x, lacc[d].x);
                                    lacc[d].y = fma(cq, pv.y, lacc[d].y);
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        }
        if (lane <= P) {
#pragma unroll
            for (int d = 0; d < ND; ++d) L[((int64_t)b * P1 + lane) * ND + d] = lacc[d];
        }
    }
}

// ----------------------------------------------------------------------------
// complex float-float times an exact float complex (a power of zeta: every
// component is 0 or a power of two, so each product below is exact)
__device__ __forceinline__ ff::C cmul_exact(ff::C a, float zx, float zy)
{
    const ff::F ax{__fmul_rn(a.re.h, zx), __fmul_rn(a.re.l, zx)}, ay{__fmul_rn(a.re.h, zy), __fmul_rn(a.re.l, zy)};
    const ff::F bx{__fmul_rn(a.im.h, zx), __fmul_rn(a.im.l, zx)}, by{__fmul_rn(a.im.h, zy), __fmul_rn(a.im.l, zy)};
    return ff::C{ff::add(ax, ff::neg(by)), ff::add(ay, bx)};
}

// M2M of one box by one warp: M(b) = sum over children of the shifted child
// multipoles (scaled form: the operator depends only on the child quadrant).
// The children are staged CB at a time (Ms [CB][P1][ND]) so that their loads
// overlap, and each staged child has its own accumulator, so the CB sums
// advance side by side (the box's M2M is on the critical path of the upward
// pass). CG: read the children with L1 bypassed (written by other blocks in
// the same launch).
template <int P, int ND, int CB, bool CG>
__device__ __forceinline__ void m2m_box_ff(const DevTree& t, const DevTables& tab, int b, float4* __restrict__ Mf,
                                           float4 (*Ms)[P + 1][ND], int lane, const ff::F minvl)
{
    constexpr int P1 = P + 1;
    ff::C tot[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) tot[d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
    for (int c0 = 0; c0 < 4; c0 += CB) {
        int chs[CB];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            chs[c] = t.child[4 * b + c0 + c];
            if (chs[c] >= 0 && lane <= P) {
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const float4* src = Mf + ((int64_t)chs[c] * P1 + lane) * ND + d;
                    Ms[c][lane][d] = CG ? __ldcg(src) : *src;
                }
            }
        }
        __syncwarp();
        if (lane <= P) {
            ff::C acc[CB][ND];
#pragma unroll
            for (int c = 0; c < CB; ++c) {
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    acc[c][d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
                    if (chs[c] < 0) continue;
                    const float4 m0 = Ms[c][0][d];
                    if (lane == 0) {
                        acc[c][d] = ff::from_float4(m0);
                    } else {
                        const float2 zl = tab.zpowf[(c0 + c) * P1 + lane];
                        const ff::F a = ff::mul(ff::F{m0.x, m0.y}, minvl);  // -M_0 / l (M_0 is real)
                        acc[c][d] = cmul_exact(ff::C{a, {0.f, 0.f}}, zl.x, zl.y);
                    }
                }
            }
            for (int k = 1; k <= lane; ++k) {
                const float2 bv = tab.Bmf[lane * P1 + k];
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    if (chs[c] < 0) continue;
                    const float2 z = tab.zpowf[(c0 + c) * P1 + lane - k];
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const ff::C mk = ff::from_float4(Ms[c][k][d]);
                        const ff::C bm{ff::mul(mk.re, ff::F{bv.x, bv.y}), ff::mul(mk.im, ff::F{bv.x, bv.y})};
                        acc[c][d] = ff::cadd(acc[c][d], cmul_exact(bm, z.x, z.y));
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < CB; ++c)
#pragma unroll
                for (int d = 0; d < ND; ++d) tot[d] = ff::cnorm(ff::cadd(tot[d], acc[c][d]));
        }
        __syncwarp();
    }
    if (lane <= P) {
#pragma unroll
        for (int d = 0; d < ND; ++d) Mf[((int64_t)b * P1 + lane) * ND + d] = ff::to_float4(tot[d]);
    }
    __syncwarp();
}

// a3/a5 on the FP32 pipes: P2M, M2M and L2L with float-float expansions (same
// operators as the FP64 kernels above; zeta powers are exact in float).
//
// P2M: u = (z - c)/R = 2 rho, rho the leaf-relative coordinate (hi/lo floats).
// With counters (one per box, zero on entry and left zero), the upward pass
// follows in the same launch: a warp that has finished a box counts itself in
// at the parent (after a fence), and the warp that completes the count computes
// the parent's M2M and carries on upwards; nothing waits.
template <int P, int ND>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_p2m_ff(DevTree t, DevTables tab, PassGeom g, const float2* __restrict__ qf, float4* __restrict__ Mf,
             int* __restrict__ counters)
{
    constexpr int P1 = P + 1;
    // per warp: the powers of the staged charges, later the children staged by M2M
    // (CB children at a time in the same space)
    constexpr int kBuf = kChunk * P1;
    constexpr int CB = kChunk / ND >= 4 ? 4 : kChunk / ND;
    static_assert(CB >= 1 && CB * ND <= kChunk, "M2M staging");
    __shared__ float4 sbuf[kWarpsPerBlock][kBuf];
    __shared__ float2 qs[kWarpsPerBlock][kChunk][ND];
    auto pwf = [&](int w, int j, int k) -> float4& { return sbuf[w][j * P1 + k]; };
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int ll = lane <= P ? lane : P;
    const ff::F minvl = ff::neg(ff::F{tab.invlf[ll].x, tab.invlf[ll].y});
    for (int li = global_warp(); li < t.nleaf; li += num_warps()) {
        const int b = t.leaves[li];
        const int s0 = g.crng[2 * b], s1 = g.crng[2 * b + 1];
        ff::C acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
        for (int base = s0; base < s1; base += kChunk) {
            const int n = min(kChunk, s1 - base);
            if (lane < n) {
                const float4 r = g.crho[base + lane];
                const ff::C u{{2.f * r.x, 2.f * r.y}, {2.f * r.z, 2.f * r.w}};
                ff::C p{{1.f, 0.f}, {0.f, 0.f}};
                pwf(wb, lane, 0) = ff::to_float4(p);
                for (int k = 1; k <= P; ++k) {
                    p = ff::cnorm(ff::cmul(p, u));
                    pwf(wb, lane, k) = ff::to_float4(p);
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) qs[wb][lane][d] = qf[(int64_t)(base + lane) * ND + d];
            }
            __syncwarp();
            if (lane <= P) {
                for (int j = 0; j < n; ++j) {
                    const float4 pv = pwf(wb, j, lane);
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const ff::F qq{qs[wb][j][d].x, qs[wb][j][d].y};
                        acc[d].re = ff::add(acc[d].re, ff::mul(qq, ff::F{pv.x, pv.y}));
                        acc[d].im = ff::add(acc[d].im, ff::mul(qq, ff::F{pv.z, pv.w}));
                    }
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = ff::cnorm(acc[d]);
            }
            __syncwarp();
        }
        if (lane <= P) {
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                ff::C m = acc[d];
                if (lane > 0) m = ff::cnorm(ff::C{ff::mul(m.re, minvl), ff::mul(m.im, minvl)});
                Mf[((int64_t)b * P1 + lane) * ND + d] = ff::to_float4(m);
            }
        }
        if (counters) {
            for (int cur = b;;) {
                const int par = t.parent[cur];
                // multipoles of levels 0 and 1 are never read (V, W and X lists start at level 2)
                if (par < 0 || t.level[par] < 2) break;
                __threadfence();  // this warp's M(cur) before its arrival at the parent
                __syncwarp();
                int old = 0;
                if (lane == 0) old = atomicAdd(&counters[par], 1);
                old = __shfl_sync(0xffffffffu, old, 0);
                int nch = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) nch += t.child[4 * par + c] >= 0 ? 1 : 0;
                if (old != nch - 1) break;  // a sibling is still running; it will carry on
                __threadfence();            // the siblings' M before reading them
                if (lane == 0) counters[par] = 0;
                m2m_box_ff<P, ND, CB, true>(t, tab, par, Mf, reinterpret_cast<float4(*)[P1][ND]>(&sbuf[wb][0]), lane, minvl);
                cur = par;
            }
        }
    }
}

template <int P, int ND>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_l2l_ff(DevTree t, DevTables tab, int b0, int b1, float4* __restrict__ Lf)
{
    constexpr int P1 = P + 1;
    __shared__ float4 Ls[kWarpsPerBlock][P1][ND];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    for (int b = b0 + global_warp(); b < b1; b += num_warps()) {
        const int p = t.parent[b];
        const int cq = (t.ixy[2 * b] & 1) | ((t.ixy[2 * b + 1] & 1) << 1);
        if (lane <= P) {
#pragma unroll
            for (int d = 0; d < ND; ++d) Ls[wb][lane][d] = Lf[((int64_t)p * P1 + lane) * ND + d];
        }
        __syncwarp();
        if (lane <= P) {
            const float2* zp = tab.zpowf + cq * P1;
            ff::C acc[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
            for (int k = lane; k <= P; ++k) {
                const float2 bv = tab.Blf[lane * P1 + k];
                const float2 z = zp[k - lane];
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const ff::C lk = ff::from_float4(Ls[wb][k][d]);
                    const ff::C bl{ff::mul(lk.re, ff::F{bv.x, bv.y}), ff::mul(lk.im, ff::F{bv.x, bv.y})};
                    acc[d] = ff::cadd(acc[d], cmul_exact(bl, z.x, z.y));
                }
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const int64_t i = ((int64_t)b * P1 + lane) * ND + d;
                Lf[i] = ff::to_float4(ff::cnorm(ff::cadd(ff::from_float4(Lf[i]), acc[d])));
            }
        }
        __syncwarp();
    }
}

// a4 on the FP32 pipes: the same M2L as k_m2l (scaled Hankel form) and the same
// X-list P2L, with multipoles, operator tables and accumulators in float-float
// (about 48 significant bits). One warp per target box, lane l owns L_l.
constexpr int kChunkF = 8;  // charges staged per step in the float-float P2L

template <int P, int ND>
struct M2LffSmem {
    static constexpr int P1 = P + 1;
    static constexpr int kA = 2 * P1 * ND;                               // V-list staging (float4), two halves
    static constexpr int kPw = kChunkF * P1;                             // P2L powers (float4)
    static constexpr int kX = kPw + (kChunkF * (ND + 1) * 2 + 3) / 4;    // + charges and logs (float2)
    static constexpr int kUnion = kA > kX ? kA : kX;
};

template <int P, int ND>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_m2l_ff(DevTree t, DevTables tab, PassGeom g, const float4* __restrict__ Mf, float4* __restrict__ Lf,
             const float2* __restrict__ qf)
{
    constexpr int P1 = P + 1;
    using S = M2LffSmem<P, ND>;
    __shared__ float2 Hs[P1 * P1];
    __shared__ float4 buf[kWarpsPerBlock][S::kUnion];  // V-list staging or P2L powers (never both at once)
    __shared__ float4 s_tab[128];
    for (int i = threadIdx.x; i < P1 * P1; i += blockDim.x) Hs[i] = tab.Hf[i];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) s_tab[i] = tab.logtab[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    float4(*As)[ND] = reinterpret_cast<float4(*)[ND]>(&buf[wb][0]);
    float4(*pw)[P1] = reinterpret_cast<float4(*)[P1]>(&buf[wb][0]);
    float2* qs = reinterpret_cast<float2*>(&buf[wb][S::kPw]);  // [kChunkF][ND]
    float2* lgs = qs + kChunkF * ND;                            // [kChunkF]
    const int ll = lane <= P ? lane : P;
    const ff::F invlf = ff::F{tab.invlf[ll].x, tab.invlf[ll].y};

    for (int b = global_warp(); b < t.nbox; b += num_warps()) {
        ff::C lacc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) lacc[d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
        const int v0 = t.v_ptr[b], v1 = t.v_ptr[b + 1];
        const int x0 = t.x_ptr[b], x1 = t.x_ptr[b + 1];
        const int bx = t.ixy[2 * b], by = t.ixy[2 * b + 1];
        const ff::F logR = ff::from_double(t.log_radius[b]);
        if constexpr (P == 16) {
            // 17 coefficients: each half-warp takes every other V-list entry, lane
            // hl of a half computes L_hl, and L_16 is summed across the half
            // (one term per lane, then a 4-step exchange); the halves are added
            // at the end, with L_16 placed in lane 16.
            const int h = lane >> 4, hl = lane & 15;
            float4(*Ah)[ND] = reinterpret_cast<float4(*)[ND]>(&buf[wb][h * P1 * ND]);
            const ff::F invh{tab.invlf[hl].x, tab.invlf[hl].y};
            const ff::F inv16{tab.invlf[16].x, tab.invlf[16].y};
            ff::C l16[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) l16[d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
            for (int it = v0; it < v1; it += 2) {
                const int e = it + h;
                const bool ok = e < v1;
                int o = 0;
                if (ok) {
                    const int C = t.v_idx[e];
                    o = (t.ixy[2 * C + 1] - by + 3) * 7 + (t.ixy[2 * C] - bx + 3);
                    const ff::C mt = ff::from_float4(tab.mtpowf[o * P1 + hl]);
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const ff::C m = ff::from_float4(Mf[((int64_t)C * P1 + hl) * ND + d]);
                        Ah[hl][d] = ff::to_float4(hl == 0 ? m : ff::cnorm(ff::cmul(m, mt)));
                    }
                    if (hl == 0) {
                        const ff::C mt16 = ff::from_float4(tab.mtpowf[o * P1 + 16]);
#pragma unroll
                        for (int d = 0; d < ND; ++d)
                            Ah[16][d] = ff::to_float4(
                                ff::cnorm(ff::cmul(ff::from_float4(Mf[((int64_t)C * P1 + 16) * ND + d]), mt16)));
                    }
                }
                __syncwarp();
                ff::C part[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) part[d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
                if (ok) {
                    ff::C acc[ND];
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
                    for (int k = 1; k <= 16; ++k) {
                        const float2 hv = Hs[hl * P1 + k];
                        const ff::F hh{hv.x, hv.y};
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            const float4 a = Ah[k][d];
                            acc[d].re = ff::add(acc[d].re, ff::mul(hh, ff::F{a.x, a.y}));
                            acc[d].im = ff::add(acc[d].im, ff::mul(hh, ff::F{a.z, a.w}));
                        }
                    }
                    if (hl == 0) {
                        const float2 lo = tab.log2of[o];
                        const ff::F lz = ff::add(logR, ff::F{lo.x, lo.y});
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            const float4 a0 = Ah[0][d];
                            lacc[d].re = ff::add(lacc[d].re, ff::add(acc[d].re, ff::mul(ff::F{a0.x, a0.y}, lz)));
                            lacc[d].im = ff::add(lacc[d].im, acc[d].im);
                        }
                    } else {
                        const ff::C tl = ff::from_float4(tab.tpowf[o * P1 + hl]);
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            const float4 a0 = Ah[0][d];
                            const ff::C a{ff::add(acc[d].re, ff::neg(ff::mul(ff::F{a0.x, a0.y}, invh))),
                                          ff::add(acc[d].im, ff::neg(ff::mul(ff::F{a0.z, a0.w}, invh)))};
                            lacc[d] = ff::cadd(lacc[d], ff::cmul(tl, ff::cnorm(a)));
                        }
                    }
#pragma unroll
                    for (int d = 0; d < ND; ++d) lacc[d] = ff::cnorm(lacc[d]);
                    // this lane's term of L_16: H[16][hl + 1] A_(hl + 1)
                    const float2 hv = Hs[16 * P1 + hl + 1];
                    const ff::F hh{hv.x, hv.y};
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const float4 a = Ah[hl + 1][d];
                        part[d] = ff::C{ff::mul(hh, ff::F{a.x, a.y}), ff::mul(hh, ff::F{a.z, a.w})};
                    }
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    for (int sh = 8; sh > 0; sh >>= 1) {
                        const ff::C other{{__shfl_xor_sync(0xffffffffu, part[d].re.h, sh, 16),
                                           __shfl_xor_sync(0xffffffffu, part[d].re.l, sh, 16)},
                                          {__shfl_xor_sync(0xffffffffu, part[d].im.h, sh, 16),
                                           __shfl_xor_sync(0xffffffffu, part[d].im.l, sh, 16)}};
                        part[d] = ff::cadd(part[d], other);
                    }
                }
                if (ok) {
                    const ff::C t16 = ff::from_float4(tab.tpowf[o * P1 + 16]);
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const float4 a0 = Ah[0][d];
                        const ff::C a{ff::add(part[d].re, ff::neg(ff::mul(ff::F{a0.x, a0.y}, inv16))),
                                      ff::add(part[d].im, ff::neg(ff::mul(ff::F{a0.z, a0.w}, inv16)))};
                        l16[d] = ff::cnorm(ff::cadd(l16[d], ff::cmul(t16, ff::cnorm(a))));
                    }
                }
                __syncwarp();
            }
            // add the halves: lanes 0..15 hold L_0..L_15, lane 16 takes L_16
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const ff::C ol{{__shfl_xor_sync(0xffffffffu, lacc[d].re.h, 16),
                                __shfl_xor_sync(0xffffffffu, lacc[d].re.l, 16)},
                               {__shfl_xor_sync(0xffffffffu, lacc[d].im.h, 16),
                                __shfl_xor_sync(0xffffffffu, lacc[d].im.l, 16)}};
                const ff::C o16{{__shfl_xor_sync(0xffffffffu, l16[d].re.h, 16),
                                 __shfl_xor_sync(0xffffffffu, l16[d].re.l, 16)},
                                {__shfl_xor_sync(0xffffffffu, l16[d].im.h, 16),
                                 __shfl_xor_sync(0xffffffffu, l16[d].im.l, 16)}};
                if (lane < 16) lacc[d] = ff::cnorm(ff::cadd(lacc[d], ol));
                else if (lane == 16) lacc[d] = ff::cnorm(ff::cadd(l16[d], o16));
            }
        } else
        for (int e = v0; e < v1; ++e) {
            const int C = t.v_idx[e];
            const int o = (t.ixy[2 * C + 1] - by + 3) * 7 + (t.ixy[2 * C] - bx + 3);
            if (lane <= P) {
                const ff::C mt = ff::from_float4(tab.mtpowf[o * P1 + lane]);
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const ff::C m = ff::from_float4(Mf[((int64_t)C * P1 + lane) * ND + d]);
                    As[lane][d] = ff::to_float4(lane == 0 ? m : ff::cnorm(ff::cmul(m, mt)));
                }
            }
            __syncwarp();
            if (lane <= P) {
                ff::C acc[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = ff::C{{0.f, 0.f}, {0.f, 0.f}};
                for (int k = 1; k <= P; ++k) {
                    const float2 hv = Hs[lane * P1 + k];
                    const ff::F h{hv.x, hv.y};
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const float4 a = As[k][d];
                        acc[d].re = ff::add(acc[d].re, ff::mul(h, ff::F{a.x, a.y}));
                        acc[d].im = ff::add(acc[d].im, ff::mul(h, ff::F{a.z, a.w}));
                    }
                }
                if (lane == 0) {
                    const float2 lo = tab.log2of[o];
                    const ff::F lz = ff::add(logR, ff::F{lo.x, lo.y});
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const float4 a0 = As[0][d];
                        lacc[d].re = ff::add(lacc[d].re, ff::add(acc[d].re, ff::mul(ff::F{a0.x, a0.y}, lz)));
                        lacc[d].im = ff::add(lacc[d].im, acc[d].im);
                    }
                } else {
                    const ff::C tl = ff::from_float4(tab.tpowf[o * P1 + lane]);
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const float4 a0 = As[0][d];
                        const ff::C a{ff::add(acc[d].re, ff::neg(ff::mul(ff::F{a0.x, a0.y}, invlf))),
                                      ff::add(acc[d].im, ff::neg(ff::mul(ff::F{a0.z, a0.w}, invlf)))};
                        lacc[d] = ff::cadd(lacc[d], ff::cmul(tl, ff::cnorm(a)));
                    }
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) lacc[d] = ff::cnorm(lacc[d]);
            }
            __syncwarp();
        }
        // P2L over X: w = (z - c_b)/side_b (exact leaf offset + scaled leaf-relative
        // coordinate), v = R_b/(z - c_b) = 1/(2w), L_l += -(q/l) v^l,
        // L_0 += q log|z - c_b| = q (1/2 log|w|^2 + log side_b)
        if (x1 > x0) {
            const ff::F logside = ff::from_double(t.log_radius[b] + 0.693147180559945309417232121458176568);
            for (int e = x0; e < x1; ++e) {
                const int C = t.x_idx[e];
                const int s0 = g.crng[2 * C], s1 = g.crng[2 * C + 1];
                const float4 xo = t.x_off[e];
                for (int base = s0; base < s1; base += kChunkF) {
                    const int n = min(kChunkF, s1 - base);
                    if (lane < n) {
                        const float4 r = g.crho[base + lane];
                        const ff::F wx = ff::shift_scale(xo.x, xo.z, r.x, r.y);
                        const ff::F wy = ff::shift_scale(xo.y, xo.z, r.z, r.w);
                        const ff::F n2 = ff::norm(ff::add(ff::mul(wx, wx), ff::mul(wy, wy)));
                        const ff::F rn = ff::recip(n2);
                        const ff::F hr = ff::F{0.5f * rn.h, 0.5f * rn.l};
                        const ff::C v{ff::norm(ff::mul(wx, hr)), ff::norm(ff::neg(ff::mul(wy, hr)))};
                        ff::C pwr{{1.f, 0.f}, {0.f, 0.f}};
                        pw[lane][0] = ff::to_float4(pwr);
                        for (int k = 1; k <= P; ++k) {
                            pwr = ff::cnorm(ff::cmul(pwr, v));
                            pw[lane][k] = ff::to_float4(pwr);
                        }
                        float Sl, lol;
                        ff::log_pair(n2.h, n2.l, s_tab, Sl, lol);
                        const ff::F lg = ff::norm(ff::add(ff::F{0.5f * Sl, 0.5f * lol}, logside));
                        lgs[lane] = make_float2(lg.h, lg.l);
#pragma unroll
                        for (int d = 0; d < ND; ++d) qs[lane * ND + d] = qf[(int64_t)(base + lane) * ND + d];
                    }
                    __syncwarp();
                    if (lane <= P) {
                        for (int j = 0; j < n; ++j) {
                            if (lane == 0) {
                                const ff::F lg{lgs[j].x, lgs[j].y};
#pragma unroll
                                for (int d = 0; d < ND; ++d)
                                    lacc[d].re = ff::add(lacc[d].re, ff::mul(ff::F{qs[j * ND + d].x, qs[j * ND + d].y}, lg));
                            } else {
                                const float4 pv = pw[j][lane];
#pragma unroll
                                for (int d = 0; d < ND; ++d) {
                                    const ff::F cq = ff::neg(ff::mul(ff::F{qs[j * ND + d].x, qs[j * ND + d].y}, invlf));
                                    lacc[d].re = ff::add(lacc[d].re, ff::mul(cq, ff::F{pv.x, pv.y}));
                                    lacc[d].im = ff::add(lacc[d].im, ff::mul(cq, ff::F{pv.z, pv.w}));
                                }
                            }
                        }
#pragma unroll
                        for (int d = 0; d < ND; ++d) lacc[d] = ff::cnorm(lacc[d]);
                    }
                    __syncwarp();
                }
            }
        }
        if (lane <= P) {
#pragma unroll
            for (int d = 0; d < ND; ++d) Lf[((int64_t)b * P1 + lane) * ND + d] = ff::to_float4(lacc[d]);
        }
    }
}

// ----------------------------------------------------------------------------
// a5: L2L from parents into the boxes of one level, one warp per child.
template <int P, int ND>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_l2l(DevTree t, DevTables tab, int b0, int b1, double2* __restrict__ L)
{
    constexpr int P1 = P + 1;
    __shared__ double2 Ls[kWarpsPerBlock][P1][ND];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    for (int b = b0 + global_warp(); b < b1; b += num_warps()) {
        const int p = t.parent[b];
        const int cq = (t.ixy[2 * b] & 1) | ((t.ixy[2 * b + 1] & 1) << 1);
        if (lane <= P) {
#pragma unroll
            for (int d = 0; d < ND; ++d) Ls[wb][lane][d] = L[((int64_t)p * P1 + lane) * ND + d];
        }
        __syncwarp();
        if (lane <= P) {
            const double2* zp = tab.zpow + cq * P1;
            double2 acc[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[d] = make_double2(0.0, 0.0);
            for (int k = lane; k <= P; ++k) {
                const double bl = tab.Bl[lane * P1 + k];
                const double2 z = zp[k - lane];
                const double2 zb = make_double2(z.x * bl, z.y * bl);
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = cfma(zb, Ls[wb][k][d], acc[d]);
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const int64_t i = ((int64_t)b * P1 + lane) * ND + d;
                L[i] = cadd(L[i], acc[d]);
            }
        }
        __syncwarp();
    }
}

// ----------------------------------------------------------------------------
// a5 + a6: per leaf, L2P + M2P over the W list + direct P2P over the U list.
// GRAD = false: psi[e][d] = Re phi(z_e). GRAD = true: psi[e][0..1][d] = grad Re phi.
template <int P, int ND, bool GRAD>
__global__ void __launch_bounds__(kLeafThreads)
    k_leaf(DevTree t, PassGeom g, const double* __restrict__ q, const double2* __restrict__ M,
           const double2* __restrict__ L, double* __restrict__ psi)
{
    constexpr int P1 = P + 1;
    __shared__ double2 Cs[P1][ND];
    __shared__ double2 sxy[kLeafThreads];
    __shared__ double sq[kLeafThreads][ND];
    const int tid = threadIdx.x;
    for (int li = blockIdx.x; li < t.nleaf; li += gridDim.x) {
        const int b = t.leaves[li];
        const int e0 = g.erng[2 * b], e1 = g.erng[2 * b + 1];
        if (e0 == e1) continue;
        const double2 cb = t.center[b];
        const double Rb = t.radius[b];
        const double invRb = 1.0 / Rb;
        const int u0 = t.u_ptr[b], u1 = t.u_ptr[b + 1];
        const int w0 = t.w_ptr[b], w1 = t.w_ptr[b + 1];
        for (int tb = e0; tb < e1; tb += kLeafThreads) {
            const int ti = tb + tid;
            const bool valid = ti < e1;
            const double2 z = valid ? g.exy[ti] : cb;
            double acc[ND], acy[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[d] = acy[d] = 0.0;

            // L2P
            __syncthreads();
            for (int i = tid; i < P1 * ND; i += kLeafThreads) (&Cs[0][0])[i] = L[(int64_t)b * P1 * ND + i];
            __syncthreads();
            if (valid) {
                const double2 u = make_double2((z.x - cb.x) * invRb, (z.y - cb.y) * invRb);
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    if (!GRAD) {
                        double2 s = Cs[P][d];
                        for (int l = P - 1; l >= 0; --l) s = cfma(s, u, Cs[l][d]);
                        acc[d] += s.x;
                    } else {
                        double2 s = make_double2(Cs[P][d].x * P, Cs[P][d].y * P);
                        for (int l = P - 1; l >= 1; --l)
                            s = cfma(s, u, make_double2(Cs[l][d].x * l, Cs[l][d].y * l));
                        acc[d] += s.x * invRb;
                        acy[d] -= s.y * invRb;
                    }
                }
            }
            // M2P over W
            for (int e = w0; e < w1; ++e) {
                const int D = t.w_idx[e];
                __syncthreads();
                for (int i = tid; i < P1 * ND; i += kLeafThreads) (&Cs[0][0])[i] = M[(int64_t)D * P1 * ND + i];
                __syncthreads();
                if (valid) {
                    const double2 cD = t.center[D];
                    const double RD = t.radius[D];
                    const double dx = z.x - cD.x, dy = z.y - cD.y;
                    const double r2 = dx * dx + dy * dy;
                    const double2 inv = make_double2(dx / r2, -dy / r2);
                    const double2 v = make_double2(inv.x * RD, inv.y * RD);
                    if (!GRAD) {
                        const double lg = 0.5 * log(r2);
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            double2 s = make_double2(0.0, 0.0);
                            for (int k = P; k >= 1; --k) s = cmul(cadd(s, Cs[k][d]), v);
                            acc[d] += fma(Cs[0][d].x, lg, s.x);
                        }
                    } else {
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            double2 s = make_double2(0.0, 0.0);
                            for (int k = P; k >= 1; --k)
                                s = cmul(cadd(s, make_double2(Cs[k][d].x * k, Cs[k][d].y * k)), v);
                            const double2 dphi = cmul(inv, make_double2(Cs[0][d].x - s.x, Cs[0][d].y - s.y));
                            acc[d] += dphi.x;
                            acy[d] -= dphi.y;
                        }
                    }
                }
            }
            // P2P over U
            for (int e = u0; e < u1; ++e) {
                const int A = t.u_idx[e];
                const int a0 = g.crng[2 * A], a1 = g.crng[2 * A + 1];
                for (int sb = a0; sb < a1; sb += kLeafThreads) {
                    const int n = min(kLeafThreads, a1 - sb);
                    __syncthreads();
                    if (tid < n) {
                        sxy[tid] = g.cxy[sb + tid];
#pragma unroll
                        for (int d = 0; d < ND; ++d) sq[tid][d] = q[(int64_t)(sb + tid) * ND + d];
                    }
                    __syncthreads();
                    if (valid) {
                        for (int j = 0; j < n; ++j) {
                            const double dx = z.x - sxy[j].x, dy = z.y - sxy[j].y;
                            if (dx == 0.0 && dy == 0.0) continue;  // coincident pair: no smooth term
                            const double r2 = dx * dx + dy * dy;
                            if (!GRAD) {
                                const double lg = 0.5 * log(r2);
#pragma unroll
                                for (int d = 0; d < ND; ++d) acc[d] = fma(sq[j][d], lg, acc[d]);
                            } else {
                                const double ir = 1.0 / r2;
                                const double gx = dx * ir, gy = dy * ir;
#pragma unroll
                                for (int d = 0; d < ND; ++d) {
                                    acc[d] = fma(sq[j][d], gx, acc[d]);
                                    acy[d] = fma(sq[j][d], gy, acy[d]);
                                }
                            }
                        }
                    }
                }
            }
            if (valid) {
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    if (!GRAD) {
                        psi[(int64_t)ti * ND + d] = acc[d];
                    } else {
                        psi[((int64_t)ti * 2 + 0) * ND + d] = acc[d];
                        psi[((int64_t)ti * 2 + 1) * ND + d] = acy[d];
                    }
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------
// a5 + a6, float-float near field. Same result as k_leaf<.., false>, but the
// direct sum over the U list runs on the FP32 pipes (64x the FP64 rate on this
// part) in float-float arithmetic: every quantity is an unevaluated sum hi + lo
// of two floats, carried with error-free transformations (TwoSum, FMA-based
// TwoProd), which keeps about 48 significant bits.
//
// Per pair, in units of the target leaf's side (so r2 stays within a few
// binades of 1):
//   dx, dy   from leaf-relative coordinates (exact leaf-centre offsets)
//   r2       = dx^2 + dy^2 (hi, lo)
//   log r2   = e ln2 + T_k + log1p(u),  r2 = 2^e m, m in [1, 2),
//              k = top 7 bits of m, u = m / c_k - 1 (|u| <= 2^-8),
//              T_k = log c_k from a 128-entry table, log1p by its series to u^5.
//            The exponent is limited to |e| <= 15 so that e * ln2_hi + T_hi is
//            exact in one float (ln2_hi and T_hi have 19 fractional bits);
//            other pairs (and only those) take an FP64 log.
//   psi     += q * log r2 (hi, lo), accumulated with TwoSum.
// Absolute error of one log r2 is below about 3e-12; the result is converted
// to FP64 once per target and combined with the leaf-size term
// log(side) * (sum of the U-list charges minus coincident ones).
// Float-float direct sum of one target over a staged tile of charges:
// ah + al += sum_k q_k log r_k'^2, coincident charges collected in qco.
// EXACT: the hi parts of target and source differ exactly in float.
template <int ND, bool EXACT>
__device__ __forceinline__ void p2p_tile(const float4 rt, const float4* __restrict__ s_rho,
                                         const float2 (*__restrict__ s_q)[ND], int n,
                                         const float4* __restrict__ s_tab, float* ah, float* al, ff::F* qco)
{
#pragma unroll 4
    for (int k = 0; k < n; ++k) {
        const float4 sr = s_rho[k];
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
        // r2 = px + py by Fast2Sum (both are >= 0, so the larger one goes first)
        const float rs = __fadd_rn(px, py);
        float re = __fsub_rn(fminf(px, py), __fsub_rn(rs, fmaxf(px, py)));
        re = __fadd_rn(re, __fadd_rn(pxe, pye));
        float S, lo;
        if (rs >= 0x1p-15f && rs < 0x1p16f) {
            ff::log_pair_fast(rs, re, s_tab, S, lo);  // (rs, re) need not be renormalised
        } else {
            if (rs == 0.0f && re == 0.0f) {  // bitwise-coincident pair: no smooth term
#pragma unroll
                for (int d = 0; d < ND; ++d) qco[d] = ff::add(qco[d], ff::F{s_q[k][d].x, s_q[k][d].y});
                continue;
            }
            const double ld = log((double)rs + (double)re);
            S = __double2float_rn(ld);
            lo = __double2float_rn(ld - (double)S);
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const float2 qq = s_q[k][d];
            const float p = __fmul_rn(qq.x, S);
            float pe = fmaf(qq.x, S, -p);
            pe = fmaf(qq.x, lo, pe);
            pe = fmaf(qq.y, S, pe);
            float sh, se;
            ff::two_sum(ah[d], p, sh, se);
            ah[d] = sh;
            al[d] = __fadd_rn(al[d], __fadd_rn(se, pe));
        }
    }
}

// Symmetric pass over one chunk of at most 32 sources of a leaf A for the 32
// targets of one warp (targets are the charge points of the warp's own leaf b,
// A != b, so no pair coincides). At step t lane l takes source (l + t) mod 32:
// it adds q_j log r^2 to its own target and q_i log r^2 (q_i the charge at its
// target) to a float-float accumulator for that source, and the accumulators
// move one lane down after each step; after 32 steps lane l holds the sum over
// the warp's targets for source l. rh, rl must be zero on entry. FULL: 32
// sources and 32 valid targets (no per-step test).
template <int ND, bool EXACT, bool FULL = false>
__device__ __forceinline__ void p2p_chunk_sym(const float4 rt, const float2* qi, bool valid_i,
                                              const float4* __restrict__ s_rho,
                                              const float2 (*__restrict__ s_q)[ND], int n, int lane,
                                              const float4* __restrict__ s_tab, float* ah, float* al, float* rh,
                                              float* rl)
{
#pragma unroll 2
    for (int t = 0; t < 32; ++t) {
        const int j = (lane + t) & 31;
        if (FULL || (valid_i && j < n)) {
            const float4 sr = s_rho[j];
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
            float S, lo;
            if (rs >= 0x1p-15f && rs < 0x1p16f) {
                ff::log_pair_fast(rs, re, s_tab, S, lo);
            } else if (rs == 0.0f && re == 0.0f) {
                S = lo = 0.0f;  // not reached for distinct leaves
            } else {
                const double ld = log((double)rs + (double)re);
                S = __double2float_rn(ld);
                lo = __double2float_rn(ld - (double)S);
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const float2 qq = s_q[j][d];
                const float p = __fmul_rn(qq.x, S);
                float pe = fmaf(qq.x, S, -p);
                pe = fmaf(qq.x, lo, pe);
                pe = fmaf(qq.y, S, pe);
                float sh, se;
                ff::two_sum(ah[d], p, sh, se);
                ah[d] = sh;
                al[d] = __fadd_rn(al[d], __fadd_rn(se, pe));
                const float r = __fmul_rn(qi[d].x, S);
                float re2 = fmaf(qi[d].x, S, -r);
                re2 = fmaf(qi[d].x, lo, re2);
                re2 = fmaf(qi[d].y, S, re2);
                ff::two_sum(rh[d], r, sh, se);
                rh[d] = sh;
                rl[d] = __fadd_rn(rl[d], __fadd_rn(se, re2));
            }
        }
        const int from = (lane + 1) & 31;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            rh[d] = __shfl_sync(0xffffffffu, rh[d], from);
            rl[d] = __shfl_sync(0xffffffffu, rl[d], from);
        }
    }
}

// Symmetric pass over the warp's own group of at most 32 points (targets and
// charges are the same points of leaf b, no two coincident): at step t = 1..16
// lane l takes point j = (l + t) mod 32 (at t = 16 only lanes l < 16, so that
// each pair is taken once), adds q_j log r^2 to its own sum and sends
// q_l log r^2 to lane j by a shuffle.
template <int ND>
__device__ __forceinline__ void p2p_diag_sym(const float4 rt, const float2* qi, bool valid_i,
                                             const float4* __restrict__ s_rho,
                                             const float2 (*__restrict__ s_q)[ND], int n, int lane,
                                             const float4* __restrict__ s_tab, float* ah, float* al)
{
    for (int t = 1; t <= 16; ++t) {
        const int j = (lane + t) & 31;
        float vh[ND], vl[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) vh[d] = vl[d] = 0.f;
        if (valid_i && j < n && (t < 16 || lane < 16)) {
            const float4 sr = s_rho[j];
            const float dxs = __fsub_rn(rt.x, sr.x), dxe = __fsub_rn(rt.y, sr.y);
            const float dys = __fsub_rn(rt.z, sr.z), dye = __fsub_rn(rt.w, sr.w);
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
            float S, lo;
            ff::log_pair(rs, re, s_tab, S, lo);
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const float2 qq = s_q[j][d];
                const float p = __fmul_rn(qq.x, S);
                float pe = fmaf(qq.x, S, -p);
                pe = fmaf(qq.x, lo, pe);
                pe = fmaf(qq.y, S, pe);
                float sh, se;
                ff::two_sum(ah[d], p, sh, se);
                ah[d] = sh;
                al[d] = __fadd_rn(al[d], __fadd_rn(se, pe));
                const float r = __fmul_rn(qi[d].x, S);
                float re2 = fmaf(qi[d].x, S, -r);
                re2 = fmaf(qi[d].x, lo, re2);
                re2 = fmaf(qi[d].y, S, re2);
                vh[d] = r;
                vl[d] = re2;
            }
        }
        const int from = (lane - t) & 31;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const float rh = __shfl_sync(0xffffffffu, vh[d], from);
            const float rl = __shfl_sync(0xffffffffu, vl[d], from);
            float sh, se;
            ff::two_sum(ah[d], rh, sh, se);
            ah[d] = sh;
            al[d] = __fadd_rn(al[d], __fadd_rn(se, rl));
        }
    }
}

template <int P, int ND, bool SYM>
__global__ void __launch_bounds__(kLeafThreads)
    k_leaf_ff(DevTree t, PassGeom g, const float2* __restrict__ qf, const float4* __restrict__ Mf,
              const float4* __restrict__ Lf, const float4* __restrict__ logtab, double* __restrict__ psi,
              int* __restrict__ work, float2* __restrict__ slots)
{
    constexpr int P1 = P + 1;
    __shared__ double2 Cs[P1][ND];
    __shared__ float4 s_L[P1 * ND];
    __shared__ float4 s_rho[kLeafThreads];
    __shared__ float2 s_q[kLeafThreads][ND];
    __shared__ float4 s_tab[128];
    // own-leaf pairs between groups g < c of 32 points: the sums for group c's
    // points made by group g's warp, [pair (g, c)][lane][d]
    constexpr bool kOwn = SYM && ND <= 2;
    static_assert(kLeafThreads == 64, "the own-leaf hand-over assumes passes of two groups of 32 targets");
    constexpr int kOwnPairs = kOwnGroups * (kOwnGroups - 1) / 2;
    __shared__ float2 s_own[kOwn ? kOwnPairs : 1][32][kOwn ? ND : 1];
    const int tid = threadIdx.x;
    for (int i = tid; i < 128; i += kLeafThreads) s_tab[i] = logtab[i];
    // persistent blocks pull leaves from a queue (leaves are stored costliest first)
    __shared__ int s_next;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_next = atomicAdd(work, 1);
        __syncthreads();
        const int li = s_next;
        if (li >= t.nleaf) break;
        const int b = SYM ? t.sym_leaves[li] : t.leaves[li];
        const int e0 = g.erng[2 * b], e1 = g.erng[2 * b + 1];
        if (e0 == e1) continue;
        const double log_side = t.log_radius[b] + 0.693147180559945309417232121458176568;
        const bool own_sym = kOwn && t.sym_own[b] != 0;  // block-uniform
        const int u0 = t.u_ptr[b], u1 = t.u_ptr[b + 1];
        const int w0 = t.w_ptr[b], w1 = t.w_ptr[b + 1];
        for (int tb = e0; tb < e1; tb += kLeafThreads) {
            const int ti = tb + tid;
            const bool valid = ti < e1;
            const float4 rt = valid ? g.erho[ti] : make_float4(0.f, 0.f, 0.f, 0.f);
            double acc[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[d] = 0.0;

            // L2P (float-float, u = (z - c)/R = 2 rho_t)
            __syncthreads();
            for (int i = tid; i < P1 * ND; i += kLeafThreads) s_L[i] = Lf[(int64_t)b * P1 * ND + i];
            __syncthreads();
            if (valid) {
                const ff::C u{{2.f * rt.x, 2.f * rt.y}, {2.f * rt.z, 2.f * rt.w}};
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    ff::C sacc = ff::from_float4(s_L[P * ND + d]);
                    for (int l = P - 1; l >= 0; --l)
                        sacc = ff::cnorm(ff::cadd(ff::cmul(sacc, u), ff::from_float4(s_L[l * ND + d])));
                    acc[d] += ff::to_double(sacc.re);
                }
            }
            // M2P over W (FP64; adaptive refinement boundaries only)
            if (w1 > w0) {
                const double2 z = valid ? g.exy[ti] : t.center[b];
                for (int e = w0; e < w1; ++e) {
                    const int D = t.w_idx[e];
                    __syncthreads();
                    for (int i = tid; i < P1 * ND; i += kLeafThreads)
                        (&Cs[0][0])[i] = ff::to_double2(ff::from_float4(Mf[(int64_t)D * P1 * ND + i]));
                    __syncthreads();
                    if (valid) {
                        const double2 cD = t.center[D];
                        const double RD = t.radius[D];
                        const double dx = z.x - cD.x, dy = z.y - cD.y;
                        const double r2 = dx * dx + dy * dy;
                        const double2 v = make_double2(dx / r2 * RD, -dy / r2 * RD);
                        const double lg = 0.5 * log(r2);
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            double2 sv = make_double2(0.0, 0.0);
                            for (int k = P; k >= 1; --k) sv = cmul(cadd(sv, Cs[k][d]), v);
                            acc[d] += fma(Cs[0][d].x, lg, sv.x);
                        }
                    }
                }
            }

            // P2P over U (float-float). Coordinates in units of leaf b's side, so
            // sum q log r = 1/2 sum q log r'^2 + log(side_b) (sum_U q - coincident q);
            // sum_U q is read from the leaves' monopoles M_0. With SYM, leaves A < b
            // are skipped (A's block sends their part through the slots) and leaves
            // A > b are summed in both directions.
            const int warp = tid >> 5, lane = tid & 31;
            const int grp = (tb - e0) / 32 + warp;  // this warp's group of 32 targets of b
            const bool grp_live = tb + 32 * warp < e1;
            float2 qi[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d)
                qi[d] = (SYM && valid) ? qf[(int64_t)ti * ND + d] : make_float2(0.f, 0.f);
            float ah[ND], al[ND];
            ff::F qu[ND], qco[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                ah[d] = al[d] = 0.f;
                qu[d] = qco[d] = ff::F{0.f, 0.f};
            }
            for (int e = u0; e < u1; ++e) {
                const int A = t.u_idx[e];
                const int a0 = g.crng[2 * A], a1 = g.crng[2 * A + 1];
                if (a0 == a1) continue;
                const float4 uo = t.u_off[e];  // exact offset of leaf A's centre and its scale, in b units
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const float4 m0 = Mf[(int64_t)A * P1 * ND + d];
                    qu[d] = ff::add(qu[d], ff::F{m0.x, m0.y});
                }
                if (SYM && A < b) continue;
                const bool rev = SYM && A > b;
                const bool own = own_sym && A == b;
                if (own && valid) {  // the coincident self pair, for the leaf-size term
#pragma unroll
                    for (int d = 0; d < ND; ++d) qco[d] = ff::add(qco[d], ff::F{qi[d].x, qi[d].y});
                }
                const int64_t sbase = rev ? t.sym_off[e] + (int64_t)grp * (a1 - a0) : 0;
                // same level or one level apart: hi parts differ exactly (both on
                // the 2^-22 grid after the exact shift/scale), so dx = (th - sh) + (tl - sl)
                const bool exact_hi = uo.z >= 0.5f && uo.z <= 2.0f;
                for (int sb = a0; sb < a1; sb += kLeafThreads) {
                    const int n = min(kLeafThreads, a1 - sb);
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
#pragma unroll
                        for (int d = 0; d < ND; ++d) s_q[tid][d] = qf[(int64_t)j * ND + d];
                    }
                    __syncthreads();
                    if (rev) {
                        if (grp_live) {  // warp-uniform
                            for (int c = 0; c < n; c += 32) {
                                const int nc = min(32, n - c);
                                float rh[ND], rl[ND];
#pragma unroll
                                for (int d = 0; d < ND; ++d) rh[d] = rl[d] = 0.f;
                                const bool full = nc == 32 && __all_sync(0xffffffffu, valid);  // warp-uniform
                                if (exact_hi && full)
                                    p2p_chunk_sym<ND, true, true>(rt, qi, valid, s_rho + c, s_q + c, nc, lane, s_tab,
                                                                  ah, al, rh, rl);
                                else if (exact_hi)
                                    p2p_chunk_sym<ND, true>(rt, qi, valid, s_rho + c, s_q + c, nc, lane, s_tab, ah,
                                                            al, rh, rl);
                                else
                                    p2p_chunk_sym<ND, false>(rt, qi, valid, s_rho + c, s_q + c, nc, lane, s_tab, ah,
                                                             al, rh, rl);
                                if (lane < nc) {
                                    const int64_t o = (sbase + (sb - a0) + c + lane) * ND;
#pragma unroll
                                    for (int d = 0; d < ND; ++d) slots[o + d] = make_float2(rh[d], rl[d]);
                                }
                            }
                        }
                    } else if (own) {
                        if constexpr (kOwn) {
                            if (grp_live) {  // warp-uniform
                                for (int c = 0; c < n; c += 32) {
                                    const int cg = (sb - a0 + c) >> 5;  // the charges' group
                                    const int nc = min(32, n - c);
                                    // pairs with a group of the same pass of 64 targets are
                                    // summed in both directions by both warps (no barrier
                                    // inside the pass); pairs with groups of later passes
                                    // are handed over through shared memory
                                    const bool same_pass = (cg >> 1) == (grp >> 1) && cg != grp;
                                    if (same_pass) {
                                        if (valid) p2p_tile<ND, true>(rt, s_rho + c, s_q + c, nc, s_tab, ah, al, qco);
                                        continue;
                                    }
                                    if (cg < grp) continue;  // that warp handed these pairs over
                                    if (cg == grp) {
                                        p2p_diag_sym<ND>(rt, qi, valid, s_rho + c, s_q + c, nc, lane, s_tab, ah, al);
                                    } else {
                                        float rh[ND], rl[ND];
#pragma unroll
                                        for (int d = 0; d < ND; ++d) rh[d] = rl[d] = 0.f;
                                        p2p_chunk_sym<ND, true>(rt, qi, valid, s_rho + c, s_q + c, nc, lane, s_tab,
                                                                ah, al, rh, rl);
                                        const int pr = cg * (cg - 1) / 2 + grp;
#pragma unroll
                                        for (int d = 0; d < ND; ++d) s_own[pr][lane][d] = make_float2(rh[d], rl[d]);
                                    }
                                }
                            }
                        }
                    } else if (valid) {
                        if (exact_hi)
                            p2p_tile<ND, true>(rt, s_rho, s_q, n, s_tab, ah, al, qco);
                        else
                            p2p_tile<ND, false>(rt, s_rho, s_q, n, s_tab, ah, al, qco);
                    }
                }
            }
            if constexpr (kOwn) {
                if (own_sym) {
                    // own-leaf sums handed over by the warps of earlier passes (written
                    // before this pass's staging barriers), in a fixed order
                    if (valid) {
                        for (int gp = 0; gp < (grp & ~1); ++gp) {
                            const int pr = grp * (grp - 1) / 2 + gp;
#pragma unroll
                            for (int d = 0; d < ND; ++d) {
                                const float2 v = s_own[pr][lane][d];
                                float sh, se;
                                ff::two_sum(ah[d], v.x, sh, se);
                                ah[d] = sh;
                                al[d] = __fadd_rn(al[d], __fadd_rn(se, v.y));
                            }
                        }
                    }
                }
            }
            if (valid) {
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double near = 0.5 * ((double)ah[d] + (double)al[d]) +
                                        log_side * (ff::to_double(qu[d]) - ff::to_double(qco[d]));
                    psi[(int64_t)ti * ND + d] = acc[d] + near;
                }
            }
        }
    }
}

// ----------------------------------------------------------------------------
// a7: out = -(1/2pi) psi (back to caller order) + Pi f, one warp per target row.
template <int ND>
__global__ void k_out_forward(int32_t n_tgt, const int32_t* __restrict__ inv, const double* __restrict__ psi,
                              const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ f, int64_t ld_f,
                              double* __restrict__ out, int64_t ld_out)
{
    const int lane = threadIdx.x & 31;
    for (int i = global_warp(); i < n_tgt; i += num_warps()) {
        double s[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) s[d] = 0.0;
        if (rowptr) {
            const int64_t k1 = rowptr[i + 1];
            for (int64_t k = rowptr[i] + lane; k < k1; k += 32) {
                const double v = val[k];
                const int32_t c = col[k];
#pragma unroll
                for (int d = 0; d < ND; ++d) s[d] = fma(v, f[d * ld_f + c], s[d]);
            }
#pragma unroll
            for (int d = 0; d < ND; ++d)
                for (int o = 16; o > 0; o >>= 1) s[d] += __shfl_xor_sync(0xffffffffu, s[d], o);
        }
        if (lane == 0) {
            const int32_t ts = inv[i];
#pragma unroll
            for (int d = 0; d < ND; ++d) out[d * ld_out + i] = fma(-kInv2Pi, psi[(int64_t)ts * ND + d], s[d]);
        }
    }
}

// transposed output: grad_f = -(1/2pi) w psi (caller order) + Pi^T g, one warp per source
template <int ND>
__global__ void k_out_adjoint(int32_t n_src, const int32_t* __restrict__ inv, const double* __restrict__ w_sorted,
                              const double* __restrict__ psi, const int64_t* __restrict__ cptr,
                              const int32_t* __restrict__ crow, const double* __restrict__ cval,
                              const double* __restrict__ g, int64_t ld_g, double* __restrict__ out,
                              int64_t ld_out)
{
    const int lane = threadIdx.x & 31;
    for (int j = global_warp(); j < n_src; j += num_warps()) {
        double s[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) s[d] = 0.0;
        if (cptr) {
            const int64_t k1 = cptr[j + 1];
            for (int64_t k = cptr[j] + lane; k < k1; k += 32) {
                const double v = cval[k];
                const int32_t r = crow[k];
#pragma unroll
                for (int d = 0; d < ND; ++d) s[d] = fma(v, g[d * ld_g + r], s[d]);
            }
#pragma unroll
            for (int d = 0; d < ND; ++d)
                for (int o = 16; o > 0; o >>= 1) s[d] += __shfl_xor_sync(0xffffffffu, s[d], o);
        }
        if (lane == 0) {
            if (psi) {
                const int32_t js = inv[j];
                const double wj = -kInv2Pi * w_sorted[js];
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + j] = fma(wj, psi[(int64_t)js * ND + d], s[d]);
            } else {  // accumulate onto out
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + j] += s[d];
            }
        }
    }
}

// grad_tgt[i] (+)= -(1/2pi) sum_d g[d][i] grad psi_d(t_i), one thread per sorted target
template <int ND>
__global__ void k_grad_out(int32_t n_tgt, int accumulate, const int32_t* __restrict__ perm,
                           const double* __restrict__ gpsi, const double* __restrict__ g, int64_t ld_g,
                           double* __restrict__ grad)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tgt; t += gridDim.x * blockDim.x) {
        const int32_t i = perm[t];
        double gx = 0.0, gy = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const double gv = g[d * ld_g + i];
            gx = fma(gv, gpsi[((int64_t)t * 2 + 0) * ND + d], gx);
            gy = fma(gv, gpsi[((int64_t)t * 2 + 1) * ND + d], gy);
        }
        gx *= -kInv2Pi;
        gy *= -kInv2Pi;
        if (accumulate) {
            grad[2 * (int64_t)i] += gx;
            grad[2 * (int64_t)i + 1] += gy;
        } else {
            grad[2 * (int64_t)i] = gx;
            grad[2 * (int64_t)i + 1] = gy;
        }
    }
}

// Adds the slots of the symmetric near field to the receiving leaves'
// potentials, one warp per leaf, slots in a fixed order (deterministic). The
// sender b summed q_i log r'^2 in b's units: the physical sum is half of it plus
// log(side_b) sum_b q, of which log(side_A) sum_b q is already in A's own
// near-field term; the rest is (log R_b - log R_A) M_0(b).
template <int P, int ND>
__global__ void k_sym_reduce(DevTree t, PassGeom g, const float2* __restrict__ slots, const float4* __restrict__ Mf,
                             double* __restrict__ psi)
{
    constexpr int P1 = P + 1;
    // one thread per evaluation point: neighbouring threads read neighbouring slots
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.n_eval; j += gridDim.x * blockDim.x) {
        const int A = t.sym_pt_leaf[j];
        const int s0 = t.sym_in_ptr[A], s1 = t.sym_in_ptr[A + 1];
        if (s0 == s1) continue;
        const int jl = j - g.erng[2 * A];
        // float-float sums on the FP32 pipes (conversions to FP64 would occupy the
        // FP64 pipe once per slot), converted once per point
        ff::F acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = ff::F{0.f, 0.f};
#pragma unroll 4
        for (int k = s0; k < s1; ++k) {
            const int64_t o = (t.sym_in_slot[k] + jl) * ND;
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const float2 v = slots[o + d];
                acc[d] = ff::add(acc[d], ff::F{v.x, v.y});
            }
        }
        double cst[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) cst[d] = 0.0;
        for (int k = t.sym_in_pptr[A]; k < t.sym_in_pptr[A + 1]; ++k) {
            const int b = t.sym_in_pbox[k];
            const double dl = t.log_radius[b] - t.log_radius[A];
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                const float4 m0 = Mf[(int64_t)b * P1 * ND + d];
                cst[d] = fma(dl, (double)m0.x + (double)m0.y, cst[d]);
            }
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) psi[(int64_t)j * ND + d] += fma(0.5, ff::to_double(acc[d]), cst[d]);
    }
}

template <int P, int ND>
cudaError_t fmm_impl(const DevTree& t, const DevTables& tab, const PassGeom& g, Workspace& ws, bool gradient,
                     bool fp64, PhaseTimer* tm, cudaStream_t s)
{
    const int threads = kWarpsPerBlock * 32;
    const bool ffp = !fp64 && !gradient;  // float-float pipeline (potential only)
    int id = tm ? tm->begin(ffp ? "upward" : "p2m") : -1;
    if (ffp) {
        // P2M and the whole M2M pass in one launch (see k_p2m_ff)
        k_p2m_ff<P, ND><<<warp_blocks(t.nleaf), threads, 0, s>>>(t, tab, g, ws.qf, ws.Mf, ws.m2m_count);
        if (tm) tm->end(id);
    } else {
        k_p2m<P, ND><<<warp_blocks(t.nleaf), threads, 0, s>>>(t, g, ws.q, ws.M);
        if (tm) tm->end(id);
        id = tm ? tm->begin("m2m") : -1;
        for (int l = t.nlevels - 2; l >= 2; --l) {  // levels 0 and 1 are never read
            const int b0 = t.level_start[l], b1 = t.level_start[l + 1];
            k_m2m<P, ND><<<warp_blocks(b1 - b0), threads, 0, s>>>(t, tab, b0, b1, ws.M);
        }
        if (tm) tm->end(id);
    }
    id = tm ? tm->begin("m2l") : -1;
    if (ffp)
        k_m2l_ff<P, ND><<<warp_blocks(t.nbox), threads, 0, s>>>(t, tab, g, ws.Mf, ws.Lf, ws.qf);
    else
        k_m2l<P, ND><<<warp_blocks(t.nbox), threads, 0, s>>>(t, tab, g, ws.M, ws.L, ws.q);
    if (tm) tm->end(id);
    id = tm ? tm->begin("l2l") : -1;
    // boxes of levels 0 and 1 have empty V and X lists, so their locals are zero
    // and the first L2L that adds anything goes into level 3
    for (int l = 3; l < t.nlevels; ++l) {
        const int b0 = t.level_start[l], b1 = t.level_start[l + 1];
        if (ffp)
            k_l2l_ff<P, ND><<<warp_blocks(b1 - b0), threads, 0, s>>>(t, tab, b0, b1, ws.Lf);
        else
            k_l2l<P, ND><<<warp_blocks(b1 - b0), threads, 0, s>>>(t, tab, b0, b1, ws.L);
    }
    if (tm) tm->end(id);
    id = tm ? tm->begin("leaf") : -1;
    const int blocks = t.nleaf < 1 ? 1 : (t.nleaf > 152 * 64 ? 152 * 64 : t.nleaf);
    if (gradient)
        k_leaf<P, ND, true><<<blocks, kLeafThreads, 0, s>>>(t, g, ws.q, ws.M, ws.L, ws.psi);
    else if (fp64)
        k_leaf<P, ND, false><<<blocks, kLeafThreads, 0, s>>>(t, g, ws.q, ws.M, ws.L, ws.psi);
    else {
        static int resident[2] = {0, 0};  // blocks of each instantiation that fit on one SM
        // the symmetric near field pays off while the shared log dominates the
        // per-pair work (one or two densities); beyond that the second
        // accumulation costs about as much as it saves
        const bool sym = t.sym && ND <= 2;
        const int si = sym ? 1 : 0;
        if (resident[si] == 0) {
            int nb = 0;
            const cudaError_t oe =
                sym ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_leaf_ff<P, ND, true>, kLeafThreads, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_leaf_ff<P, ND, false>, kLeafThreads, 0);
            if (oe != cudaSuccess || nb < 1) nb = 1;
            resident[si] = nb;
        }
        int sms = 152;
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int pblocks = std::max(1, std::min(t.nleaf, sms * resident[si]));
        cudaMemsetAsync(ws.work, 0, sizeof(int), s);
        if (sym) {
            k_leaf_ff<P, ND, true><<<pblocks, kLeafThreads, 0, s>>>(t, g, ws.qf, ws.Mf, ws.Lf, tab.logtab, ws.psi,
                                                                   ws.work, ws.slots);
            const int rblocks = std::max(1, std::min((g.n_eval + 255) / 256, 152 * 32));
            k_sym_reduce<P, ND><<<rblocks, 256, 0, s>>>(t, g, ws.slots, ws.Mf, ws.psi);
        } else {
            k_leaf_ff<P, ND, false><<<pblocks, kLeafThreads, 0, s>>>(t, g, ws.qf, ws.Mf, ws.Lf, tab.logtab, ws.psi,
                                                                    ws.work, nullptr);
        }
    }
    if (tm) tm->end(id);
    return cudaGetLastError();
}

template <int P>
cudaError_t fmm_p(int nd, const DevTree& t, const DevTables& tab, const PassGeom& g, Workspace& ws, bool grad,
                  bool fp64, PhaseTimer* tm, cudaStream_t s)
{
    switch (nd) {
        case 1: return fmm_impl<P, 1>(t, tab, g, ws, grad, fp64, tm, s);
        case 2: return fmm_impl<P, 2>(t, tab, g, ws, grad, fp64, tm, s);
        case 4: return fmm_impl<P, 4>(t, tab, g, ws, grad, fp64, tm, s);
        case 8: return fmm_impl<P, 8>(t, tab, g, ws, grad, fp64, tm, s);
        default: return cudaErrorInvalidValue;
    }
}

int grid_1d(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

}  // namespace

bool p_supported(int P) { return P == 16 || P == 24 || P == 30; }

cudaError_t launch_charges(int nd, int32_t n, const int32_t* perm, const double* w_sorted, const double* f,
                           int64_t ld_f, double* q, float2* qf, cudaStream_t s)
{
    const int blocks = grid_1d((int64_t)n * nd, 256);
    switch (nd) {
        case 1: k_charges<1><<<blocks, 256, 0, s>>>(n, perm, w_sorted, f, ld_f, q, qf); break;
        case 2: k_charges<2><<<blocks, 256, 0, s>>>(n, perm, w_sorted, f, ld_f, q, qf); break;
        case 4: k_charges<4><<<blocks, 256, 0, s>>>(n, perm, w_sorted, f, ld_f, q, qf); break;
        case 8: k_charges<8><<<blocks, 256, 0, s>>>(n, perm, w_sorted, f, ld_f, q, qf); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fmm_potential(int P, int nd, const DevTree& t, const DevTables& tab, const PassGeom& g,
                                 Workspace& ws, bool gradient, bool fp64, PhaseTimer* timer, cudaStream_t s)
{
    switch (P) {
        case 16: return fmm_p<16>(nd, t, tab, g, ws, gradient, fp64, timer, s);
        case 24: return fmm_p<24>(nd, t, tab, g, ws, gradient, fp64, timer, s);
        case 30: return fmm_p<30>(nd, t, tab, g, ws, gradient, fp64, timer, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_out_forward(int nd, int32_t n_tgt, const int32_t* tgt_inv, const double* psi,
                               const int64_t* rowptr, const int32_t* col, const double* val, const double* f,
                               int64_t ld_f, double* out, int64_t ld_out, cudaStream_t s)
{
    const int blocks = warp_blocks(n_tgt), threads = kWarpsPerBlock * 32;
    switch (nd) {
        case 1: k_out_forward<1><<<blocks, threads, 0, s>>>(n_tgt, tgt_inv, psi, rowptr, col, val, f, ld_f, out, ld_out); break;
        case 2: k_out_forward<2><<<blocks, threads, 0, s>>>(n_tgt, tgt_inv, psi, rowptr, col, val, f, ld_f, out, ld_out); break;
        case 4: k_out_forward<4><<<blocks, threads, 0, s>>>(n_tgt, tgt_inv, psi, rowptr, col, val, f, ld_f, out, ld_out); break;
        case 8: k_out_forward<8><<<blocks, threads, 0, s>>>(n_tgt, tgt_inv, psi, rowptr, col, val, f, ld_f, out, ld_out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_out_adjoint(int nd, int32_t n_src, const int32_t* src_inv, const double* w_sorted,
                               const double* psi, const int64_t* cptr, const int32_t* crow, const double* cval,
                               const double* g, int64_t ld_g, double* out, int64_t ld_out, cudaStream_t s)
{
    const int blocks = warp_blocks(n_src), threads = kWarpsPerBlock * 32;
    switch (nd) {
        case 1: k_out_adjoint<1><<<blocks, threads, 0, s>>>(n_src, src_inv, w_sorted, psi, cptr, crow, cval, g, ld_g, out, ld_out); break;
        case 2: k_out_adjoint<2><<<blocks, threads, 0, s>>>(n_src, src_inv, w_sorted, psi, cptr, crow, cval, g, ld_g, out, ld_out); break;
        case 4: k_out_adjoint<4><<<blocks, threads, 0, s>>>(n_src, src_inv, w_sorted, psi, cptr, crow, cval, g, ld_g, out, ld_out); break;
        case 8: k_out_adjoint<8><<<blocks, threads, 0, s>>>(n_src, src_inv, w_sorted, psi, cptr, crow, cval, g, ld_g, out, ld_out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_grad_out(int nd, bool accumulate, int32_t n_tgt, const int32_t* tgt_perm, const double* gpsi,
                            const double* g, int64_t ld_g, double* grad, cudaStream_t s)
{
    const int blocks = grid_1d(n_tgt, 256);
    const int acc = accumulate ? 1 : 0;
    switch (nd) {
        case 1: k_grad_out<1><<<blocks, 256, 0, s>>>(n_tgt, acc, tgt_perm, gpsi, g, ld_g, grad); break;
        case 2: k_grad_out<2><<<blocks, 256, 0, s>>>(n_tgt, acc, tgt_perm, gpsi, g, ld_g, grad); break;
        case 4: k_grad_out<4><<<blocks, 256, 0, s>>>(n_tgt, acc, tgt_perm, gpsi, g, ld_g, grad); break;
        case 8: k_grad_out<8><<<blocks, 256, 0, s>>>(n_tgt, acc, tgt_perm, gpsi, g, ld_g, grad); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vp
