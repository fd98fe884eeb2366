// FMM kernels (Laplace kernel) in IEEE float64 arithmetic, shaped for GB300's
// narrow FP64 pipe (2 DFMA per clock per SM): every kernel keeps all 32 lanes
// of its FP64 instructions busy and spends as few FP64 operations per unit of
// work as the arithmetic allows; integer, shared-memory and shuffle work is
// cheap beside them and is used freely. This is the default arithmetic of
// libvp (arXiv 2203.05933: the smooth-quadrature point sum of
// Eq. Tk_smooth_quad evaluated by a point FMM, Sec. 4).
//
// Conventions as in vp_fmm.cu: psi(z) = Re sum_j q_j log(z - z_j), expansions
// scaled by the box half-side R (M_k = a_k / R^k, L_l = b_l R^l), the same
// scaled translation operators.
//
// Near field. Coordinates are the absolute float64 node coordinates (as in the
// direct sum), so dx, dy are the exact differences of the inputs for nearby
// points. log r^2 comes from an own table-driven logarithm (the method of
// P. T. P. Tang, "Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 16(4), 1990): with r^2 = 2^e m and c_k
// the table point nearest m (spacing 2^-12),
//     log r^2 = e log 2 + T_k + log1p(u),   u = m s_k - 1,   T_k = -log s_k,
// where s_k = RN(1/c_k) is a float64 and T_k is its exact logarithm rounded
// once, so the split is exact whatever the rounding of s_k; |u| <= 2^-13 and
// log1p(u) = u (1 - u/2 + u^2/3) has truncation error below 2^-54. u is one FMA
// of r^2 with s_k 2^-e (the power of two is applied to s_k's exponent field by
// an integer add, exactly); the sum e log 2 + T_k is one addition of two table
// values, and the last multiplication of the series is fused with the final
// addition: log r^2 = fma(u, 1 - u/2 + u^2/3, e log 2 + T_k). That is 5 FP64
// operations per logarithm. Error: the roundings of e log 2, T_k and their sum
// (each at most half an ulp of numbers below max(1, |e| log 2)) plus the final
// rounding, so |error| <= 2^-52 max(1, |e| log 2) + half an ulp of the result:
// about one ulp of log r^2 wherever |log r^2| >= 1, an absolute 2^-52 near
// r^2 = 1 (tested against CUDA's log through the public API). With the squares
// and differences, one directed pair costs 10 FP64 operations; a pair
// evaluated once for both directions costs 11.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "vp_fixed.cuh"
#include "vp_internal.h"

namespace vp {
namespace {

constexpr int kW64 = 4;             // warps per block of the expansion kernels
// Warps per block of the near-field kernels. Each block holds one 64 KB copy of
// the logarithm's table, so shared memory caps the resident blocks: at one or
// two densities (64 registers) 16-warp blocks give 2 blocks, 32 warps per SM,
// against 3 blocks of 8 warps; more densities need more registers than a
// 512-thread block allows and keep 8 warps.
template <int ND>
constexpr int leaf_warps64()
{
    return ND <= 2 ? 16 : 8;
}
constexpr int kGradWarps64 = 8;  // warps per block of the near-field gradient kernel
constexpr int kEBias = 64;          // exponent table covers e in [-64, 63]

__device__ __forceinline__ double2 cmul64(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// a * b + c
__device__ __forceinline__ double2 cfma64(double2 a, double2 b, double2 c)
{
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

__device__ __forceinline__ int gwarp() { return (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); }
__device__ __forceinline__ int nwarps() { return (int)((gridDim.x * blockDim.x) >> 5); }

// CUDA's log for the pairs outside the table's exponent range (kept out of line:
// it is not met on the hot path).
__device__ __noinline__ double log_r2_slow(double r2) { return r2 == 0.0 ? 0.0 : log(r2); }

// log(r2) by the table-driven method above. tab[k] = (s_k, T_k), etab[e + 64] =
// e log 2. r2 == 0 (a bitwise-coincident pair) gives 0 (no smooth term);
// r2 outside [2^-64, 2^63] takes CUDA's log (not met by nodes of a domain of
// size O(1) unless two of them are within 2^-32 of each other).
__device__ __forceinline__ double log_r2(double r2, const double2* __restrict__ tab, const double* __restrict__ etab)
{
    const int hi = __double2hiint(r2);
    const int h = hi + (1 << (19 - kLog64Bits));       // round m to the nearest table point
    const int e = (h >> 20) - 1023;                      // exponent of 2^e c_k
    const int k = (h >> (20 - kLog64Bits)) & ((1 << kLog64Bits) - 1);
    const double2 sk = tab[k];
    const int ei = min(max(e + kEBias, 0), 2 * kEBias - 1);
    const double s = __hiloint2double(__double2hiint(sk.x) - (e << 20), __double2loint(sk.x));  // s_k 2^-e
    const double u = fma(r2, s, -1.0);
    const double b = fma(u, fma(u, 0x1.5555555555555p-2, -0.5), 1.0);  // 1 - u/2 + u^2/3
    double L = fma(u, b, etab[ei] + sk.y);
    if ((unsigned)(e + kEBias) >= (unsigned)(2 * kEBias)) L = log_r2_slow(r2);
    return L;
}

// Logarithm in fixed point on the integer pipes (the table method of log_r2,
// P. T. P. Tang 1990, with integer arithmetic): for x = X 2^(e - 62), X in
// [2^62, 2^63), returns Lp with log x = Lp 2^-60 + E log 2 (E = e, or e + 1
// when X rounds up to the next power of two). The table point c_k = 1 + k
// 2^-12 nearest x's mantissa is chosen from X's bits; tab[k] = (S_k, T_k) with
// S_k = round(2^62 / c_k) and T_k = round(-log(S_k 2^-62) 2^60), so that
// log x = E log 2 + T_k 2^-60 + log1p(u) exactly for u = (X S_k) 2^-124 - 1,
// |u| <= 2^-13, whatever the rounding of S_k. X S_k is a 125-bit product;
// u is kept as U = u 2^75 and log1p(u) = u (1 - u (1/2 - u (1/3 - u/4))) is
// evaluated by four high-half 64-bit products (truncation below 2^-65, each
// product's rounding below 2^-59). No floating-point operation.
__device__ __forceinline__ long long log_fix(unsigned long long X, int e, const longlong2* __restrict__ tab, int& E)
{
    unsigned long long kr = ((X >> (61 - kLog64Bits)) + 1ULL) >> 1;  // 2^12 + k, rounded; 2^13 on a carry
    const int carry = (int)(kr >> (kLog64Bits + 1));
    if (carry) {
        X >>= 1;
        kr = 1ULL << kLog64Bits;
    }
    E = e + carry;
    const longlong2 st = tab[kr - (1ULL << kLog64Bits)];
    // U = X S_k - 2^124 (|U| < 2^112) and u75 = U >> 49, from the product's halves
    const unsigned long long plo = X * (unsigned long long)st.x;
    const long long phi = (long long)(__umul64hi(X, (unsigned long long)st.x) - (1ULL << 60));
    const long long u75 = (long long)(((unsigned long long)phi << 15) | (plo >> 49));
    const long long t0 = 0x1555555555555555LL - (u75 >> 15);              // (1/3 - u/4) 2^62
    const long long t1 = (1LL << 61) - (__mul64hi(u75, t0) >> 11);        // (1/2 - u t0) 2^62
    const long long t2 = (1LL << 62) - (__mul64hi(u75, t1) >> 11);        // (1 - u t1) 2^62
    return st.y + (__mul64hi(u75, t2) >> 13);                              // (T_k + u t2) 2^60
}

// log of a positive float64 through log_fix (two conversions and an FMA)
__device__ __forceinline__ double log_via_fix(double r2, const longlong2* __restrict__ tab)
{
    const long long bits = __double_as_longlong(r2);
    const int eb = (int)((bits >> 52) & 0x7ff);
    if (r2 <= 0.0 || eb == 0 || eb == 0x7ff) return r2 == 0.0 ? 0.0 : log(r2);
    const unsigned long long X = (((unsigned long long)bits & 0xfffffffffffffULL) | 0x10000000000000ULL) << 10;
    int E;
    const long long Lp = log_fix(X, eb - 1023, tab, E);
    return fma((double)E, 0.693147180559945309417232121458, (double)Lp * 0x1p-60);
}

// log r^2 of two points on the integer grid 2^-sigma (|dx|, |dy| < 2^62), in
// fixed point: log r^2 = Lp 2^-60 + Ep log 2. dx^2 + dy^2 is formed exactly in
// 128-bit integers and its leading 63 bits go to log_fix (truncation below
// 2^-62 relative); Ep = E - 2 sigma. r^2 = 0 (coincident points) gives 0, 0.
__device__ __forceinline__ long long log_r2_int(long long dx, long long dy, const longlong2* __restrict__ tab,
                                                int two_sigma, int& Ep)
{
    const unsigned long long ax = (unsigned long long)(dx < 0 ? -dx : dx);
    const unsigned long long ay = (unsigned long long)(dy < 0 ? -dy : dy);
    const unsigned long long l1 = ax * ax, l2 = ay * ay;
    const unsigned long long lo = l1 + l2;
    const unsigned long long hi = __umul64hi(ax, ax) + __umul64hi(ay, ay) + (lo < l1 ? 1ULL : 0ULL);
    if ((hi | lo) == 0ULL) {
        Ep = 0;
        return 0;
    }
    const int n = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // leading one
    const int sh = n - 62;
    unsigned long long X;
    if (sh <= 0)
        X = lo << (-sh);
    else if (sh < 64)
        X = (lo >> sh) | (hi << (64 - sh));
    else
        X = hi >> (sh - 64);
    int E;
    const long long Lp = log_fix(X, n, tab, E);
    Ep = E - two_sigma;
    return Lp;
}

// ----------------------------------------------------------------------------
// a5 + a6: near field, L2P and W-list M2P of one leaf per warp (persistent
// warps pull leaves from a queue, costliest first). Lane i holds one
// evaluation point of the current group of 32; the sources of each U-list leaf
// are staged 32 at a time in the warp's shared buffer.
// SYM (evaluation points are the charge points, same tree order): leaves
// A < b are skipped, A == b is summed directed (coincident pairs give 0), and
// for A > b each distance is evaluated once: at step t lane l takes source
// (l + t) mod 32, adds q_j log r^2 to its own point and q_i log r^2 to an
// accumulator for that source, which moves one lane down each step; after 32
// steps lane l holds the group's sum for source l and writes it to the slot of
// (b, A, group), added to A's points by k_sym_reduce64 in a fixed order.
template <int ND>
struct LeafStage64 {
    double2 xy[32];
    double q[32][ND];
};

template <int ND>
struct LeafStageFix {
    longlong2 xy[32];  // integer coordinates (PassGeom::cfix)
    double q[32][ND];
};

template <int P, int ND, bool SYM>
__global__ void __launch_bounds__(leaf_warps64<ND>() * 32)
    k_leaf64(DevTree t, PassGeom g, const double* __restrict__ q, const double2* __restrict__ M,
             const double2* __restrict__ L, const double2* __restrict__ logtab, const double* __restrict__ etab_g,
             double* __restrict__ psi, int* __restrict__ work, double* __restrict__ slots)
{
    constexpr int P1 = P + 1;
    extern __shared__ __align__(16) unsigned char smem64[];
    double2* tab = reinterpret_cast<double2*>(smem64);                       // [1 << kLog64Bits]
    double* etab = reinterpret_cast<double*>(tab + (1 << kLog64Bits));       // [2 * kEBias]
    LeafStage64<ND>* stage = reinterpret_cast<LeafStage64<ND>*>(etab + 2 * kEBias);
    for (int i = threadIdx.x; i < (1 << kLog64Bits); i += blockDim.x) tab[i] = logtab[i];
    for (int i = threadIdx.x; i < 2 * kEBias; i += blockDim.x) etab[i] = etab_g[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    LeafStage64<ND>& st = stage[threadIdx.x >> 5];

    for (;;) {
        int li = 0;
        if (lane == 0) li = atomicAdd(work, 1);
        li = __shfl_sync(0xffffffffu, li, 0);
        if (li >= t.nleaf) break;
        const int b = SYM ? t.sym_leaves[li] : t.leaves[li];
        const int e0 = g.erng[2 * b], e1 = g.erng[2 * b + 1];
        if (e0 == e1) continue;
        const double2 cb = t.center[b];
        const int u0 = t.u_ptr[b], u1 = t.u_ptr[b + 1];
        const int w0 = t.w_ptr[b], w1 = t.w_ptr[b + 1];
        for (int gb = e0; gb < e1; gb += 32) {
            const int grp = (gb - e0) >> 5;
            // directed sums: a group of fewer than 32 points is shared by ksplit
            // sub-groups of lanes that divide the sources among them (masked lanes
            // would cost FP64 issue slots all the same); their partial sums are
            // added by shuffles at the end
            const int gcount = min(32, e1 - gb);
            const int ksplit = SYM ? 1 : 32 / gcount;
            const int sub = SYM ? 0 : lane / gcount;
            const int ti = SYM ? gb + lane : gb + lane % gcount;
            const bool valid = SYM ? ti < e1 : sub < ksplit;
            const double2 z = valid ? g.exy[ti] : cb;
            double acc[ND], near[ND], qi[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                acc[d] = 0.0;
                near[d] = 0.0;
                qi[d] = (SYM && valid) ? q[(int64_t)ti * ND + d] : 0.0;
            }
            // L2P: Re sum_l L_l u^l, u = (z - c)/R, from the point's stored powers
            {
                const double2* Lb = L + (int64_t)b * P1 * ND;
                const double2* up = g.epow + (int64_t)(valid ? ti : e0) * P;
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = Lb[d].x;
#pragma unroll 4
                for (int l = 1; l <= P; ++l) {
                    const double2 ul = up[l - 1];
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const double2 Ll = Lb[l * ND + d];
                        acc[d] = fma(Ll.x, ul.x, fma(-Ll.y, ul.y, acc[d]));
                    }
                }
            }
            // M2P over W: M_0 log|z - c| + Re sum_k M_k v^k, v = R/(z - c)
            for (int e = w0; e < w1; ++e) {
                const int D = t.w_idx[e];
                const double2 cD = t.center[D];
                const double RD = t.radius[D];
                const double dx = z.x - cD.x, dy = z.y - cD.y;
                const double r2 = fma(dx, dx, dy * dy);
                const double2 v = make_double2(dx / r2 * RD, -dy / r2 * RD);
                const double lg = 0.5 * log_r2(r2, tab, etab);
                const double2* MD = M + (int64_t)D * P1 * ND;
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    double2 s = make_double2(0.0, 0.0);
#pragma unroll 2
                    for (int k = P; k >= 1; --k) {
                        const double2 m = MD[k * ND + d];
                        s = cmul64(make_double2(s.x + m.x, s.y + m.y), v);
                    }
                    acc[d] += fma(MD[d].x, lg, s.x);
                }
            }
            // P2P over U
            for (int e = u0; e < u1; ++e) {
                const int A = t.u_idx[e];
                if (SYM && A < b) continue;
                const int a0 = g.crng[2 * A], a1 = g.crng[2 * A + 1];
                const bool rev = SYM && A > b;
                const int64_t sbase = rev ? t.sym_off[e] + (int64_t)grp * (a1 - a0) : 0;
                for (int c = a0; c < a1; c += 32) {
                    const int n = min(32, a1 - c);
                    __syncwarp();
                    if (lane < n) {
                        st.xy[lane] = g.cxy[c + lane];
#pragma unroll
                        for (int d = 0; d < ND; ++d) st.q[lane][d] = q[(int64_t)(c + lane) * ND + d];
                    }
                    __syncwarp();
                    if (rev) {
                        double rv[ND];
#pragma unroll
                        for (int d = 0; d < ND; ++d) rv[d] = 0.0;
                        if (n == 32 && __all_sync(0xffffffffu, valid)) {
#pragma unroll 2
                            for (int s = 0; s < 32; ++s) {
                                const int j = (lane + s) & 31;
                                const double2 sp = st.xy[j];
                                const double dx = z.x - sp.x, dy = z.y - sp.y;
                                const double Lg = log_r2(fma(dx, dx, dy * dy), tab, etab);
#pragma unroll
                                for (int d = 0; d < ND; ++d) {
                                    near[d] = fma(st.q[j][d], Lg, near[d]);
                                    rv[d] = fma(qi[d], Lg, rv[d]);
                                    rv[d] = __shfl_sync(0xffffffffu, rv[d], (lane + 1) & 31);
                                }
                            }
                        } else {
                            for (int s = 0; s < 32; ++s) {
                                const int j = (lane + s) & 31;
                                if (valid && j < n) {
                                    const double2 sp = st.xy[j];
                                    const double dx = z.x - sp.x, dy = z.y - sp.y;
                                    const double Lg = log_r2(fma(dx, dx, dy * dy), tab, etab);
#pragma unroll
                                    for (int d = 0; d < ND; ++d) {
                                        near[d] = fma(st.q[j][d], Lg, near[d]);
                                        rv[d] = fma(qi[d], Lg, rv[d]);
                                    }
                                }
#pragma unroll
                                for (int d = 0; d < ND; ++d) rv[d] = __shfl_sync(0xffffffffu, rv[d], (lane + 1) & 31);
                            }
                        }
                        if (lane < n) {
                            const int64_t o = (sbase + (c - a0) + lane) * ND;
#pragma unroll
                            for (int d = 0; d < ND; ++d) slots[o + d] = rv[d];
                        }
                    } else if (valid) {
#pragma unroll 4
                        for (int j = sub; j < n; j += ksplit) {
                            const double2 sp = st.xy[j];
                            const double dx = z.x - sp.x, dy = z.y - sp.y;
                            const double Lg = log_r2(fma(dx, dx, dy * dy), tab, etab);
#pragma unroll
                            for (int d = 0; d < ND; ++d) near[d] = fma(st.q[j][d], Lg, near[d]);
                        }
                    }
                }
            }
            for (int sg = 1; sg < ksplit; ++sg) {  // warp-uniform
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double v = __shfl_down_sync(0xffffffffu, near[d], sg * gcount);
                    if (sub == 0) near[d] += v;
                }
            }
            if (valid && sub == 0) {
#pragma unroll
                for (int d = 0; d < ND; ++d) psi[(int64_t)ti * ND + d] = fma(0.5, near[d], acc[d]);
            }
        }
    }
}

// a5 + a6, directed (evaluation points are not the charge points of a
// symmetric plan): one leaf per warp from the persistent queue. First the far
// part of each evaluation point of the leaf (L2P + W-list M2P, one point per
// lane) is written to psi. Then the near field: the charge points of all U-list
// leaves form one stream, staged 32 at a time; the leaf's T points and K
// interleaved subsets of each 32-point chunk share the lanes (lane = a K + kap
// takes point a of the pass and chunk positions kap, kap + K, ...), in
// ceil(T K / 32) passes over the stream, K in {1, 2, 4, 8, 16} chosen per leaf
// for the fewest lane-steps (every lane of an FP64 instruction costs an issue
// slot, busy or not). A pair: r^2 from the points' integer coordinates in
// 128-bit integers, its logarithm in fixed point (log_r2_int: log r^2 = Lp
// 2^-60 + Ep log 2), both parts joined in one 64-bit fixed-point value L =
// Lp 2^(sL - 60) + Ep round(log 2 2^sL) (sL chosen per plan so that |L| <
// 2^63), converted once and accumulated in float64: q_j L_j with one FMA, the
// factor 2^-sL applied per point. The K partial sums of a point are added by
// shuffles and psi += near / 2 (the log is of r^2).
template <int P, int ND>
__global__ void __launch_bounds__(leaf_warps64<ND>() * 32)
    k_leaf64d(DevTree t, PassGeom g, const double* __restrict__ q, const double2* __restrict__ M,
              const double2* __restrict__ L, const longlong2* __restrict__ logtab, int two_sigma, int sL,
              long long ln2_sL, double* __restrict__ psi, int* __restrict__ work)
{
    constexpr int P1 = P + 1;
    extern __shared__ __align__(16) unsigned char smem64d[];
    longlong2* tab = reinterpret_cast<longlong2*>(smem64d);                  // [1 << kLog64Bits] (S_k, T_k)
    LeafStageFix<ND>* stage =
        reinterpret_cast<LeafStageFix<ND>*>(smem64d + (size_t)(1 << kLog64Bits) * sizeof(longlong2) +
                                            2 * kEBias * sizeof(double));
    for (int i = threadIdx.x; i < (1 << kLog64Bits); i += blockDim.x) tab[i] = logtab[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    LeafStageFix<ND>& st = stage[threadIdx.x >> 5];

    for (;;) {
        int li = 0;
        if (lane == 0) li = atomicAdd(work, 1);
        li = __shfl_sync(0xffffffffu, li, 0);
        if (li >= t.nleaf) break;
        const int b = t.leaves[li];
        const int e0 = g.erng[2 * b], e1 = g.erng[2 * b + 1];
        if (e0 == e1) continue;
        const int T = e1 - e0;
        const int u0 = t.u_ptr[b], u1 = t.u_ptr[b + 1];
        const int w0 = t.w_ptr[b], w1 = t.w_ptr[b + 1];
        // far part: L2P (Re sum_l L_l u^l, u = (z - c)/R, from the point's stored
        // powers) and M2P over W (M_0 log|z - c| + Re sum_k M_k v^k, v = R/(z - c))
        for (int i = lane; i < T; i += 32) {
            const double2 z = g.exy[e0 + i];
            double acc[ND];
            const double2* Lb = L + (int64_t)b * P1 * ND;
            const double2* up = g.epow + (int64_t)(e0 + i) * P;  // u^l, u = (z - c)/R
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[d] = Lb[d].x;
#pragma unroll 4
            for (int l = 1; l <= P; ++l) {
                const double2 ul = up[l - 1];
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double2 Ll = Lb[l * ND + d];
                    acc[d] = fma(Ll.x, ul.x, fma(-Ll.y, ul.y, acc[d]));
                }
            }
            for (int e = w0; e < w1; ++e) {
                const int D = t.w_idx[e];
                const double2 cD = t.center[D];
                const double RD = t.radius[D];
                const double dx = z.x - cD.x, dy = z.y - cD.y;
                const double r2 = fma(dx, dx, dy * dy);
                const double2 v = make_double2(dx / r2 * RD, -dy / r2 * RD);
                const double lg = 0.5 * log_via_fix(r2, tab);
                const double2* MD = M + (int64_t)D * P1 * ND;
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    double2 sm = make_double2(0.0, 0.0);
#pragma unroll 2
                    for (int k = P; k >= 1; --k) {
                        const double2 m = MD[k * ND + d];
                        sm = cmul64(make_double2(sm.x + m.x, sm.y + m.y), v);
                    }
                    acc[d] += fma(MD[d].x, lg, sm.x);
                }
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) psi[(int64_t)(e0 + i) * ND + d] = acc[d];
        }
        __syncwarp();  // the far parts before other lanes add to them
        int S = 0;
        for (int e = u0; e < u1; ++e) {
            const int A = t.u_idx[e];
            S += g.crng[2 * A + 1] - g.crng[2 * A];
        }
        if (S == 0) continue;
        // position p of the U-list stream -> charge index, from the cursor (entry
        // ecur whose first position is ebase <= p)
        auto charge_at = [&](int ecur, int ebase, int p) -> int {
            int e = ecur, pos = p - ebase;
            int A = t.u_idx[e];
            int a0 = g.crng[2 * A], len = g.crng[2 * A + 1] - a0;
            while (pos >= len) {
                pos -= len;
                A = t.u_idx[++e];
                a0 = g.crng[2 * A];
                len = g.crng[2 * A + 1] - a0;
            }
            return a0 + pos;
        };
        auto advance = [&](int& ecur, int& ebase, int p) {  // cursor to the entry holding position p
            for (;;) {
                const int A = t.u_idx[ecur];
                const int len = g.crng[2 * A + 1] - g.crng[2 * A];
                if (ebase + len > p || ecur + 1 >= u1) break;
                ebase += len;
                ++ecur;
            }
        };
        // the split with the fewest lane-steps
        const int full = S >> 5, rem = S & 31;
        int K = 1;
        long long best = -1;
        for (int kk = 1; kk <= 16; kk <<= 1) {
            const long long steps = (long long)((T * kk + 31) / 32) * (full * (32 / kk) + (rem + kk - 1) / kk);
            if (best < 0 || steps < best) {
                best = steps;
                K = kk;
            }
        }
        const int per = 32 / K;  // points per pass
        const int a = lane / K, kap = lane % K;
        for (int p0 = 0; p0 < T; p0 += per) {
            const int ti = p0 + a;
            const bool valid = ti < T;
            const longlong2 z = valid ? g.efix[e0 + ti] : make_longlong2(0, 0);
            double near[ND];  // sum q L, L in units of 2^-sL
#pragma unroll
            for (int d = 0; d < ND; ++d) near[d] = 0.0;
            int ecur = u0, ebase = 0;
            for (int c0 = 0; c0 < S; c0 += 32) {
                const int n = min(32, S - c0);
                __syncwarp();
                if (lane < n) {
                    const int j = charge_at(ecur, ebase, c0 + lane);
                    st.xy[lane] = g.cfix[j];
#pragma unroll
                    for (int d = 0; d < ND; ++d) st.q[lane][d] = q[(int64_t)j * ND + d];
                }
                advance(ecur, ebase, c0 + 32);
                __syncwarp();
                if (valid) {
#pragma unroll 4
                    for (int j = kap; j < n; j += K) {
                        const longlong2 sp = st.xy[j];
                        int Ep;
                        const long long Lp = log_r2_int(z.x - sp.x, z.y - sp.y, tab, two_sigma, Ep);
                        const double Lv = (double)((Lp >> (60 - sL)) + (long long)Ep * ln2_sL);
#pragma unroll
                        for (int d = 0; d < ND; ++d) near[d] = fma(st.q[j][d], Lv, near[d]);
                    }
                }
            }
            for (int off = 1; off < K; off <<= 1) {  // warp-uniform
#pragma unroll
                for (int d = 0; d < ND; ++d) near[d] += __shfl_xor_sync(0xffffffffu, near[d], off);
            }
            if (valid && kap == 0) {
                const double half = ldexp(0.5, -sL);
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    double* o = psi + (int64_t)(e0 + ti) * ND + d;
                    *o = fma(half, near[d], *o);
                }
            }
        }
    }
}

// 1/r2 by two Newton-Raphson steps (y <- y + y (1 - r2 y)) from the hardware's
// approximate float64 reciprocal (rcp.approx.ftz.f64, relative error about
// 2^-22): after two steps the relative error is at the rounding level. Four
// FP64 operations. r2 > 0 and normal.
__device__ __forceinline__ double recip_r2(double r2)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(r2));
    double e = fma(-r2, y, 1.0);
    y = fma(y, e, y);
    e = fma(-r2, y, 1.0);
    return fma(y, e, y);
}

// a8 (target gradient): grad Re phi at the evaluation points, psi[(e * 2 + c) * ND + d]
// (c = 0: d/dx, 1: d/dy), one leaf per warp as in k_leaf64 (directed):
//   L2P  d/dz sum_l L_l u^l = (1/R) sum_l l L_l u^(l-1)  -> (Re, -Im)
//   M2P  d/dz [M_0 log(z - c) + sum_k M_k v^k] = (M_0 - sum_k k M_k v^k) / (z - c)
//   P2P  sum_j q_j (z - z_j) / |z - z_j|^2   (coincident pairs skipped)
// One directed pair costs 11 FP64 operations (differences, r^2, the reciprocal,
// q / r^2 and two accumulations).
template <int P, int ND>
__global__ void __launch_bounds__(kGradWarps64 * 32)
    k_leaf_grad64(DevTree t, PassGeom g, const double* __restrict__ q, const double2* __restrict__ M,
                  const double2* __restrict__ L, double* __restrict__ psi, int* __restrict__ work)
{
    constexpr int P1 = P + 1;
    __shared__ LeafStage64<ND> stage[kGradWarps64];
    const int lane = threadIdx.x & 31;
    LeafStage64<ND>& st = stage[threadIdx.x >> 5];
    for (;;) {
        int li = 0;
        if (lane == 0) li = atomicAdd(work, 1);
        li = __shfl_sync(0xffffffffu, li, 0);
        if (li >= t.nleaf) break;
        const int b = t.leaves[li];
        const int e0 = g.erng[2 * b], e1 = g.erng[2 * b + 1];
        if (e0 == e1) continue;
        const double2 cb = t.center[b];
        const double invRb = 1.0 / t.radius[b];
        const int u0 = t.u_ptr[b], u1 = t.u_ptr[b + 1];
        const int w0 = t.w_ptr[b], w1 = t.w_ptr[b + 1];
        for (int gb = e0; gb < e1; gb += 32) {
            // a group of fewer than 32 points is shared by ksplit sub-groups of lanes
            // that divide the sources among them (as in k_leaf64)
            const int gcount = min(32, e1 - gb);
            const int ksplit = 32 / gcount;
            const int sub = lane / gcount;
            const int ti = gb + lane % gcount;
            const bool valid = sub < ksplit;
            const double2 z = valid ? g.exy[ti] : cb;
            double gx[ND], gy[ND];
            {
                const double2 u = make_double2((z.x - cb.x) * invRb, (z.y - cb.y) * invRb);
                const double2* Lb = L + (int64_t)b * P1 * ND;
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double2 lp = Lb[P * ND + d];
                    double2 s = make_double2(lp.x * P, lp.y * P);
#pragma unroll 4
                    for (int l = P - 1; l >= 1; --l) {
                        const double2 c = Lb[l * ND + d];
                        s = cfma64(s, u, make_double2(c.x * l, c.y * l));
                    }
                    gx[d] = s.x * invRb;
                    gy[d] = -s.y * invRb;
                }
            }
            for (int e = w0; e < w1; ++e) {
                const int D = t.w_idx[e];
                const double2 cD = t.center[D];
                const double RD = t.radius[D];
                const double dx = z.x - cD.x, dy = z.y - cD.y;
                const double ir = recip_r2(fma(dx, dx, dy * dy));
                const double2 inv = make_double2(dx * ir, -dy * ir);  // 1/(z - c)
                const double2 v = make_double2(inv.x * RD, inv.y * RD);
                const double2* MD = M + (int64_t)D * P1 * ND;
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    double2 s = make_double2(0.0, 0.0);
#pragma unroll 2
                    for (int k = P; k >= 1; --k) {
                        const double2 m = MD[k * ND + d];
                        s = cmul64(make_double2(fma(m.x, (double)k, s.x), fma(m.y, (double)k, s.y)), v);
                    }
                    const double2 dphi = cmul64(inv, make_double2(MD[d].x - s.x, MD[d].y - s.y));
                    gx[d] += dphi.x;
                    gy[d] -= dphi.y;
                }
            }
            double nx[ND], ny[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) nx[d] = ny[d] = 0.0;
            for (int e = u0; e < u1; ++e) {
                const int A = t.u_idx[e];
                const int a0 = g.crng[2 * A], a1 = g.crng[2 * A + 1];
                for (int c = a0; c < a1; c += 32) {
                    const int n = min(32, a1 - c);
                    __syncwarp();
                    if (lane < n) {
                        st.xy[lane] = g.cxy[c + lane];
#pragma unroll
                        for (int d = 0; d < ND; ++d) st.q[lane][d] = q[(int64_t)(c + lane) * ND + d];
                    }
                    __syncwarp();
                    if (valid) {
#pragma unroll 4
                        for (int j = sub; j < n; j += ksplit) {
                            const double2 sp = st.xy[j];
                            const double dx = z.x - sp.x, dy = z.y - sp.y;
                            const double r2 = fma(dx, dx, dy * dy);
                            const double ir = r2 == 0.0 ? 0.0 : recip_r2(r2);  // coincident: no term
#pragma unroll
                            for (int d = 0; d < ND; ++d) {
                                const double qr = st.q[j][d] * ir;
                                nx[d] = fma(qr, dx, nx[d]);
                                ny[d] = fma(qr, dy, ny[d]);
                            }
                        }
                    }
                }
            }
            for (int sg = 1; sg < ksplit; ++sg) {  // warp-uniform
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double vx = __shfl_down_sync(0xffffffffu, nx[d], sg * gcount);
                    const double vy = __shfl_down_sync(0xffffffffu, ny[d], sg * gcount);
                    if (sub == 0) {
                        nx[d] += vx;
                        ny[d] += vy;
                    }
                }
            }
            if (valid && sub == 0) {
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    psi[((int64_t)ti * 2 + 0) * ND + d] = gx[d] + nx[d];
                    psi[((int64_t)ti * 2 + 1) * ND + d] = gy[d] + ny[d];
                }
            }
        }
    }
}

// Adds the symmetric near field's slots to the receiving points, one thread per
// point, slots in a fixed order (deterministic results).
template <int ND>
__global__ void k_sym_reduce64(DevTree t, PassGeom g, const double* __restrict__ slots, double* __restrict__ psi)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.n_eval; j += gridDim.x * blockDim.x) {
        const int A = t.sym_pt_leaf[j];
        const int s0 = t.sym_in_ptr[A], s1 = t.sym_in_ptr[A + 1];
        if (s0 == s1) continue;
        const int jl = j - g.erng[2 * A];
        double acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = 0.0;
#pragma unroll 4
        for (int k = s0; k < s1; ++k) {
            const int64_t o = (t.sym_in_slot[k] + jl) * ND;
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[d] += slots[o + d];
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) psi[(int64_t)j * ND + d] = fma(0.5, acc[d], psi[(int64_t)j * ND + d]);
    }
}

// component c of (sgn i)^m (X + i Y)
__device__ __forceinline__ __int128 quarter_turn(__int128 X, __int128 Y, int m, int sgn, int c)
{
    __int128 re, im;
    switch (m & 3) {
        case 0: re = X, im = Y; break;
        case 1: re = -Y, im = X; break;
        case 2: re = -X, im = -Y; break;
        default: re = Y, im = -X; break;
    }
    __int128 v = c ? im : re;
    return (sgn < 0 && (m & 1)) ? -v : v;
}

// a 128-bit integer from the lane `lane ^ o` of `mask`
__device__ __forceinline__ __int128 shfl_xor_i128(unsigned mask, __int128 v, int o)
{
    const long long hi = __shfl_xor_sync(mask, (long long)(v >> 64), o);
    const unsigned long long lo = __shfl_xor_sync(mask, (unsigned long long)v, o);
    return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
}

// ----------------------------------------------------------------------------
// a3: P2M, one warp per leaf: lane k sums q_j u_j^k over the leaf's points (u =
// (z - c)/R), the powers read from the plan's per-point table (formed once, the
// geometry being static); lane 0 sums q_j. Scaled: M_k = -(1/k) sum_j q_j u_j^k.
template <int P, int ND>
__global__ void __launch_bounds__(kW64 * 32)
    k_p2m64(DevTree t, PassGeom g, const double* __restrict__ q, double2* __restrict__ M)
{
    constexpr int P1 = P + 1;
    const int lane = threadIdx.x & 31;
    const double sc = lane == 0 ? 1.0 : -1.0 / (double)lane;
    for (int li = gwarp(); li < t.nleaf; li += nwarps()) {
        const int b = t.leaves[li];
        const int s0 = g.crng[2 * b], s1 = g.crng[2 * b + 1];
        double2 acc[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[d] = make_double2(0.0, 0.0);
        if (lane <= P) {
#pragma unroll 4
            for (int j = s0; j < s1; ++j) {
                const double2 pv = lane == 0 ? make_double2(1.0, 0.0) : g.cpow[(int64_t)j * P + lane - 1];
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double qv = q[(int64_t)j * ND + d];
                    acc[d].x = fma(qv, pv.x, acc[d].x);
                    acc[d].y = fma(qv, pv.y, acc[d].y);
                }
            }
#pragma unroll
            for (int d = 0; d < ND; ++d)
                M[((int64_t)b * P1 + lane) * ND + d] = make_double2(acc[d].x * sc, acc[d].y * sc);
        }
    }
}

// a3: M2M into the non-leaf boxes of one level (levels from the deepest up),
// exactly, on the integer pipes. With zeta = s/2 the offset of child c from the
// parent's centre over the parent half-side, s = sx + i sy (sx, sy = +-1 by
// quadrant), the scaled M2M of the child's multipole M is
//   B_l = -M_0 zeta^l / l + sum_{k=1..l} C(l-1, k-1) 2^-k M_k zeta^(l-k)   (l >= 1),
//   B_0 = M_0,
// which factors (2^-k zeta^(l-k) = 2^-l s^l s^-k, s^-1 = conj(s)/2) as
//   a_k = conj(s)^k 2^-k M_k,  beta_n = sum_{j<=n} C(n, j) a_{j+1},
//   B_l = 2^-l s^l (beta_{l-1} - M_0 / l).
// conj(s)^k 2^-k and 2^-l s^l are quarter turns times powers of two (times
// conj(s) or s for odd powers, one addition), beta is the binomial transform of
// a (P(P-1)/2 additions, real and imaginary parts apart). In 128-bit fixed point
// with one scale 2^F per parent and density, from the exponents of the four
// children's coefficients so that every partial sum stays below 2^125, all of it
// is exact (M_0 / l by an integer division, to one unit of 2^-F): the parent's
// coefficients are the correctly rounded sums of the four translations. Eight
// lanes per parent: lane 2c + r of the group carries the real (r = 0) or
// imaginary (r = 1) sums of child c; partners swap by shuffles, the children's
// sums are added by shuffles, and the lanes of child 0 store. A parent with an
// infinity or NaN among its children's coefficients takes the float64 table
// m2m[c][l][k] = C(l-1, k-1) 2^-k zeta_c^(l-k) (k >= 1), -zeta_c^l / l (k = 0).
constexpr int kM2MThreads = 128;

template <int P, int ND>
__global__ void __launch_bounds__(kM2MThreads)
    k_m2m64(DevTree t, DevTables tab, int b0, int b1, double2* __restrict__ M)
{
    constexpr int P1 = P + 1;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int g8 = (int)(gid & 7), c = g8 >> 1, r = g8 & 1;
    const int64_t bi = b0 + (gid >> 3);
    if (bi >= b1) return;  // the whole group of eight leaves together
    const int b = (int)bi;
    if (t.is_leaf[b]) return;
    const unsigned grp = 0xffu << ((threadIdx.x & 31) & ~7);
    const int ch = t.child[4 * b + c];
    const int sx = (c & 1) ? 1 : -1, sy = (c & 2) ? 1 : -1, sg = sx * sy;
    const double2* Mc = M + (int64_t)(ch >= 0 ? ch : 0) * P1 * ND;
    double* Mb = reinterpret_cast<double*>(M + (int64_t)b * P1 * ND);
#pragma unroll 1
    for (int d = 0; d < ND; ++d) {
        // H = max(e_0, max_{k>=1} (e_k - floor(k/2))) over the four children,
        // |Re M_k|, |Im M_k| < 2^e_k (a missing child: zeros)
        int H = -1021;
        bool finite = true;
        if (ch >= 0) {
#pragma unroll
            for (int k = 0; k <= P; ++k) {
                const double2 v = Mc[k * ND + d];
                const unsigned e = max(max(exponent_field(v.x), exponent_field(v.y)), 1u);
                finite = finite && e < 0x7ffu;
                H = max(H, (int)e - 1022 - k / 2);
            }
        }
        H = max(H, __shfl_xor_sync(grp, H, 2));
        H = max(H, __shfl_xor_sync(grp, H, 4));
        finite = __all_sync(grp, finite);
        if (!finite) {
            const double2* tc = tab.m2m64 + (size_t)c * P1 * P1;
            for (int l = 0; l <= P; ++l) {
                double acc = 0.0;
                if (ch >= 0) {
                    if (l == 0) {
                        acc = r ? Mc[d].y : Mc[d].x;
                    } else {
                        for (int k = 0; k <= l; ++k) {
                            const double2 z = tc[l * P1 + k], v = Mc[k * ND + d];
                            acc += r ? z.x * v.y + z.y * v.x : z.x * v.x - z.y * v.y;
                        }
                    }
                }
                acc += __shfl_xor_sync(grp, acc, 2);
                acc += __shfl_xor_sync(grp, acc, 4);
                if (c == 0) Mb[(l * ND + d) * 2 + r] = acc;
            }
            continue;
        }
        // every partial sum and the four children's total: below
        // 4 sqrt2 (2^(P-1) P + 1) 2^(H + 1/2) <= 2^(H + P + 7) for P <= 30
        const int F = 118 - P - H;
        __int128 a[P];  // a[j] = a_{j+1}, then beta_j
#pragma unroll
        for (int k = 1; k <= P; ++k) {
            const double2 v = ch >= 0 ? Mc[k * ND + d] : make_double2(0.0, 0.0);
            const int m = k >> 1;
            __int128 X, Y;
            if ((k & 1) == 0) {
                X = fixed128(v.x, F - m);
                Y = fixed128(v.y, F - m);
            } else {  // times conj(s)
                const __int128 x = fixed128(v.x, F - m - 1), y = fixed128(v.y, F - m - 1);
                X = (sx > 0 ? x : -x) + (sy > 0 ? y : -y);
                Y = (sx > 0 ? y : -y) - (sy > 0 ? x : -x);
            }
            a[k - 1] = quarter_turn(X, Y, m, -sg, r);
        }
        // binomial transform: beta_n = sum_{j<=n} C(n, j) a_{j+1}
#pragma unroll
        for (int i = 1; i < P; ++i)
#pragma unroll
            for (int j = P - 1; j >= i; --j) a[j] += a[j - 1];
        const double2 m0 = ch >= 0 ? Mc[d] : make_double2(0.0, 0.0);
        const __int128 q0 = fixed128(r ? m0.y : m0.x, F);
        {  // B_0 = sum of the children's M_0
            __int128 v = q0;
            v += shfl_xor_i128(grp, v, 2);
            v += shfl_xor_i128(grp, v, 4);
            if (c == 0) Mb[d * 2 + r] = int128_ldexp(v, -F);
        }
#pragma unroll
        for (int l = 1; l <= P; ++l) {
            const __int128 mine = a[l - 1] - q0 / (__int128)l;
            const __int128 other = shfl_xor_i128(grp, mine, 1);
            const __int128 Cx = r ? other : mine, Cy = r ? mine : other;
            const int m = l >> 1;
            __int128 X = Cx, Y = Cy;
            int sc = -F - m;
            if (l & 1) {  // times s
                X = (sx > 0 ? Cx : -Cx) - (sy > 0 ? Cy : -Cy);
                Y = (sy > 0 ? Cx : -Cx) + (sx > 0 ? Cy : -Cy);
                sc -= 1;
            }
            __int128 v = quarter_turn(X, Y, m, sg, r);
            v += shfl_xor_i128(grp, v, 2);
            v += shfl_xor_i128(grp, v, 4);
            if (c == 0) Mb[(l * ND + d) * 2 + r] = int128_ldexp(v, sc);
        }
    }
}

// ----------------------------------------------------------------------------
// a4: M2L over the V list plus P2L over the X list, one warp per target box.
//
// For a V-list entry with source box C and offset o (t = R/z0 from the offset
// table) the local coefficients of the target box receive
//   L_l += t^l Y_l,   Y_l = sum_{k=0..P} H[l][k] A_k,   l = 1..P,
//   A_k = M_k (-t)^k (k >= 1), A_0 = M_0, H[l][k] = C(l+k-1, k-1), H[l][0] = -1/l,
//   Re L_0 += M_0 log|z0| + sum_{k>=1} Re A_k.
// With tau = 2^-1.5 and the scaled operands H'[l][k] = H[l][k] tau^k, A'_k =
// M_k (-t/tau)^k (so that H' A' = H A term by term), both operands are bounded:
// |A'_k| <= sum |q| / k because |t| <= 1/4 and the scaled multipole satisfies
// |M_k| <= sum |q| 2^(k/2) / k, and every H'[l][k] t^l u^l (|u| <= sqrt 2 at an
// evaluation point) is at most 2^-1.5.
//
// The products Y = H' A' run on the tensor cores, exactly: each operand is
// rounded to 62-bit fixed point (H' per row, A' per column, with a power-of-two
// scale) and split into eight signed 8-bit digits, x = sum_j d_j 2^(8 (7 - j));
// a digit is an integer of at most 8 significant bits and so exact in bf16.
// mma.sync m16n8k16 (bf16 inputs, f32 accumulation) forms for each level n the
// sum S_n = sum_{i+j=n} Hd_i Ad_j over k: products of two digits are at most
// 2^14 and |S_n| < 2^22, so every partial sum is an integer below 2^24 and the
// f32 accumulation is exact. Levels n <= 7 are kept (36 digit products; the rest
// lie below 2^-62 of the operands' scales per term) and combined in 64-bit
// integers, Y = sum_n S_n 2^(40 - 8n) (S_6, S_7 rounded down by 8 and 16 bits),
// converted once to float64 and scaled by a power of two folded into t^l. The
// result differs from the exact product of the float64 operands by about 2^-55
// of (row maximum x column maximum), the size of float64 rounding in the same
// (P + 1)-term sum; with the bounds above that is below 2^-55 * 2^-1.5 * sum |q|
// in the potential per V-list pair. The float64 work left per pair is A' (one
// complex multiply per k), the conversions and t^l Y_l: about 11 P operations
// against 2 P^2 + 10 P for the sum itself.
//
// A warp takes G entries at a time (8 tensor columns per n-tile: real and
// imaginary parts of G entries x ND densities), forms A' (item (entry, k) per
// lane), the column exponents (shared-memory maximum), the digits of A' into
// its shared tile, then per 16-row m-tile the 28 digit products of levels 0-6
// (two k-steps each), and adds t^l Y_l into the lane's rows (fragment row
// groups) and column pair. The X list (P2L) then adds
//   L_0 += q log|z - c|,  L_l -= (q / l) v^l,  v = R/(z - c),
// with lane l owning L_l; kXB sources at a time (lane j forms the powers of v_j).
constexpr int kSl = 8;   // 8-bit digits per operand
constexpr int kHs = 40;  // row stride (bf16 elements) of the digit tiles: conflict-free fragment loads
constexpr int kXB = 16;  // X-list sources per batch
constexpr size_t kHdBytes = (size_t)kSl * 32 * kHs * sizeof(uint16_t);

template <int P, int ND>
struct M2LTShape {
    static constexpr int P1 = P + 1;
    static constexpr int MT = (P + 15) / 16;           // m-tiles of 16 rows (l = 1..P)
    static constexpr int NT = ND <= 4 ? 1 : ND / 4;    // n-tiles of 8 columns
    static constexpr int NCOL = 8 * NT;
    static constexpr int G = NCOL / (2 * ND);          // V-list entries per group
    static constexpr int RA = (G * P + 31) / 32;       // rounds of the A' items (entry, k = 1..P)
    static constexpr int RS = (NCOL * P1 + 31) / 32;   // rounds of the digit items (column, k = 0..P)
    // per-warp shared memory: A' [G][P1][ND] double2 and the digits [kSl][NCOL][kHs]
    // bf16 for the V list, the same space for the X list's powers [kXB][P1] double2;
    // charges and logs [kXB][ND + 1] double; column exponents [G ND], entry offsets [G]
    static constexpr size_t kAs = (size_t)G * P1 * ND * 16;
    static constexpr size_t kBt = (size_t)kSl * NCOL * kHs * 2;
    static constexpr size_t kPw = (size_t)kXB * P1 * 16;
    static constexpr size_t kR1 = kAs + kBt > kPw ? kAs + kBt : kPw;
    static constexpr size_t kQl = (((size_t)kXB * (ND + 1) * 8) + 15) & ~(size_t)15;
    static constexpr size_t kEx = (((size_t)(G * ND + G) * 4) + 15) & ~(size_t)15;
    static constexpr size_t kWarp = kR1 + kQl + kEx;
};

template <int P, int ND>
size_t m2l64_smem()
{
    return kHdBytes + 128 + (size_t)kW64 * M2LTShape<P, ND>::kWarp;
}

// unbiased binary exponent of |x| (a large negative sentinel for zero)
__device__ __forceinline__ int expo64(double x)
{
    const int E = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
    return E == 0 ? -4000 : E - 1023;
}

// round(x 2^(62 - e)) for |x| < 2^(e - 1), by integer operations on the bits of
// x: |result| < 2^61 (zero and subnormal x give 0)
__device__ __forceinline__ long long fixed62(double x, int e)
{
    const long long bits = __double_as_longlong(x);
    const int E = (int)((bits >> 52) & 0x7ff);
    if (E == 0) return 0;
    const long long mant = (bits & 0xfffffffffffffLL) | 0x10000000000000LL;
    const int sh = E - 1075 + 62 - e;  // x 2^(62 - e) = mant 2^sh, sh <= 8
    long long X;
    if (sh >= 0)
        X = mant << sh;
    else if (sh < -62)
        X = 0;
    else
        X = (mant + (1LL << (-sh - 1))) >> (-sh);
    return bits < 0 ? -X : X;
}

// bf16 bit pattern of an integer |d| <= 2^8 (exact): through the f32 value
// 1.5 2^23 + d, whose unit in the last place is 1
__device__ __forceinline__ uint16_t bf16_digit(int d)
{
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return (uint16_t)(__float_as_uint(f) >> 16);
}

// integer value of an f32 holding an integer |v| < 2^22 (same device as above)
__device__ __forceinline__ long long int_of_f32(float v)
{
    return (long long)(__float_as_int(v + 12582912.0f) - 0x4B400000);
}

// v 2^sc by the exponent field (0 below the normal range)
__device__ __forceinline__ double scale_pow2(double v, int sc)
{
    const long long bits = __double_as_longlong(v);
    const int E = (int)((bits >> 52) & 0x7ff);
    const int En = E + sc;
    if (E == 0 || En <= 0) return 0.0;
    if (En >= 2047) return ldexp(v, sc);
    return __longlong_as_double(bits + (long long)sc * (1LL << 52));
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int P, int ND>
__global__ void __launch_bounds__(kW64 * 32, ND <= 2 ? 4 : 2)
    k_m2l64(DevTree t, DevTables tab, PassGeom g, const double2* __restrict__ M, double2* __restrict__ L,
            const double* __restrict__ q, const double2* __restrict__ logtab, const double* __restrict__ etab)
{
    using S = M2LTShape<P, ND>;
    constexpr int P1 = S::P1, MT = S::MT, NT = S::NT, NCOL = S::NCOL, G = S::G, RA = S::RA, RS = S::RS;
    extern __shared__ __align__(16) unsigned char smem_m2l[];
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;  // fragment row group, column pair
    uint16_t* Hd = reinterpret_cast<uint16_t*>(smem_m2l);           // [kSl][32][kHs]
    int* eHs = reinterpret_cast<int*>(smem_m2l + kHdBytes);         // [32]
    unsigned char* wbase = smem_m2l + kHdBytes + 128 + (size_t)wb * S::kWarp;
    double2* As = reinterpret_cast<double2*>(wbase);                // [G][P1][ND]
    uint16_t* Bt = reinterpret_cast<uint16_t*>(wbase + S::kAs);     // [kSl][NCOL][kHs]
    double2* pws = reinterpret_cast<double2*>(wbase);                               // [kXB][P1] (X list)
    double* qls = reinterpret_cast<double*>(wbase + S::kR1);                         // [kXB][ND + 1]
    int* em = reinterpret_cast<int*>(wbase + S::kR1 + S::kQl);                       // [G ND]
    int* eo = em + G * ND;                                                                // [G]
    for (int i = threadIdx.x; i < (int)(kHdBytes / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(Hd)[i] = tab.m2lh[i];
    for (int i = threadIdx.x; i < 32; i += blockDim.x) eHs[i] = tab.m2le[i];
    for (int i = lane; i < (int)(S::kBt / 4); i += 32) reinterpret_cast<uint32_t*>(Bt)[i] = 0u;  // k padding stays 0
    __syncthreads();

    // this lane's A' items: entry slot and coefficient k = 1..P per round, and tau^k
    int it_s[RA], it_k[RA];
    double tauk[RA];
#pragma unroll
    for (int r = 0; r < RA; ++r) {
        const int f = r * 32 + lane;
        const bool on = f < G * P;
        it_s[r] = on ? f / P : -1;
        it_k[r] = on ? f % P + 1 : 1;
        tauk[r] = tab.tau_pow[it_k[r]];
    }

    for (int b = gwarp(); b < t.nbox; b += nwarps()) {
        double2 lacc[2 * MT][NT];
#pragma unroll
        for (int i = 0; i < 2 * MT; ++i)
#pragma unroll
            for (int n = 0; n < NT; ++n) lacc[i][n] = make_double2(0.0, 0.0);
        double l0d[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) l0d[d] = 0.0;
        const int v0 = t.v_ptr[b], v1 = t.v_ptr[b + 1];
        const int bx = t.ixy[2 * b], by = t.ixy[2 * b + 1];
        const double logR = t.log_radius[b];
        for (int e0 = v0; e0 < v1; e0 += G) {
            __syncwarp();
            if (lane < G * ND) em[lane] = -4000;
            if (lane < G) eo[lane] = -1;
            __syncwarp();
            // A'_k of the G entries (item (s, k) per lane and round), the column
            // exponents, and this lane's share of Re L_0
#pragma unroll
            for (int r = 0; r < RA; ++r) {
                const int s = it_s[r], k = it_k[r];
                int exd[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) exd[d] = -4000;
                const int e = e0 + s;
                if (s >= 0 && e < v1) {
                    const int C = t.v_idx[e];
                    const int o = (t.ixy[2 * C + 1] - by + 3) * 7 + (t.ixy[2 * C] - bx + 3);
                    const double2 mt = tab.mtpow_s[o * P1 + k];
                    const double2* MC = M + (int64_t)C * P1 * ND;
                    if (k == 1) eo[s] = o;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const double2 a = cmul64(MC[k * ND + d], mt);
                        As[(s * P1 + k) * ND + d] = a;
                        l0d[d] = fma(a.x, tauk[r], l0d[d]);
                        exd[d] = max(expo64(a.x), expo64(a.y));
                        if (k == 1) {
                            const double2 m0 = MC[d];
                            As[(s * P1) * ND + d] = m0;
                            l0d[d] = fma(m0.x, logR + tab.log2o[o], l0d[d]);
                            exd[d] = max(exd[d], max(expo64(m0.x), expo64(m0.y)));
                        }
                    }
                } else if (s >= 0) {
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        As[(s * P1 + k) * ND + d] = make_double2(0.0, 0.0);
                        if (k == 1) As[(s * P1) * ND + d] = make_double2(0.0, 0.0);
                    }
                }
                // maximum over the lanes of one entry (consecutive lanes of the round):
                // a segmented reduction downwards, the segment's first lane publishes
                bool same[5];
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    const int s2 = __shfl_down_sync(0xffffffffu, s, 1 << i);
                    same[i] = lane + (1 << i) < 32 && s2 == s;
                }
                const int sp = __shfl_up_sync(0xffffffffu, s, 1);
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    int m = exd[d];
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        const int v = __shfl_down_sync(0xffffffffu, m, 1 << i);
                        if (same[i]) m = max(m, v);
                    }
                    if (s >= 0 && (lane == 0 || sp != s)) atomicMax(&em[s * ND + d], m);
                }
            }
            __syncwarp();
            // digits of A': item (column c, k), column c = (s ND + d) 2 + (0: real, 1: imaginary)
#pragma unroll
            for (int r = 0; r < RS; ++r) {
                const int f = r * 32 + lane;
                if (f >= NCOL * P1) continue;
                const int c = f / P1, k = f % P1, sd = c >> 1;
                const double2 a = As[((sd / ND) * P1 + k) * ND + sd % ND];
                long long X = fixed62((c & 1) ? a.y : a.x, em[sd] + 2);
                uint16_t* dst = Bt + (size_t)c * kHs + k;
#pragma unroll
                for (int j = kSl - 1; j >= 1; --j) {
                    const int dj = (int)(signed char)(X & 0xff);
                    dst[(size_t)j * NCOL * kHs] = bf16_digit(dj);
                    X = (X - dj) >> 8;
                }
                dst[0] = bf16_digit((int)X);
            }
            __syncwarp();
            // Y = H' A' on the tensor cores, level by level, then L_l += t^l Y_l
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                uint32_t bfr[kSl][2][2];
#pragma unroll
                for (int j = 0; j < kSl; ++j)
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint16_t* col = Bt + ((size_t)j * NCOL + 8 * nt + gq) * kHs + 16 * ks + 2 * tq;
                        bfr[j][ks][0] = *reinterpret_cast<const uint32_t*>(col);
                        bfr[j][ks][1] = *reinterpret_cast<const uint32_t*>(col + 8);
                    }
                const int sd = 4 * nt + tq;  // this lane's column pair
                const int o = eo[sd / ND];
                const int eA = em[sd] + 2;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    float acc[kSl][4];
#pragma unroll
                    for (int n = 0; n < kSl; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                        for (int i = 0; i < kSl; ++i) {
                            const uint16_t* hr = Hd + ((size_t)i * 32 + 16 * mt + gq) * kHs + 16 * ks + 2 * tq;
                            const uint32_t a0 = *reinterpret_cast<const uint32_t*>(hr);
                            const uint32_t a1 = *reinterpret_cast<const uint32_t*>(hr + 8 * kHs);
                            const uint32_t a2 = *reinterpret_cast<const uint32_t*>(hr + 8);
                            const uint32_t a3 = *reinterpret_cast<const uint32_t*>(hr + 8 * kHs + 8);
#pragma unroll
                            for (int j = 0; j + i < kSl; ++j)
                                mma_bf16_16816(acc[i + j], a0, a1, a2, a3, bfr[j][ks][0], bfr[j][ks][1]);
                        }
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int row = 16 * mt + 8 * h + gq, l = row + 1;
                        if (l > P || o < 0) continue;
                        long long yr = 0, yi = 0;
#pragma unroll
#pragma unroll
                        for (int n = 0; n < 6; ++n) {
                            yr += int_of_f32(acc[n][2 * h]) * (1LL << (40 - 8 * n));
                            yi += int_of_f32(acc[n][2 * h + 1]) * (1LL << (40 - 8 * n));
                        }
                        yr += (int_of_f32(acc[6][2 * h]) >> 8) + (int_of_f32(acc[7][2 * h]) >> 16);
                        yi += (int_of_f32(acc[6][2 * h + 1]) >> 8) + (int_of_f32(acc[7][2 * h + 1]) >> 16);
                        const int sc = eHs[row] + eA - 52;
                        const double2 tl = tab.tpow[o * P1 + l];
                        const double2 ts = make_double2(scale_pow2(tl.x, sc), scale_pow2(tl.y, sc));
                        lacc[2 * mt + h][nt] = cfma64(ts, make_double2((double)yr, (double)yi), lacc[2 * mt + h][nt]);
                    }
                }
            }
        }
        // the column pairs of one density are summed over the lanes that hold
        // them (tq with the same (4 nt + tq) mod ND), then lane l takes L_l
#pragma unroll
        for (int i = 0; i < 2 * MT; ++i)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int off = ND; off < 4; off <<= 1) {
                    lacc[i][n].x += __shfl_xor_sync(0xffffffffu, lacc[i][n].x, off);
                    lacc[i][n].y += __shfl_xor_sync(0xffffffffu, lacc[i][n].y, off);
                }
        __syncwarp();
        if (tq < ND) {
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int l = 16 * mt + 8 * h + gq + 1;
                    if (l > P) continue;
#pragma unroll
                    for (int n = 0; n < NT; ++n) As[l * ND + (4 * n + tq) % ND] = lacc[2 * mt + h][n];
                }
        }
        __syncwarp();
        double2 lo[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            double s0 = l0d[d];
            for (int off = 16; off > 0; off >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, off);
            lo[d] = make_double2(0.0, 0.0);
            if (lane == 0)
                lo[d].x = s0;
            else if (lane <= P)
                lo[d] = As[lane * ND + d];
        }
        // X list (P2L), lane l <= P owns L_l
        const int x0 = t.x_ptr[b], x1 = t.x_ptr[b + 1];
        if (x1 > x0) {
            const double2 c = t.center[b];
            const double Rb = t.radius[b];
            const double inv_ll = (lane == 0 || lane > P) ? 0.0 : 1.0 / (double)lane;
            for (int e = x0; e < x1; ++e) {
                const int Cx = t.x_idx[e];
                const int s0 = g.crng[2 * Cx], s1 = g.crng[2 * Cx + 1];
                for (int base = s0; base < s1; base += kXB) {
                    const int n = min(kXB, s1 - base);
                    __syncwarp();
                    if (lane < n) {
                        const double2 z = g.cxy[base + lane];
                        const double dx = z.x - c.x, dy = z.y - c.y;
                        const double r2 = fma(dx, dx, dy * dy);
                        const double sc = Rb / r2;
                        const double2 v = make_double2(dx * sc, -dy * sc);
                        double2 pw = make_double2(1.0, 0.0);
                        pws[lane * P1] = pw;
                        for (int k = 1; k <= P; ++k) {
                            pw = cmul64(pw, v);
                            pws[lane * P1 + k] = pw;
                        }
#pragma unroll
                        for (int d = 0; d < ND; ++d) qls[lane * (ND + 1) + d] = q[(int64_t)(base + lane) * ND + d];
                        qls[lane * (ND + 1) + ND] = 0.5 * log_r2(r2, logtab, etab);
                    }
                    __syncwarp();
                    if (lane <= P) {
                        for (int j = 0; j < n; ++j) {
                            if (lane == 0) {
#pragma unroll
                                for (int d = 0; d < ND; ++d)
                                    lo[d].x = fma(qls[j * (ND + 1) + d], qls[j * (ND + 1) + ND], lo[d].x);
                            } else {
                                const double2 pv = pws[j * P1 + lane];
#pragma unroll
                                for (int d = 0; d < ND; ++d) {
                                    const double cq = -qls[j * (ND + 1) + d] * inv_ll;
                                    lo[d].x = fma(cq, pv.x, lo[d].x);
                                    lo[d].y = fma(cq, pv.y, lo[d].y);
                                }
                            }
                        }
                    }
                }
            }
            // the powers shared the digit tile's space: zero its k padding again
            __syncwarp();
            for (int i = lane; i < kSl * NCOL * (32 - P1); i += 32)
                Bt[(i / (32 - P1)) * kHs + P1 + i % (32 - P1)] = 0;
        }
        if (lane <= P) {
#pragma unroll
            for (int d = 0; d < ND; ++d) L[((int64_t)b * P1 + lane) * ND + d] = lo[d];
        }
    }
}

// ----------------------------------------------------------------------------
// a5: L2L into the boxes of one level, exactly, on the integer pipes. With
// zeta = s/2 the child's centre offset over the parent half-side, s = sx + i sy
// (sx, sy = +-1 by quadrant), the scaled translation
//   L'_l = sum_{k>=l} C(k, l) 2^-l zeta^(k-l) L_k
// factors as a_k = s^k 2^-k L_k, b_l = sum_{k>=l} C(k, l) a_k, L'_l = conj(s)^l 2^-l b_l
// (2^-l zeta^-l = s^-l and s^-1 = conj(s)/2). Since s^2 = 2 i sx sy, s^k 2^-k is
// (i sx sy)^m 2^-m for k = 2m and (i sx sy)^m s 2^-(m+1) for k = 2m + 1: a_k and
// L'_l take sign changes, swaps, one addition and power-of-two scales; b is the
// Taylor shift of a by 1 (P(P+1)/2 additions, real and imaginary parts apart).
// In 128-bit fixed point with one scale 2^F per parent and density, chosen from
// the exponents of L so that every partial sum stays below 2^125 (a partial sum
// of the shift is at most sum_k 2^k |a_k| = sum_k 2^(k/2) |L_k|), all of it is
// exact and only the conversions round: L'_l is the correctly rounded value of
// the translation of the parent's coefficients, with no FP64 instruction but
// the final addition. Two lanes per child box: lane c of the pair carries the
// real (c = 0) or imaginary (c = 1) sums and the pair swaps them by one shuffle
// per coefficient at the end. A parent holding an infinity or NaN takes the
// float64 table (l2l[c][l][k] = C(k, l) 2^-l zeta_c^(k-l)) instead.
constexpr int kL2LThreads = 128;


template <int P, int ND>
__global__ void __launch_bounds__(kL2LThreads)
    k_l2l64(DevTree t, DevTables tab, int b0, int b1, double2* __restrict__ L)
{
    constexpr int P1 = P + 1;
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int c = (int)(gid & 1);
    const int64_t bi = b0 + (gid >> 1);
    // a pair past the level's end repeats its last box and stores nothing
    const bool live = bi < b1;
    const int b = live ? (int)bi : b1 - 1;
    const unsigned pair = 3u << ((threadIdx.x & 31) & ~1);
    const int p = t.parent[b];
    const int cq = (t.ixy[2 * b] & 1) | ((t.ixy[2 * b + 1] & 1) << 1);
    const int sx = (cq & 1) ? 1 : -1, sy = (cq & 2) ? 1 : -1, sg = sx * sy;
    const double2* Lp = L + (int64_t)p * P1 * ND;
    double* Lc = reinterpret_cast<double*>(L + (int64_t)b * P1 * ND);
#pragma unroll 1
    for (int d = 0; d < ND; ++d) {
        // G = max_k (ceil(k/2) + e_k), |Re L_k|, |Im L_k| < 2^e_k
        int G = -(1 << 20);
        bool finite = true;
#pragma unroll
        for (int k = 0; k <= P; ++k) {
            const double2 v = Lp[k * ND + d];
            const unsigned e = max(max(exponent_field(v.x), exponent_field(v.y)), 1u);
            finite = finite && e < 0x7ffu;
            G = max(G, (k + 1) / 2 + (int)e - 1022);
        }
        if (!finite) {
            const double2* tc = tab.l2l64 + (size_t)cq * P1 * P1;
            for (int l = 0; l <= P; ++l) {
                double acc = 0.0;
                for (int k = l; k <= P; ++k) {
                    const double2 z = tc[l * P1 + k], v = Lp[k * ND + d];
                    acc += c ? z.x * v.y + z.y * v.x : z.x * v.x - z.y * v.y;
                }
                if (live) Lc[(l * ND + d) * 2 + c] += acc;
            }
            continue;
        }
        // sum_k 2^(k/2) |L_k| < (P + 1) 2^(G + 1) <= 2^(G + 6), so F = 119 - G keeps
        // every partial sum below 2^125
        const int F = 119 - G;
        __int128 a[P1];
#pragma unroll
        for (int k = 0; k <= P; ++k) {
            const double2 v = Lp[k * ND + d];
            const int m = k >> 1;
            __int128 X, Y;
            if ((k & 1) == 0) {
                X = fixed128(v.x, F - m);
                Y = fixed128(v.y, F - m);
            } else {  // times s
                const __int128 x = fixed128(v.x, F - m - 1), y = fixed128(v.y, F - m - 1);
                X = (sx > 0 ? x : -x) - (sy > 0 ? y : -y);
                Y = (sy > 0 ? x : -x) + (sx > 0 ? y : -y);
            }
            a[k] = quarter_turn(X, Y, m, sg, c);
        }
        // Taylor shift by 1: b_l = sum_{k>=l} C(k, l) a_k
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int j = P - 1; j >= i; --j) a[j] += a[j + 1];
#pragma unroll
        for (int l = 0; l <= P; ++l) {
            const __int128 other = shfl_xor_i128(pair, a[l], 1);
            const __int128 Bx = c ? other : a[l], By = c ? a[l] : other;
            const int m = l >> 1;
            __int128 X = Bx, Y = By;
            int sc = -F - m;
            if (l & 1) {  // times conj(s)
                X = (sx > 0 ? Bx : -Bx) + (sy > 0 ? By : -By);
                Y = (sx > 0 ? By : -By) - (sy > 0 ? Bx : -Bx);
                sc -= 1;
            }
            const __int128 v = quarter_turn(X, Y, m, -sg, c);
            if (live) Lc[(l * ND + d) * 2 + c] += int128_ldexp(v, sc);
        }
    }
}

// ----------------------------------------------------------------------------
int blocks_for_warps(int64_t nwork, int warps_per_block)
{
    int64_t b = (nwork + warps_per_block - 1) / warps_per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

int device_sms()
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, n = 152;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            sms = n;
        else
            sms = 152;
    }
    return sms;
}

template <int ND>
size_t leaf_smem()
{
    return (size_t)(1 << kLog64Bits) * sizeof(double2) + 2 * kEBias * sizeof(double) +
           (size_t)leaf_warps64<ND>() * std::max(sizeof(LeafStage64<ND>), sizeof(LeafStageFix<ND>));
}

template <int P, int ND>
cudaError_t fmm64_impl(const DevTree& t, const DevTables& tab, const PassGeom& g, Workspace& ws, bool gradient,
                       PhaseTimer* tm, cudaStream_t s)
{
    const int threads = kW64 * 32;
    // one-time opt-in to the dynamic shared memory of this instantiation
    static bool attr_done = false;
    static int leaf_resident[2] = {0, 0};
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_m2l64<P, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)m2l64_smem<P, ND>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_leaf64<P, ND, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)leaf_smem<ND>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_leaf64d<P, ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)leaf_smem<ND>());
        if (e != cudaSuccess) return e;
        for (int si = 0; si < 2; ++si) {
            int nb = 0;
            e = si ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_leaf64<P, ND, true>, leaf_warps64<ND>() * 32, leaf_smem<ND>())
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_leaf64d<P, ND>, leaf_warps64<ND>() * 32, leaf_smem<ND>());
            if (e != cudaSuccess) return e;
            leaf_resident[si] = std::max(1, nb);
        }
        attr_done = true;
    }
    int id = tm ? tm->begin("upward") : -1;
    k_p2m64<P, ND><<<blocks_for_warps(t.nleaf, kW64), threads, 0, s>>>(t, g, ws.q, ws.M);
    // M2M level by level from the deepest parents up; multipoles of levels 0 and 1
    // are never read
    for (int l = t.nlevels - 2; l >= 2; --l) {
        const int b0 = t.level_start[l], b1 = t.level_start[l + 1];
        if (b1 <= b0) continue;
        const int64_t lanes = 8 * (int64_t)(b1 - b0);
        k_m2m64<P, ND><<<(int)((lanes + kM2MThreads - 1) / kM2MThreads), kM2MThreads, 0, s>>>(t, tab, b0, b1, ws.M);
    }
    if (tm) tm->end(id);
    id = tm ? tm->begin("m2l") : -1;
    k_m2l64<P, ND><<<blocks_for_warps(t.nbox, kW64), threads, m2l64_smem<P, ND>(), s>>>(t, tab, g, ws.M, ws.L, ws.q,
                                                                                       tab.log64, tab.elog64);
    if (tm) tm->end(id);
    id = tm ? tm->begin("l2l") : -1;
    // boxes of levels 0 and 1 have empty V and X lists, so the first L2L that
    // adds anything goes into level 3
    for (int l = 3; l < t.nlevels; ++l) {
        const int b0 = t.level_start[l], b1 = t.level_start[l + 1];
        if (b1 <= b0) continue;
        const int64_t lanes = 2 * (int64_t)(b1 - b0);
        k_l2l64<P, ND><<<(int)((lanes + kL2LThreads - 1) / kL2LThreads), kL2LThreads, 0, s>>>(t, tab, b0, b1, ws.L);
    }
    if (tm) tm->end(id);
    id = tm ? tm->begin("leaf") : -1;
    if (gradient) {
        const int gblocks = std::max(1, std::min((t.nleaf + kGradWarps64 - 1) / kGradWarps64, device_sms() * 4));
        cudaMemsetAsync(ws.work, 0, sizeof(int), s);
        k_leaf_grad64<P, ND><<<gblocks, kGradWarps64 * 32, 0, s>>>(t, g, ws.q, ws.M, ws.L, ws.psi, ws.work);
        if (tm) tm->end(id);
        return cudaGetLastError();
    }
    const bool sym = t.sym;
    const int si = sym ? 1 : 0;
    constexpr int lw = leaf_warps64<ND>();
    const int lblocks = std::max(1, std::min((t.nleaf + lw - 1) / lw, device_sms() * leaf_resident[si]));
    cudaMemsetAsync(ws.work, 0, sizeof(int), s);
    double* slots = reinterpret_cast<double*>(ws.slots);  // the slot buffer holds 8 bytes per slot and density
    if (sym) {
        k_leaf64<P, ND, true><<<lblocks, lw * 32, leaf_smem<ND>(), s>>>(t, g, ws.q, ws.M, ws.L, tab.log64,
                                                                                 tab.elog64, ws.psi, ws.work, slots);
        const int rblocks = std::max(1, std::min((g.n_eval + 255) / 256, 152 * 32));
        k_sym_reduce64<ND><<<rblocks, 256, 0, s>>>(t, g, slots, ws.psi);
    } else {
        // the fixed-point log's scale: |Lp 2^(sL-60) + Ep log 2 2^sL| < 2^63 for |Ep| <= max(2 sigma, 127)
        const int maxE = std::max(2 * g.fix_sigma, 127);
        int sL = 60;
        while (sL > 40 && std::ldexp((double)maxE * 0.6931471805599453 + 1.0, sL) >= 0x1p62) --sL;
        const long long ln2_sL = std::llround(std::ldexp(0.693147180559945309417232121458176568L, sL));
        k_leaf64d<P, ND><<<lblocks, lw * 32, leaf_smem<ND>(), s>>>(t, g, ws.q, ws.M, ws.L, tab.logint,
                                                                            2 * g.fix_sigma, sL, ln2_sL, ws.psi,
                                                                            ws.work);
    }
    if (tm) tm->end(id);
    return cudaGetLastError();
}

template <int P>
cudaError_t fmm64_p(int nd, const DevTree& t, const DevTables& tab, const PassGeom& g, Workspace& ws, bool gradient,
                    PhaseTimer* tm, cudaStream_t s)
{
    switch (nd) {
        case 1: return fmm64_impl<P, 1>(t, tab, g, ws, gradient, tm, s);
        case 2: return fmm64_impl<P, 2>(t, tab, g, ws, gradient, tm, s);
        case 4: return fmm64_impl<P, 4>(t, tab, g, ws, gradient, tm, s);
        case 8: return fmm64_impl<P, 8>(t, tab, g, ws, gradient, tm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_fmm64(int P, int nd, const DevTree& t, const DevTables& tab, const PassGeom& g, Workspace& ws,
                         bool gradient, PhaseTimer* timer, cudaStream_t s)
{
    switch (P) {
        case 16: return fmm64_p<16>(nd, t, tab, g, ws, gradient, timer, s);
        case 24: return fmm64_p<24>(nd, t, tab, g, ws, gradient, timer, s);
        case 30: return fmm64_p<30>(nd, t, tab, g, ws, gradient, timer, s);
        default: return cudaErrorInvalidValue;
    }
}


namespace {
// Powers u^k, k = 1..P, of each point relative to its leaf, u = (z - c)/R (c
// the leaf's center, R its half side), [n][P] in tree order: the geometry is
// static, so they are formed once per plan and serve as the P2M input where
// the points carry charges and as the L2P input where they are evaluated. The
// same products as P2M formed on the fly (u, then p <- p u). One warp per leaf.
template <int P>
__global__ void k_point_powers(DevTree t, const int32_t* __restrict__ rng, const double2* __restrict__ xy,
                               double2* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    for (int li = gwarp(); li < t.nleaf; li += nwarps()) {
        const int b = t.leaves[li];
        const int s0 = rng[2 * b], s1 = rng[2 * b + 1];
        const double2 c = t.center[b];
        const double invR = 1.0 / t.radius[b];
        for (int j = s0 + lane; j < s1; j += 32) {
            const double2 z = xy[j];
            const double2 u = make_double2((z.x - c.x) * invR, (z.y - c.y) * invR);
            double2 pk = u;
            double2* o = out + (int64_t)j * P;
            o[0] = pk;
            for (int k = 2; k <= P; ++k) {
                pk = cmul64(pk, u);
                o[k - 1] = pk;
            }
        }
    }
}
}  // namespace

cudaError_t launch_point_powers(int P, const DevTree& t, const int32_t* rng, const double2* xy, double2* out,
                                cudaStream_t s)
{
    if (t.nleaf == 0) return cudaSuccess;
    const int blocks = blocks_for_warps(t.nleaf, kW64);
    switch (P) {
        case 16: k_point_powers<16><<<blocks, kW64 * 32, 0, s>>>(t, rng, xy, out); break;
        case 24: k_point_powers<24><<<blocks, kW64 * 32, 0, s>>>(t, rng, xy, out); break;
        case 30: k_point_powers<30><<<blocks, kW64 * 32, 0, s>>>(t, rng, xy, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// M2M table of order P: m2m[c][l][k] = C(l-1, k-1) 2^-k zeta_c^(l-k) for 1 <= k <= l,
// m2m[c][l][0] = -zeta_c^l / l (l >= 1), zero elsewhere; zeta_c = ((c & 1 ? 1 : -1) +
// i (c & 2 ? 1 : -1)) / 2 is the child-centre offset over the parent half-side. The
// binomial products are exact in float64 (dyadic zeta powers), the 1/l terms rounded once.
std::vector<double2> make_m2m64_table(int P)
{
    const int P1 = P + 1;
    std::vector<double2> tab((size_t)4 * P1 * P1, make_double2(0.0, 0.0));
    for (int c = 0; c < 4; ++c) {
        const double zx = (c & 1) ? 0.5 : -0.5, zy = (c & 2) ? 0.5 : -0.5;
        std::vector<double2> zp((size_t)P1);
        zp[0] = make_double2(1.0, 0.0);
        for (int m = 1; m <= P; ++m)
            zp[(size_t)m] = make_double2(zp[(size_t)m - 1].x * zx - zp[(size_t)m - 1].y * zy,
                                         zp[(size_t)m - 1].x * zy + zp[(size_t)m - 1].y * zx);
        for (int l = 1; l <= P; ++l) {
            double2* row = tab.data() + ((size_t)c * P1 + l) * P1;
            row[0] = make_double2(-zp[(size_t)l].x / l, -zp[(size_t)l].y / l);
            double binom = 1.0;  // C(l-1, k-1), k = 1
            for (int k = 1; k <= l; ++k) {
                const double w = std::ldexp(binom, -k);
                row[k] = make_double2(w * zp[(size_t)(l - k)].x, w * zp[(size_t)(l - k)].y);
                binom = binom * (double)(l - k) / (double)k;  // C(l-1, k) (exact: integers below 2^53)
            }
        }
    }
    return tab;
}

// Tables of the tensor-core M2L of order P (see k_m2l64), tau = 2^-1.5:
//   hd [8][32][40] bf16 digits of H'[l][k] (row l - 1, column k = 0..P; zero
//      padding), H'[l][0] = -1/l, H'[l][k] = C(l+k-1, k-1) tau^k;
//   eh [32] row exponents e with |H'[l][k]| < 2^(e - 1), H' ~ X 2^(e - 62);
//   mts [49][P1] (-t_o / tau)^k, t_o = 1/(2 (ox + i oy)) (zero for near offsets);
//   taup [P1] tau^k.
// Computed in long double; the digits are the balanced base-256 digits of the
// 62-bit fixed-point value, most significant first.
static uint64_t binom_u64_host(int n, int k)
{
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;  // exact at every step
    return r;
}

void make_m2l_tensor_tables(int P, std::vector<uint16_t>& hd, std::vector<int32_t>& eh, std::vector<double2>& mts,
                            std::vector<double>& taup)
{
    const int P1 = P + 1;
    const long double tau = 0.353553390593273762200422181052424519642L;  // 2^-1.5
    std::vector<long double> tp((size_t)P1);
    tp[0] = 1.0L;
    for (int k = 1; k <= P; ++k) tp[(size_t)k] = tp[(size_t)k - 1] * tau;
    taup.assign((size_t)P1, 0.0);
    for (int k = 0; k <= P; ++k) taup[(size_t)k] = (double)tp[(size_t)k];
    hd.assign((size_t)kSl * 32 * kHs, 0);
    eh.assign(32, 0);
    auto bf16_bits = [](int d) -> uint16_t {  // exact: |d| <= 256
        const float f = (float)d;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return (uint16_t)(u >> 16);
    };
    for (int l = 1; l <= P; ++l) {
        std::vector<long double> row((size_t)P1);
        long double mx = 0.0L;
        for (int k = 0; k <= P; ++k) {
            row[(size_t)k] = k == 0 ? -1.0L / (long double)l : (long double)binom_u64_host(l + k - 1, k - 1) * tp[(size_t)k];
            mx = std::max(mx, std::fabs(row[(size_t)k]));
        }
        const int e = std::ilogb(mx) + 2;
        eh[(size_t)l - 1] = e;
        for (int k = 0; k <= P; ++k) {
            long long X = std::llround(std::ldexp(row[(size_t)k], 62 - e));
            int dg[kSl];
            for (int j = kSl - 1; j >= 1; --j) {
                const int dj = (int)(signed char)(X & 0xff);
                dg[j] = dj;
                X = (X - dj) / 256;
            }
            dg[0] = (int)X;
            for (int j = 0; j < kSl; ++j) hd[((size_t)j * 32 + (l - 1)) * kHs + k] = bf16_bits(dg[j]);
        }
    }
    mts.assign((size_t)49 * P1, make_double2(0.0, 0.0));
    for (int oy = -3; oy <= 3; ++oy)
        for (int ox = -3; ox <= 3; ++ox) {
            if (std::max(std::abs(ox), std::abs(oy)) < 2) continue;
            const long double den = 2.0L * (long double)(ox * ox + oy * oy);
            // -t / tau, t = (ox - i oy) / den
            const long double ur = -(long double)ox / den / tau, ui = (long double)oy / den / tau;
            long double pr = 1.0L, pi = 0.0L;
            const int o = (oy + 3) * 7 + (ox + 3);
            for (int k = 0; k <= P; ++k) {
                mts[(size_t)o * P1 + k] = make_double2((double)pr, (double)pi);
                const long double nr = pr * ur - pi * ui, ni = pr * ui + pi * ur;
                pr = nr;
                pi = ni;
            }
        }
}

// L2L table of order P: l2l[c][l][k] = C(k, l) 2^-l zeta_c^(k-l) for k >= l (exact in
// float64: dyadic zeta powers, integer binomials below 2^53), zero elsewhere.
std::vector<double2> make_l2l64_table(int P)
{
    const int P1 = P + 1;
    std::vector<double2> tab((size_t)4 * P1 * P1, make_double2(0.0, 0.0));
    for (int c = 0; c < 4; ++c) {
        const double zx = (c & 1) ? 0.5 : -0.5, zy = (c & 2) ? 0.5 : -0.5;
        std::vector<double2> zp((size_t)P1);
        zp[0] = make_double2(1.0, 0.0);
        for (int m = 1; m <= P; ++m)
            zp[(size_t)m] = make_double2(zp[(size_t)m - 1].x * zx - zp[(size_t)m - 1].y * zy,
                                         zp[(size_t)m - 1].x * zy + zp[(size_t)m - 1].y * zx);
        for (int l = 0; l <= P; ++l) {
            double binom = 1.0;  // C(k, l), k = l
            for (int k = l; k <= P; ++k) {
                const double w = std::ldexp(binom, -l);
                tab[((size_t)c * P1 + l) * P1 + k] = make_double2(w * zp[(size_t)(k - l)].x, w * zp[(size_t)(k - l)].y);
                binom = binom * (double)(k + 1) / (double)(k + 1 - l);  // C(k + 1, l)
            }
        }
    }
    return tab;
}

// Host tables of the FP64 logarithm: tab[k] = (s_k, T_k) with c_k = 1 + k 2^-B,
// s_k = RN(1/c_k), T_k = -log(s_k) rounded once from extended precision
// (long double: at least 64 significant bits on the targets this builds for);
// etab[i] = (i - 64) log 2.
// The fixed-point logarithm's table (log_fix): S_k = round(2^62 / c_k), c_k = 1 +
// k 2^-12, and T_k = round(-log(S_k 2^-62) 2^60), in long double.
std::vector<longlong2> make_logint_table()
{
    const int n = 1 << kLog64Bits;
    std::vector<longlong2> tab((size_t)n);
    for (int k = 0; k < n; ++k) {
        const long double c = 1.0L + std::ldexp((long double)k, -kLog64Bits);
        const long double S = std::nearbyint(std::ldexp(1.0L, 62) / c);
        const long double T = -std::log(std::ldexp(S, -62));
        tab[(size_t)k] = make_longlong2((long long)S, (long long)std::llround(std::ldexp(T, 60)));
    }
    return tab;
}

void make_log64_tables(std::vector<double2>& tab, std::vector<double>& etab)
{
    const int n = 1 << kLog64Bits;
    tab.resize((size_t)n);
    for (int k = 0; k < n; ++k) {
        const double c = 1.0 + std::ldexp((double)k, -kLog64Bits);  // exact
        const double sk = 1.0 / c;
        const long double T = -std::log((long double)sk);
        tab[(size_t)k] = make_double2(sk, (double)T);
    }
    const long double ln2 = 0.693147180559945309417232121458176568L;
    etab.resize(2 * kEBias);
    for (int i = 0; i < 2 * kEBias; ++i) etab[(size_t)i] = (double)((long double)(i - kEBias) * ln2);
}

}  // namespace vp
