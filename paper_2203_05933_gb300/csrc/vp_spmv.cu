// Correction apply (a7): out = -(1/2pi) psi + Pi f, the sparse map of the
// per-cell corrections "accurate minus smooth" (arXiv 2203.05933, Sec. 4,
// paragraph after Eq. nsrcs): float64 plans as exact fixed-point sums on the
// integer pipes (k_out_grouped64, the default), float-float plans on the FP32
// pipes (k_out_grouped, VP_FLAG_FF).
//
// The rows of one cell share their column list (every node of a cell couples
// to the nodes of the same near cells), so the plan stores each distinct
// column list once per group of consecutive rows. One block per group gathers
// x[:, cols] once into shared memory; each warp then streams its rows' values
// (8 bytes per nonzero, coalesced). HBM traffic is one read of the values plus
// the outputs.
#include <cuda_runtime.h>

#include <algorithm>

#include "vp_ff.cuh"
#include "vp_fixed.cuh"
#include "vp_internal.h"

namespace vp {
namespace {

constexpr double kInv2PiG = 0.159154943091895335768883763372514362;
constexpr int kGroupThreads = 256;
constexpr int kGroupSmemBytes = 96 * 1024;
static_assert((kGroupSmemBytes / (8 * (int)sizeof(float2))) % 2 == 0, "even staging capacity for 8 densities");

__global__ void k_to_ff_rows(int64_t total, int32_t n, const double* __restrict__ x, int64_t ld_x,
                             float2* __restrict__ xf)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = i / n, j = i % n;
        const ff::F v = ff::from_double(x[d * ld_x + j]);
        xf[i] = make_float2(v.h, v.l);
    }
}

// The rows of one group, one warp per row: U independent accumulators per
// density keep U 16-byte value loads in flight per lane (four for one or two
// densities; two beyond, where each value is reused ND times and registers are
// the scarcer resource). STAGED: x[:, cols] sits in shared memory (F, density
// d at F + d * smem_m); else it is gathered from xf.
template <int ND, bool STAGED>
__device__ __forceinline__ void grouped_rows(const DevGroupedCSR& A, int r0, int r1, int64_t c0, int m, int smem_m,
                                             const float2* __restrict__ F, const int32_t* __restrict__ inv,
                                             const double* __restrict__ w_sorted, const double* __restrict__ psi,
                                             const float2* __restrict__ xf, int64_t ld_xf, double* __restrict__ out,
                                             int64_t ld_out, int mode, int lane, int warp, int nw)
{
    constexpr int U = ND >= 4 ? 2 : 4;
    const int np = (m + 1) >> 1;  // value pairs per row (the padding value is zero)
    for (int r = r0 + warp; r < r1; r += nw) {
        const float4* vrow = reinterpret_cast<const float4*>(A.vf + A.rowptr[r]);  // rows start on 16 bytes
        ff::F acc[U][ND];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[u][d] = ff::F{0.f, 0.f};
        for (int q0 = lane; q0 < np; q0 += 32 * U) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + 32 * u;
                v[u] = q < np ? vrow[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = q0 + 32 * u;
                if (q < np) {
                    const int k = 2 * q;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        float4 x;
                        if (STAGED) {
                            x = *reinterpret_cast<const float4*>(F + d * smem_m + k);
                        } else {
                            const float2 x0 = xf[d * ld_xf + A.cols[c0 + k]];
                            const float2 x1 = k + 1 < m ? xf[d * ld_xf + A.cols[c0 + k + 1]] : make_float2(0.f, 0.f);
                            x = make_float4(x0.x, x0.y, x1.x, x1.y);
                        }
                        acc[u][d] = ff::add(acc[u][d], ff::mul(ff::F{v[u].x, v[u].y}, ff::F{x.x, x.y}));
                        acc[u][d] = ff::add(acc[u][d], ff::mul(ff::F{v[u].z, v[u].w}, ff::F{x.z, x.w}));
                    }
                }
            }
        }
#pragma unroll
        for (int u = 1; u < U; ++u)
#pragma unroll
            for (int d = 0; d < ND; ++d) acc[0][d] = ff::add(acc[0][d], acc[u][d]);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            for (int o = 16; o > 0; o >>= 1) {
                const float h = __shfl_xor_sync(0xffffffffu, acc[0][d].h, o);
                const float l = __shfl_xor_sync(0xffffffffu, acc[0][d].l, o);
                acc[0][d] = ff::add(acc[0][d], ff::F{h, l});
            }
        }
        if (lane == 0) {
            if (mode == kOutWithPsi) {
                const int32_t ri = inv[r];
                const double wv = w_sorted ? w_sorted[ri] : 1.0;
#pragma unroll
                for (int d = 0; d < ND; ++d)
                    out[d * ld_out + r] = fma(-kInv2PiG * wv, psi[(int64_t)ri * ND + d], ff::to_double(acc[0][d]));
            } else if (mode == kOutAccumulate) {
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + r] += ff::to_double(acc[0][d]);
            } else {
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + r] = ff::to_double(acc[0][d]);
            }
        }
    }
}

template <int ND>
__global__ void __launch_bounds__(kGroupThreads)
    k_out_grouped(DevGroupedCSR A, int smem_m, const int32_t* __restrict__ inv, const double* __restrict__ w_sorted,
                  const double* __restrict__ psi, const float2* __restrict__ xf, int64_t ld_xf,
                  double* __restrict__ out, int64_t ld_out, int mode)
{
    // [ND][smem_m] (smem_m even): lanes read consecutive pairs of columns of one density
    extern __shared__ __align__(16) float2 F[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int gi = blockIdx.x; gi < A.ngroups; gi += gridDim.x) {
        const int r0 = A.g_r0[gi], r1 = A.g_r0[gi + 1];
        const int64_t c0 = A.g_c0[gi];
        const int m = (int)(A.g_c0[gi + 1] - c0);
        const bool staged = m + (m & 1) <= smem_m;
        __syncthreads();
        if (staged) {
            for (int i = threadIdx.x; i < m * ND; i += blockDim.x) {
                const int k = i % m, d = i / m;
                F[d * smem_m + k] = xf[d * ld_xf + A.cols[c0 + k]];
            }
            if ((m & 1) && threadIdx.x < ND) F[threadIdx.x * smem_m + m] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (staged)
            grouped_rows<ND, true>(A, r0, r1, c0, m, smem_m, F, inv, w_sorted, psi, xf, ld_xf, out, ld_out, mode, lane,
                                   warp, nw);
        else
            grouped_rows<ND, false>(A, r0, r1, c0, m, smem_m, F, inv, w_sorted, psi, xf, ld_xf, out, ld_out, mode,
                                    lane, warp, nw);
    }
}

// Float64 plans. The values are stored in per-row fixed point (A.vi, A.vexp:
// v = V 2^vexp[r], |V| <= 2^52, as the 26-bit pieces {V mod 2^26, V >> 26}); one
// block per group stages x at the group's columns and puts each density in
// fixed point too (X = x 2^(52-e), e from the largest staged |x|, so |X| <=
// 2^52 and the rounding is at most 2^-53 of that largest value). A nonzero then
// costs four 32x32-bit multiply-adds into three 64-bit sums (the products of the
// high pieces, the cross products, the low pieces), each exact; per row the lane
// sums combine into one exact 128-bit integer, which is rounded to float64 once
// (to nearest). So the row's result is the rounded exact sum of the stored
// products, and the integer pipes carry the work that would otherwise take one
// DFMA per nonzero (the FP64 unit, 2 per clock per SM on GB300, is slower than
// the values stream from HBM); the conversions in and out of fixed point are
// integer operations on the bits too (vp_fixed.cuh). Eight lanes share a row
// (four rows per warp at a time); the rows of a group read the same staged
// columns (broadcast).
//
// Groups whose columns do not fit the staging buffer, longer than kFixMaxM, or
// whose x holds a non-finite value take the float64 loop instead: the same
// stored values, each converted back to float64 exactly, one DFMA per nonzero.
constexpr int kRowLanes64 = 8;
// Block size: one group per block at a time, so small blocks (many resident per
// SM, each with its own staging buffer) keep more value loads in flight than
// large ones waiting at their barriers; with more densities the rows do more
// work per value and larger blocks share one staging.
template <int ND>
constexpr int group64_threads()
{
    return ND == 1 ? 64 : ND == 2 ? 128 : 256;
}
// the longest column list staged (longer groups, and for eight densities those
// beyond kGroupSmemBytes, take the float64 loop from global memory)
constexpr int kStage64MaxM = 3072;
// the longest column list of the fixed-point loop: a lane then sums at most 512
// products, which keeps every 64-bit partial sum below 2^63
constexpr int kFixMaxM = 4096;

// c + a b, 32 x 32 -> 64-bit signed
__device__ __forceinline__ long long mad_wide(int a, int b, long long c)
{
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

template <int ND>
__device__ __forceinline__ void store_row64(int r, const double* v, const int32_t* __restrict__ inv,
                                            const double* __restrict__ w_sorted, const double* __restrict__ psi,
                                            double* __restrict__ out, int64_t ld_out, int mode)
{
    if (mode == kOutWithPsi) {
        const int32_t ri = inv[r];
        const double wv = w_sorted ? w_sorted[ri] : 1.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) out[d * ld_out + r] = fma(-kInv2PiG * wv, psi[(int64_t)ri * ND + d], v[d]);
    } else if (mode == kOutAccumulate) {
#pragma unroll
        for (int d = 0; d < ND; ++d) out[d * ld_out + r] += v[d];
    } else {
#pragma unroll
        for (int d = 0; d < ND; ++d) out[d * ld_out + r] = v[d];
    }
}

// The fixed-point loop: X[d * smem_m + k] = {X mod 2^26, X >> 26} of density d at
// column k (even smem_m, a zero after odd m), x = X 2^xsc[d].
template <int ND>
__device__ __forceinline__ void grouped_rows_fix(const DevGroupedCSR& A, int r0, int r1, int m, int smem_m,
                                                 const int2* __restrict__ X, const int* __restrict__ xsc,
                                                 const int32_t* __restrict__ inv, const double* __restrict__ w_sorted,
                                                 const double* __restrict__ psi, double* __restrict__ out,
                                                 int64_t ld_out, int mode, int lane, int warp, int nw)
{
    constexpr int RPW = 32 / kRowLanes64;  // rows per warp at a time
    constexpr int U = ND <= 2 ? 8 : 2;     // value pairs per lane in flight
    const int li = lane % kRowLanes64, sub = lane / kRowLanes64;
    const int np = (m + 1) >> 1;  // value pairs per row (the padding value is zero)
    for (int rb = r0 + warp * RPW; rb < r1; rb += nw * RPW) {
        const int r = rb + sub;
        const bool live = r < r1;
        long long hh[ND], md[ND], ll[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) hh[d] = md[d] = ll[d] = 0;
        if (live) {
            const int4* vrow = reinterpret_cast<const int4*>(A.vi + A.rowptr[r]);  // rows start on 16 bytes
            for (int q0 = li; q0 < np; q0 += U * kRowLanes64) {
                int4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int qp = q0 + u * kRowLanes64;
                    v[u] = qp < np ? __ldcs(vrow + qp) : make_int4(0, 0, 0, 0);  // streamed once
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int qp = q0 + u * kRowLanes64;
                    if (qp >= np) continue;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        const int4 xv = *reinterpret_cast<const int4*>(X + d * smem_m + 2 * qp);
                        ll[d] = mad_wide(v[u].x, xv.x, ll[d]);
                        ll[d] = mad_wide(v[u].z, xv.z, ll[d]);
                        md[d] = mad_wide(v[u].x, xv.y, md[d]);
                        md[d] = mad_wide(v[u].y, xv.x, md[d]);
                        md[d] = mad_wide(v[u].z, xv.w, md[d]);
                        md[d] = mad_wide(v[u].w, xv.z, md[d]);
                        hh[d] = mad_wide(v[u].y, xv.y, hh[d]);
                        hh[d] = mad_wide(v[u].w, xv.w, hh[d]);
                    }
                }
            }
        }
        double res[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            // the lane's sum hh 2^52 + md 2^26 + ll, then the row's eight lanes, in 128 bits
            __int128 t = ((__int128)hh[d] << 52) + ((__int128)md[d] << 26) + (__int128)ll[d];
#pragma unroll
            for (int o = kRowLanes64 / 2; o > 0; o >>= 1) {
                const long long th = __shfl_xor_sync(0xffffffffu, (long long)(t >> 64), o);
                const unsigned long long tl = __shfl_xor_sync(0xffffffffu, (unsigned long long)t, o);
                t += ((__int128)th << 64) | (__int128)tl;
            }
            res[d] = live ? int128_ldexp(t, A.vexp[r] + xsc[d]) : 0.0;
        }
        if (live && li == 0) store_row64<ND>(r, res, inv, w_sorted, psi, out, ld_out, mode);
    }
}

// The float64 loop over the same values (V converted exactly, the row's scale
// applied to the sum). STAGED: x[:, cols] as float64 in F; else gathered from x.
template <int ND, bool STAGED>
__device__ __forceinline__ void grouped_rows64(const DevGroupedCSR& A, int r0, int r1, int64_t c0, int m, int smem_m,
                                               const double* __restrict__ F, const int32_t* __restrict__ inv,
                                               const double* __restrict__ w_sorted, const double* __restrict__ psi,
                                               const double* __restrict__ x, int64_t ld_x, double* __restrict__ out,
                                               int64_t ld_out, int mode, int lane, int warp, int nw)
{
    constexpr int RPW = 32 / kRowLanes64;
    constexpr int U = ND <= 2 ? 4 : 2;
    const int li = lane % kRowLanes64, sub = lane / kRowLanes64;
    const int np = (m + 1) >> 1;
    for (int rb = r0 + warp * RPW; rb < r1; rb += nw * RPW) {
        const int r = rb + sub;
        const bool live = r < r1;
        double acc0[ND], acc1[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc0[d] = acc1[d] = 0.0;
        if (live) {
            const int4* vrow = reinterpret_cast<const int4*>(A.vi + A.rowptr[r]);
            for (int q0 = li; q0 < np; q0 += U * kRowLanes64) {
                int4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int qp = q0 + u * kRowLanes64;
                    v[u] = qp < np ? __ldcs(vrow + qp) : make_int4(0, 0, 0, 0);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int qp = q0 + u * kRowLanes64;
                    if (qp >= np) continue;
                    const int k = 2 * qp;
                    const double v0 = (double)(((long long)v[u].y << 26) + v[u].x);  // |V| <= 2^52: exact
                    const double v1 = (double)(((long long)v[u].w << 26) + v[u].z);
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        double2 xv;
                        if (STAGED) {
                            xv = *reinterpret_cast<const double2*>(F + d * smem_m + k);
                        } else {
                            xv.x = x[d * ld_x + A.cols[c0 + k]];
                            xv.y = k + 1 < m ? x[d * ld_x + A.cols[c0 + k + 1]] : 0.0;
                        }
                        acc0[d] = fma(v0, xv.x, acc0[d]);
                        acc1[d] = fma(v1, xv.y, acc1[d]);
                    }
                }
            }
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            double a = acc0[d] + acc1[d];
#pragma unroll
            for (int o = kRowLanes64 / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            acc0[d] = live ? ldexp(a, A.vexp[r]) : 0.0;
        }
        if (live && li == 0) store_row64<ND>(r, acc0, inv, w_sorted, psi, out, ld_out, mode);
    }
}

template <int ND>
__global__ void __launch_bounds__(group64_threads<ND>())
    k_out_grouped64(DevGroupedCSR A, int smem_m, const int32_t* __restrict__ inv, const double* __restrict__ w_sorted,
                    const double* __restrict__ psi, const double* __restrict__ x, int64_t ld_x,
                    double* __restrict__ out, int64_t ld_out, int mode)
{
    // [ND][smem_m] (smem_m even): x at the group's columns, density-major, as
    // float64 and then (same 8 bytes) in fixed point
    extern __shared__ __align__(16) double F64[];
    __shared__ unsigned xe[ND];  // the largest biased exponent of the staged x, per density
    __shared__ int xsc[ND];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int gi = blockIdx.x; gi < A.ngroups; gi += gridDim.x) {
        const int r0 = A.g_r0[gi], r1 = A.g_r0[gi + 1];
        const int64_t c0 = A.g_c0[gi];
        const int m = (int)(A.g_c0[gi + 1] - c0);
        const bool staged = m + (m & 1) <= smem_m;
        __syncthreads();  // the previous group's rows are done with F64, xe, xsc
        if (threadIdx.x < ND) xe[threadIdx.x] = 0u;
        __syncthreads();
        if (staged) {
            // four columns per thread at a time: their indices, then their x values
            constexpr int G = 4;
            unsigned em[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) em[d] = 0u;
            for (int k0 = threadIdx.x; k0 < m; k0 += G * blockDim.x) {
                int c[G];
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int k = k0 + j * blockDim.x;
                    c[j] = k < m ? A.cols[c0 + k] : -1;
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    double v[G];
#pragma unroll
                    for (int j = 0; j < G; ++j) v[j] = c[j] >= 0 ? x[d * ld_x + c[j]] : 0.0;
#pragma unroll
                    for (int j = 0; j < G; ++j) {
                        if (c[j] < 0) continue;
                        F64[d * smem_m + k0 + j * blockDim.x] = v[j];
                        em[d] = max(em[d], exponent_field(v[j]));
                    }
                }
            }
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                em[d] = __reduce_max_sync(0xffffffffu, em[d]);
                if (lane == 0) atomicMax(&xe[d], em[d]);
            }
            if ((m & 1) && threadIdx.x < ND) F64[threadIdx.x * smem_m + m] = 0.0;  // also the fixed-point zero
        }
        __syncthreads();
        if (!staged) {
            grouped_rows64<ND, false>(A, r0, r1, c0, m, smem_m, F64, inv, w_sorted, psi, x, ld_x, out, ld_out, mode,
                                      lane, warp, nw);
            continue;
        }
        bool fix = m <= kFixMaxM;
#pragma unroll
        for (int d = 0; d < ND; ++d) fix = fix && xe[d] < 0x7ffu;  // no infinity or NaN staged
        if (!fix) {
            grouped_rows64<ND, true>(A, r0, r1, c0, m, smem_m, F64, inv, w_sorted, psi, x, ld_x, out, ld_out, mode,
                                     lane, warp, nw);
            continue;
        }
        // in place, each element by the thread that staged it: |x| < 2^e, e = E - 1022
        // for the largest biased exponent E (E = 0: zeros and subnormals, e = -1021)
        int2* X = reinterpret_cast<int2*>(F64);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const int e = (int)max(xe[d], 1u) - 1022;
            for (int k = threadIdx.x; k < m; k += blockDim.x) {
                const long long q = fixed52(F64[d * smem_m + k], e);
                X[d * smem_m + k] = make_int2((int)(q & 0x3ffffff), (int)(q >> 26));
            }
            if (threadIdx.x == 0) xsc[d] = e - 52;
        }
        __syncthreads();
        grouped_rows_fix<ND>(A, r0, r1, m, smem_m, X, xsc, inv, w_sorted, psi, out, ld_out, mode, lane, warp, nw);
    }
}

template <int ND>
cudaError_t launch_grouped64_nd(const DevGroupedCSR& A, const int32_t* inv, const double* w_sorted, const double* psi,
                                const double* x, int64_t ld_x, double* out, int64_t ld_out, int mode, int max_blocks,
                                cudaStream_t s)
{
    // staging sized to the longest column list (even), at most kStage64MaxM columns
    // and kGroupSmemBytes
    int smem_m = A.max_m + (A.max_m & 1);
    if (smem_m > kStage64MaxM) smem_m = kStage64MaxM;
    if (smem_m > (kGroupSmemBytes / (ND * (int)sizeof(double)) & ~1)) smem_m = kGroupSmemBytes / (ND * (int)sizeof(double)) & ~1;
    if (smem_m < 2) smem_m = 2;
    const size_t bytes = (size_t)smem_m * ND * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_out_grouped64<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    constexpr int threads = group64_threads<ND>();
    const int cap = max_blocks > 0 ? max_blocks : 152 * (2048 / threads);
    int blocks = A.ngroups < cap ? A.ngroups : cap;
    if (blocks < 1) blocks = 1;
    k_out_grouped64<ND><<<blocks, threads, bytes, s>>>(A, smem_m, inv, w_sorted, psi, x, ld_x, out, ld_out, mode);
    return cudaGetLastError();
}

// out[d][r] += -(1/2pi) w psi[inv[r]][d], w = w_sorted[inv[r]] or 1 (the smooth part added
// to a correction computed on its own)
template <int ND>
__global__ void k_add_psi(int32_t n, const int32_t* __restrict__ inv, const double* __restrict__ w_sorted,
                          const double* __restrict__ psi, double* __restrict__ out, int64_t ld_out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n * ND;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)(i / ND);
        const int d = (int)(i - (int64_t)r * ND);
        const int32_t ri = inv[r];
        const double wv = w_sorted ? w_sorted[ri] : 1.0;
        out[d * ld_out + r] = fma(-kInv2PiG * wv, psi[(int64_t)ri * ND + d], out[d * ld_out + r]);
    }
}

template <int ND>
cudaError_t launch_grouped_nd(const DevGroupedCSR& A, const int32_t* inv, const double* w_sorted, const double* psi,
                              const float2* xf, int64_t ld_xf, double* out, int64_t ld_out, int mode, int max_blocks,
                              cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_out_grouped<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kGroupSmemBytes);
    if (e != cudaSuccess) return e;
    // the staged columns of density d start at F + d * smem_m and are read as 16-byte
    // pairs: smem_m must be even (the capacity below is)
    int smem_m = kGroupSmemBytes / (ND * (int)sizeof(float2));
    const int want = A.max_m + (A.max_m & 1);
    if (want < smem_m) smem_m = want;
    if (smem_m < 2) smem_m = 2;
    const size_t bytes = (size_t)smem_m * ND * sizeof(float2);
    const int cap = max_blocks > 0 ? max_blocks : 152 * 16;
    int blocks = A.ngroups < cap ? A.ngroups : cap;
    if (blocks < 1) blocks = 1;
    k_out_grouped<ND><<<blocks, kGroupThreads, bytes, s>>>(A, smem_m, inv, w_sorted, psi, xf, ld_xf, out, ld_out,
                                                          mode);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_to_ff_rows(int nd, int32_t n, const double* x, int64_t ld_x, float2* xf, cudaStream_t s)
{
    const int64_t total = (int64_t)nd * n;
    if (total == 0) return cudaSuccess;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    k_to_ff_rows<<<(int)blocks, 256, 0, s>>>(total, n, x, ld_x, xf);
    return cudaGetLastError();
}

cudaError_t launch_out_grouped(int nd, const DevGroupedCSR& A, const int32_t* inv, const double* w_sorted,
                               const double* psi, const float2* xf, int64_t ld_xf, double* out, int64_t ld_out,
                               int mode, int max_blocks, cudaStream_t s)
{
    switch (nd) {
        case 1: return launch_grouped_nd<1>(A, inv, w_sorted, psi, xf, ld_xf, out, ld_out, mode, max_blocks, s);
        case 2: return launch_grouped_nd<2>(A, inv, w_sorted, psi, xf, ld_xf, out, ld_out, mode, max_blocks, s);
        case 4: return launch_grouped_nd<4>(A, inv, w_sorted, psi, xf, ld_xf, out, ld_out, mode, max_blocks, s);
        case 8: return launch_grouped_nd<8>(A, inv, w_sorted, psi, xf, ld_xf, out, ld_out, mode, max_blocks, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_out_grouped64(int nd, const DevGroupedCSR& A, const int32_t* inv, const double* w_sorted,
                                 const double* psi, const double* x, int64_t ld_x, double* out, int64_t ld_out,
                                 int mode, int max_blocks, cudaStream_t s)
{
    switch (nd) {
        case 1: return launch_grouped64_nd<1>(A, inv, w_sorted, psi, x, ld_x, out, ld_out, mode, max_blocks, s);
        case 2: return launch_grouped64_nd<2>(A, inv, w_sorted, psi, x, ld_x, out, ld_out, mode, max_blocks, s);
        case 4: return launch_grouped64_nd<4>(A, inv, w_sorted, psi, x, ld_x, out, ld_out, mode, max_blocks, s);
        case 8: return launch_grouped64_nd<8>(A, inv, w_sorted, psi, x, ld_x, out, ld_out, mode, max_blocks, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_add_psi(int nd, int32_t n, const int32_t* inv, const double* w_sorted, const double* psi,
                           double* out, int64_t ld_out, cudaStream_t s)
{
    const int64_t total = (int64_t)nd * n;
    if (total == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 32);
    switch (nd) {
        case 1: k_add_psi<1><<<blocks, 256, 0, s>>>(n, inv, w_sorted, psi, out, ld_out); break;
        case 2: k_add_psi<2><<<blocks, 256, 0, s>>>(n, inv, w_sorted, psi, out, ld_out); break;
        case 4: k_add_psi<4><<<blocks, 256, 0, s>>>(n, inv, w_sorted, psi, out, ld_out); break;
        case 8: k_add_psi<8><<<blocks, 256, 0, s>>>(n, inv, w_sorted, psi, out, ld_out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vp
