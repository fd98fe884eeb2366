// Correction apply (a7): out = -(1/2pi) psi + Pi f, the sparse map of the
// per-cell corrections "accurate minus smooth" (arXiv 2203.05933, Sec. 4,
// paragraph after Eq. nsrcs): in float64 (k_out_grouped64, the default) or on
// the FP32 pipes in float-float arithmetic (k_out_grouped, VP_FLAG_FF).
//
// The rows of one cell share their column list (every node of a cell couples
// to the nodes of the same near cells), so the plan stores each distinct
// column list once per group of consecutive rows. One block per group gathers
// x[:, cols] once into shared memory as hi/lo floats; each warp then streams
// its rows' values (8 bytes per nonzero, coalesced) and accumulates with
// TwoProd/TwoSum. HBM traffic is one read of the values plus the outputs.
#include <cuda_runtime.h>

#include <algorithm>

#include "vp_ff.cuh"
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

// Float64 form (float64 plans): values A.vd (8 bytes per nonzero, rows padded to
// even lengths, so each row starts on 16 bytes), one DFMA per nonzero and
// density. Eight lanes share a row (four rows per warp at a time), so that the
// closing reduction costs three shuffle-adds per row against a row length of a
// few hundred; the rows of a group read the same staged columns (broadcast).
constexpr int kRowLanes64 = 8;

template <int ND, bool STAGED>
__device__ __forceinline__ void grouped_rows64(const DevGroupedCSR& A, int r0, int r1, int64_t c0, int m, int smem_m,
                                               const double* __restrict__ F, const int32_t* __restrict__ inv,
                                               const double* __restrict__ w_sorted, const double* __restrict__ psi,
                                               const double* __restrict__ x, int64_t ld_x, double* __restrict__ out,
                                               int64_t ld_out, int mode, int lane, int warp, int nw)
{
    constexpr int RPW = 32 / kRowLanes64;  // rows per warp at a time
    const int li = lane % kRowLanes64, sub = lane / kRowLanes64;
    const int np = (m + 1) >> 1;  // value pairs per row (the padding value is zero)
    for (int rb = r0 + warp * RPW; rb < r1; rb += nw * RPW) {
        const int r = rb + sub;
        const bool live = r < r1;
        // U value pairs per lane in flight (loads issued before the arithmetic)
        constexpr int U = ND <= 2 ? 4 : 2;
        double acc0[ND], acc1[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) acc0[d] = acc1[d] = 0.0;
        if (live) {
            const double2* vrow = reinterpret_cast<const double2*>(A.vd + A.rowptr[r]);
            for (int q0 = li; q0 < np; q0 += U * kRowLanes64) {
                double2 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int qp = q0 + u * kRowLanes64;
                    v[u] = qp < np ? __ldcs(vrow + qp) : make_double2(0.0, 0.0);  // streamed once
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int qp = q0 + u * kRowLanes64;
                    if (qp >= np) continue;
                    const int k = 2 * qp;
#pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        double2 xv;
                        if (STAGED) {
                            xv = *reinterpret_cast<const double2*>(F + d * smem_m + k);
                        } else {
                            xv.x = x[d * ld_x + A.cols[c0 + k]];
                            xv.y = k + 1 < m ? x[d * ld_x + A.cols[c0 + k + 1]] : 0.0;
                        }
                        acc0[d] = fma(v[u].x, xv.x, acc0[d]);
                        acc1[d] = fma(v[u].y, xv.y, acc1[d]);
                    }
                }
            }
        }
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            double a = acc0[d] + acc1[d];
#pragma unroll
            for (int o = kRowLanes64 / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            acc0[d] = a;
        }
        if (live && li == 0) {
            if (mode == kOutWithPsi) {
                const int32_t ri = inv[r];
                const double wv = w_sorted ? w_sorted[ri] : 1.0;
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + r] = fma(-kInv2PiG * wv, psi[(int64_t)ri * ND + d], acc0[d]);
            } else if (mode == kOutAccumulate) {
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + r] += acc0[d];
            } else {
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + r] = acc0[d];
            }
        }
    }
}

template <int ND>
__global__ void __launch_bounds__(kGroupThreads)
    k_out_grouped64(DevGroupedCSR A, int smem_m, const int32_t* __restrict__ inv, const double* __restrict__ w_sorted,
                    const double* __restrict__ psi, const double* __restrict__ x, int64_t ld_x,
                    double* __restrict__ out, int64_t ld_out, int mode)
{
    // [ND][smem_m] (smem_m even): x at the group's columns, density-major
    extern __shared__ __align__(16) double F64[];
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
                F64[d * smem_m + k] = x[d * ld_x + A.cols[c0 + k]];
            }
            if ((m & 1) && threadIdx.x < ND) F64[threadIdx.x * smem_m + m] = 0.0;
        }
        __syncthreads();
        if (staged)
            grouped_rows64<ND, true>(A, r0, r1, c0, m, smem_m, F64, inv, w_sorted, psi, x, ld_x, out, ld_out, mode,
                                     lane, warp, nw);
        else
            grouped_rows64<ND, false>(A, r0, r1, c0, m, smem_m, F64, inv, w_sorted, psi, x, ld_x, out, ld_out, mode,
                                      lane, warp, nw);
    }
}

template <int ND>
cudaError_t launch_grouped64_nd(const DevGroupedCSR& A, const int32_t* inv, const double* w_sorted, const double* psi,
                                const double* x, int64_t ld_x, double* out, int64_t ld_out, int mode, int max_blocks,
                                cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_out_grouped64<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kGroupSmemBytes);
    if (e != cudaSuccess) return e;
    int smem_m = kGroupSmemBytes / (ND * (int)sizeof(double));
    smem_m &= ~1;
    const int want = A.max_m + (A.max_m & 1);
    if (want < smem_m) smem_m = want;
    if (smem_m < 2) smem_m = 2;
    const size_t bytes = (size_t)smem_m * ND * sizeof(double);
    const int cap = max_blocks > 0 ? max_blocks : 152 * 16;
    int blocks = A.ngroups < cap ? A.ngroups : cap;
    if (blocks < 1) blocks = 1;
    k_out_grouped64<ND><<<blocks, kGroupThreads, bytes, s>>>(A, smem_m, inv, w_sorted, psi, x, ld_x, out, ld_out,
                                                            mode);
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
