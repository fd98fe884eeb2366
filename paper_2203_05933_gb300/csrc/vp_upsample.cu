// Oversampled smooth quadrature on the GPU (Sec. 2, "Oversampled smooth
// quadratures", Eq. Tk_smooth_quad; Sec. 4.2): the density is sampled at the
// p-nodes of each cell and interpolated to the cell's q-nodes by the fixed
// matrix of its type, f_q = O_{p,q} f_p, in the same pass that turns values
// into FMM charges (q-node weight times value, written in tree order as FP64
// and as a hi/lo float pair). The transpose, used by the adjoint, applies O^T
// to the FMM result at the q-nodes of each cell.
//
// One block per cell (grid-stride over cells). Tensor-product types
// (O = A kron B, boxes) take two small products through shared memory:
// 2 (pa qb pb + qa qb pa) flops per cell and density instead of 2 n_q n_p.

#include <cuda_runtime.h>
#include <stdint.h>

#include "vp_internal.h"

namespace vp {
namespace {

constexpr int kUpsThreads = 128;
constexpr double kInv2PiU = 0.159154943091895335768883763372514362;

template <int ND>
__global__ void __launch_bounds__(kUpsThreads)
    k_ups_charges(DevUpsample u, const int32_t* __restrict__ inv, const double* __restrict__ w,
                  const double* __restrict__ f, int64_t ld_f, double* __restrict__ q, float2* __restrict__ qf)
{
    extern __shared__ double sm[];
    double* fs = sm;                       // [ND][max_p]
    double* tmp = sm + ND * u.max_p;       // [ND][max_tmp]
    for (int c = blockIdx.x; c < u.n_cells; c += gridDim.x) {
        const int t = u.cell_type[c];
        const int* ti = u.tinfo + 8 * t;
        const int kind = ti[0], nq = ti[1], np = ti[2];
        const int64_t f0 = u.f_start[c], s0 = u.src_start[c];
        __syncthreads();
        for (int i = threadIdx.x; i < np * ND; i += blockDim.x) {
            const int d = i / np, k = i - d * np;
            fs[d * u.max_p + k] = f[d * ld_f + f0 + k];
        }
        __syncthreads();
        if (kind == 1) {
            const int pa = ti[4], qb = ti[5], pb = ti[6];  // ti[3] = qa enters through nq = qa qb
            const double* A = u.mats + u.toff[2 * t];
            const double* B = u.mats + u.toff[2 * t + 1];
            // tmp[d][ia][rb] = sum_ib B[rb][ib] f[d][ia][ib]
            for (int i = threadIdx.x; i < pa * qb; i += blockDim.x) {
                const int ia = i / qb, rb = i - ia * qb;
                double acc[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = 0.0;
                for (int ib = 0; ib < pb; ++ib) {
                    const double bv = B[rb * pb + ib];
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = fma(bv, fs[d * u.max_p + ia * pb + ib], acc[d]);
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) tmp[d * u.max_tmp + i] = acc[d];
            }
            __syncthreads();
            // y[d][ra][rb] = sum_ia A[ra][ia] tmp[d][ia][rb]
            for (int r = threadIdx.x; r < nq; r += blockDim.x) {
                const int ra = r / qb, rb = r - ra * qb;
                double acc[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = 0.0;
                for (int ia = 0; ia < pa; ++ia) {
                    const double av = A[ra * pa + ia];
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = fma(av, tmp[d * u.max_tmp + ia * qb + rb], acc[d]);
                }
                const int32_t pos = inv[s0 + r];
                const double wv = w[pos];
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double v = wv * acc[d];
                    q[(int64_t)pos * ND + d] = v;
                    const float hi = __double2float_rn(v);
                    qf[(int64_t)pos * ND + d] = make_float2(hi, __double2float_rn(v - (double)hi));
                }
            }
        } else {
            const double* O = u.mats + u.toff[2 * t];
            for (int r = threadIdx.x; r < nq; r += blockDim.x) {
                double acc[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = 0.0;
                for (int k = 0; k < np; ++k) {
                    const double ov = O[(int64_t)r * np + k];
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = fma(ov, fs[d * u.max_p + k], acc[d]);
                }
                const int32_t pos = inv[s0 + r];
                const double wv = w[pos];
#pragma unroll
                for (int d = 0; d < ND; ++d) {
                    const double v = wv * acc[d];
                    q[(int64_t)pos * ND + d] = v;
                    const float hi = __double2float_rn(v);
                    qf[(int64_t)pos * ND + d] = make_float2(hi, __double2float_rn(v - (double)hi));
                }
            }
        }
    }
}

template <int ND>
__global__ void __launch_bounds__(kUpsThreads)
    k_ups_adjoint(DevUpsample u, const int32_t* __restrict__ inv, const double* __restrict__ w,
                  const double* __restrict__ psi, double* __restrict__ out, int64_t ld_out)
{
    extern __shared__ double sm[];
    double* us = sm;                       // [ND][max_q]
    double* tmp = sm + ND * u.max_q;       // [ND][max_tmp]
    for (int c = blockIdx.x; c < u.n_cells; c += gridDim.x) {
        const int t = u.cell_type[c];
        const int* ti = u.tinfo + 8 * t;
        const int kind = ti[0], nq = ti[1], np = ti[2];
        const int64_t f0 = u.f_start[c], s0 = u.src_start[c];
        __syncthreads();
        for (int r = threadIdx.x; r < nq; r += blockDim.x) {
            const int32_t pos = inv[s0 + r];
            const double wv = -kInv2PiU * w[pos];
#pragma unroll
            for (int d = 0; d < ND; ++d) us[d * u.max_q + r] = wv * psi[(int64_t)pos * ND + d];
        }
        __syncthreads();
        if (kind == 1) {
            const int qa = ti[3], pa = ti[4], qb = ti[5], pb = ti[6];
            const double* A = u.mats + u.toff[2 * t];
            const double* B = u.mats + u.toff[2 * t + 1];
            // tmp[d][ia][rb] = sum_ra A[ra][ia] u[d][ra][rb]
            for (int i = threadIdx.x; i < pa * qb; i += blockDim.x) {
                const int ia = i / qb, rb = i - ia * qb;
                double acc[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = 0.0;
                for (int ra = 0; ra < qa; ++ra) {
                    const double av = A[ra * pa + ia];
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = fma(av, us[d * u.max_q + ra * qb + rb], acc[d]);
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) tmp[d * u.max_tmp + i] = acc[d];
            }
            __syncthreads();
            // out[d][ia][ib] = sum_rb B[rb][ib] tmp[d][ia][rb]
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                const int ia = i / pb, ib = i - ia * pb;
                double acc[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = 0.0;
                for (int rb = 0; rb < qb; ++rb) {
                    const double bv = B[rb * pb + ib];
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = fma(bv, tmp[d * u.max_tmp + ia * qb + rb], acc[d]);
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + f0 + i] = acc[d];
            }
        } else {
            const double* O = u.mats + u.toff[2 * t];
            for (int i = threadIdx.x; i < np; i += blockDim.x) {
                double acc[ND];
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[d] = 0.0;
                for (int r = 0; r < nq; ++r) {
                    const double ov = O[(int64_t)r * np + i];
#pragma unroll
                    for (int d = 0; d < ND; ++d) acc[d] = fma(ov, us[d * u.max_q + r], acc[d]);
                }
#pragma unroll
                for (int d = 0; d < ND; ++d) out[d * ld_out + f0 + i] = acc[d];
            }
        }
    }
}

int ups_blocks(const DevUpsample& u)
{
    int b = u.n_cells < 152 * 16 ? u.n_cells : 152 * 16;
    return b < 1 ? 1 : b;
}

template <int ND>
cudaError_t ups_charges_nd(const DevUpsample& u, const int32_t* inv, const double* w, const double* f, int64_t ld_f,
                           double* q, float2* qf, cudaStream_t s)
{
    const size_t bytes = sizeof(double) * ND * (size_t)(u.max_p + u.max_tmp);
    cudaError_t e = cudaFuncSetAttribute(k_ups_charges<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_ups_charges<ND><<<ups_blocks(u), kUpsThreads, bytes, s>>>(u, inv, w, f, ld_f, q, qf);
    return cudaGetLastError();
}

template <int ND>
cudaError_t ups_adjoint_nd(const DevUpsample& u, const int32_t* inv, const double* w, const double* psi, double* out,
                           int64_t ld_out, cudaStream_t s)
{
    const size_t bytes = sizeof(double) * ND * (size_t)(u.max_q + u.max_tmp);
    cudaError_t e = cudaFuncSetAttribute(k_ups_adjoint<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_ups_adjoint<ND><<<ups_blocks(u), kUpsThreads, bytes, s>>>(u, inv, w, psi, out, ld_out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ups_charges(int nd, const DevUpsample& u, const int32_t* inv, const double* w_sorted,
                               const double* f, int64_t ld_f, double* q, float2* qf, cudaStream_t s)
{
    if (u.n_cells == 0) return cudaSuccess;
    switch (nd) {
        case 1: return ups_charges_nd<1>(u, inv, w_sorted, f, ld_f, q, qf, s);
        case 2: return ups_charges_nd<2>(u, inv, w_sorted, f, ld_f, q, qf, s);
        case 4: return ups_charges_nd<4>(u, inv, w_sorted, f, ld_f, q, qf, s);
        case 8: return ups_charges_nd<8>(u, inv, w_sorted, f, ld_f, q, qf, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ups_adjoint(int nd, const DevUpsample& u, const int32_t* inv, const double* w_sorted,
                               const double* psi, double* out, int64_t ld_out, cudaStream_t s)
{
    if (u.n_cells == 0) return cudaSuccess;
    switch (nd) {
        case 1: return ups_adjoint_nd<1>(u, inv, w_sorted, psi, out, ld_out, s);
        case 2: return ups_adjoint_nd<2>(u, inv, w_sorted, psi, out, ld_out, s);
        case 4: return ups_adjoint_nd<4>(u, inv, w_sorted, psi, out, ld_out, s);
        case 8: return ups_adjoint_nd<8>(u, inv, w_sorted, psi, out, ld_out, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vp
