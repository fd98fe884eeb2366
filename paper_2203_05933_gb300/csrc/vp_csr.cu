// Device-side construction of the grouped correction matrix and its transposed
// product (a7 and the Pi^T g term of a8; Pi is the sparse map of the per-cell
// corrections "accurate minus smooth", arXiv 2203.05933, Sec. 4, paragraph
// after Eq. nsrcs).
//
// The rows of one cell couple to the same near cells, so consecutive rows with
// identical column lists form a group with one stored column list and a dense
// block of values (rows padded to even lengths). The plan builds this layout on
// the device straight from the caller's CSR: a check kernel (columns in range,
// finite values), a row-equality flag per row (the host turns the flags into
// group boundaries), a gather of each group's column list, and a copy of the
// values into the padded layout (per-row fixed point for float64 plans, hi/lo
// floats for float-float plans). No transposed copy of the values is made: Pi^T g is computed per
// group as the transposed block product into a buffer of partial sums (one
// entry per stored column position), then gathered per column over the
// positions where it appears, in ascending order (deterministic).
#include <cuda_runtime.h>

#include "vp_ff.cuh"
#include "vp_fixed.cuh"
#include "vp_internal.h"

namespace vp {
namespace {

constexpr double kInv2PiC = 0.159154943091895335768883763372514362;

int grid_for(int64_t n, int per_block)
{
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

// err bit 1: a column outside [0, ncols); bit 2: a non-finite value
__global__ void k_csr_check(int64_t nnz, const int32_t* __restrict__ col, const double* __restrict__ val, int64_t ncols,
                            int* __restrict__ err)
{
    int bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = col[k];
        if (c < 0 || (int64_t)c >= ncols) bad |= 1;
        if (!isfinite(val[k])) bad |= 2;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (bad && (threadIdx.x & 31) == 0) atomicOr(err, bad);
}

// same[i] = 1 when row i has the length and the columns of row i - 1 (one warp per row)
__global__ void k_row_same(int64_t nrows, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           uint8_t* __restrict__ same)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < nrows; i += warps) {
        bool eq = false;
        if (i > 0) {
            const int64_t a0 = rowptr[i - 1], a1 = rowptr[i], b1 = rowptr[i + 1];
            eq = (a1 - a0) == (b1 - a1);
            if (eq) {
                bool diff = false;
                for (int64_t k = lane; k < a1 - a0; k += 32) diff |= col[a0 + k] != col[a1 + k];
                eq = !__any_sync(0xffffffffu, diff);
            }
        }
        if (lane == 0) same[i] = eq ? 1 : 0;
    }
}

// cols[g_c0[g] + k] = col[rowptr[g_r0[g]] + k] (one warp per group)
__global__ void k_group_cols(int32_t ngroups, const int32_t* __restrict__ g_r0, const int64_t* __restrict__ g_c0,
                             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             int32_t* __restrict__ cols)
{
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ngroups; g += warps) {
        const int64_t src = rowptr[g_r0[g]], dst = g_c0[g], m = g_c0[g + 1] - g_c0[g];
        for (int64_t k = lane; k < m; k += 32) cols[dst + k] = col[src + k];
    }
}

// values into the padded layout (row r at prow[r], length padded to even with a
// zero) as hi/lo floats
__global__ void k_pad_values(int64_t nrows, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ prow,
                             const double* __restrict__ val, float2* __restrict__ vf)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nrows; r += warps) {
        const int64_t a = rowptr[r], len = rowptr[r + 1] - a, o = prow[r], plen = prow[r + 1] - o;
        for (int64_t k = lane; k < plen; k += 32) {
            const ff::F f = ff::from_double(k < len ? val[a + k] : 0.0);
            vf[o + k] = make_float2(f.h, f.l);
        }
    }
}

// The same layout in per-row fixed point (one warp per row): with E the largest
// biased exponent among the row's values and e = max(E, 1) - 1022 (so every
// |v| < 2^e, and 2^(e-1) <= max |v| for a normal maximum), V = v 2^(52-e)
// rounded to the nearest integer: |V| <= 2^52 and the rounding error is at most
// 2^-53 of 2^e, i.e. 2^-52 of the row's largest value (the row's own float64
// rounding is 2^-53 of it); vexp[r] = e - 52. Stored as {V mod 2^26, V >> 26}:
// the product kernel multiplies 26-bit pieces (exact 64-bit products) and keeps
// its sums exact.
__global__ void k_fix_values(int64_t nrows, const int64_t* __restrict__ rowptr, const int64_t* __restrict__ prow,
                             const double* __restrict__ val, int2* __restrict__ vi, int32_t* __restrict__ vexp)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nrows; r += warps) {
        const int64_t a = rowptr[r], len = rowptr[r + 1] - a, o = prow[r], plen = prow[r + 1] - o;
        unsigned em = 0u;
        for (int64_t k = lane; k < len; k += 32) em = max(em, exponent_field(val[a + k]));
        em = __reduce_max_sync(0xffffffffu, em);
        const int e = (int)max(em, 1u) - 1022;
        for (int64_t k = lane; k < plen; k += 32) {
            const long long V = k < len ? fixed52(val[a + k], e) : 0LL;
            vi[o + k] = make_int2((int)(V & 0x3ffffff), (int)(V >> 26));
        }
        if (lane == 0) vexp[r] = e - 52;
    }
}

// ----------------------------------------------------------------------------
// Pi^T x: partial[p][d] = sum_{r in group} V[r][k] x[d][r], p = g_c0[g] + k
// (one block per group; threads over the group's columns, rows in order).
constexpr int kAdjThreads = 128;
constexpr int kAdjRows = 64;  // rows of x staged per step

template <int ND, bool F64>
__global__ void __launch_bounds__(kAdjThreads)
    k_adj_partial(DevGroupedCSR A, const double* __restrict__ x, int64_t ld_x, double* __restrict__ partial)
{
    // x of the staged rows: float64 times the row's fixed-point scale (the values
    // are then the exact integers V), or as hi/lo floats for the float-float
    // values (converted once per row here, not once per nonzero)
    __shared__ double xs[kAdjRows][ND];
    float2(*xf)[ND] = reinterpret_cast<float2(*)[ND]>(&xs[0][0]);
    for (int g = blockIdx.x; g < A.ngroups; g += gridDim.x) {
        const int r0 = A.g_r0[g], r1 = A.g_r0[g + 1];
        const int64_t p0 = A.g_c0[g];
        const int m = (int)(A.g_c0[g + 1] - p0);
        for (int k0 = 0; k0 < m; k0 += kAdjThreads) {
            const int k = k0 + threadIdx.x;
            double acc[ND];
            ff::F facc[ND];
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                acc[d] = 0.0;
                facc[d] = ff::F{0.f, 0.f};
            }
            for (int rb = r0; rb < r1; rb += kAdjRows) {
                const int nr = min(kAdjRows, r1 - rb);
                __syncthreads();
                for (int i = threadIdx.x; i < nr * ND; i += kAdjThreads) {
                    const int rr = i / ND, d = i % ND;
                    const double xv = x[d * ld_x + rb + rr];
                    if (F64) {
                        xs[rr][d] = ldexp(xv, A.vexp[rb + rr]);  // the row's scale, exact
                    } else {
                        const ff::F f = ff::from_double(xv);
                        xf[rr][d] = make_float2(f.h, f.l);
                    }
                }
                __syncthreads();
                if (k < m) {
                    for (int rr = 0; rr < nr; ++rr) {
                        const int64_t o = A.rowptr[rb + rr] + k;
                        if (F64) {
                            const int2 vv = A.vi[o];
                            const double v = (double)(((long long)vv.y << 26) + vv.x);  // |V| <= 2^52: exact
#pragma unroll
                            for (int d = 0; d < ND; ++d) acc[d] = fma(v, xs[rr][d], acc[d]);
                        } else {
                            const float2 v = A.vf[o];
#pragma unroll
                            for (int d = 0; d < ND; ++d)
                                facc[d] = ff::add(facc[d], ff::mul(ff::F{v.x, v.y}, ff::F{xf[rr][d].x, xf[rr][d].y}));
                        }
                    }
                }
            }
            if (k < m) {
#pragma unroll
                for (int d = 0; d < ND; ++d) partial[(p0 + k) * ND + d] = F64 ? acc[d] : ff::to_double(facc[d]);
            }
        }
    }
}

// out[d][c] = sum over the positions p of column c (ascending) of partial[p][d],
// combined with the smooth part as in the forward product (mode).
template <int ND>
__global__ void k_adj_gather(int64_t ncols, const int64_t* __restrict__ inc_ptr, const int64_t* __restrict__ inc_pos,
                             const double* __restrict__ partial, const int32_t* __restrict__ inv,
                             const double* __restrict__ w_sorted, const double* __restrict__ psi, double* __restrict__ out,
                             int64_t ld_out, int mode)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncols; c += (int64_t)gridDim.x * blockDim.x) {
        double s[ND];
#pragma unroll
        for (int d = 0; d < ND; ++d) s[d] = 0.0;
        for (int64_t i = inc_ptr[c]; i < inc_ptr[c + 1]; ++i) {
            const int64_t p = inc_pos[i];
#pragma unroll
            for (int d = 0; d < ND; ++d) s[d] += partial[p * ND + d];
        }
        if (mode == kOutWithPsi) {
            const int32_t ci = inv[c];
            const double wv = w_sorted ? w_sorted[ci] : 1.0;
#pragma unroll
            for (int d = 0; d < ND; ++d) out[d * ld_out + c] = fma(-kInv2PiC * wv, psi[(int64_t)ci * ND + d], s[d]);
        } else if (mode == kOutAccumulate) {
#pragma unroll
            for (int d = 0; d < ND; ++d) out[d * ld_out + c] += s[d];
        } else {
#pragma unroll
            for (int d = 0; d < ND; ++d) out[d * ld_out + c] = s[d];
        }
    }
}

template <int ND>
cudaError_t adj_nd(const DevGroupedCSR& A, bool f64, const double* x, int64_t ld_x, double* partial,
                   const int32_t* inv, const double* w_sorted, const double* psi, double* out, int64_t ld_out, int mode,
                   int max_blocks, cudaStream_t s)
{
    const int cap = max_blocks > 0 ? max_blocks : 152 * 16;
    const int blocks = std::max(1, std::min(A.ngroups, cap));
    if (A.ngroups > 0) {
        if (f64)
            k_adj_partial<ND, true><<<blocks, kAdjThreads, 0, s>>>(A, x, ld_x, partial);
        else
            k_adj_partial<ND, false><<<blocks, kAdjThreads, 0, s>>>(A, x, ld_x, partial);
    }
    const int gb = max_blocks > 0 ? std::max(1, std::min(max_blocks, grid_for(A.adj_ncols, 256)))
                                  : grid_for(A.adj_ncols, 256);
    k_adj_gather<ND><<<gb, 256, 0, s>>>(A.adj_ncols, A.inc_ptr, A.inc_pos, partial, inv, w_sorted, psi, out, ld_out,
                                        mode);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_csr_check(int64_t nnz, const int32_t* col, const double* val, int64_t ncols, int* err,
                             cudaStream_t s)
{
    if (nnz == 0) return cudaSuccess;
    k_csr_check<<<grid_for(nnz, 256 * 8), 256, 0, s>>>(nnz, col, val, ncols, err);
    return cudaGetLastError();
}

cudaError_t launch_row_same(int64_t nrows, const int64_t* rowptr, const int32_t* col, uint8_t* same, cudaStream_t s)
{
    if (nrows == 0) return cudaSuccess;
    k_row_same<<<grid_for(nrows, 8), 256, 0, s>>>(nrows, rowptr, col, same);
    return cudaGetLastError();
}

cudaError_t launch_group_cols(int32_t ngroups, const int32_t* g_r0, const int64_t* g_c0, const int64_t* rowptr,
                              const int32_t* col, int32_t* cols, cudaStream_t s)
{
    if (ngroups == 0) return cudaSuccess;
    k_group_cols<<<grid_for(ngroups, 8), 256, 0, s>>>(ngroups, g_r0, g_c0, rowptr, col, cols);
    return cudaGetLastError();
}

cudaError_t launch_pad_values(int64_t nrows, const int64_t* rowptr, const int64_t* prow, const double* val,
                              float2* vf, cudaStream_t s)
{
    if (nrows == 0) return cudaSuccess;
    k_pad_values<<<grid_for(nrows, 8), 256, 0, s>>>(nrows, rowptr, prow, val, vf);
    return cudaGetLastError();
}

cudaError_t launch_fix_values(int64_t nrows, const int64_t* rowptr, const int64_t* prow, const double* val, int2* vi,
                              int32_t* vexp, cudaStream_t s)
{
    if (nrows == 0) return cudaSuccess;
    k_fix_values<<<grid_for(nrows, 8), 256, 0, s>>>(nrows, rowptr, prow, val, vi, vexp);
    return cudaGetLastError();
}

cudaError_t launch_adj_grouped(int nd, const DevGroupedCSR& A, bool f64, const double* x, int64_t ld_x,
                               double* partial, const int32_t* inv, const double* w_sorted, const double* psi,
                               double* out, int64_t ld_out, int mode, int max_blocks, cudaStream_t s)
{
    switch (nd) {
        case 1: return adj_nd<1>(A, f64, x, ld_x, partial, inv, w_sorted, psi, out, ld_out, mode, max_blocks, s);
        case 2: return adj_nd<2>(A, f64, x, ld_x, partial, inv, w_sorted, psi, out, ld_out, mode, max_blocks, s);
        case 4: return adj_nd<4>(A, f64, x, ld_x, partial, inv, w_sorted, psi, out, ld_out, mode, max_blocks, s);
        case 8: return adj_nd<8>(A, f64, x, ld_x, partial, inv, w_sorted, psi, out, ld_out, mode, max_blocks, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vp
