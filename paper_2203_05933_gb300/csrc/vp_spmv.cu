// Correction apply (a7): out = -(1/2pi) psi + Pi f, the sparse map of the
// per-cell corrections "accurate minus smooth" (arXiv 2203.05933, Sec. 4,
// paragraph after Eq. nsrcs), on the FP32 pipes in float-float arithmetic.
//
// The rows of one cell share their column list (every node of a cell couples
// to the nodes of the same near cells), so the plan stores each distinct
// column list once per group of consecutive rows. One block per group gathers
// x[:, cols] once into shared memory as hi/lo floats; each warp then streams
// its rows' values (8 bytes per nonzero, coalesced) and accumulates with
// TwoProd/TwoSum. HBM traffic is one read of the values plus the outputs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "vp_ff.cuh"
#include "vp_internal.h"

namespace vp {
namespace {

constexpr double kInv2PiG = 0.159154943091895335768883763372514362;
constexpr int kGroupThreads = 256;
constexpr int kGroupSmemBytes = 96 * 1024;

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

template <int ND>
__global__ void __launch_bounds__(kGroupThreads)
    k_out_grouped(DevGroupedCSR A, int smem_m, const int32_t* __restrict__ inv, const double* __restrict__ w_sorted,
                  const double* __restrict__ psi, const float2* __restrict__ xf, int64_t ld_xf,
                  double* __restrict__ out, int64_t ld_out)
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
        const int np = (m + 1) >> 1;  // value pairs per row (the padding value is zero)
        for (int r = r0 + warp; r < r1; r += nw) {
            const float4* vrow = reinterpret_cast<const float4*>(A.vf + A.rowptr[r]);  // rows start on 16 bytes
            // four independent accumulators per density keep four 16-byte loads in flight per lane
            ff::F acc[4][ND];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[u][d] = ff::F{0.f, 0.f};
            for (int q0 = lane; q0 < np; q0 += 128) {
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + 32 * u;
                    v[u] = q < np ? vrow[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int q = q0 + 32 * u;
                    if (q < np) {
                        const int k = 2 * q;
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            float4 x;
                            if (staged) {
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
            for (int d = 0; d < ND; ++d)
                acc[0][d] = ff::add(ff::add(acc[0][d], acc[1][d]), ff::add(acc[2][d], acc[3][d]));
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                for (int o = 16; o > 0; o >>= 1) {
                    const float h = __shfl_xor_sync(0xffffffffu, acc[0][d].h, o);
                    const float l = __shfl_xor_sync(0xffffffffu, acc[0][d].l, o);
                    acc[0][d] = ff::add(acc[0][d], ff::F{h, l});
                }
            }
            if (lane == 0) {
                if (psi) {
                    const int32_t ri = inv[r];
                    const double wv = w_sorted ? w_sorted[ri] : 1.0;
#pragma unroll
                    for (int d = 0; d < ND; ++d)
                        out[d * ld_out + r] = fma(-kInv2PiG * wv, psi[(int64_t)ri * ND + d], ff::to_double(acc[0][d]));
                } else {  // accumulate onto out
#pragma unroll
                    for (int d = 0; d < ND; ++d) out[d * ld_out + r] += ff::to_double(acc[0][d]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The same product with the values streamed into shared memory by the Tensor
// Memory Accelerator (cp.async.bulk, completion counted on an mbarrier), in
// runs of whole rows of one group, kTmaStages runs in flight per block: the
// copies of the next runs proceed while the warps reduce the current one from
// shared memory. Rows are padded to even lengths, so every run starts on a
// 16-byte boundary and has a multiple of 16 bytes. A wait that does not
// complete within its bound sets *err and ends the block.
constexpr int kTmaStages = 3;
constexpr int kTmaStageBytes = 32 * 1024;
constexpr int kTmaStageElems = kTmaStageBytes / 8;
constexpr long long kTmaWaitBound = 1LL << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// rows of group g that fit in one stage
__device__ __forceinline__ int tma_rows(const DevGroupedCSR& A, int g, int r)
{
    const int m = (int)(A.g_c0[g + 1] - A.g_c0[g]);
    const int mp = m + (m & 1);
    const int rpc = mp > 0 ? max(1, kTmaStageElems / mp) : 1 << 30;
    return min(rpc, A.g_r0[g + 1] - r);
}

template <int ND>
__global__ void __launch_bounds__(kGroupThreads)
    k_out_grouped_tma(DevGroupedCSR A, int smem_m, const int32_t* __restrict__ inv,
                      const double* __restrict__ w_sorted, const double* __restrict__ psi,
                      const float2* __restrict__ xf, int64_t ld_xf, double* __restrict__ out, int64_t ld_out,
                      int* __restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* stage = (float2*)smem_raw;                                        // [kTmaStages][kTmaStageElems]
    float2* F = (float2*)(smem_raw + (size_t)kTmaStages * kTmaStageBytes);   // [ND][smem_m]
    __shared__ __align__(8) uint64_t full[kTmaStages];
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int G = A.ngroups;
    if (tid == 0) {
        for (int s = 0; s < kTmaStages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();
    // producer cursor (thread 0): next run to load
    int pg = blockIdx.x, pr = pg < G ? A.g_r0[pg] : 0;
    auto produce = [&](int s) {
        while (pg < G && pr >= A.g_r0[pg + 1]) {
            pg += gridDim.x;
            if (pg < G) pr = A.g_r0[pg];
        }
        if (pg >= G) return;
        const int nr = tma_rows(A, pg, pr);
        const int64_t v0 = A.rowptr[pr], v1 = A.rowptr[pr + nr];
        const uint32_t bytes = (uint32_t)((v1 - v0) * 8);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&full[s], bytes);
        if (bytes > 0) bulk_copy_g2s(stage + (size_t)s * kTmaStageElems, A.vf + v0, bytes, &full[s]);
        pr += nr;
    };
    if (tid == 0)
        for (int s = 0; s < kTmaStages; ++s) produce(s);
    int cg = blockIdx.x, cr = cg < G ? A.g_r0[cg] : 0, last_g = -1;
    for (int c = 0;; ++c) {
        while (cg < G && cr >= A.g_r0[cg + 1]) {
            cg += gridDim.x;
            if (cg < G) cr = A.g_r0[cg];
        }
        if (cg >= G) break;
        const int s = c % kTmaStages;
        const uint32_t parity = (uint32_t)((c / kTmaStages) & 1);
        const int m = (int)(A.g_c0[cg + 1] - A.g_c0[cg]);
        const int mp = m + (m & 1);
        const int nr = tma_rows(A, cg, cr);
        if (cg != last_g) {  // block-uniform: gather x[:, cols] of the new group
            const int64_t c0 = A.g_c0[cg];
            for (int i = tid; i < m * ND; i += blockDim.x) {
                const int k = i % m, d = i / m;
                F[d * smem_m + k] = xf[d * ld_xf + A.cols[c0 + k]];
            }
            last_g = cg;
        }
        bool ok = false;
        for (long long it = 0; it < kTmaWaitBound && !ok; ++it) ok = mbar_try_wait(&full[s], parity);
        if (!ok) s_fail = 1;
        __syncthreads();  // F complete; every thread saw the run arrive (or a wait gave up)
        if (s_fail) {
            if (tid == 0) atomicExch(err, 1);
            return;
        }
        const float2* V = stage + (size_t)s * kTmaStageElems;
        for (int i = warp; i < nr; i += nw) {
            const float2* vr = V + (size_t)i * mp;
            ff::F acc[4][ND];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int d = 0; d < ND; ++d) acc[u][d] = ff::F{0.f, 0.f};
            for (int k0 = lane; k0 < m; k0 += 128) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = k0 + 32 * u;
                    if (k < m) {
                        const float2 v = vr[k];
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            const float2 x = F[d * smem_m + k];
                            acc[u][d] = ff::add(acc[u][d], ff::mul(ff::F{v.x, v.y}, ff::F{x.x, x.y}));
                        }
                    }
                }
            }
#pragma unroll
            for (int d = 0; d < ND; ++d)
                acc[0][d] = ff::add(ff::add(acc[0][d], acc[1][d]), ff::add(acc[2][d], acc[3][d]));
#pragma unroll
            for (int d = 0; d < ND; ++d) {
                for (int o = 16; o > 0; o >>= 1) {
                    const float h = __shfl_xor_sync(0xffffffffu, acc[0][d].h, o);
                    const float l = __shfl_xor_sync(0xffffffffu, acc[0][d].l, o);
                    acc[0][d] = ff::add(acc[0][d], ff::F{h, l});
                }
            }
            if (lane == 0) {
                const int r = cr + i;
                if (psi) {
                    const int32_t ri = inv[r];
                    const double wv = w_sorted ? w_sorted[ri] : 1.0;
#pragma unroll
                    for (int d = 0; d < ND; ++d)
                        out[d * ld_out + r] = fma(-kInv2PiG * wv, psi[(int64_t)ri * ND + d], ff::to_double(acc[0][d]));
                } else {
#pragma unroll
                    for (int d = 0; d < ND; ++d) out[d * ld_out + r] += ff::to_double(acc[0][d]);
                }
            }
        }
        __syncthreads();  // stage s and F are free
        if (tid == 0) produce(s);
        cr += nr;
    }
}

template <int ND>
cudaError_t launch_grouped_nd(const DevGroupedCSR& A, const int32_t* inv, const double* w_sorted, const double* psi,
                              const float2* xf, int64_t ld_xf, double* out, int64_t ld_out, int* err, cudaStream_t s)
{
    // bulk-copy path (kept for matrices whose rows are long enough to fill its stages;
    // with rows of a few hundred values the register-streaming kernel below is faster)
    if (err && A.ngroups > 0 && A.max_m >= kTmaStageElems / 2 && (int64_t)(A.max_m + 1) * 8 <= kTmaStageBytes && ((uintptr_t)A.vf % 16) == 0) {
        const int smem_m = A.max_m < 1 ? 1 : A.max_m;
        const size_t bytes = (size_t)kTmaStages * kTmaStageBytes + (size_t)smem_m * ND * sizeof(float2);
        if (bytes <= 200 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_out_grouped_tma<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)bytes);
            if (e != cudaSuccess) return e;
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_out_grouped_tma<ND>, kGroupThreads, bytes) !=
                    cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            int sms = 152, dev = 0;
            if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const int blocks = std::min(A.ngroups, sms * per_sm);
            k_out_grouped_tma<ND><<<blocks, kGroupThreads, bytes, s>>>(A, smem_m, inv, w_sorted, psi, xf, ld_xf, out,
                                                                      ld_out, err);
            return cudaGetLastError();
        }
    }
    cudaError_t e = cudaFuncSetAttribute(k_out_grouped<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kGroupSmemBytes);
    if (e != cudaSuccess) return e;
    int smem_m = kGroupSmemBytes / (ND * (int)sizeof(float2));
    if (A.max_m < smem_m) smem_m = A.max_m;
    if (smem_m < 1) smem_m = 1;
    const size_t bytes = (size_t)smem_m * ND * sizeof(float2);
    int blocks = A.ngroups < 152 * 16 ? A.ngroups : 152 * 16;
    if (blocks < 1) blocks = 1;
    k_out_grouped<ND><<<blocks, kGroupThreads, bytes, s>>>(A, smem_m, inv, w_sorted, psi, xf, ld_xf, out, ld_out);
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
                               int* err, cudaStream_t s)
{
    switch (nd) {
        case 1: return launch_grouped_nd<1>(A, inv, w_sorted, psi, xf, ld_xf, out, ld_out, err, s);
        case 2: return launch_grouped_nd<2>(A, inv, w_sorted, psi, xf, ld_xf, out, ld_out, err, s);
        case 4: return launch_grouped_nd<4>(A, inv, w_sorted, psi, xf, ld_xf, out, ld_out, err, s);
        case 8: return launch_grouped_nd<8>(A, inv, w_sorted, psi, xf, ld_xf, out, ld_out, err, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace vp
