// Allocation-free evaluation for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need the volume potential: code running while a CUDA graph is
// being captured by someone else's allocator policy, plug-ins whose host
// application owns every device allocation, or embedded users that must not
// grow the device footprint after start-up. vp_eval_direct_static serves them:
// it evaluates the same quantity as vp_eval (smooth-rule point sum plus the
// correction matrix) by direct summation over all sources, without a plan, and
// keeps its intermediate charges and partial sums in a fixed file-scope device
// array instead of allocating. The paper has no counterpart; it is a
// convenience variant of the direct (P2P) kernel for small problems.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "vp.h"

namespace vp {
void set_last_error(const std::string& msg);  // defined with the rest of the ABI (vp_api.cu)
}

namespace {

constexpr double kInv2PiS = 0.159154943091895335768883763372514362;
constexpr int kStaticThreads = 128;
constexpr int kMaxSplit = 32;
constexpr int kMaxDevices = 64;

// The shared scratch: every GPU that loads the library holds it until exit.
static __device__ __align__(256) double g_vp_static_scratch[VP_STATIC_SCRATCH_DOUBLES];

std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {};

// q[j] = w[j] f[j]
__global__ void k_static_charges(int64_t n, const double* __restrict__ w, const double* __restrict__ f,
                                 double* __restrict__ q)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        q[j] = w[j] * f[j];
}

// partial[s][i] = sum over source slice s of q_j log|t_i - r_j| (coincident pairs skipped)
__global__ void __launch_bounds__(kStaticThreads)
    k_static_partial(int64_t n_src, const double2* __restrict__ src, const double* __restrict__ q, int64_t n_tgt,
                     const double2* __restrict__ tgt, int64_t chunk, double* __restrict__ partial)
{
    __shared__ double2 sxy[kStaticThreads];
    __shared__ double sq[kStaticThreads];
    const int64_t i = blockIdx.x * (int64_t)kStaticThreads + threadIdx.x;
    const bool valid = i < n_tgt;
    const double2 t = valid ? tgt[i] : make_double2(0.0, 0.0);
    const int64_t j0 = blockIdx.y * chunk;
    const int64_t j1 = j0 + chunk < n_src ? j0 + chunk : n_src;
    double acc = 0.0;
    for (int64_t b = j0; b < j1; b += kStaticThreads) {
        const int n = (int)(j1 - b < kStaticThreads ? j1 - b : kStaticThreads);
        __syncthreads();
        if (threadIdx.x < n) {
            sxy[threadIdx.x] = src[b + threadIdx.x];
            sq[threadIdx.x] = q[b + threadIdx.x];
        }
        __syncthreads();
        if (valid) {
            for (int k = 0; k < n; ++k) {
                const double dx = t.x - sxy[k].x, dy = t.y - sxy[k].y;
                if (dx == 0.0 && dy == 0.0) continue;
                acc = fma(sq[k], 0.5 * log(dx * dx + dy * dy), acc);
            }
        }
    }
    if (valid) partial[blockIdx.y * n_tgt + i] = acc;
}

// out[i] = -(1/2pi) sum_s partial[s][i] + sum_k val[k] f[col[k]], one warp per row
__global__ void k_static_reduce(int64_t n_tgt, int nsplit, const double* __restrict__ partial,
                                const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ f, double* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n_tgt; i += warps) {
        double s = 0.0;
        if (rowptr) {
            for (int64_t k = rowptr[i] + lane; k < rowptr[i + 1]; k += 32) s = fma(val[k], f[col[k]], s);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            double p = 0.0;
            for (int sp = 0; sp < nsplit; ++sp) p += partial[sp * n_tgt + i];
            out[i] = fma(-kInv2PiS, p, s);
        }
    }
}

vp_status static_fail(vp_status st, const std::string& m)
{
    vp::set_last_error(m);
    return st;
}

// Device address of the scratch array for the current device. It is looked up
// with that device current on every call made outside a stream capture (the
// lookup allocates nothing, and a fresh lookup stays valid after the module was
// reloaded, e.g. after cudaDeviceReset); a call made while `s` is being
// captured reuses the address of the device's last uncaptured call.
vp_status static_scratch(cudaStream_t s, double** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(VP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return static_fail(VP_ERR_UNSUPPORTED, "device ordinal above 63");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return static_fail(VP_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (cs != cudaStreamCaptureStatusNone && !g_static_ptr[dev])
        return static_fail(VP_ERR_STATE, "first call on this device made inside a stream capture: call once outside "
                                         "the capture first");
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_vp_static_scratch);
        if (e != cudaSuccess || !p)
            return static_fail(VP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_static_ptr[dev] = (double*)p;
    }
    *out = g_static_ptr[dev];
    return VP_OK;
}

}  // namespace

extern "C" vp_status vp_eval_direct_static(int64_t n_src, const double* src_xy, const double* w, int32_t ndens,
                                           const double* f, int64_t ld_f, int64_t n_tgt, const double* tgt_xy,
                                           const int64_t* corr_rowptr, const int32_t* corr_col,
                                           const double* corr_val, double* out, int64_t ld_out, void* stream)
{
    vp::set_last_error("");
    if (n_src < 0 || n_tgt < 0 || ndens < 0) return static_fail(VP_ERR_ARG, "negative size");
    if (ndens == 0 || n_tgt == 0) return VP_OK;
    if (!out || !tgt_xy || (n_src > 0 && (!src_xy || !w || !f)))
        return static_fail(VP_ERR_ARG, "NULL input or output");
    if (ld_f < n_src || ld_out < n_tgt) return static_fail(VP_ERR_ARG, "leading dimension too small");
    if (corr_rowptr && n_src > 0 && (!corr_col || !corr_val)) return static_fail(VP_ERR_ARG, "NULL CSR array");
    // a correction needs source values to multiply (its rows are not read here, see below)
    if (corr_rowptr && n_src == 0) return static_fail(VP_ERR_ARG, "correction matrix given with n_src == 0");
    // the kernels read the points as 16-byte (double2) vectors
    if ((((uintptr_t)src_xy) | ((uintptr_t)tgt_xy)) & 15u)
        return static_fail(VP_ERR_ARG, "src_xy and tgt_xy must be 16-byte aligned");
    // scratch layout per density pass: q [n_src] then partial [nsplit][n_tgt]
    int64_t nsplit = (n_src + 4095) / 4096;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > kMaxSplit) nsplit = kMaxSplit;
    while (nsplit > 1 && n_src + nsplit * n_tgt > (int64_t)VP_STATIC_SCRATCH_DOUBLES) --nsplit;
    if (n_src + nsplit * n_tgt > (int64_t)VP_STATIC_SCRATCH_DOUBLES)
        return static_fail(VP_ERR_ARG, "problem too large for the static scratch: n_src + n_tgt must not exceed "
                                       "VP_STATIC_SCRATCH_DOUBLES");
    double* scratch = nullptr;
    vp_status st = static_scratch((cudaStream_t)stream, &scratch);
    if (st != VP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    double* q = scratch;
    double* partial = scratch + n_src;
    const int64_t chunk = n_src > 0 ? (n_src + nsplit - 1) / nsplit : 1;
    const dim3 grid((unsigned)((n_tgt + kStaticThreads - 1) / kStaticThreads), (unsigned)nsplit);
    for (int32_t d = 0; d < ndens; ++d) {
        const double* fd = f ? f + (int64_t)d * ld_f : nullptr;
        if (n_src > 0) {
            const int cb = (int)((n_src + 255) / 256 < 4096 ? (n_src + 255) / 256 : 4096);
            k_static_charges<<<cb, 256, 0, s>>>(n_src, w, fd, q);
        }
        k_static_partial<<<grid, kStaticThreads, 0, s>>>(n_src, (const double2*)src_xy, q, n_tgt,
                                                         (const double2*)tgt_xy, chunk, partial);
        const int rb = (int)((n_tgt + 3) / 4 < 4096 ? (n_tgt + 3) / 4 : 4096);
        k_static_reduce<<<rb, 128, 0, s>>>(n_tgt, (int)nsplit, partial, corr_rowptr, corr_col, corr_val, fd,
                                           out + (int64_t)d * ld_out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return static_fail(VP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    }
    return VP_OK;
}
