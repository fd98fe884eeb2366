// Throughput calibration for the roofline denominators: how many FP64 and FP32
// fused multiply-adds per second this GPU sustains at its current clocks, from
// chains of independent FMAs in every lane of a full grid. The paper has no
// counterpart; the evaluation path never calls this.
#include <cuda_runtime.h>

#include <string>

#include "vp.h"

namespace vp {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kCalThreads = 256;
constexpr int kCalBlocksPerSm = 8;

// 8 independent chains per lane; the result is stored so the work is not removed
template <typename T>
__global__ void __launch_bounds__(kCalThreads) k_fma_chain(T* out, int iters, T a, T b)
{
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
cudaError_t time_fma(int blocks, int iters, T* buf, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* tflops)
{
    float best = 0.f;
    for (int rep = 0; rep < 3; ++rep) {  // the first launch also warms the clocks up
        cudaError_t e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) return e;
        k_fma_chain<T><<<blocks, kCalThreads, 0, s>>>(buf, iters, (T)0.999999, (T)1e-7);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    *tflops = 2.0 * 8.0 * (double)iters * blocks * kCalThreads / (best * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace

extern "C" vp_status vp_measure_peaks(double* fp64_tflops, double* fp32_tflops, void* stream)
{
    if (!fp64_tflops || !fp32_tflops) {
        vp::set_last_error("NULL output");
        return VP_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * kCalBlocksPerSm;
    void* buf = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&buf, (size_t)blocks * kCalThreads * sizeof(double));
    if (e != cudaSuccess) {
        vp::set_last_error(std::string("vp_measure_peaks: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = time_fma<double>(blocks, 2048, (double*)buf, s, e0, e1, fp64_tflops);
    if (e == cudaSuccess) e = time_fma<float>(blocks, 65536, (float*)buf, s, e0, e1, fp32_tflops);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) {
        vp::set_last_error(std::string("vp_measure_peaks: ") + cudaGetErrorString(e));
        return VP_ERR_CUDA;
    }
    return VP_OK;
}
