// Throughput calibration for the roofline denominators: how many FP64 and FP32
// fused multiply-adds per second this GPU sustains at its current clocks, from
// chains of independent FMAs in every lane of a full grid; optionally the FP64
// tensor instruction (mma.sync m8n8k4 f64), the bf16 warp-level tensor
// instruction (mma.sync m16n8k16, f32 accumulation) and the int8 one
// (mma.sync m16n8k32, s32 accumulation) in the same way. The paper
// has no counterpart; the evaluation path never calls this.
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

// 4 independent chains of m8n8k4 f64 tensor products per warp (512 flops each)
__global__ void __launch_bounds__(kCalThreads) k_dmma_chain(double* out, int iters, double a, double b)
{
    double c[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[k][0]), "+d"(c[k][1])
                         : "d"(a), "d"(b));
    }
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) r += c[k][0] + c[k][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// 4 independent chains of m16n8k16 bf16 tensor products, f32 accumulation (4096 flops each)
__global__ void __launch_bounds__(kCalThreads) k_bf16mma_chain(double* out, int iters, unsigned a, unsigned b)
{
    float c[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[k][j] = 0.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile(
                "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                "{%0, %1, %2, %3};"
                : "+f"(c[k][0]), "+f"(c[k][1]), "+f"(c[k][2]), "+f"(c[k][3])
                : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
    }
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) r += c[k][0] + c[k][1] + c[k][2] + c[k][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// 4 independent chains of m16n8k32 int8 tensor products, s32 accumulation (8192 ops each)
__global__ void __launch_bounds__(kCalThreads) k_s8mma_chain(double* out, int iters, unsigned a, unsigned b)
{
    int c[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) c[k][j] = 0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                "{%0, %1, %2, %3};"
                : "+r"(c[k][0]), "+r"(c[k][1]), "+r"(c[k][2]), "+r"(c[k][3])
                : "r"(a), "r"(a), "r"(a), "r"(a), "r"(b), "r"(b));
    }
    int r = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) r += c[k][0] + c[k][1] + c[k][2] + c[k][3];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (double)r;
}

// kind: 0 FP64 FMA, 1 FP32 FMA, 2 f64 mma, 3 bf16 mma, 4 int8 mma
template <typename T>
cudaError_t time_fma(int blocks, int iters, T* buf, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* tflops,
                     int kind = -1)
{
    float best = 0.f;
    for (int rep = 0; rep < 3; ++rep) {  // the first launch also warms the clocks up
        cudaError_t e = cudaEventRecord(e0, s);
        if (e != cudaSuccess) return e;
        if (kind == 2)
            k_dmma_chain<<<blocks, kCalThreads, 0, s>>>((double*)buf, iters, 0.999999, 1e-7);
        else if (kind == 3)
            k_bf16mma_chain<<<blocks, kCalThreads, 0, s>>>((double*)buf, iters, 0x3f803f80u, 0x00010001u);
        else if (kind == 4)
            k_s8mma_chain<<<blocks, kCalThreads, 0, s>>>((double*)buf, iters, 0x01010101u, 0x01010101u);
        else
            k_fma_chain<T><<<blocks, kCalThreads, 0, s>>>(buf, iters, (T)0.999999, (T)1e-7);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    // flops per thread and iteration: 8 FMAs; 4 mma of 512 or 4096 flops per warp
    const double per = kind == 2 ? 4.0 * 512.0 / 32.0
                     : (kind == 3 ? 4.0 * 4096.0 / 32.0 : (kind == 4 ? 4.0 * 8192.0 / 32.0 : 16.0));
    *tflops = per * (double)iters * blocks * kCalThreads / (best * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace

extern "C" vp_status vp_measure_peaks(double* fp64_tflops, double* fp32_tflops, double* dmma_tflops,
                                      double* bf16_mma_tflops, double* s8_mma_tops, void* stream)
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
    if (e == cudaSuccess && dmma_tflops) e = time_fma<double>(blocks, 1024, (double*)buf, s, e0, e1, dmma_tflops, 2);
    if (e == cudaSuccess && bf16_mma_tflops)
        e = time_fma<double>(blocks, 16384, (double*)buf, s, e0, e1, bf16_mma_tflops, 3);
    if (e == cudaSuccess && s8_mma_tops) e = time_fma<double>(blocks, 16384, (double*)buf, s, e0, e1, s8_mma_tops, 4);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess) {
        vp::set_last_error(std::string("vp_measure_peaks: ") + cudaGetErrorString(e));
        return VP_ERR_CUDA;
    }
    return VP_OK;
}
