// Throughput probe for the roofline denominators on this GPU (not part of libvp): FP64 FMA,
// FP32 FMA, FP64 mma.sync (m8n8k4 and m16n8k4), CUDA FP64 log, FP32 logf and __logf.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 probe_peaks.cu -o probe && ./probe
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("CUDA err %s at %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

__global__ void k_dfma(double* out, int iters, double a, double b){
  double x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for(int i=0;i<iters;i++){
    x0=fma(x0,a,b);x1=fma(x1,a,b);x2=fma(x2,a,b);x3=fma(x3,a,b);
    x4=fma(x4,a,b);x5=fma(x5,a,b);x6=fma(x6,a,b);x7=fma(x7,a,b);
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void k_ffma(float* out, int iters, float a, float b){
  float x0=threadIdx.x, x1=x0+1, x2=x0+2, x3=x0+3, x4=x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for(int i=0;i<iters;i++){
    x0=fmaf(x0,a,b);x1=fmaf(x1,a,b);x2=fmaf(x2,a,b);x3=fmaf(x3,a,b);
    x4=fmaf(x4,a,b);x5=fmaf(x5,a,b);x6=fmaf(x6,a,b);x7=fmaf(x7,a,b);
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=x0+x1+x2+x3+x4+x5+x6+x7;
}
__global__ void k_dmma884(double* out, int iters){
  double a=threadIdx.x*1e-3, b=1.0+threadIdx.x*1e-4;
  double c0[4]={0,0,0,0}, c1[4]={0,0,0,0};
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int j=0;j<2;j++){
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
        : "+d"(c0[2*j]), "+d"(c0[2*j+1]) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
        : "+d"(c1[2*j]), "+d"(c1[2*j+1]) : "d"(a), "d"(b));
    }
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=c0[0]+c0[1]+c0[2]+c0[3]+c1[0]+c1[1]+c1[2]+c1[3];
}
__global__ void k_dmma1684(double* out, int iters){
  double a0=threadIdx.x*1e-3, a1=a0+1e-3, b=1.0+threadIdx.x*1e-4;
  double c[4][4]={};
  for(int i=0;i<iters;i++){
    #pragma unroll
    for(int j=0;j<4;j++){
      asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3]) : "d"(a0), "d"(a1), "d"(b));
    }
  }
  double s=0; for(int j=0;j<4;j++) for(int k=0;k<4;k++) s+=c[j][k];
  out[blockIdx.x*blockDim.x+threadIdx.x]=s;
}
__global__ void k_dlog(double* out, int iters){
  double x=1.0+threadIdx.x*1e-3, s0=0,s1=0,s2=0,s3=0;
  for(int i=0;i<iters;i++){
    s0+=log(x); s1+=log(x+0.5); s2+=log(x+1.5); s3+=log(x+2.5); x+=1e-7;
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=s0+s1+s2+s3;
}
__global__ void k_flog(float* out, int iters){
  float x=1.0f+threadIdx.x*1e-3f, s0=0,s1=0,s2=0,s3=0;
  for(int i=0;i<iters;i++){
    s0+=logf(x); s1+=logf(x+0.5f); s2+=logf(x+1.5f); s3+=logf(x+2.5f); x+=1e-6f;
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=s0+s1+s2+s3;
}
__global__ void k_flog_fast(float* out, int iters){
  float x=1.0f+threadIdx.x*1e-3f, s0=0,s1=0,s2=0,s3=0;
  for(int i=0;i<iters;i++){
    s0+=__logf(x); s1+=__logf(x+0.5f); s2+=__logf(x+1.5f); s3+=__logf(x+2.5f); x+=1e-6f;
  }
  out[blockIdx.x*blockDim.x+threadIdx.x]=s0+s1+s2+s3;
}
int main(){
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p,0));
  printf("device %s sm_%d%d SMs %d l2 %d MB smem/block optin %zu\n", p.name,p.major,p.minor,p.multiProcessorCount,p.l2CacheSize>>20,p.sharedMemPerBlockOptin);
  int blocks=p.multiProcessorCount*8, threads=256; size_t n=(size_t)blocks*threads;
  double* dout; CK(cudaMalloc(&dout,n*sizeof(double)));
  cudaEvent_t e0,e1; cudaEventCreate(&e0); cudaEventCreate(&e1); float ms;
  for(int rep=0;rep<2;rep++){
  { int it=4096; k_dfma<<<blocks,threads>>>(dout,16,1.0000001,1e-9); cudaEventRecord(e0); k_dfma<<<blocks,threads>>>(dout,it,1.0000001,1e-9); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    printf("DFMA: %.1f GFLOP/s (%.3f ms)\n", 2.0*8*it*n/(ms*1e6), ms); }
  { int it=65536; k_ffma<<<blocks,threads>>>((float*)dout,16,1.0000001f,1e-9f); cudaEventRecord(e0); k_ffma<<<blocks,threads>>>((float*)dout,it,1.0000001f,1e-9f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    printf("FFMA: %.1f GFLOP/s (%.3f ms)\n", 2.0*8*it*n/(ms*1e6), ms); }
  { int it=1024; k_dmma884<<<blocks,threads>>>(dout,4); cudaEventRecord(e0); k_dmma884<<<blocks,threads>>>(dout,it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    double warps=n/32.0; printf("DMMA m8n8k4: %.1f GFLOP/s (%.3f ms)\n", warps*it*4*(2.0*8*8*4)/(ms*1e6), ms); }
  { int it=512; k_dmma1684<<<blocks,threads>>>(dout,4); cudaEventRecord(e0); k_dmma1684<<<blocks,threads>>>(dout,it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    double warps=n/32.0; printf("DMMA m16n8k4: %.1f GFLOP/s (%.3f ms)\n", warps*it*4*(2.0*16*8*4)/(ms*1e6), ms); }
  { int it=512; k_dlog<<<blocks,threads>>>(dout,4); cudaEventRecord(e0); k_dlog<<<blocks,threads>>>(dout,it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    printf("FP64 log: %.2f Glog/s (%.3f ms)\n", 4.0*it*n/(ms*1e6), ms); }
  { int it=8192; k_flog<<<blocks,threads>>>((float*)dout,4); cudaEventRecord(e0); k_flog<<<blocks,threads>>>((float*)dout,it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    printf("FP32 logf: %.2f Glog/s (%.3f ms)\n", 4.0*it*n/(ms*1e6), ms); }
  { int it=8192; k_flog_fast<<<blocks,threads>>>((float*)dout,4); cudaEventRecord(e0); k_flog_fast<<<blocks,threads>>>((float*)dout,it); cudaEventRecord(e1); CK(cudaEventSynchronize(e1)); cudaEventElapsedTime(&ms,e0,e1);
    printf("FP32 __logf: %.2f Glog/s (%.3f ms)\n", 4.0*it*n/(ms*1e6), ms); }
  }
  CK(cudaGetLastError());
  return 0;
}
