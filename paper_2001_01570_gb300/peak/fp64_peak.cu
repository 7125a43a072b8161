// FP64 throughput of this GPU, the denominator of the stage kernels' roofline
// (they are bound by the FP64 pipe).  Eight independent chains per thread, 8
// CTAs of 256 threads per SM, CUDA events around one launch after a warm-up
// launch.  Rates in G operations per second; FMA counts as one operation here
// (the roofline uses 2 flops per FMA).  Also: DADD, FP32 FFMA, and the FP64
// divide, correctly rounded reciprocal, sqrt, exp and erfc as called from CUDA
// code, and a DFMA occupancy sweep.
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096
__global__ void k_dfma(double* out, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < ITERS; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void k_dadd(double* out, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < ITERS; ++i) {
    x0 = x0 + a; x1 = x1 + a; x2 = x2 + a; x3 = x3 + a; x4 = x4 + b; x5 = x5 + b; x6 = x6 + b; x7 = x7 + b;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void k_ffma(float* out, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < ITERS; ++i) {
    x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
__global__ void k_ddiv(double* out, double a) {
  double x0 = 1.0 + threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS / 8; ++i) { x0 = a / x0 + 1.0; x1 = a / x1 + 1.0; x2 = a / x2 + 1.0; x3 = a / x3 + 1.0; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_rcp(double* out, double a) {
  double x0 = 1.0 + threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS / 8; ++i) { x0 = __drcp_rn(x0) + a; x1 = __drcp_rn(x1) + a; x2 = __drcp_rn(x2) + a; x3 = __drcp_rn(x3) + a; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_sqrt(double* out, double a) {
  double x0 = 1.0 + threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
  for (int i = 0; i < ITERS / 8; ++i) { x0 = sqrt(x0) + a; x1 = sqrt(x1) + a; x2 = sqrt(x2) + a; x3 = sqrt(x3) + a; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_exp(double* out, double a) {
  double x0 = -1.0 - threadIdx.x * 1e-3, x1 = x0 - 1, x2 = x0 - 2, x3 = x0 - 3;
  for (int i = 0; i < ITERS / 8; ++i) { x0 = -exp(x0) - a; x1 = -exp(x1) - a; x2 = -exp(x2) - a; x3 = -exp(x3) - a; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
__global__ void k_erfc(double* out, double a) {
  double x0 = 0.1 + threadIdx.x * 1e-4, x1 = x0 + 0.5, x2 = x0 + 1, x3 = x0 - 1.5;
  for (int i = 0; i < ITERS / 8; ++i) { x0 = erfc(x0) * a; x1 = erfc(x1) * a; x2 = erfc(x2) * a; x3 = erfc(x3) * a; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3;
}
int main() {
  int nsm = 0; cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  int clk = 0; cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
  printf("SMs %d clock(kHz) %d\n", nsm, clk);
  int blocks = nsm * 8, threads = 256;
  double* d; cudaMalloc(&d, (size_t)blocks * threads * sizeof(double));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  double n = (double)blocks * threads;
#define RUN(name, launch, ops) \
  launch; cudaDeviceSynchronize(); cudaEventRecord(e0); launch; cudaEventRecord(e1); cudaEventSynchronize(e1); \
  cudaEventElapsedTime(&ms, e0, e1); printf("%-6s %8.3f ms  %10.3f Gop/s  (%s)\n", name, ms, n * (ops) / (ms * 1e6), cudaGetErrorString(cudaGetLastError()));
  RUN("dfma", (k_dfma<<<blocks, threads>>>(d, 0.999, 1e-3)), 8.0 * ITERS)
  RUN("dadd", (k_dadd<<<blocks, threads>>>(d, 0.999, 1e-3)), 8.0 * ITERS)
  RUN("ffma", (k_ffma<<<blocks, threads>>>((float*)d, 0.999f, 1e-3f)), 8.0 * ITERS)
  RUN("ddiv", (k_ddiv<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  RUN("drcp", (k_rcp<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  RUN("dsqrt", (k_sqrt<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  RUN("dexp", (k_exp<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  RUN("derfc", (k_erfc<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  // occupancy sweep of dfma: blocks per SM
  for (int bps = 1; bps <= 8; bps *= 2) for (int th = 64; th <= 256; th *= 2) {
    int b = nsm * bps; double nn = (double)b * th;
    k_dfma<<<b, th>>>(d, 0.999, 1e-3); cudaDeviceSynchronize();
    cudaEventRecord(e0); k_dfma<<<b, th>>>(d, 0.999, 1e-3); cudaEventRecord(e1); cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("dfma blocks/SM %d threads %3d : %8.3f Gop/s\n", bps, th, nn * 8.0 * ITERS / (ms * 1e6));
  }
  cudaFree(d);
  return 0;
}
