// FP64 throughput of this GPU, the denominator of the stage kernels' roofline
// (they are bound by the FP64 pipe).  Throughput loops of DFMA, DADD, DMUL and
// half-and-half mixes: independent chains per thread, operands in registers,
// a runtime trip count, CUDA events around one launch after a warm-up launch;
// thread 0 of block 0 also reads clock64() and %globaltimer at its start and
// end, which gives the SM clock during the loop and the rate per SM and cycle.
// Rates in G operations per second; FMA counts as one operation here (the
// roofline uses 2 flops per FMA).  Also: FP32 FFMA, and the FP64 divide,
// correctly rounded reciprocal, sqrt, exp and erfc as called from CUDA code,
// and a DFMA occupancy sweep.
#include <cstdio>
#include <cuda_runtime.h>
#define ITERS 4096

struct Clk { unsigned long long c0, c1, t0, t1; };
__device__ __forceinline__ unsigned long long global_ns()
{
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// OP 0: x = fma(x, a, b); 1: x = x + b; 2: x = x * a; 3: fma and mul on
// alternate chains; 4: fma and add on alternate chains; 5: fma(x, 0.99999, b)
// with a compile-time multiplicand; 6: x * 0.99999; 7: x + b written as
// fma(x, one, b) and 8: x * a written as fma(x, a, nzero), with one = 1.0 and
// nzero = -0.0 read from shared memory
template <int OP, int CH>
__global__ void k_fp64(double* out, Clk* clk, double a, double b, int iters)
{
  const unsigned long long c0 = clock64(), t0 = global_ns();
  __shared__ double s_k[2];
  if (threadIdx.x == 0) { s_k[0] = 1.0; s_k[1] = -0.0; }
  __syncthreads();
  const double one = ((volatile double*)s_k)[0], nzero = ((volatile double*)s_k)[1];
  const double ar = a + threadIdx.x * 1e-15, br = b + threadIdx.x * 1e-15;
  double x[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) x[c] = 1.0 + threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (OP == 0 || ((OP == 3 || OP == 4) && (c & 1) == 0)) x[c] = fma(x[c], ar, br);
      else if (OP == 1 || OP == 4) x[c] = x[c] + br;
      else if (OP == 2 || OP == 3) x[c] = x[c] * ar;
      else if (OP == 5) x[c] = fma(x[c], 0.99999, br);
      else if (OP == 6) x[c] = x[c] * 0.99999;
      else if (OP == 7) x[c] = fma(x[c], one, br);
      else x[c] = fma(x[c], ar, nzero);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) { clk->c0 = c0; clk->c1 = clock64(); clk->t0 = t0; clk->t1 = global_ns(); }
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
  printf("SMs %d max clock(kHz) %d\n", nsm, clk);
  int blocks = nsm * 8, threads = 256;
  double* d; cudaMalloc(&d, (size_t)blocks * threads * sizeof(double));
  Clk* dclk; cudaMalloc(&dclk, sizeof(Clk));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  float ms;
  double n = (double)blocks * threads;
  // FP64 loops: rate, SM clock of block 0 during the loop, rate per SM and cycle
#define RUN64(name, OP, CH, nb, nt, iters) {                                                          \
    k_fp64<OP, CH><<<nb, nt>>>(d, dclk, 0.99999, 1e-3, iters); cudaDeviceSynchronize();               \
    cudaEventRecord(e0); k_fp64<OP, CH><<<nb, nt>>>(d, dclk, 0.99999, 1e-3, iters); cudaEventRecord(e1); \
    cudaEventSynchronize(e1); cudaEventElapsedTime(&ms, e0, e1);                                       \
    Clk h; cudaMemcpy(&h, dclk, sizeof(Clk), cudaMemcpyDeviceToHost);                                  \
    const double ops = (double)(nb) * (nt) * (CH) * (double)(iters);                                   \
    const double mhz = 1e3 * (double)(h.c1 - h.c0) / (double)(h.t1 - h.t0);                            \
    printf("%-24s %8.3f ms  %10.3f Gop/s  SM clock %7.1f MHz  %.3f per SM per cycle  (%s)\n", name, ms,  \
           ops / (ms * 1e6), mhz, ops / (ms * 1e-3) / (nsm * mhz * 1e6), cudaGetErrorString(cudaGetLastError())); }
  RUN64("dfma", 0, 8, blocks, threads, ITERS)
  RUN64("dadd", 1, 8, blocks, threads, ITERS)
  RUN64("dmul", 2, 8, blocks, threads, ITERS)
  RUN64("dfma+dmul", 3, 8, blocks, threads, ITERS)
  RUN64("dfma+dadd", 4, 8, blocks, threads, ITERS)
  RUN64("dfma, 0.4 s", 0, 8, blocks, threads, ITERS * 25)
  RUN64("dfma, immediate mult.", 5, 8, blocks, threads, ITERS)
  RUN64("dmul by immediate", 6, 8, blocks, threads, ITERS)
  RUN64("add as fma(x, one, b)", 7, 8, blocks, threads, ITERS)
  RUN64("mul as fma(x, a, nzero)", 8, 8, blocks, threads, ITERS)
#define RUN(name, launch, ops) \
  launch; cudaDeviceSynchronize(); cudaEventRecord(e0); launch; cudaEventRecord(e1); cudaEventSynchronize(e1); \
  cudaEventElapsedTime(&ms, e0, e1); printf("%-24s %8.3f ms  %10.3f Gop/s  (%s)\n", name, ms, n * (ops) / (ms * 1e6), cudaGetErrorString(cudaGetLastError()));
  RUN("ffma", (k_ffma<<<blocks, threads>>>((float*)d, 0.999f, 1e-3f)), 8.0 * ITERS)
  RUN("ddiv", (k_ddiv<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  RUN("drcp", (k_rcp<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  RUN("dsqrt", (k_sqrt<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  RUN("dexp", (k_exp<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  RUN("derfc", (k_erfc<<<blocks, threads>>>(d, 0.7)), 4.0 * ITERS / 8)
  // occupancy sweep of dfma: CTAs per SM x threads per CTA, and the chain count
  for (int bps = 1; bps <= 8; bps *= 2)
    for (int th = 64; th <= 256; th *= 2) {
      char name[64];
      snprintf(name, sizeof(name), "dfma %d CTA/SM x %d", bps, th);
      RUN64(name, 0, 8, nsm * bps, th, ITERS)
    }
  RUN64("dfma 4 chains", 0, 4, blocks, threads, 2 * ITERS)
  RUN64("dfma 2 chains", 0, 2, blocks, threads, 4 * ITERS)
  RUN64("dfma 1 chain", 0, 1, blocks, threads, 8 * ITERS)
  cudaFree(d); cudaFree(dclk);
  return 0;
}
