// cgks_diag.cu -- libcgks_diag: checks of the flux kernels' own math routines
// against CUDA's, and the FP64 throughput of the GPU that the kernels' roofline
// divides by.  Not part of the solver's C ABI (include/cgks.h); the test suite
// and the benchmark call it.
//
//   cgks_diag_exp_neg_maxulp   exp_neg (cgks_flux.cuh: Tang's table-driven e^x,
//                              x <= 0) against CUDA's exp, largest difference in
//                              units in the last place over n arguments
//   cgks_diag_rcp_maxulp       RegK::rcp (cgks_device.cuh: rcp.approx + two
//                              Newton-Raphson steps) against __drcp_rn
//   cgks_diag_erfc_maxrel      erfc_scaled (the erfcx table of cgks_erfcx_table.h
//                              times exp_neg(-t^2)) against CUDA's erfc, largest
//                              relative difference over t in [0, 26]
//   cgks_diag_fp64_rate        throughput of one FP64 operation (DFMA with
//                              register operands -- the issue form the kernels
//                              use --, DADD, DMUL, immediate operands, divide,
//                              exp, erfc), with the SM clock read during the loop
// All return 0 on success or the cudaError_t of the failing call.
#include "../cgks_flux.cuh"

#include <cuda_runtime.h>

namespace {

using namespace cgks;

__constant__ FluxFixed kDiagFixed = make_flux_fixed();

// the coefficient table as the stage kernel builds it (fixed part, 2^(j/32))
__device__ __forceinline__ RegK diag_table(double* s_fk)
{
    for (int i = threadIdx.x; i < FK_NFIX; i += blockDim.x) s_fk[i] = kDiagFixed.v[i];
    if (threadIdx.x < 32) s_fk[FK_EXP2 + threadIdx.x] = exp2((double)threadIdx.x * (1.0 / 32.0));
    __syncthreads();
    return RegK{s_fk, ((volatile const double*)s_fk)[FK_ONE], ((volatile const double*)s_fk)[FK_NZERO]};
}

__device__ __forceinline__ unsigned long long ulp_diff(double a, double b)
{
    long long d = __double_as_longlong(a) - __double_as_longlong(b);
    return (unsigned long long)(d < 0 ? -d : d);
}

// arguments: half of them uniform in [-700, 0], the other half dense near 0
__global__ void exp_kernel(unsigned long long* maxulp, int n)
{
    __shared__ double s_fk[FK_NFIX2];
    const RegK r = diag_table(s_fk);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = -700.0 * ((double)i / (double)n);
    if (i & 1) x = -(double)(i % 100000) * 1e-5;
    atomicMax(maxulp, ulp_diff(exp_neg(r, x), exp(x)));
}

// every mantissa pattern of a stride through [1, 2), scaled by 1e-150 and
// 1e+150, both signs
__global__ void rcp_kernel(unsigned long long* maxulp, int n)
{
    __shared__ double s_fk[FK_NFIX2];
    const RegK r = diag_table(s_fk);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long mant = ((unsigned long long)i * 0x0000001000000001ULL) & 0x000FFFFFFFFFFFFFULL;
    double x = __longlong_as_double((long long)(0x3FF0000000000000ULL | mant));
    x *= (i & 1) ? 1e150 : 1e-150;
    if (i & 2) x = -x;
    atomicMax(maxulp, ulp_diff(r.rcp(x), __drcp_rn(x)));
}

// relative difference as the bits of a non-negative double (ordered like the value)
__global__ void erfc_kernel(unsigned long long* maxrel_bits, int n)
{
    __shared__ double s_fk[FK_NFIX2];
    const RegK r = diag_table(s_fk);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double t = 26.0 * ((double)i / (double)n);
    const double e = exp_neg(r, -(t * t));
    const double ref = erfc(t);
    const double got = erfc_scaled(r, t, e);
    const double rel = ref > 0.0 ? fabs(got - ref) / ref : fabs(got);
    atomicMax(maxrel_bits, (unsigned long long)__double_as_longlong(rel));
}

constexpr int kChains = 8;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// kChains independent chains per thread of one FP64 operation:
//   0 fma(x, a, b), all operands in registers      1 x + b (DADD)
//   2 x * a (DMUL)                                 3 fma(x, 0.99999, b), immediate multiplicand
//   4 x + b written as fma(x, one, b)              5 x * a written as fma(x, a, nzero)
//   6 a / x + 1 (divide)                           7 -exp(x) - b (CUDA's exp)
//   8 erfc(x) * a (CUDA's erfc)                    9 rsqrt(x) + b (CUDA's rsqrt)
// with one = 1.0 and nzero = -0.0 read from shared memory through volatile loads
// (the register forms of RegK)
template <int OP>
__global__ void fp64_kernel(double* out, unsigned long long* clk, double a, double b, int iters)
{
    const unsigned long long c0 = clock64(), t0 = global_ns();
    __shared__ double s_k[2];
    if (threadIdx.x == 0) { s_k[0] = 1.0; s_k[1] = -0.0; }
    __syncthreads();
    const double one = ((volatile double*)s_k)[0], nzero = ((volatile double*)s_k)[1];
    const double ar = a + threadIdx.x * 1e-15, br = b + threadIdx.x * 1e-15;
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = OP == 7 ? -1.0 - threadIdx.x * 1e-3 - c : (OP == 8 ? 0.1 + threadIdx.x * 1e-4 + 0.3 * c
                                                                 : 1.0 + threadIdx.x * 1e-3 + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (OP == 0) x[c] = fma(x[c], ar, br);
            if (OP == 1) x[c] = x[c] + br;
            if (OP == 2) x[c] = x[c] * ar;
            if (OP == 3) x[c] = fma(x[c], 0.99999, br);
            if (OP == 4) x[c] = fma(x[c], one, br);
            if (OP == 5) x[c] = fma(x[c], ar, nzero);
            if (OP == 6) x[c] = ar / x[c] + 1.0;
            if (OP == 7) x[c] = -exp(x[c]) - br;
            if (OP == 8) x[c] = erfc(x[c]) * ar;
            if (OP == 9) x[c] = rsqrt(x[c]) + br;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = c0;
        clk[1] = clock64();
        clk[2] = t0;
        clk[3] = global_ns();
    }
}

void launch_fp64(int op, int blocks, int threads, double* d, unsigned long long* clk, double a, double b, int iters)
{
    switch (op) {
    case 0: fp64_kernel<0><<<blocks, threads>>>(d, clk, a, b, iters); break;
    case 1: fp64_kernel<1><<<blocks, threads>>>(d, clk, a, b, iters); break;
    case 2: fp64_kernel<2><<<blocks, threads>>>(d, clk, a, b, iters); break;
    case 3: fp64_kernel<3><<<blocks, threads>>>(d, clk, a, b, iters); break;
    case 4: fp64_kernel<4><<<blocks, threads>>>(d, clk, a, b, iters); break;
    case 5: fp64_kernel<5><<<blocks, threads>>>(d, clk, a, b, iters); break;
    case 6: fp64_kernel<6><<<blocks, threads>>>(d, clk, a, b, iters); break;
    case 7: fp64_kernel<7><<<blocks, threads>>>(d, clk, a, b, iters); break;
    case 8: fp64_kernel<8><<<blocks, threads>>>(d, clk, a, b, iters); break;
    default: fp64_kernel<9><<<blocks, threads>>>(d, clk, a, b, iters); break;
    }
}

template <typename F>
cudaError_t run_max(F launch, unsigned long long* host_out)
{
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        launch(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e;
}

}  // namespace

extern "C" {

int cgks_diag_exp_neg_maxulp(int n, unsigned long long* maxulp)
{
    if (n <= 0 || !maxulp) return (int)cudaErrorInvalidValue;
    return (int)run_max([n](unsigned long long* d) { exp_kernel<<<(n + 255) / 256, 256>>>(d, n); }, maxulp);
}

int cgks_diag_rcp_maxulp(int n, unsigned long long* maxulp)
{
    if (n <= 0 || !maxulp) return (int)cudaErrorInvalidValue;
    return (int)run_max([n](unsigned long long* d) { rcp_kernel<<<(n + 255) / 256, 256>>>(d, n); }, maxulp);
}

int cgks_diag_erfc_maxrel(int n, double* maxrel)
{
    if (n <= 0 || !maxrel) return (int)cudaErrorInvalidValue;
    unsigned long long bits = 0;
    cudaError_t e = run_max([n](unsigned long long* d) { erfc_kernel<<<(n + 255) / 256, 256>>>(d, n); }, &bits);
    *maxrel = __builtin_bit_cast(double, bits);
    return (int)e;
}

// Throughput of FP64 operation `op` (numbered as for fp64_kernel): out[0] G
// operations per second, out[1] per SM and cycle, out[2] the SM clock in MHz
// during the loop (one warm-up launch, then one timed launch of 8 CTAs of 256
// threads per SM).
int cgks_diag_fp64_rate(int op, int iters, double out[3])
{
    if (op < 0 || op > 9 || iters <= 0 || !out) return (int)cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int blocks = 8 * nsm, threads = 256;
    double* d = nullptr;
    unsigned long long* clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&d, (size_t)blocks * threads * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&clk, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    unsigned long long h[4] = {};
    if (e == cudaSuccess) {
        launch_fp64(op, blocks, threads, d, clk, 0.99999, 1e-3, iters);
        cudaEventRecord(e0);
        launch_fp64(op, blocks, threads, d, clk, 0.99999, 1e-3, iters);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
        const double ops = (double)blocks * threads * kChains * (double)iters;
        const double mhz = 1e3 * (double)(h[1] - h[0]) / (double)(h[3] - h[2]);
        out[0] = ops / (ms * 1e6);
        out[1] = ops / (ms * 1e-3) / (nsm * mhz * 1e6);
        out[2] = mhz;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    cudaFree(clk);
    return (int)e;
}

}  // extern "C"
