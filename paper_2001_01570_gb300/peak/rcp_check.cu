// The kernels' reciprocal (RegK::rcp in csrc/cgks_device.cuh): the hardware
// approximation rcp.approx.ftz.f64 refined by two Newton-Raphson steps
// y <- y + y (1 - x y).  This program checks it against CUDA's correctly
// rounded __drcp_rn on 4.2 million arguments (every mantissa pattern of a
// stride through [1, 2), scaled by 1e-150 and 1e+150, both signs) and times
// both in a throughput loop.  Prints the largest difference in units in the
// last place and the rates.
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ double rcp_nr(double x, double one)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, one);
    y = fma(y, e, y);
    e = fma(-x, y, one);
    return fma(y, e, y);
}

__global__ void check(unsigned long long* maxulp, int n)
{
    __shared__ double s_one;
    if (threadIdx.x == 0) s_one = 1.0;
    __syncthreads();
    const double one = *(volatile double*)&s_one;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long mant = ((unsigned long long)i * 0x0000001000000001ULL) & 0x000FFFFFFFFFFFFFULL;
    double x = __longlong_as_double((long long)(0x3FF0000000000000ULL | mant));
    x *= (i & 1) ? 1e150 : 1e-150;
    if (i & 2) x = -x;
    long long d = __double_as_longlong(rcp_nr(x, one)) - __double_as_longlong(__drcp_rn(x));
    if (d < 0) d = -d;
    atomicMax(maxulp, (unsigned long long)d);
}

template <int NR>
__global__ void rate(double* out, double a, int iters)
{
    __shared__ double s_one;
    if (threadIdx.x == 0) s_one = 1.0;
    __syncthreads();
    const double one = *(volatile double*)&s_one;
    double x[4];
    for (int c = 0; c < 4; ++c) x[c] = 1.0 + threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = fma(NR ? rcp_nr(x[c], one) : __drcp_rn(x[c]), a, one);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] + x[1] + x[2] + x[3];
}

int main()
{
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    const int n = 1 << 22, blocks = nsm * 4, threads = 256, iters = 1024;
    unsigned long long* m;
    double* d;
    cudaMalloc(&m, sizeof(unsigned long long));
    cudaMalloc(&d, (size_t)blocks * threads * sizeof(double));
    cudaMemset(m, 0, sizeof(unsigned long long));
    check<<<(n + 255) / 256, 256>>>(m, n);
    unsigned long long h = 0;
    cudaMemcpy(&h, m, sizeof(h), cudaMemcpyDeviceToHost);
    printf("rcp.approx + 2 Newton steps vs __drcp_rn over %d arguments: max difference %llu ulp (%s)\n", n, h,
           cudaGetErrorString(cudaGetLastError()));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int nr = 0; nr < 2; ++nr) {
        float ms;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0);
            if (nr) rate<1><<<blocks, threads>>>(d, 0.37, iters);
            else rate<0><<<blocks, threads>>>(d, 0.37, iters);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        printf("%-28s %10.2f G reciprocals/s (%s)\n", nr ? "rcp.approx + 2 Newton steps" : "__drcp_rn",
               (double)blocks * threads * 4.0 * iters / (ms * 1e6), cudaGetErrorString(cudaGetLastError()));
    }
    cudaFree(m);
    cudaFree(d);
    return 0;
}
