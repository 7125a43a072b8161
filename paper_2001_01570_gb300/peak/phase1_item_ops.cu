// FP64 operation count of one phase-1 item of the stage kernels (one variable of
// one face-row record): the linear reconstruction alone (outer rows) and with the
// WENO-Z pair (inner rows), with the same device functions and scalings as the
// stage kernel, on random data.  Run under ncu with the FP64 op counters: one
// launch per kind, 65536 items each.
#include "../csrc/cgks_device.cuh"
#include <cstdio>
#include <vector>
#include <random>
using namespace cgks;

__global__ void probe(const double* __restrict__ in, double* __restrict__ out, int n, int inner, double h, double ih, double eps)
{
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= n) return;
    double Q[4], S[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) { Q[c] = in[c * n + it]; S[c] = h * in[(4 + c) * n + it]; }
    double v, hvx, h2vxx;
    linear_recon(Q[0], Q[1], Q[2], Q[3], S[0], S[1], S[2], S[3], v, hvx, h2vxx);
    out[0 * n + it] = v;
    out[1 * n + it] = hvx * ih;
    out[2 * n + it] = h2vxx * ih * ih;
    if (inner) {
        double vl, sl, vr, sr;
        weno_pair(Q[0], Q[1], Q[2], Q[3], S[0], S[1], S[2], S[3], eps, vl, sl, vr, sr);
        out[3 * n + it] = vl; out[4 * n + it] = vr; out[5 * n + it] = sl * ih; out[6 * n + it] = sr * ih;
    }
}

int main()
{
    const int n = 1 << 16;
    std::vector<double> h_in(8 * (size_t)n);
    std::mt19937_64 g(1);
    std::uniform_real_distribution<double> U(0.5, 1.5);
    for (auto& x : h_in) x = U(g);
    double *d_in, *d_out;
    cudaMalloc(&d_in, 8 * (size_t)n * sizeof(double));
    cudaMalloc(&d_out, 7 * (size_t)n * sizeof(double));
    cudaMemcpy(d_in, h_in.data(), 8 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
    for (int inner = 0; inner < 2; ++inner) probe<<<n / 256, 256>>>(d_in, d_out, n, inner, 0.01, 100.0, 1e-6);
    cudaError_t e = cudaDeviceSynchronize();
    printf("n=%d status=%s\n", n, cudaGetErrorString(e));
    cudaFree(d_in); cudaFree(d_out);
    return e == cudaSuccess ? 0 : 1;
}
