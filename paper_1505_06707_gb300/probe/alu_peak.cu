// FMA throughput probe: the FP32 and FP64 arithmetic rates of the device,
// measured the way the step kernels use them (independent dependency chains
// of fused multiply-adds per thread, every SM filled).  It corroborates the
// ALU peaks that the benchmark derives from unit counts and clocks; it is not
// part of the method.
//
//   int alu_fma_rate(int fp64, int iters, double* flops_per_s, double* ms)
//
// Launches 8 x (SM count) CTAs of 256 threads; each thread runs 8 chains of
// `iters` FMAs (2 flops each).  Returns 0, or the CUDA error code.
#include <cuda_runtime.h>

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T b, T c) {
    T a0 = (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
    T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a0 = a0 * b + c; a1 = a1 * b + c; a2 = a2 * b + c; a3 = a3 * b + c;
            a4 = a4 * b + c; a5 = a5 * b + c; a6 = a6 * b + c; a7 = a7 * b + c;
        }
    }
    const T s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
    if (s == (T)-12345.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <typename T>
int run(int iters, double* flops, double* ms_out) {
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int blocks = 8 * nsm, threads = 256;
    T* out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(T) * blocks * threads)) != cudaSuccess) return (int)e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T b = (T)0.999999, c = (T)1e-7;
    fma_chains<T><<<blocks, threads>>>(out, iters / 8, b, c);     // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) fma_chains<T><<<blocks, threads>>>(out, iters, b, c);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return (int)e;
    const double fl = 5.0 * 2.0 * 8.0 * 4.0 * (double)iters * blocks * threads;
    *flops = fl / (ms * 1e-3);
    *ms_out = ms / 5.0;
    return 0;
}

}  // namespace

extern "C" int alu_fma_rate(int fp64, int iters, double* flops_per_s, double* ms) {
    if (!flops_per_s || !ms || iters <= 0) return -1;
    return fp64 ? run<double>(iters, flops_per_s, ms) : run<float>(iters, flops_per_s, ms);
}
