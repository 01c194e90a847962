// FMA-throughput microbenchmark: the denominators of the ALU rooflines
// (FP32 and FP64 fused multiply-add rates of the device it runs on).
#include <cuda_runtime.h>

#include "../../include/jk.h"

namespace {
template <typename T>
__global__ void fma_chain(T *out, T a, T b, int iters)
{
    // eight independent chains per thread keep the FMA pipe full
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = x0 * a + b;
            x1 = x1 * a + b;
            x2 = x2 * a + b;
            x3 = x3 * a + b;
            x4 = x4 * a + b;
            x5 = x5 * a + b;
            x6 = x6 * a + b;
            x7 = x7 * a + b;
        }
    }
    T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
    if (s == T(-1.2345)) out[threadIdx.x] = s;  // keeps the chains live; never true
}

template <typename T>
int run(double *tflops)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    T *out = nullptr;
    if (cudaMalloc(&out, 1024 * sizeof(T)) != cudaSuccess) return JK_ERR_OOM;
    const int blocks = sms * 8, threads = 256, iters = 2048;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_chain<T><<<blocks, threads>>>(out, T(0.999999), T(1e-7), 64);
    cudaEventRecord(e0);
    fma_chain<T><<<blocks, threads>>>(out, T(0.999999), T(1e-7), iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return cudaGetLastError() == cudaSuccess ? JK_OK : JK_ERR_CUDA;
}
}  // namespace

extern "C" int jk_microbench_fma(int fp64, double *tflops)
{
    if (!tflops) return JK_ERR_INVALID;
    return fp64 ? run<double>(tflops) : run<float>(tflops);
}
