// lgt_diag.cu -- measurement helpers: peak FP64 FMA throughput of the device,
// from 16 independent dependent-FMA chains per thread on a full-device grid.
#include "lgt_internal.h"

namespace lgt {

__global__ void __launch_bounds__(256) fp64_fma_kernel(double* out, double b, double c, int iters) {
    double a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = 1e-9 * threadIdx.x + k;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    if (s == 123456.789) out[0] = s;  // keeps the chains alive
}

cudaError_t fp64_peak_kernel_run(double* flops, double* seconds) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    double* out = nullptr;
    if ((e = cudaMalloc(&out, sizeof(double))) != cudaSuccess) return e;
    const int blocks = sms * 8, threads = 256, iters = 4096;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    fp64_fma_kernel<<<blocks, threads>>>(out, 0.9999999, 1e-7, iters);  // warm-up
    cudaEventRecord(a);
    const int reps = 3;
    for (int r = 0; r < reps; ++r) fp64_fma_kernel<<<blocks, threads>>>(out, 0.9999999, 1e-7, iters);
    cudaEventRecord(b);
    e = cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    *seconds = ms * 1e-3;
    *flops = 2.0 * 16.0 * iters * (double)blocks * threads * reps / (*seconds);
    return cudaGetLastError();
}

}  // namespace lgt
