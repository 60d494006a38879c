// fp64_probe.cu -- measured FP64 throughput of the chip (roofline denominator).
//
// Every thread runs eight independent DFMA chains x <- x * b + c; b = 1 - 2^-20
// and c = 2^-30 keep the values bounded and normal.  FLOPs = 2 per DFMA.  The
// grid fills every SM several times over so the FP64 pipes, not latency, set
// the rate.
#include <cuda_runtime.h>

#include "pq_kernels.h"

namespace pqi {

__global__ void __launch_bounds__(256) fp64_probe_kernel(int64_t iters, double* sink)
{
    const double b = 1.0 - 0x1p-20, c = 0x1p-30;
    double x0 = 1.0 + threadIdx.x * 0x1p-12, x1 = x0 + 0.125, x2 = x0 + 0.25, x3 = x0 + 0.375;
    double x4 = x0 + 0.5, x5 = x0 + 0.625, x6 = x0 + 0.75, x7 = x0 + 0.875;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x0 = __fma_rn(x0, b, c);
            x1 = __fma_rn(x1, b, c);
            x2 = __fma_rn(x2, b, c);
            x3 = __fma_rn(x3, b, c);
            x4 = __fma_rn(x4, b, c);
            x5 = __fma_rn(x5, b, c);
            x6 = __fma_rn(x6, b, c);
            x7 = __fma_rn(x7, b, c);
        }
    }
    double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == -1.0)  // never true; keeps the chains alive
        sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t fp64_probe(int64_t iters, double* flops_per_s, double* ms, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    const int threads = 256, blocks = sms * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    fp64_probe_kernel<<<blocks, threads, 0, st>>>(iters / 16 + 1, nullptr);  // warm-up
    cudaEventRecord(a, st);
    fp64_probe_kernel<<<blocks, threads, 0, st>>>(iters, nullptr);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    float t = 0.0f;
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess)
        return e;
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const double flops = 2.0 * 32.0 * (double)iters * (double)threads * (double)blocks;
    *ms = (double)t;
    *flops_per_s = flops / ((double)t * 1e-3);
    return cudaSuccess;
}

}  // namespace pqi
