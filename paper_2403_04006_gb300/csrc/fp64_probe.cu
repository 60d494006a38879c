// fp64_probe.cu -- measured FP64 throughput of the chip (roofline denominator).
//
// Every thread runs eight independent DFMA chains x <- x * b + c; b = 1 - 2^-20
// and c = 2^-30 keep the values bounded and normal.  FLOPs = 2 per DFMA.  The
// grid fills every SM several times over so the FP64 pipes, not latency, set
// the rate.
//
// The sweep (pq_probe_fp64_sweep) runs the same kind of chains for DFMA, DADD
// or DMUL at a chosen number of resident warps per SM and independent chains
// per thread: it shows how many warps saturate the FP64 pipe and whether
// dependency latency matters, which decides how the permanent kernels are
// laid out.
#include <cuda_runtime.h>

#include "../../include/pq.h"
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

template <int CH, int OP>
__global__ void fp64_sweep_kernel(int64_t iters, double* sink)
{
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c)
        x[c] = 1.0 + threadIdx.x * 0x1p-20 + c * 0x1p-7;
    const double b = 1.0 - 0x1p-20, cst = 0x1p-30;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                if (OP == 0)
                    x[c] = __fma_rn(x[c], b, cst);
                else if (OP == 1)
                    x[c] = __dadd_rn(x[c], cst);
                else
                    x[c] = __dmul_rn(x[c], b);
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
        s += x[c];
    if (s == -1.0)  // never true; keeps the chains alive
        sink[threadIdx.x] = s;
}

template <int CH, int OP>
static cudaError_t sweep_launch(unsigned blocks, unsigned threads, int64_t iters, cudaStream_t st)
{
    fp64_sweep_kernel<CH, OP><<<blocks, threads, 0, st>>>(iters, nullptr);
    return cudaGetLastError();
}

template <int OP>
static cudaError_t sweep_dispatch(int chains, unsigned blocks, unsigned threads, int64_t iters,
                                  cudaStream_t st)
{
    switch (chains) {
    case 1: return sweep_launch<1, OP>(blocks, threads, iters, st);
    case 2: return sweep_launch<2, OP>(blocks, threads, iters, st);
    case 4: return sweep_launch<4, OP>(blocks, threads, iters, st);
    default: return sweep_launch<8, OP>(blocks, threads, iters, st);
    }
}

// One block of warps_per_sm warps per SM (two blocks of half as many above
// 32 warps); lane operations per second per SM.
cudaError_t fp64_sweep(int op, int warps_per_sm, int chains, int64_t iters, double* rate,
                       cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return e;
    unsigned threads = 32u * (unsigned)warps_per_sm, blocks = (unsigned)sms;
    if (threads > 1024) {
        blocks = (unsigned)sms * (threads / 1024);
        threads = 1024;
    }
    auto run = [&](int64_t it) {
        return op == 0 ? sweep_dispatch<0>(chains, blocks, threads, it, st)
                       : op == 1 ? sweep_dispatch<1>(chains, blocks, threads, it, st)
                                 : sweep_dispatch<2>(chains, blocks, threads, it, st);
    };
    if ((e = run(iters / 8 + 1)) != cudaSuccess)  // warm-up
        return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    e = run(iters);
    cudaEventRecord(b, st);
    if (e == cudaSuccess)
        e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess)
        return e;
    const double ops = 4.0 * chains * (double)iters * threads * blocks;
    *rate = ops / ((double)ms * 1e-3) / sms;
    return cudaSuccess;
}

}  // namespace pqi

extern "C" int pq_probe_fp64_sweep(int32_t op, int32_t warps_per_sm, int32_t chains, int64_t iters,
                                   double* lane_ops_per_sm_per_s, void* stream)
{
    if (!lane_ops_per_sm_per_s || iters <= 0 || op < 0 || op > 2 || warps_per_sm < 1 ||
        warps_per_sm > 64 || (chains != 1 && chains != 2 && chains != 4 && chains != 8))
        return pqi::report(PQ_ERR_ARG, "op in 0..2, warps_per_sm in 1..64, chains 1/2/4/8");
    const cudaError_t e = pqi::fp64_sweep(op, warps_per_sm, chains, iters, lane_ops_per_sm_per_s,
                                          (cudaStream_t)stream);
    return e == cudaSuccess ? PQ_OK : pqi::report(PQ_ERR_CUDA, cudaGetErrorString(e));
}
