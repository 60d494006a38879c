// fp64_sweep.cu -- throughput of the GB300 FP64 pipe against warps per SM and
// independent dependency chains per thread, for DFMA, DADD and DMUL.
//
// Prints lane operations per clock per SM (clock = the device's maximum SM
// clock).  Used to decide what bounds the permanent kernels: how many warps
// per SM saturate the FP64 pipe and whether dependency latency matters.
#include <cstdio>

#include <cuda_runtime.h>

template <int CH, int OP>
__global__ void sweep_kernel(long iters, double* sink)
{
    double x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c)
        x[c] = 1.0 + threadIdx.x * 1e-6 + c * 0.01;
    const double b = 1.0 - 0x1p-20, cst = 0x1p-30;
    for (long i = 0; i < iters; ++i) {
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
    double s = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c)
        s += x[c];
    if (s == -1.0)  // never true: keeps the chains alive
        sink[threadIdx.x] = s;
}

template <int CH, int OP>
static double lane_ops_per_sm_per_s(int sms, int warps_per_sm, long iters)
{
    int threads = 32 * warps_per_sm, blocks = sms;
    if (threads > 1024) {
        blocks = sms * (threads / 1024);
        threads = 1024;
    }
    sweep_kernel<CH, OP><<<blocks, threads>>>(iters / 8 + 1, nullptr);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    sweep_kernel<CH, OP><<<blocks, threads>>>(iters, nullptr);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const double ops = 4.0 * CH * (double)iters * threads * blocks;
    return ops / (ms * 1e-3) / sms;
}

template <int OP>
static void row(const char* name, int sms, int w, long it, double hz)
{
    const double r1 = lane_ops_per_sm_per_s<1, OP>(sms, w, it);
    const double r2 = lane_ops_per_sm_per_s<2, OP>(sms, w, it);
    const double r4 = lane_ops_per_sm_per_s<4, OP>(sms, w, it);
    const double r8 = lane_ops_per_sm_per_s<8, OP>(sms, w, it);
    printf("%s warps/SM %2d  lane-ops/clk/SM: ch1 %.3f ch2 %.3f ch4 %.3f ch8 %.3f\n", name, w,
           r1 / hz, r2 / hz, r4 / hz, r8 / hz);
}

int main()
{
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    printf("sms %d max_clock_khz %d\n", sms, clk);
    const long it = 20000;
    const double hz = clk * 1e3;
    const int W[] = {1, 2, 4, 8, 12, 16, 32, 64};
    for (int w : W)
        row<0>("dfma", sms, w, it, hz);
    for (int w : W)
        row<1>("dadd", sms, w, it, hz);
    for (int w : W)
        row<2>("dmul", sms, w, it, hz);
    const cudaError_t e = cudaGetLastError();
    printf("status %s\n", cudaGetErrorString(e));
    return e == cudaSuccess ? 0 : 1;
}
