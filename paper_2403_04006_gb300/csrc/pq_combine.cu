// pq_combine.cu -- the exchange step of a permanent batch split over ranks:
// the shards' unscaled double-double partial sums of the Glynn terms
// (pq_permanent_partials) are added in shard order and scaled by
// 2^{-(n-1)}, the normalisation of the BB/FG formula (Sec. 4.2).
//
// The same arithmetic runs on the device (one thread per permanent) and on
// the host (for partials gathered into host memory), so both give the same
// bits: additions only (TwoSum of the high parts, the error and both low
// parts gathered into the low part, as the kernels' lane reductions do) and
// an exact power-of-two scaling.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/pq.h"
#include "pq_kernels.h"

namespace pqi {

__host__ __device__ inline void combine_two_sum(double a, double b, double& s, double& e)
{
    s = a + b;
    const double bv = s - a;
    const double av = s - bv;
    e = (a - av) + (b - bv);
}

// Permanent p of a batch of `batch`: parts[(r * batch + p) * 4 + {re hi, re lo,
// im hi, im lo}] for shards r = 0 .. R-1.
__host__ __device__ inline double2 combine_one(const double* parts, int R, int64_t batch,
                                               int64_t p, int n)
{
    const double* q = parts + 4 * p;
    double rh = q[0], rl = q[1], ih = q[2], il = q[3];
    for (int r = 1; r < R; ++r) {
        q = parts + ((int64_t)r * batch + p) * 4;
        double s, e;
        combine_two_sum(rh, q[0], s, e);
        rh = s;
        rl = (rl + q[1]) + e;
        combine_two_sum(ih, q[2], s, e);
        ih = s;
        il = (il + q[3]) + e;
    }
    const int sh = n > 0 ? 1 - n : 0;
    return make_double2(scalbn(rh + rl, sh), scalbn(ih + il, sh));
}

__global__ void combine_partials_kernel(const double* parts, int R, int64_t batch,
                                        const int32_t* n, double2* out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < batch;
         p += (int64_t)gridDim.x * blockDim.x)
        out[p] = combine_one(parts, R, batch, p, n[p]);
}

}  // namespace pqi

using namespace pqi;

extern "C" int pq_combine_partials(const double* parts, int32_t nshards, int64_t batch,
                                   const int32_t* n, pq_c128* out, void* stream)
{
    if (batch < 0 || nshards < 1)
        return report(PQ_ERR_ARG, "batch < 0 or fewer than one shard");
    if (batch == 0)
        return PQ_OK;
    if (!parts || !n || !out)
        return report(PQ_ERR_ARG, "null argument");
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return report(PQ_ERR_CUDA, "no CUDA device");
    const int threads = 256;
    int64_t blocks = (batch + threads - 1) / threads;
    if (blocks > 8L * sms)
        blocks = 8L * sms;
    combine_partials_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        parts, nshards, batch, n, reinterpret_cast<double2*>(out));
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PQ_OK : report(PQ_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" int pq_combine_partials_host(const double* parts, int32_t nshards, int64_t batch,
                                        const int32_t* n, pq_c128* out)
{
    if (batch < 0 || nshards < 1)
        return report(PQ_ERR_ARG, "batch < 0 or fewer than one shard");
    if (batch == 0)
        return PQ_OK;
    if (!parts || !n || !out)
        return report(PQ_ERR_ARG, "null argument");
    for (int64_t p = 0; p < batch; ++p) {
        if (n[p] < 0 || n[p] > PQ_MAX_N)
            return report(PQ_ERR_ARG, "photon number outside [0, PQ_MAX_N]");
        const double2 v = combine_one(parts, nshards, batch, p, n[p]);
        out[p].re = v.x;
        out[p].im = v.y;
    }
    return PQ_OK;
}
