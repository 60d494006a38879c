// pq_diag.cu -- host-side runs of device helpers, for tests without a GPU.
#include <algorithm>
#include <cmath>

#include "../../include/pq.h"
#include "pq_device.cuh"
#include "pq_fixsum.cuh"

extern "C" int pq_gray_walk(const int32_t* radix, int32_t ndig, int64_t steps, int32_t* digit,
                            int32_t* dir)
{
    if (!radix || ndig < 0 || ndig > pqi::kMaxLowDigits || steps < 0 ||
        (steps > 0 && (!digit || !dir)))
        return PQ_ERR_ARG;
    pqi::LowWalk w;
    w.v = 0;
    w.g = 0;
    w.dir = 0;
    w.radm1 = 0;
    w.topp = 0;
    int64_t total = 1;
    for (int d = 0; d < ndig; ++d) {
        if (radix[d] < 2 || radix[d] > pqi::kMaxLowRadix)
            return PQ_ERR_ARG;
        w.radm1 |= uint64_t(radix[d] - 1) << (4 * d);
        total *= radix[d];
    }
    if (steps > total - 1)
        return PQ_ERR_ARG;  // the walk covers exactly total codes
    for (int64_t s = 0; s < steps; ++s) {
        int up;
        digit[s] = pqi::low_step(w, up);
        dir[s] = up;
    }
    return PQ_OK;
}

// The forward kernels' exact warp sum, run on the host: the same conversion,
// the same 26-bit limbs added as 32-bit words (as redux.sync adds them) and
// the same conversion back, over n <= 32 lanes.
extern "C" int pq_fixsum_host(const double* hi, const double* lo, int32_t n, double* out)
{
    if (n < 0 || n > 32 || !out || (n > 0 && (!hi || !lo)))
        return PQ_ERR_ARG;
    int emax = 1;
    for (int q = 0; q < n; ++q) {
        if (!std::isfinite(hi[q]) || !std::isfinite(lo[q]))
            return PQ_ERR_ARG;
        emax = std::max(emax, std::max(pqi::fix_exp(hi[q]), pqi::fix_exp(lo[q])));
    }
    uint32_t sum[4] = {0, 0, 0, 0};
    int32_t top = 0;
    for (int q = 0; q < n; ++q) {
        uint32_t limb[4];
        int32_t t;
        pqi::fix_limbs(pqi::fix_of(hi[q], emax) + pqi::fix_of(lo[q], emax), limb, t);
        for (int w = 0; w < 4; ++w)
            sum[w] += limb[w];
        top += t;
    }
    pqi::fix_to_dd(pqi::fix_from_limbs(sum, top), emax, out[0], out[1]);
    return PQ_OK;
}

// The same sum on the device, by one warp: lane q adds hi[q] + lo[q] (zero
// beyond n) and writes its copy of the result to out[2q], out[2q + 1].
__global__ void fixsum_probe_kernel(const double* hi, const double* lo, int n, double* out)
{
    const int lane = threadIdx.x;
    const double h = lane < n ? hi[lane] : 0.0;
    const double l = lane < n ? lo[lane] : 0.0;
    double sh, sl;
    pqi::warp_fix_sum(h, l, sh, sl);
    out[2 * lane] = sh;
    out[2 * lane + 1] = sl;
}

extern "C" int pq_fixsum_device(const double* hi, const double* lo, int32_t n, double* out,
                                void* stream)
{
    if (n < 0 || n > 32 || !out || (n > 0 && (!hi || !lo)))
        return PQ_ERR_ARG;
    fixsum_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(hi, lo, n, out);
    return cudaGetLastError() == cudaSuccess ? PQ_OK : PQ_ERR_CUDA;
}
