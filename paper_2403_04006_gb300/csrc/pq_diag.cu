// pq_diag.cu -- host-side runs of device helpers, for tests without a GPU.
#include "../../include/pq.h"
#include "pq_device.cuh"

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
