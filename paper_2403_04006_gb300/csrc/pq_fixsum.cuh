// pq_fixsum.cuh -- exact sums of double-double values over a warp in integer
// arithmetic, for the forward kernels' lane reduction and task combination.
//
// Every value x = +-M 2^(e - 1075) (M the 53-bit significand, e the biased
// exponent) is an integer multiple of 2^(E - 1075 - kFixFrac), where E is the
// largest exponent among the values summed: it becomes the 128-bit integer
// +-M 2^(e - E + kFixFrac).  Bits below the unit are dropped (truncated
// towards zero), an error below 2^-116 of the largest value, far below the
// double-double rounding (2^-106) it replaces.  With kFixFrac = 64 a value
// takes at most 53 + 64 + 1 bits and a warp's 64 values (hi and lo of 32
// lanes) at most 124, inside a signed 128-bit integer.  The warp adds five
// 26-bit limbs of each lane's integer with redux.sync (sums below 2^31, no
// carry is lost) and recombines them, so the sum is exact and independent of
// the order; the result goes back to a double-double by truncating to 53 and
// 53 more bits.  Integer, shift and redux instructions only: on GB300 the FP64
// pipe is the walk's bottleneck, and the double-double tree this replaces took
// 56 FP64 operations per lane and task.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

namespace pqi {

constexpr int kFixFrac = 64;  // fraction bits below the largest value's last significand bit

typedef __int128 fix128;
typedef unsigned __int128 ufix128;

__host__ __device__ __forceinline__ uint64_t fix_bits(double x)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    std::memcpy(&b, &x, sizeof(b));
    return b;
#endif
}

__host__ __device__ __forceinline__ double fix_double(uint64_t b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double x;
    std::memcpy(&x, &b, sizeof(x));
    return x;
#endif
}

// Biased exponent of x as the summation sees it (subnormals and zero: 1).
__host__ __device__ __forceinline__ int fix_exp(double x)
{
    const uint64_t b = fix_bits(x);
    const int e = (int)((b >> 52) & 0x7ff);
    return e == 0 ? 1 : e;
}

// x as an integer in units of 2^(emax - 1075 - kFixFrac); emax >= fix_exp(x).
__host__ __device__ __forceinline__ fix128 fix_of(double x, int emax)
{
    const uint64_t b = fix_bits(x);
    const int e = (int)((b >> 52) & 0x7ff);
    uint64_t m = b & 0xfffffffffffffull;
    if (e != 0)
        m |= 0x10000000000000ull;
    const int s = (e == 0 ? 1 : e) - emax + kFixFrac;  // <= kFixFrac
    ufix128 u;
    if (s >= 0)
        u = (ufix128)m << s;
    else
        u = (s > -64) ? (ufix128)(m >> (-s)) : (ufix128)0;
    const fix128 v = (fix128)u;
    return (b >> 63) ? -v : v;
}

// Five limbs of 26 bits (the last signed) whose weighted sum is v.
__host__ __device__ __forceinline__ void fix_limbs(fix128 v, uint32_t (&lo)[4], int32_t& top)
{
    const ufix128 u = (ufix128)v;
    lo[0] = (uint32_t)(u & 0x3ffffff);
    lo[1] = (uint32_t)((u >> 26) & 0x3ffffff);
    lo[2] = (uint32_t)((u >> 52) & 0x3ffffff);
    lo[3] = (uint32_t)((u >> 78) & 0x3ffffff);
    top = (int32_t)(v >> 104);  // arithmetic shift: bits 104 .. 127 with the sign
}

__host__ __device__ __forceinline__ fix128 fix_from_limbs(const uint32_t (&lo)[4], int32_t top)
{
    fix128 v = (fix128)top;
    v = (v << 26) + (fix128)lo[3];
    v = (v << 26) + (fix128)lo[2];
    v = (v << 26) + (fix128)lo[1];
    v = (v << 26) + (fix128)lo[0];
    return v;
}

// Index of the highest set bit of u != 0.
__host__ __device__ __forceinline__ int fix_msb(ufix128 u)
{
    const uint64_t h = (uint64_t)(u >> 64), l = (uint64_t)u;
#ifdef __CUDA_ARCH__
    return h ? 127 - __clzll((long long)h) : 63 - __clzll((long long)l);
#else
    return h ? 127 - __builtin_clzll(h) : 63 - __builtin_clzll(l);
#endif
}

// The double (-1)^neg m 2^(f - 1075) for 2^52 <= m < 2^53 and f in
// [-600, 2646], built from its bits; outside the normal exponents it is built
// 600 binades nearer and scaled by an exact power of two (one rounding, into
// the subnormals or to infinity).
__host__ __device__ __forceinline__ double fix_make_double(bool neg, uint64_t m, int f)
{
    const int adj = f < 1 ? 600 : (f > 2046 ? -600 : 0);
    const uint64_t b =
        ((uint64_t)neg << 63) | ((uint64_t)(f + adj) << 52) | (m & 0xfffffffffffffull);
    const double d = fix_double(b);
    if (adj == 0)
        return d;
    return adj > 0 ? d * 0x1p-600 : d * 0x1p600;
}

// v (units 2^(emax - 1075 - kFixFrac)) as hi + lo: hi its leading 53 bits,
// lo the leading 53 bits of the rest (both truncated, same sign).
__host__ __device__ __forceinline__ void fix_to_dd(fix128 v, int emax, double& hi, double& lo)
{
    hi = lo = 0.0;
    if (v == 0)
        return;
    const bool neg = v < 0;
    ufix128 u = neg ? (ufix128)(-v) : (ufix128)v;
    const int base = emax - kFixFrac;
    int p = fix_msb(u);
    uint64_t m;
    ufix128 rest = 0;
    if (p >= 52) {
        m = (uint64_t)(u >> (p - 52));
        rest = u - ((ufix128)m << (p - 52));
    } else {
        m = (uint64_t)u << (52 - p);
    }
    hi = fix_make_double(neg, m, p - 52 + base);
    if (rest == 0)
        return;
    p = fix_msb(rest);
    m = p >= 52 ? (uint64_t)(rest >> (p - 52)) : (uint64_t)rest << (52 - p);
    lo = fix_make_double(neg, m, p - 52 + base);
}

#ifdef __CUDACC__
// Exact sum of hi + lo over the 32 lanes of a warp (all lanes call it); every
// lane receives the sum as a double-double.  A non-finite value anywhere in
// the warp (an overflowing input) is summed in plain FP64 instead, so that
// infinities and NaNs reach the output as they would through FP64 addition.
__device__ __forceinline__ void warp_fix_sum(double hi, double lo, double& shi, double& slo)
{
    const bool nonfinite = ((fix_bits(hi) >> 52) & 0x7ff) == 0x7ff ||
                           ((fix_bits(lo) >> 52) & 0x7ff) == 0x7ff;
    if (__any_sync(0xffffffffu, nonfinite)) {
        double t = hi + lo;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            t += __shfl_xor_sync(0xffffffffu, t, off);
        shi = t;
        slo = 0.0;
        return;
    }
    const int e = max(fix_exp(hi), fix_exp(lo));
    const int emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
    const fix128 v = fix_of(hi, emax) + fix_of(lo, emax);
    uint32_t limb[4];
    int32_t top;
    fix_limbs(v, limb, top);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        limb[q] = __reduce_add_sync(0xffffffffu, limb[q]);
    top = __reduce_add_sync(0xffffffffu, top);
    fix_to_dd(fix_from_limbs(limb, top), emax, shi, slo);
}
#endif

}  // namespace pqi
