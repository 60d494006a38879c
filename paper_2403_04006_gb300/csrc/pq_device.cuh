// pq_device.cuh -- device helpers shared by the forward and backward kernels:
// double-double accumulation, complex FP64 products, the
// warp-uniform mixed-radix Gray walk and the per-task shared-memory staging.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pq_internal.h"

namespace pqi {

// ---------------------------------------------------------------- dd numbers
struct dd2 {  // complex double-double: (hi, lo) for the real and imaginary parts
    double rh, rl, ih, il;
};

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e)
{
    s = __dadd_rn(a, b);
    e = __dsub_rn(b, __dsub_rn(s, a));
}

// TwoSum with the operands ordered by magnitude first: comparing the bit
// patterns without their sign bits as integers orders finite doubles by
// absolute value, on the integer pipe; once |big| >= |small|, Dekker's
// Fast2Sum is exact with three FP64 operations instead of TwoSum's six.
__device__ __forceinline__ void two_sum_ord(double a, double b, double& s, double& e)
{
    const unsigned long long ma = (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
    const unsigned long long mb = (unsigned long long)__double_as_longlong(b) & 0x7fffffffffffffffull;
    const bool ge = ma >= mb;
    const double big = ge ? a : b;
    const double small = ge ? b : a;
    s = __dadd_rn(big, small);
    e = __dsub_rn(small, __dsub_rn(s, big));
}

// hi + lo += x (compensated; lo collects the exact rounding errors)
__device__ __forceinline__ void dd_acc(double& hi, double& lo, double x)
{
    double s, e;
    two_sum_ord(hi, x, s, e);
    hi = s;
    lo = __dadd_rn(lo, e);
}

// (ah, al) + (bh, bl), renormalised
__device__ __forceinline__ void dd_add(double& ah, double& al, double bh, double bl)
{
    double s, e, t, f;
    two_sum_ord(ah, bh, s, e);
    two_sum_ord(al, bl, t, f);
    e = __dadd_rn(e, t);
    fast_two_sum(s, e, s, e);
    e = __dadd_rn(e, f);
    fast_two_sum(s, e, ah, al);
}

// (h, l) * w for a double w
__device__ __forceinline__ void dd_mul_d(double& h, double& l, double w)
{
    double p = __dmul_rn(h, w);
    double e = __fma_rn(h, w, -p);
    e = __fma_rn(l, w, e);
    fast_two_sum(p, e, h, l);
}

// ---------------------------------------------------------------- complex FP64
// p * s with two DMUL and two DFMA
__device__ __forceinline__ double2 cmul(double2 p, double2 s)
{
    double2 r;
    r.x = __fma_rn(p.x, s.x, -__dmul_rn(p.y, s.y));
    r.y = __fma_rn(p.x, s.y, __dmul_rn(p.y, s.x));
    return r;
}

// acc += p * s (NEG: acc -= p * s) with four DFMA and no separate product
template <bool NEG>
__device__ __forceinline__ void cfma_acc(double2& acc, double2 p, double2 s)
{
    if (NEG) {
        acc.x = __fma_rn(-p.x, s.x, acc.x);
        acc.x = __fma_rn(p.y, s.y, acc.x);
        acc.y = __fma_rn(-p.x, s.y, acc.y);
        acc.y = __fma_rn(-p.y, s.x, acc.y);
    } else {
        acc.x = __fma_rn(p.x, s.x, acc.x);
        acc.x = __fma_rn(-p.y, s.y, acc.x);
        acc.y = __fma_rn(p.x, s.y, acc.y);
        acc.y = __fma_rn(p.y, s.x, acc.y);
    }
}

// ---------------------------------------------------------------- binomials
// Exact C(top, g) for the small tops of low digits (top <= 14).
__host__ __device__ __forceinline__ uint64_t binom_u64(int top, int g)
{
    uint64_t r = 1;
    for (int i = 1; i <= g; ++i)
        r = r * (uint64_t)(top - g + i) / (uint64_t)i;
    return r;
}

// C(top, g) for top, g < 16 (the low digits), Pascal's triangle built at
// compile time.  On the device the walk reads it from constant memory with a
// warp-uniform index instead of dividing 64-bit integers at every step.
struct BinomTable16 {
    uint16_t v[16][16];
};
constexpr BinomTable16 make_binom16()
{
    BinomTable16 t{};
    for (int n = 0; n < 16; ++n) {
        t.v[n][0] = 1;
        for (int g = 1; g <= n; ++g)
            t.v[n][g] = (uint16_t)(t.v[n - 1][g - 1] + (g < n ? t.v[n - 1][g] : 0));
    }
    return t;
}
static __constant__ BinomTable16 c_binom16 = make_binom16();

__host__ __device__ __forceinline__ uint64_t binom_small(int top, int g)
{
#ifdef __CUDA_ARCH__
    return c_binom16.v[top][g];
#else
    return binom_u64(top, g);
#endif
}

// C(top, g) in double (exact while it stays below 2^53).
__device__ __forceinline__ double binom_f64(int top, int g)
{
    double r = 1.0;
    for (int i = 1; i <= g; ++i)
        r = r * (double)(top - g + i) / (double)i;
    return r;
}

// ---------------------------------------------------------------- metadata views
struct MetaView {
    const int32_t* ridx;
    const int32_t* cidx;
    const int32_t* rmul;
    const int32_t* cmul;
    const int32_t* drow;
    const int32_t* drad;
    const int32_t* dtop;
    const int32_t* ecnt;
};

__device__ __forceinline__ MetaView meta_view(const int32_t* pool, const PermDesc& D)
{
    MetaView m;
    m.ridx = pool + D.meta;
    m.cidx = m.ridx + D.k;
    m.rmul = m.cidx + D.l;
    m.cmul = m.rmul + D.k;
    m.drow = m.cmul + D.l;
    m.drad = m.drow + D.ndig;
    m.dtop = m.drad + D.ndig;
    m.ecnt = m.dtop + D.ndig;
    return m;
}

// ---------------------------------------------------------------- task guards
// The checks a task passes before any of its data is used (the error record
// of pq_internal.h): the permanent it names, its part, the descriptor's sizes
// against the launch's shared-memory layout (kmax rows, ld columns, jmax low
// digits), the digit counts against the walk's limits, and the descriptor's
// indices into the metadata pool, the partial slots and the outputs.
// nslots < 0: the caller indexes its own slots (no slot check).  Returns 0 or
// the error code.  The guard reads the descriptor through the L2 path into a
// copy of its own, so the task's code loads what it needs afterwards and no
// descriptor stays live in registers across the task.
__device__ __forceinline__ int32_t task_guard(const Task& t, const PermDesc* desc, int64_t nperm,
                                           int64_t nmeta, int64_t nslots, int kmax, int ld,
                                           int jmax)
{
    if (t.perm < 0 || (int64_t)t.perm >= nperm)
        return kErrTaskPerm;
    PermDesc D = desc[t.perm];
    if (D.k < 0 || D.l < 0 || D.k > kmax || D.l > ld)
        return kErrDescLayout;
    if (D.J < 0 || D.J > jmax || D.J > kMaxLowDigits || D.ndig < D.J || D.ndig > 64)
        return kErrDescDigits;
    if (D.meta < 0 || (int64_t)D.meta + meta_size(D.k, D.l, D.ndig) > nmeta || D.out < 0 ||
        (int64_t)D.out >= nperm || D.ntasks < 1)
        return kErrDescIndex;
    if (nslots >= 0 && (D.slot0 < 0 || (int64_t)D.slot0 + D.ntasks > nslots))
        return kErrDescIndex;
    const int64_t q = (int64_t)t.part - D.part0;
    if (q < 0 || q >= D.ntasks)
        return kErrTaskPart;
    return 0;
}

// Keep the first failure: the code, then the task's index in the list.
__device__ __forceinline__ void record_error(int32_t* err, int32_t code, int64_t ti)
{
    if (atomicCAS(err, 0, code) == 0)
        atomicExch(err + 1, (int32_t)ti);
}

// Warp-uniform state of the walk over the J low digits of a chunk.  Digit d
// occupies bits [4d, 4d+4) of v (odometer value) and g (Gray value).
struct LowWalk {
    uint64_t v, g;      // packed digits
    uint32_t dir;       // bit d set: digit d currently moves down
    uint64_t radm1;     // packed radix - 1 of each low digit
    uint64_t topp;      // packed binomial tops of the low digits
};

// Advance one Gray step; returns the changed digit and sets up = +1/-1.
__host__ __device__ __forceinline__ int low_step(LowWalk& w, int& up)
{
    int d = 0;
    while (((w.v >> (4 * d)) & 15u) == ((w.radm1 >> (4 * d)) & 15u)) {
        w.v &= ~(uint64_t(15) << (4 * d));
        w.dir ^= (1u << d);
        ++d;
    }
    w.v += uint64_t(1) << (4 * d);
    if ((w.dir >> d) & 1u) {
        up = -1;
        w.g -= uint64_t(1) << (4 * d);
    } else {
        up = 1;
        w.g += uint64_t(1) << (4 * d);
    }
    return d;
}

// prod_{d<J} C(top_d, g_d) for the current low Gray value
__host__ __device__ __forceinline__ uint64_t low_weight(const LowWalk& w, int J)
{
    uint64_t r = 1;
    for (int d = 0; d < J; ++d) {
        int g = int((w.g >> (4 * d)) & 15u);
        int top = int((w.topp >> (4 * d)) & 15u);
        if (g)
            r *= binom_small(top, g);
    }
    return r;
}

}  // namespace pqi
