// glynn_fwd.cu -- forward kernels: permanents with repeated rows and columns by
// the BB/FG formula over a mixed-radix Gray code (paper Sec. 4.2, "Boson
// Sampling"; Eq. (per_def) for the permanent, Eq. (BS_prob) for the
// probabilities written by the final reduction).
//
// One thread walks one chunk of the Gray code.  On GB300 the FP64 pipe (1.68
// lane operations per clock per SM, saturated by four warps whatever their
// dependency chains) is the only resource the walk loads, so the kernel is
// written to issue exactly the FP64 instructions the method needs and nothing
// else into that pipe:
//   * every lane's column sums S_j = sum_i (r_i - 2 g_i) b_ij live in shared
//     memory, lane-major (one 16-byte complex per lane per column, so a warp
//     access is conflict-free); the loops over columns are plain runtime loops,
//     never unrolled against a bound and never if-converted, so no predicated-
//     off or speculative FP64 instruction takes a pipe slot;
//   * a Gray step changes one row's sign count by +-1 for all lanes at once:
//     S_j += -+2 b_ij, one DFMA per real component, b read as a broadcast;
//   * product columns are sorted by non-increasing multiplicity, so
//     prod_j S_j^{c_j} = prod_m P(n_m) with P(q) = S_0 ... S_{q-1}: l - 1
//     complex products for P(l) plus one per extra prefix, instead of n - 1;
//     the last product is fused into the running sum (four DFMA);
//   * the sign (-1)^step alternates, so pairs of terms are unrolled with the
//     sign folded into the DFMA operands; the binomial weight of the low
//     digits changes only when a digit of radix > 2 moves, so a run of equally
//     weighted terms is summed unweighted and weighted once (two DFMA);
//   * every 32 terms the FP64 running sum is folded into a double-double
//     accumulator with TwoSum.
// A warp task is up to 32 chunks of one permanent (one per lane).  The lanes'
// sums are added exactly, in 128-bit integers (pq_fixsum.cuh), and the tasks
// of one permanent in task order by the warp that finishes last, so results
// do not depend on scheduling.
#include <cuda_runtime.h>

#include "pq_device.cuh"
#include "pq_fixsum.cuh"
#include "pq_kernels.h"

namespace pqi {

// Shared memory of one warp: base matrix (kmax x ld complex), base column sums
// (ld complex), column sums of the 32 lanes (ld x 32 complex), low-digit rows
// (16 ints), extra-factor counts (ld ints).
__host__ __device__ inline int warp_smem_bytes(int kmax, int ld)
{
    int bytes = (kmax * ld + ld + 32 * ld) * 16 + (16 + ld) * 4;
    return (bytes + 15) & ~15;
}

struct WarpSmem {
    double2* M;       // kmax x ld
    double2* base;    // ld
    double2* S;       // ld x 32, S[j * 32 + lane]
    int32_t* lowrow;  // 16
    int32_t* ecnt;    // ld
    int ld;
    __device__ WarpSmem(unsigned char* raw, int kmax, int ld_)
    {
        ld = ld_;
        M = reinterpret_cast<double2*>(raw);
        base = M + kmax * ld;
        S = base + ld;
        lowrow = reinterpret_cast<int32_t*>(S + 32 * ld);
        ecnt = lowrow + 16;
    }
};

// Copy the oriented base matrix of permanent D into shared memory and form
// base_j = sum_i r_i b_ij (all Gray digits at zero).
template <class SM>
__device__ void stage_perm(const ExecArgs& a, const PermDesc& D, const MetaView& mv, SM& sm,
                           int lane)
{
    const int k = D.k, l = D.l;
    for (int e = lane; e < k * l; e += kWarp) {
        const int i = e / l, j = e - i * l;
        const int64_t off = D.src_off + (int64_t)mv.ridx[i] * D.si + (int64_t)mv.cidx[j] * D.sj;
        sm.M[i * sm.ld + j] = a.src[off];
    }
    for (int d = lane; d < D.J; d += kWarp)
        sm.lowrow[d] = mv.drow[d];
    for (int j = lane; j < l; j += kWarp)
        sm.ecnt[j] = mv.ecnt[j];
    __syncwarp();
    for (int j = lane; j < l; j += kWarp) {
        double2 s = make_double2(0.0, 0.0);
        for (int i = 0; i < k; ++i) {
            const double r = (double)mv.rmul[i];
            const double2 b = sm.M[i * sm.ld + j];
            s.x = __fma_rn(r, b.x, s.x);
            s.y = __fma_rn(r, b.y, s.y);
        }
        sm.base[j] = s;
    }
    __syncwarp();
}

// One Glynn term: acc +-= prod_j S_j^{c_j} (S = this lane's column sums,
// stride 32).  unit: every c_j = 1; jf: first column with an extra prefix.
// The low-digit weight is applied by the caller, once per run of terms that
// share it.
template <bool NEG>
__device__ __forceinline__ void glynn_term(const double2* S, int l, bool unit, int jf,
                                           const int32_t* ecnt, double2& acc)
{
    if (unit) {
        if (l == 1) {  // n = 1: the product is S_0 itself
            acc.x = NEG ? __dsub_rn(acc.x, S[0].x) : __dadd_rn(acc.x, S[0].x);
            acc.y = NEG ? __dsub_rn(acc.y, S[0].y) : __dadd_rn(acc.y, S[0].y);
            return;
        }
        double2 p = S[0];
#pragma unroll 1
        for (int j = 1; j < l - 1; ++j)
            p = cmul(p, S[j * 32]);
        cfma_acc<NEG>(acc, p, S[(l - 1) * 32]);
        return;
    }
    // P(q) for q = 1 .. l in `pre`, extra prefixes multiplied into `ex`
    double2 pre = S[0];
#pragma unroll 1
    for (int j = 1; j <= jf; ++j)
        pre = cmul(pre, S[j * 32]);
    double2 ex = pre;
#pragma unroll 1
    for (int e = 1; e < ecnt[jf]; ++e)
        ex = cmul(ex, pre);
#pragma unroll 1
    for (int j = jf + 1; j < l; ++j) {
        pre = cmul(pre, S[j * 32]);
#pragma unroll 1
        for (int e = 0; e < ecnt[j]; ++e)
            ex = cmul(ex, pre);
    }
    cfma_acc<NEG>(acc, pre, ex);
}

// One Gray step of the warp-uniform low walk: every lane's S += -+2 b_row.
// Returns true when the changed digit has radix > 2, i.e. when the low-digit
// weight prod_d C(top_d, g_d) changes (a radix-2 digit has weight C(1, g) = 1).
__device__ __forceinline__ bool glynn_step(LowWalk& wk, const WarpSmem& sm, double2* S, int l)
{
    int up;
    const int d = low_step(wk, up);
    const double2* Mr = sm.M + sm.lowrow[d] * sm.ld;
    const double delta = up > 0 ? -2.0 : 2.0;  // x = r - 2g
#pragma unroll 1
    for (int j = 0; j < l; ++j) {
        const double2 b = Mr[j];
        double2 s = S[j * 32];
        s.x = __fma_rn(delta, b.x, s.x);
        s.y = __fma_rn(delta, b.y, s.y);
        S[j * 32] = s;
    }
    return ((wk.radm1 >> (4 * d)) & 15u) > 1u;
}

// A run of equally weighted terms ends: run += wlow * acc, and the walk's new
// weight becomes wlow.
__device__ __forceinline__ void reweight(const LowWalk& wk, int J, double& wlow, double2& acc,
                                         double2& run)
{
    run.x = __fma_rn(wlow, acc.x, run.x);
    run.y = __fma_rn(wlow, acc.y, run.y);
    acc = make_double2(0.0, 0.0);
    wlow = (double)low_weight(wk, J);
}

// Write per = 2^{-(n-1)} * sum, and |per|^2 * norm; a sharded plan writes
// its unscaled double-double sum instead.
__device__ __forceinline__ void finalize(const ExecArgs& a, const PermDesc& D, dd2 v)
{
    if (a.out_partial) {
        double* o = a.out_partial + 4 * (int64_t)D.out;
        if (D.trivial) {
            o[0] = 1.0;
            o[1] = o[2] = o[3] = 0.0;
        } else {
            o[0] = v.rh;
            o[1] = v.rl;
            o[2] = v.ih;
            o[3] = v.il;
        }
        return;
    }
    double re, im;
    if (D.trivial) {
        re = 1.0;
        im = 0.0;
    } else {
        double h, e;
        fast_two_sum(v.rh, v.rl, h, e);
        re = scalbn(h + e, 1 - D.n);
        fast_two_sum(v.ih, v.il, h, e);
        im = scalbn(h + e, 1 - D.n);
    }
    if (a.out_amp)
        a.out_amp[D.out] = make_double2(re, im);
    if (a.out_prob)
        a.out_prob[D.out] = (re * re + im * im) * D.norm;
}

__device__ void combine_task(const ExecArgs& a, const Task& t, const PermDesc& D, dd2 res, int lane);

// The task's sum: every lane's chunk sum (rh + rl, ih + il) times its
// high-digit weight (-1)^neg whigh_u (zero for a lane without a chunk), added
// over the warp exactly in integer arithmetic (pq_fixsum.cuh); every lane gets
// it.  When no lane's weight is above 1 the weight is a sign, applied to the
// bit patterns, and the double-double product (14 FP64 operations) is skipped.
__device__ __forceinline__ dd2 task_sum(double rh, double rl, double ih, double il,
                                        uint64_t whigh_u, bool neg, bool active)
{
    if (__any_sync(0xffffffffu, active && whigh_u != 1)) {
        double w = active ? (double)whigh_u : 0.0;
        if (neg)
            w = -w;
        fast_two_sum(rh, rl, rh, rl);
        fast_two_sum(ih, il, ih, il);
        dd_mul_d(rh, rl, w);
        dd_mul_d(ih, il, w);
    } else if (!active) {
        rh = rl = ih = il = 0.0;
    } else if (neg) {
        const uint64_t s = 1ull << 63;
        rh = fix_double(fix_bits(rh) ^ s);
        rl = fix_double(fix_bits(rl) ^ s);
        ih = fix_double(fix_bits(ih) ^ s);
        il = fix_double(fix_bits(il) ^ s);
    }
    dd2 res;
    warp_fix_sum(rh, rl, res.rh, res.rl);
    warp_fix_sum(ih, il, res.ih, res.il);
    return res;
}

__device__ void process_task(const ExecArgs& a, const Task& t, WarpSmem& sm, int& staged, int lane)
{
    const PermDesc D = a.desc[t.perm];
    const MetaView mv = meta_view(a.meta, D);
    const int l = D.l, J = D.J, ndig = D.ndig;
    dd2 res = {0.0, 0.0, 0.0, 0.0};

    if (!D.trivial) {
        if (staged != t.perm) {
            __syncwarp();
            stage_perm(a, D, mv, sm, lane);
            staged = t.perm;
        }
        // ---- this lane's chunk: decode the high digits, start the column sums
        const int64_t chunk0 = (int64_t)t.part * kWarp;
        const bool active = chunk0 + lane < D.nchunks;
        int64_t c = active ? (chunk0 + lane) : 0;
        double2* S = sm.S + lane;
#pragma unroll 1
        for (int j = 0; j < l; ++j)
            S[j * 32] = sm.base[j];
        uint64_t whigh_u = 1;
        int gpar = 0;
#pragma unroll 1
        for (int d = J; d < ndig; ++d) {
            const int rad = mv.drad[d];
            const int g = (int)(c % rad);
            c /= rad;
            if (g == 0)  // no sign flip in this row: nothing to do (for the whole warp, often)
                continue;
            const double2* Mr = sm.M + mv.drow[d] * sm.ld;
            const double coef = (double)(-2 * g);
#pragma unroll 1
            for (int j = 0; j < l; ++j) {
                const double2 b = Mr[j];
                double2 s = S[j * 32];
                s.x = __fma_rn(coef, b.x, s.x);
                s.y = __fma_rn(coef, b.y, s.y);
                S[j * 32] = s;
            }
            whigh_u *= binom_u64(mv.dtop[d], g);
            gpar += g;
        }

        // ---- warp-uniform walk over the low digits
        LowWalk wk;
        wk.v = 0;
        wk.g = 0;
        wk.dir = 0;
        wk.radm1 = 0;
        wk.topp = 0;
        for (int d = 0; d < J; ++d) {
            wk.radm1 |= uint64_t(mv.drad[d] - 1) << (4 * d);
            wk.topp |= uint64_t(mv.dtop[d]) << (4 * d);
        }
        const bool weighted = D.weighted != 0;
        const bool unit = D.jf < 0;
        const int jf = D.jf;
        // acc: the terms since the weight last changed (unweighted); run: the
        // weighted sum since the last fold; every 32 terms run (or, for an
        // unweighted permanent, acc) is folded into the double-double rh/rl,
        // ih/il.  The weight changes only when a digit of radix > 2 moves, so
        // it costs 2 DFMA per change instead of 2 DMUL per term.
        double wlow = 1.0;
        double2 acc = make_double2(0.0, 0.0), run = make_double2(0.0, 0.0);
        double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
        const int64_t L = D.L;
        int64_t s = 0;
        int blk = 0;
#pragma unroll 1
        while (s < L) {
            glynn_term<false>(S, l, unit, jf, sm.ecnt, acc);
            if (++s < L) {
                if (glynn_step(wk, sm, S, l) && weighted)
                    reweight(wk, J, wlow, acc, run);
                glynn_term<true>(S, l, unit, jf, sm.ecnt, acc);
                if (++s < L && glynn_step(wk, sm, S, l) && weighted)
                    reweight(wk, J, wlow, acc, run);
            }
            if (++blk == 16) {
                blk = 0;
                if (weighted) {
                    run.x = __fma_rn(wlow, acc.x, run.x);
                    run.y = __fma_rn(wlow, acc.y, run.y);
                    acc = run;
                    run = make_double2(0.0, 0.0);
                }
                dd_acc(rh, rl, acc.x);
                dd_acc(ih, il, acc.y);
                acc = make_double2(0.0, 0.0);
            }
        }
        if (weighted) {
            run.x = __fma_rn(wlow, acc.x, run.x);
            run.y = __fma_rn(wlow, acc.y, run.y);
            acc = run;
        }
        dd_acc(rh, rl, acc.x);
        dd_acc(ih, il, acc.y);
        res = task_sum(rh, rl, ih, il, whigh_u, (gpar & 1) != 0, active);
    }
    combine_task(a, t, D, res, lane);
}

// The task's sum res (the same on every lane) goes to the permanent's output
// if the permanent has one task; otherwise to its slot, and the warp that
// writes the last slot adds the slots in task order.
__device__ void combine_task(const ExecArgs& a, const Task& t, const PermDesc& D, dd2 res, int lane)
{
    if (D.ntasks <= 1) {
        if (lane == 0)
            finalize(a, D, res);
        return;
    }
    int last = 0;
    if (lane == 0) {
        double* pp = a.partials + 4 * (int64_t)(D.slot0 + t.part - D.part0);
        pp[0] = res.rh;
        pp[1] = res.rl;
        pp[2] = res.ih;
        pp[3] = res.il;
        __threadfence();
        const int old = atomicAdd(a.counters + 1 + t.perm, 1);
        last = (old == D.ntasks - 1);
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last)
        return;
    __threadfence();
    dd2 tot = {0.0, 0.0, 0.0, 0.0};
    for (int q = lane; q < D.ntasks; q += kWarp) {
        const double* pp = a.partials + 4 * (int64_t)(D.slot0 + q);
        dd_add(tot.rh, tot.rl, __ldcg(pp + 0), __ldcg(pp + 1));
        dd_add(tot.ih, tot.il, __ldcg(pp + 2), __ldcg(pp + 3));
    }
    warp_fix_sum(tot.rh, tot.rl, tot.rh, tot.rl);
    warp_fix_sum(tot.ih, tot.il, tot.ih, tot.il);
    if (lane == 0)
        finalize(a, D, tot);
}

// ---------------------------------------------------------------- register-resident walk
// For product sides of at most kFwdRegMaxLd columns a lane keeps its column
// sums in registers, in a walk instantiated for even column bounds NL and
// launched once per class of permanents (at most NL product columns).
// Columns 0 .. l-2 live in registers 0 .. l-2 and the last column l-1 in
// register NL-1; the registers between are padding whose sum stays exactly
// 1 + 0i (its base-matrix entries are staged as zeros and its extra-prefix
// count as 0).  So no FP64 instruction of the walk depends on l: every column
// loop runs over all NL registers without a test, and a padding column costs
// its products by 1, which are exact (a test per column made the compiler
// predicate the FP64 work, and predicated-off instructions took 40-55% of
// the FP64 pipe).  The products are formed in the order of the shared-memory
// walk, so both give the same bits.  A warp's shared memory holds the base
// matrix and its column sums in register order and the small integer arrays.
__host__ __device__ inline int reg_warp_smem_bytes(int kmax, int ld)
{
    int bytes = (kmax * ld + ld) * 16 + (16 + ld) * 4;
    return (bytes + 15) & ~15;
}

struct RegSmem {
    double2* M;       // kmax x ld, register order
    double2* base;    // ld, register order
    int32_t* lowrow;  // 16
    int32_t* ecnt;    // ld, register order
    int ld;
    __device__ RegSmem(unsigned char* raw, int kmax, int ld_)
    {
        ld = ld_;
        M = reinterpret_cast<double2*>(raw);
        base = M + kmax * ld;
        lowrow = reinterpret_cast<int32_t*>(base + ld);
        ecnt = lowrow + 16;
    }
};

// Register of product column j of a permanent with l columns.
template <int NL>
__device__ __forceinline__ int reg_of(int j, int l)
{
    return j == l - 1 ? NL - 1 : j;
}

// Stage permanent D for the register walk: base matrix and base column sums
// in register order (padding: entries 0, sum 1 + 0i), extra-prefix counts in
// register order (padding: 0).  sm.ld = NL.
template <int NL>
__device__ void stage_perm_reg(const ExecArgs& a, const PermDesc& D, const MetaView& mv,
                               RegSmem& sm, int lane)
{
    const int k = D.k, l = D.l;
    for (int e = lane; e < k * NL; e += kWarp) {
        const int i = e / NL, r = e - i * NL;
        double2 v = make_double2(0.0, 0.0);
        const int j = r == NL - 1 ? l - 1 : r;
        if (r == NL - 1 || r < l - 1) {
            const int64_t off =
                D.src_off + (int64_t)mv.ridx[i] * D.si + (int64_t)mv.cidx[j] * D.sj;
            v = a.src[off];
        }
        sm.M[e] = v;
    }
    for (int d = lane; d < D.J; d += kWarp)
        sm.lowrow[d] = mv.drow[d];
    for (int r = lane; r < NL; r += kWarp)
        sm.ecnt[r] = r == NL - 1 ? mv.ecnt[l - 1] : (r < l - 1 ? mv.ecnt[r] : 0);
    __syncwarp();
    for (int r = lane; r < NL; r += kWarp) {
        double2 s = make_double2(0.0, 0.0);
        if (r == NL - 1 || r < l - 1) {
            for (int i = 0; i < k; ++i) {
                const double rm = (double)mv.rmul[i];
                const double2 b = sm.M[i * NL + r];
                s.x = __fma_rn(rm, b.x, s.x);
                s.y = __fma_rn(rm, b.y, s.y);
            }
        } else {
            s = make_double2(1.0, 0.0);
        }
        sm.base[r] = s;
    }
    __syncwarp();
}

// S += coef * (row Mr), every register (padding entries are zero).
template <int NL>
__device__ __forceinline__ void reg_add_row(double2 (&S)[NL], const double2* Mr, double coef)
{
#pragma unroll
    for (int r = 0; r < NL; ++r) {
        const double2 b = Mr[r];
        S[r].x = __fma_rn(coef, b.x, S[r].x);
        S[r].y = __fma_rn(coef, b.y, S[r].y);
    }
}

// One term, as glynn_term: acc +-= prod_j S_j^{c_j}.  jr = register of the
// first column with an extra prefix (-1: every c_j = 1); ec = extra-prefix
// counts in register order.
template <int NL, bool NEG>
__device__ __forceinline__ void reg_term(const double2 (&S)[NL], int jr, const int (&ec)[NL],
                                         double2& acc)
{
    if (jr < 0) {
        double2 p = S[0];
#pragma unroll
        for (int r = 1; r < NL - 1; ++r)
            p = cmul(p, S[r]);
        cfma_acc<NEG>(acc, p, S[NL - 1]);
        return;
    }
    // P(q) = S_0 ... S_{q-1} for every column; at the first column with an
    // extra prefix ex starts as that prefix, and each extra multiplies it in
    double2 pre = S[0], ex = S[0];
#pragma unroll
    for (int r = 0; r < NL; ++r) {
        if (r > 0)
            pre = cmul(pre, S[r]);
        ex = r == jr ? pre : ex;
        const int e0 = r == jr ? 1 : 0;
#pragma unroll 1
        for (int e = e0; e < ec[r]; ++e)
            ex = cmul(ex, pre);
    }
    cfma_acc<NEG>(acc, pre, ex);
}

// One Gray step, as glynn_step, on the register column sums.
template <int NL>
__device__ __forceinline__ bool reg_step(LowWalk& wk, const RegSmem& sm, double2 (&S)[NL])
{
    int up;
    const int d = low_step(wk, up);
    reg_add_row(S, sm.M + sm.lowrow[d] * NL, up > 0 ? -2.0 : 2.0);
    return ((wk.radm1 >> (4 * d)) & 15u) > 1u;
}

// The walk of this lane's chunk c (as in process_task); returns the task's
// sum over the warp (task_sum).
template <int NL>
__device__ __forceinline__ dd2 reg_walk(const PermDesc& D, const MetaView& mv, const RegSmem& sm,
                                        int64_t c, bool active)
{
    const int l = D.l, J = D.J, ndig = D.ndig;
    double2 S[NL];
    int ec[NL];
#pragma unroll
    for (int r = 0; r < NL; ++r) {
        S[r] = sm.base[r];
        ec[r] = sm.ecnt[r];
    }
    const int jr = D.jf < 0 ? -1 : reg_of<NL>(D.jf, l);
    uint64_t whigh_u = 1;
    int gpar = 0;
#pragma unroll 1
    for (int d = J; d < ndig; ++d) {
        const int rad = mv.drad[d];
        const int g = (int)(c % rad);
        c /= rad;
        if (g == 0)
            continue;
        reg_add_row(S, sm.M + mv.drow[d] * NL, (double)(-2 * g));
        whigh_u *= binom_u64(mv.dtop[d], g);
        gpar += g;
    }

    LowWalk wk;
    wk.v = 0;
    wk.g = 0;
    wk.dir = 0;
    wk.radm1 = 0;
    wk.topp = 0;
    for (int d = 0; d < J; ++d) {
        wk.radm1 |= uint64_t(mv.drad[d] - 1) << (4 * d);
        wk.topp |= uint64_t(mv.dtop[d]) << (4 * d);
    }
    const bool weighted = D.weighted != 0;
    double wlow = 1.0;
    double2 acc = make_double2(0.0, 0.0), run = make_double2(0.0, 0.0);
    double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
    const int64_t L = D.L;
    int64_t s = 0;
    int blk = 0;
#pragma unroll 1
    while (s < L) {
        reg_term<NL, false>(S, jr, ec, acc);
        if (++s < L) {
            if (reg_step(wk, sm, S) && weighted)
                reweight(wk, J, wlow, acc, run);
            reg_term<NL, true>(S, jr, ec, acc);
            if (++s < L && reg_step(wk, sm, S) && weighted)
                reweight(wk, J, wlow, acc, run);
        }
        if (++blk == 16) {
            blk = 0;
            if (weighted) {
                run.x = __fma_rn(wlow, acc.x, run.x);
                run.y = __fma_rn(wlow, acc.y, run.y);
                acc = run;
                run = make_double2(0.0, 0.0);
            }
            dd_acc(rh, rl, acc.x);
            dd_acc(ih, il, acc.y);
            acc = make_double2(0.0, 0.0);
        }
    }
    if (weighted) {
        run.x = __fma_rn(wlow, acc.x, run.x);
        run.y = __fma_rn(wlow, acc.y, run.y);
        acc = run;
    }
    dd_acc(rh, rl, acc.x);
    dd_acc(ih, il, acc.y);
    return task_sum(rh, rl, ih, il, whigh_u, (gpar & 1) != 0, active);
}

template <int NL>
__device__ void process_task_reg(const ExecArgs& a, const Task& t, RegSmem& sm, int& staged,
                                 int lane)
{
    const PermDesc D = a.desc[t.perm];
    const MetaView mv = meta_view(a.meta, D);
    dd2 res = {0.0, 0.0, 0.0, 0.0};
    if (!D.trivial) {
        if (staged != t.perm) {
            __syncwarp();
            stage_perm_reg<NL>(a, D, mv, sm, lane);
            staged = t.perm;
        }
        const int64_t chunk0 = (int64_t)t.part * kWarp;
        const bool active = chunk0 + lane < D.nchunks;
        res = reg_walk<NL>(D, mv, sm, active ? (chunk0 + lane) : 0, active);
    }
    combine_task(a, t, D, res, lane);
}

// The register-resident kernel of column bound NL: tasks as in
// glynn_fwd_kernel, each of a permanent with at most NL product columns (a
// task beyond that is skipped and recorded as a layout error).  The batched
// method launches one such kernel per column class, so that the warps of an
// SM run one instantiation of the walk: warps running different ones (a
// single kernel dispatching on l) ran 1.6 times slower.
template <int NL>
__global__ void __launch_bounds__(256, 1) glynn_fwd_reg_kernel(ExecArgs a, int64_t t_begin,
                                                             int64_t t_end, int kmax, int ld,
                                                             int queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (NL > ld) {  // the launch's shared-memory rows are narrower than this class's
        if (threadIdx.x == 0)
            record_error(a.err, kErrDescLayout, t_begin);
        return;
    }
    RegSmem sm(smem_raw + warp * reg_warp_smem_bytes(kmax, ld), kmax, NL);
    int staged = -1;
    auto run = [&](int64_t ti) {
        const Task t = a.tasks[ti];
        const int32_t bad = task_guard(t, a.desc, a.nperm, a.nmeta, a.nslots, kmax,
                                       ld < NL ? ld : NL, kMaxLowDigits);
        if (bad) {
            if (lane == 0)
                record_error(a.err, bad, ti);
            return;
        }
        process_task_reg<NL>(a, t, sm, staged, lane);
    };
    if (!queue) {
        const int64_t ti = t_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
        if (ti < t_end)
            run(ti);
        return;
    }
    for (;;) {
        int q = 0;
        if (lane == 0)
            q = atomicAdd(a.counters, 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        const int64_t ti = t_begin + q;
        if (ti >= t_end)
            break;
        run(ti);
    }
}

// Task ti of the list, once its guards pass (a failing task is skipped and
// recorded in the error record).
__device__ __forceinline__ void run_task(const ExecArgs& a, int64_t ti, WarpSmem& sm, int kmax,
                                         int ld, int& staged, int lane)
{
    const Task t = a.tasks[ti];
    const int32_t bad = task_guard(t, a.desc, a.nperm, a.nmeta, a.nslots, kmax, ld, kMaxLowDigits);
    if (bad) {
        if (lane == 0)
            record_error(a.err, bad, ti);
        return;
    }
    process_task(a, t, sm, staged, lane);
}

// Tasks [t_begin, t_end) of the list.  queue != 0: every warp pulls tasks from
// the global counter until the range is exhausted (persistent launch of a
// whole batch); queue == 0: warp w of block b takes task t_begin + b * wpb + w
// (one launch per permanent, the plain method).
__global__ void __launch_bounds__(256, 2) glynn_fwd_kernel(ExecArgs a, int64_t t_begin,
                                                         int64_t t_end, int kmax, int ld,
                                                         int queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem sm(smem_raw + warp * warp_smem_bytes(kmax, ld), kmax, ld);
    int staged = -1;
    if (!queue) {
        const int64_t ti = t_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
        if (ti < t_end)
            run_task(a, ti, sm, kmax, ld, staged, lane);
        return;
    }
    for (;;) {
        int q = 0;
        if (lane == 0)
            q = atomicAdd(a.counters, 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        const int64_t ti = t_begin + q;
        if (ti >= t_end)
            break;
        run_task(a, ti, sm, kmax, ld, staged, lane);
    }
}

// All column classes in one persistent launch: each task runs the
// instantiation of its own class.
__global__ void __launch_bounds__(256, 1) glynn_fwd_reg_mixed_kernel(ExecArgs a, int64_t t_begin,
                                                                     int64_t t_end, int kmax,
                                                                     int ld, int queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* raw = smem_raw + warp * reg_warp_smem_bytes(kmax, ld);
    int staged = -1, staged_nl = 0;
    auto run = [&](int64_t ti) {
        const Task t = a.tasks[ti];
        const int32_t bad =
            task_guard(t, a.desc, a.nperm, a.nmeta, a.nslots, kmax, ld, kMaxLowDigits);
        if (bad) {
            if (lane == 0)
                record_error(a.err, bad, ti);
            return;
        }
        const int l = a.desc[t.perm].l;
        const int nl = l <= 4 ? 4 : l + (l & 1);
        if (nl > ld) {  // the class's rows do not fit the launch's layout
            if (lane == 0)
                record_error(a.err, kErrDescLayout, ti);
            return;
        }
        if (nl != staged_nl)
            staged = -1;  // the staged layout depends on the class
        staged_nl = nl;
        switch (nl) {
#define PQ_REG_CASE(N)                                   \
    case N: {                                            \
        RegSmem sm(raw, kmax, N);                        \
        process_task_reg<N>(a, t, sm, staged, lane);     \
        break;                                           \
    }
            PQ_REG_CASE(4)
            PQ_REG_CASE(6)
            PQ_REG_CASE(8)
            PQ_REG_CASE(10)
            PQ_REG_CASE(12)
            PQ_REG_CASE(14)
            PQ_REG_CASE(16)
            PQ_REG_CASE(18)
            PQ_REG_CASE(20)
#undef PQ_REG_CASE
        default:
            break;
        }
    };
    if (!queue) {
        const int64_t ti = t_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
        if (ti < t_end)
            run(ti);
        return;
    }
    for (;;) {
        int q = 0;
        if (lane == 0)
            q = atomicAdd(a.counters, 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        const int64_t ti = t_begin + q;
        if (ti >= t_end)
            break;
        run(ti);
    }
}

// ---------------------------------------------------------------- host side
int fwd_smem_per_warp(int kmax, int ld) { return warp_smem_bytes(kmax, ld); }

int fwd_regs_per_thread(int)
{
    cudaFuncAttributes at{};
    return cudaFuncGetAttributes(&at, glynn_fwd_kernel) == cudaSuccess ? at.numRegs : 255;
}

// Raise (never lower) the kernel's dynamic shared-memory limit: plans made
// earlier with larger workspaces must keep launching.
cudaError_t fwd_prepare(int, int smem_bytes)
{
    cudaFuncAttributes at{};
    cudaError_t e = cudaFuncGetAttributes(&at, glynn_fwd_kernel);
    if (e != cudaSuccess)
        return e;
    if (at.maxDynamicSharedSizeBytes >= smem_bytes)
        return cudaSuccess;
    return cudaFuncSetAttribute(glynn_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes);
}

cudaError_t fwd_launch_persistent(int ld, const ExecArgs& a, int kmax, int blocks, int wpb,
                                  cudaStream_t st)
{
    const int smem = wpb * warp_smem_bytes(kmax, ld);
    glynn_fwd_kernel<<<blocks, 32 * wpb, smem, st>>>(a, 0, a.ntasks, kmax, ld, 1);
    return cudaGetLastError();
}

cudaError_t fwd_launch_plain(int ld, const ExecArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                             int wpb, cudaStream_t st)
{
    const int smem = wpb * warp_smem_bytes(kmax, ld);
    const int64_t nt = t_end - t_begin;
    const unsigned grid = (unsigned)((nt + wpb - 1) / wpb);
    glynn_fwd_kernel<<<grid, 32 * wpb, smem, st>>>(a, t_begin, t_end, kmax, ld, 0);
    return cudaGetLastError();
}

// ---- register-resident walk
int fwd_reg_class_of(int l) { return l <= 4 ? 4 : l + (l & 1); }

int fwd_reg_smem_per_warp(int kmax, int ld) { return reg_warp_smem_bytes(kmax, ld); }

static const void* fwd_reg_kernel_for(int nl)
{
    switch (nl) {
    case 4: return (const void*)glynn_fwd_reg_kernel<4>;
    case 6: return (const void*)glynn_fwd_reg_kernel<6>;
    case 8: return (const void*)glynn_fwd_reg_kernel<8>;
    case 10: return (const void*)glynn_fwd_reg_kernel<10>;
    case 12: return (const void*)glynn_fwd_reg_kernel<12>;
    case 14: return (const void*)glynn_fwd_reg_kernel<14>;
    case 16: return (const void*)glynn_fwd_reg_kernel<16>;
    case 18: return (const void*)glynn_fwd_reg_kernel<18>;
    case 20: return (const void*)glynn_fwd_reg_kernel<20>;
    default: return nullptr;
    }
}

int fwd_reg_regs_per_thread(int nl)
{
    cudaFuncAttributes at{};
    const void* f = fwd_reg_kernel_for(nl);
    return (f && cudaFuncGetAttributes(&at, f) == cudaSuccess) ? at.numRegs : 255;
}

cudaError_t fwd_reg_prepare(int nl, int smem_bytes)
{
    const void* f = fwd_reg_kernel_for(nl);
    if (!f)
        return cudaErrorInvalidValue;
    cudaFuncAttributes at{};
    cudaError_t e = cudaFuncGetAttributes(&at, f);
    if (e != cudaSuccess)
        return e;
    if (at.maxDynamicSharedSizeBytes >= smem_bytes)
        return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

int fwd_reg_mixed_regs_per_thread()
{
    cudaFuncAttributes at{};
    return cudaFuncGetAttributes(&at, glynn_fwd_reg_mixed_kernel) == cudaSuccess ? at.numRegs
                                                                                : 255;
}

cudaError_t fwd_reg_mixed_prepare(int smem_bytes)
{
    cudaFuncAttributes at{};
    cudaError_t e = cudaFuncGetAttributes(&at, glynn_fwd_reg_mixed_kernel);
    if (e != cudaSuccess)
        return e;
    if (at.maxDynamicSharedSizeBytes >= smem_bytes)
        return cudaSuccess;
    return cudaFuncSetAttribute(glynn_fwd_reg_mixed_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

cudaError_t fwd_reg_mixed_launch(const ExecArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                                 int ld, unsigned grid, int wpb, int queue, cudaStream_t st)
{
    glynn_fwd_reg_mixed_kernel<<<grid, 32 * wpb, wpb * reg_warp_smem_bytes(kmax, ld), st>>>(
        a, t_begin, t_end, kmax, ld, queue);
    return cudaGetLastError();
}

template <int NL>
static void fwd_reg_launch_nl(const ExecArgs& a, int64_t t_begin, int64_t t_end, int kmax, int ld,
                              unsigned grid, int wpb, int queue, cudaStream_t st)
{
    glynn_fwd_reg_kernel<NL><<<grid, 32 * wpb, wpb * reg_warp_smem_bytes(kmax, ld), st>>>(
        a, t_begin, t_end, kmax, ld, queue);
}

cudaError_t fwd_reg_launch(int nl, const ExecArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                           int ld, unsigned grid, int wpb, int queue, cudaStream_t st)
{
    switch (nl) {
    case 4: fwd_reg_launch_nl<4>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    case 6: fwd_reg_launch_nl<6>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    case 8: fwd_reg_launch_nl<8>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    case 10: fwd_reg_launch_nl<10>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    case 12: fwd_reg_launch_nl<12>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    case 14: fwd_reg_launch_nl<14>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    case 16: fwd_reg_launch_nl<16>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    case 18: fwd_reg_launch_nl<18>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    case 20: fwd_reg_launch_nl<20>(a, t_begin, t_end, kmax, ld, grid, wpb, queue, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pqi
