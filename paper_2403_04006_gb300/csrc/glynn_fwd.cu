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
//     sign folded into the DFMA operands; binomial weights of low digits with
//     radix > 2 scale one factor (two DMUL);
//   * every 16 terms the FP64 running sum is folded into a double-double
//     accumulator with TwoSum.
// A warp task is up to 32 chunks of one permanent (one per lane).  Lanes are
// reduced in a fixed tree order and the tasks of one permanent in task order
// by the warp that finishes last, so results do not depend on scheduling.
#include <cuda_runtime.h>

#include "pq_device.cuh"
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
__device__ void stage_perm(const ExecArgs& a, const PermDesc& D, const MetaView& mv,
                           WarpSmem& sm, int lane)
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
        double whigh = active ? (double)whigh_u : 0.0;
        if (gpar & 1)
            whigh = -whigh;

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
        fast_two_sum(rh, rl, rh, rl);
        fast_two_sum(ih, il, ih, il);
        dd_mul_d(rh, rl, whigh);
        dd_mul_d(ih, il, whigh);
        res.rh = rh;
        res.rl = rl;
        res.ih = ih;
        res.il = il;
        res = warp_sum_dd2(res);
    }

    // ---- combine tasks of this permanent
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
    tot = warp_sum_dd2(tot);
    if (lane == 0)
        finalize(a, D, tot);
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
__global__ void __launch_bounds__(256) glynn_fwd_kernel(ExecArgs a, int64_t t_begin,
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

}  // namespace pqi
