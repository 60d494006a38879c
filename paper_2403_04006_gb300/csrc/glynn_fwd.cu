// glynn_fwd.cu -- forward kernels: permanents with repeated rows and columns by
// the BB/FG formula over a mixed-radix Gray code (paper Sec. 4.2, "Boson
// Sampling"; Eq. (per_def) for the permanent, Eq. (BS_prob) for the
// probabilities written by the final reduction).
//
// One thread walks one chunk of the Gray code:
//   * column sums S_j = sum_i (r_i - 2 g_i) b_ij live in registers as complex
//     FP64 (the template LMAX bounds the product-side columns);
//   * every step changes one row's sign count by +-1, so every S_j moves by
//     -+2 b_ij: one DFMA per real component, with b read from shared memory
//     (the same row for all lanes of the warp: a broadcast);
//   * the term prod_j S_j^{c_j} is a chain of complex FP64 products whose
//     last factor is fused into the running sum (four DFMA);
//   * the sign (-1)^step alternates, so pairs of terms are unrolled with the
//     sign folded into the DFMA operands; binomial weights of low digits with
//     radix > 2 scale the first factor;
//   * every 16 terms the FP64 running sum is folded into a double-double
//     accumulator with TwoSum.
// A warp task is up to 32 chunks of one permanent; lanes are reduced in a
// fixed tree order, tasks of one permanent in task order by the warp that
// finishes last, so results do not depend on scheduling.
#include <cuda_runtime.h>

#include "pq_device.cuh"
#include "pq_kernels.h"

namespace pqi {

// Shared memory of one warp: matrix (kmax x LMAX complex), base column sums
// (LMAX complex), low-digit rows (16 ints), column multiplicities (LMAX ints).
__host__ __device__ inline int warp_smem_bytes(int kmax, int lmax)
{
    int bytes = (kmax * lmax + lmax) * 16 + (16 + lmax) * 4;
    return (bytes + 15) & ~15;
}

template <int LMAX>
struct WarpSmem {
    double2* M;
    double2* base;
    int32_t* lowrow;
    int32_t* cm;
    __device__ WarpSmem(unsigned char* raw, int kmax)
    {
        M = reinterpret_cast<double2*>(raw);
        base = M + kmax * LMAX;
        lowrow = reinterpret_cast<int32_t*>(base + LMAX);
        cm = lowrow + 16;
    }
};

// Copy the oriented base matrix of permanent D into shared memory and form
// base_j = sum_i r_i b_ij (all Gray digits at zero).
template <int LMAX>
__device__ void stage_perm(const ExecArgs& a, const PermDesc& D, const MetaView& mv,
                           WarpSmem<LMAX>& sm, int lane)
{
    const int k = D.k, l = D.l;
    for (int e = lane; e < k * l; e += kWarp) {
        int i = e / l, j = e - i * l;
        int64_t off = D.src_off + (int64_t)mv.ridx[i] * D.si + (int64_t)mv.cidx[j] * D.sj;
        sm.M[i * LMAX + j] = a.src[off];
    }
    for (int d = lane; d < D.J; d += kWarp)
        sm.lowrow[d] = mv.drow[d];
    for (int j = lane; j < LMAX; j += kWarp)
        sm.cm[j] = (j < l) ? mv.cmul[j] : 0;
    __syncwarp();
    for (int j = lane; j < l; j += kWarp) {
        double2 s = make_double2(0.0, 0.0);
        for (int i = 0; i < k; ++i) {
            double r = (double)mv.rmul[i];
            double2 b = sm.M[i * LMAX + j];
            s.x = __fma_rn(r, b.x, s.x);
            s.y = __fma_rn(r, b.y, s.y);
        }
        sm.base[j] = s;
    }
    __syncwarp();
}

// One Glynn term: acc +-= w * prod_j S_j^{c_j}.
template <int LMAX, bool NEG>
__device__ __forceinline__ void glynn_term(const double2 (&S)[LMAX], int l, int n,
                                           const int32_t* cm, bool weighted, double w,
                                           double2& acc)
{
    if (n == 1) {  // a single entry: the product is S_0 itself
        acc.x = NEG ? __dsub_rn(acc.x, S[0].x) : __dadd_rn(acc.x, S[0].x);
        acc.y = NEG ? __dsub_rn(acc.y, S[0].y) : __dadd_rn(acc.y, S[0].y);
        return;
    }
    double2 p = S[0];
    if (weighted) {
        p.x = __dmul_rn(p.x, w);
        p.y = __dmul_rn(p.y, w);
    }
    // Column tests are bit tests: written as j == l - 1 the compiler sinks the
    // fused step out of the unrolled loop as S[l - 1], a dynamic index that
    // sends S to local memory.
    const uint64_t lastbit = uint64_t(1) << (l - 1);
    const uint64_t colmask = (lastbit << 1) - 1;
#pragma unroll
    for (int j = 0; j < LMAX; ++j) {
        const uint64_t bit = uint64_t(1) << j;
        if (colmask & bit) {
            int cnt = cm[j] - (j == 0 ? 1 : 0) - ((lastbit & bit) ? 1 : 0);
            for (int e = 0; e < cnt; ++e)
                p = cmul(p, S[j]);
            if (lastbit & bit)
                cfma_acc<NEG>(acc, p, S[j]);
        }
    }
}

// One Gray step of the warp-uniform low walk: update S by -+2 b_row.
template <int LMAX>
__device__ __forceinline__ void glynn_step(LowWalk& wk, const WarpSmem<LMAX>& sm, int l, int J,
                                           bool weighted, double2 (&S)[LMAX], double& wlow)
{
    int up;
    int d = low_step(wk, up);
    const double2* Mr = sm.M + sm.lowrow[d] * LMAX;
    const double delta = up > 0 ? -2.0 : 2.0;  // x = r - 2g
#pragma unroll
    for (int j = 0; j < LMAX; ++j) {
        if (j < l) {
            double2 b = Mr[j];
            S[j].x = __fma_rn(delta, b.x, S[j].x);
            S[j].y = __fma_rn(delta, b.y, S[j].y);
        }
    }
    if (weighted && ((wk.radm1 >> (4 * d)) & 15u) > 1u)
        wlow = (double)low_weight(wk, J);
}

// Write per = 2^{-(n-1)} * sum, and |per|^2 * norm.
__device__ __forceinline__ void finalize(const ExecArgs& a, const PermDesc& D, dd2 v)
{
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

template <int LMAX>
__device__ void process_task(const ExecArgs& a, const Task& t, WarpSmem<LMAX>& sm, int& staged,
                             int lane)
{
    const PermDesc D = a.desc[t.perm];
    const MetaView mv = meta_view(a.meta, D);
    const int l = D.l, n = D.n, J = D.J, ndig = D.ndig;
    dd2 res = {0.0, 0.0, 0.0, 0.0};

    if (!D.trivial) {
        if (staged != t.perm) {
            __syncwarp();
            stage_perm<LMAX>(a, D, mv, sm, lane);
            staged = t.perm;
        }
        // ---- this lane's chunk: decode the high digits, start the column sums
        const int64_t chunk0 = (int64_t)t.part * kWarp;
        const bool active = chunk0 + lane < D.nchunks;
        int64_t c = active ? (chunk0 + lane) : 0;
        double2 S[LMAX];
#pragma unroll
        for (int j = 0; j < LMAX; ++j)
            S[j] = (j < l) ? sm.base[j] : make_double2(0.0, 0.0);
        uint64_t whigh_u = 1;
        int gpar = 0;
        for (int d = J; d < ndig; ++d) {
            int rad = mv.drad[d];
            int g = (int)(c % rad);
            c /= rad;
            const double2* Mr = sm.M + mv.drow[d] * LMAX;
            const double coef = -2.0 * (double)g;
#pragma unroll
            for (int j = 0; j < LMAX; ++j) {
                if (j < l) {
                    double2 b = Mr[j];
                    S[j].x = __fma_rn(coef, b.x, S[j].x);
                    S[j].y = __fma_rn(coef, b.y, S[j].y);
                }
            }
            if (g) {
                whigh_u *= binom_u64(mv.dtop[d], g);
                gpar += g;
            }
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
        double wlow = 1.0;
        double2 acc = make_double2(0.0, 0.0);
        double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
        const int64_t L = D.L;
        int64_t s = 0;
        int blk = 0;
        while (s < L) {
            glynn_term<LMAX, false>(S, l, n, sm.cm, weighted, wlow, acc);
            if (++s < L) {
                glynn_step<LMAX>(wk, sm, l, J, weighted, S, wlow);
                glynn_term<LMAX, true>(S, l, n, sm.cm, weighted, wlow, acc);
                if (++s < L)
                    glynn_step<LMAX>(wk, sm, l, J, weighted, S, wlow);
            }
            if (++blk == 8) {
                blk = 0;
                dd_acc(rh, rl, acc.x);
                dd_acc(ih, il, acc.y);
                acc = make_double2(0.0, 0.0);
            }
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
        double* pp = a.partials + 4 * (int64_t)(D.slot0 + t.part);
        pp[0] = res.rh;
        pp[1] = res.rl;
        pp[2] = res.ih;
        pp[3] = res.il;
        __threadfence();
        int old = atomicAdd(a.counters + 1 + t.perm, 1);
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

// Persistent: every warp pulls tasks from a global queue until it is empty.
template <int LMAX>
__global__ void __launch_bounds__(256) glynn_fwd_persistent(ExecArgs a, int kmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<LMAX> sm(smem_raw + warp * warp_smem_bytes(kmax, LMAX), kmax);
    int staged = -1;
    for (;;) {
        int ti = 0;
        if (lane == 0)
            ti = atomicAdd(a.counters, 1);
        ti = __shfl_sync(0xffffffffu, ti, 0);
        if (ti >= a.ntasks)
            break;
        Task t = a.tasks[ti];
        process_task<LMAX>(a, t, sm, staged, lane);
    }
}

// Plain: tasks [t_begin, t_end) of one permanent, one warp each.
template <int LMAX>
__global__ void __launch_bounds__(256) glynn_fwd_plain(ExecArgs a, int64_t t_begin, int64_t t_end,
                                                       int kmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<LMAX> sm(smem_raw + warp * warp_smem_bytes(kmax, LMAX), kmax);
    int staged = -1;
    int64_t ti = t_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (ti >= t_end)
        return;
    Task t = a.tasks[ti];
    process_task<LMAX>(a, t, sm, staged, lane);
}

// ---------------------------------------------------------------- host side
template <int LMAX>
static cudaError_t set_smem_attrs(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(glynn_fwd_persistent<LMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(glynn_fwd_plain<LMAX>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int fwd_smem_per_warp(int kmax, int lmax) { return warp_smem_bytes(kmax, lmax); }

cudaError_t fwd_prepare(int lmax, int smem_bytes)
{
    switch (lmax) {
    case 8: return set_smem_attrs<8>(smem_bytes);
    case 16: return set_smem_attrs<16>(smem_bytes);
    case 24: return set_smem_attrs<24>(smem_bytes);
    case 32: return set_smem_attrs<32>(smem_bytes);
    case 40: return set_smem_attrs<40>(smem_bytes);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fwd_launch_persistent(int lmax, const ExecArgs& a, int kmax, int blocks, int wpb,
                                  cudaStream_t st)
{
    const int smem = wpb * warp_smem_bytes(kmax, lmax);
    const dim3 grid(blocks), block(32 * wpb);
    switch (lmax) {
    case 8: glynn_fwd_persistent<8><<<grid, block, smem, st>>>(a, kmax); break;
    case 16: glynn_fwd_persistent<16><<<grid, block, smem, st>>>(a, kmax); break;
    case 24: glynn_fwd_persistent<24><<<grid, block, smem, st>>>(a, kmax); break;
    case 32: glynn_fwd_persistent<32><<<grid, block, smem, st>>>(a, kmax); break;
    case 40: glynn_fwd_persistent<40><<<grid, block, smem, st>>>(a, kmax); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t fwd_launch_plain(int lmax, const ExecArgs& a, int64_t t_begin, int64_t t_end,
                             int kmax, int wpb, cudaStream_t st)
{
    const int smem = wpb * warp_smem_bytes(kmax, lmax);
    const int64_t nt = t_end - t_begin;
    const dim3 grid((unsigned)((nt + wpb - 1) / wpb)), block(32 * wpb);
    switch (lmax) {
    case 8: glynn_fwd_plain<8><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax); break;
    case 16: glynn_fwd_plain<16><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax); break;
    case 24: glynn_fwd_plain<24><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax); break;
    case 32: glynn_fwd_plain<32><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax); break;
    case 40: glynn_fwd_plain<40><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pqi
