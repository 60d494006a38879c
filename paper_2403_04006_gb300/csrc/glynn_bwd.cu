// glynn_bwd.cu -- gradient of the permanent with respect to the base matrix,
// in the same Gray-code pass as the permanent itself.
//
// With per = 2^{-(n-1)} sum_t w_t prod_j S_j(t)^{c_j} and
// S_j = sum_i x_i b_ij, x_i = r_i - 2 g_i, the derivative is
//   G_ij = d per / d b_ij = 2^{-(n-1)} sum_t w_t x_i(t) Q_j(t),
//   Q_j  = c_j S_j^{c_j - 1} prod_{j' != j} S_{j'}^{c_{j'}},
// which counts every copy of b_ij in the expanded matrix.  Q_j comes from
// prefix and suffix products of the column powers (no division, so S_j = 0
// is harmless).  Product columns arrive sorted by non-increasing
// multiplicity, so the columns with c_j >= 2 are the first n2 and the loops
// are split at n2 instead of testing c_j per column.
//
// Accumulation per thread over one chunk: A_j = sum_t w_t Q_j(t).  Rows whose
// x_i is constant in the chunk (high digits, rows without a digit) contribute
// x_i A_j.  A low-digit row changes x_i by Delta at some steps tau; then
//   sum_t x_i(t) R_j(t) = x_i(end) A_j - sum_tau Delta A_j(before tau),
// so only the changed row's correction C_ij += Delta A_j is updated per step:
// O(l) work per term instead of O(k l).  At the end of a task the lanes are
// contracted in a fixed order (lane-parallel over the k x l entries), tasks of
// one permanent are summed in task order by the warp that finishes last, and
// the result is multiplied by the upstream gradient (PyTorch convention:
// grad_b = grad_per * conj(G)).
//
// As in the forward kernel, every per-lane array lives in shared memory,
// lane-major, and every loop over columns is a runtime loop, so the FP64 pipe
// (the only loaded resource on GB300) sees no predicated or speculative work.
#include <cuda_runtime.h>

#include "pq_device.cuh"
#include "pq_kernels.h"

namespace pqi {

// Row stride (in elements) of the lane-major per-lane arrays: 33, not 32, so
// that the end-of-task contraction, where lane e reads element (j(e), q) for
// a fixed q, spreads over the banks instead of hitting one bank 32 times.
constexpr int kLS = 33;

// Per-warp shared memory: ld = product-column bound, jb = low digits of the
// plan's chunks, n2 = repeated product columns at most (powers are kept only
// for those).  Layout: base matrix M (kmax x ld), base column sums (ld), the
// lanes' accumulators A (ld x kLS) and corrections C (jb x ld x kLS), then a
// region that the walk uses for the column sums S, prefixes P and powers PW,
// FULL, and that the end-of-task contraction reuses for the lanes' row
// multipliers X (kmax x kLS doubles) and the correction sums V (jb x ld),
// then the weights wh (32) and small integer arrays.
__host__ __device__ inline long bwd_walk_region_bytes(int kmax, int ld, int jb, int n2)
{
    const long walk = 16L * kLS * (2L * ld + 2L * n2);
    const long contraction = ((8L * kLS * kmax + 15) & ~15L) + 16L * jb * ld;
    return walk > contraction ? walk : contraction;
}

__host__ __device__ inline int bwd_warp_smem_bytes(int kmax, int ld, int jb, int n2)
{
    long bytes = 16L * (kmax * ld + ld + kLS * (long)ld + kLS * (long)jb * ld) +
                 bwd_walk_region_bytes(kmax, ld, jb, n2) + 8L * 32 + 4L * (16 + ld + kmax);
    return (int)((bytes + 15) & ~15L);
}

struct BwdSmem {
    double2* M;       // kmax x ld
    double2* base;    // ld
    double2* A;       // ld x kLS (lane-major: element (j, lane) at j * kLS + lane)
    double2* C;       // jb x ld x kLS
    double2* S;       // ld x kLS        -- walk region
    double2* P;       // ld x kLS
    double2* PW;      // n2 x kLS
    double2* FULL;    // n2 x kLS
    double* X;        // kmax x kLS      -- the same region at the end of a task
    double2* V;       // jb x ld
    double* wh;       // 32
    int32_t* lowrow;  // 16
    int32_t* cm;      // ld
    int32_t* rowdig;  // kmax: low digit of each row, or -1
    int ld;
    __device__ BwdSmem(unsigned char* raw, int kmax, int ld_, int jb, int n2)
    {
        ld = ld_;
        M = reinterpret_cast<double2*>(raw);
        base = M + kmax * ld;
        A = base + ld;
        C = A + kLS * ld;
        S = C + kLS * jb * ld;
        P = S + kLS * ld;
        PW = P + kLS * ld;
        FULL = PW + kLS * n2;
        X = reinterpret_cast<double*>(S);
        V = reinterpret_cast<double2*>(reinterpret_cast<unsigned char*>(S) +
                                       ((8L * kLS * kmax + 15) & ~15L));
        wh = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(S) +
                                       bwd_walk_region_bytes(kmax, ld, jb, n2));
        lowrow = reinterpret_cast<int32_t*>(wh + 32);
        cm = lowrow + 16;
        rowdig = cm + ld;
    }
};

__device__ __forceinline__ void acc_scaled(double2* a, double s, double2 q)
{
    double2 v = *a;
    v.x = __fma_rn(s, q.x, v.x);
    v.y = __fma_rn(s, q.y, v.y);
    *a = v;
}

// A_j += ws * Q_j for this lane's column sums.  All pointers are lane-offset
// with stride kLS.  n2 = number of leading columns with c_j >= 2, for which
// PW_j = c_j S_j^{c_j - 1} (the derivative of the column power) and FULL_j =
// S_j^{c_j} are formed first.  The prefixes P_j = prod_{j' < j} S_{j'}^{c_{j'}}
// are stored; the suffix sw = ws prod_{j' > j} S_{j'}^{c_{j'}} carries the
// term's weight, so that every column's accumulation A_j += P_j sw (times PW_j
// for a repeated column) is one fused complex multiply-add.
//
// Every loop over columns loads the next column's operands from shared
// memory before it computes the current one (the index of the last column
// is reused instead of reading past it): with only a few warps per SM
// sub-partition a load waited for inside the loop would leave the FP64 pipe
// idle.
__device__ __forceinline__ void bwd_term(const double2* S, double2* P, double2* PW, double2* FULL,
                                         double2* A, int l, int n2, const int32_t* cm, double ws)
{
    if (l == 1) {
        if (n2 == 0) {  // n = 1: d per / d b = 1
            A[0].x = __dadd_rn(A[0].x, ws);
            return;
        }
        double2 q = S[0];  // c_0 S_0^{c_0 - 1}
#pragma unroll 1
        for (int e = 2; e < cm[0]; ++e)
            q = cmul(q, S[0]);
        acc_scaled(A, ws * (double)cm[0], q);
        return;
    }
    // powers of the repeated columns
    if (n2 > 0) {
        double2 sn = S[0];
        int cn = cm[0];
#pragma unroll 1
        for (int j = 0; j < n2; ++j) {
            const double2 s = sn;
            const int c = cn;
            const int jn = j + 1 < n2 ? j + 1 : j;
            sn = S[jn * kLS];
            cn = cm[jn];
            double2 pw = s;
#pragma unroll 1
            for (int e = 2; e < c; ++e)
                pw = cmul(pw, s);
            FULL[j * kLS] = cmul(pw, s);
            const double cd = (double)c;
            PW[j * kLS] = make_double2(__dmul_rn(cd, pw.x), __dmul_rn(cd, pw.y));
        }
    }
    // prefix P_j = prod_{j' < j} S_{j'}^{c_{j'}}, j = 1 .. l-1: FULL for the
    // repeated columns among 1 .. l-2, then S
    double2 run = (n2 > 0) ? FULL[0] : S[0];
    P[kLS] = run;
    const int na = n2 < l - 1 ? n2 : l - 1;
    if (na > 1) {
        double2 fn = FULL[kLS];
#pragma unroll 1
        for (int j = 1; j < na; ++j) {
            const double2 f = fn;
            fn = FULL[(j + 1 < na ? j + 1 : j) * kLS];
            run = cmul(run, f);
            P[(j + 1) * kLS] = run;
        }
    }
    {
        const int j0 = na > 1 ? na : 1;
        if (j0 < l - 1) {
            double2 sn = S[j0 * kLS];
#pragma unroll 1
            for (int j = j0; j < l - 1; ++j) {
                const double2 sv = sn;
                sn = S[(j + 1 < l - 1 ? j + 1 : j) * kLS];
                run = cmul(run, sv);
                P[(j + 1) * kLS] = run;
            }
        }
    }
    // suffix pass, last column first
    double2 sw;
    {
        const int j = l - 1;
        double2 q = P[j * kLS];
        double2 f;
        if (j < n2) {
            q = cmul(q, PW[j * kLS]);
            f = FULL[j * kLS];
        } else {
            f = S[j * kLS];
        }
        acc_scaled(A + j * kLS, ws, q);
        sw = make_double2(__dmul_rn(ws, f.x), __dmul_rn(ws, f.y));
    }
    // columns l-2 .. max(n2, 1) with c_j = 1
    {
        const int jlo = n2 > 1 ? n2 : 1;
        int j = l - 2;
        if (j >= jlo) {
            double2 pn = P[j * kLS], an = A[j * kLS], sn = S[j * kLS];
#pragma unroll 1
            for (; j >= jlo; --j) {
                const double2 pv = pn, sv = sn;
                double2 av = an;
                const int jn = j - 1 >= jlo ? j - 1 : j;
                pn = P[jn * kLS];
                an = A[jn * kLS];
                sn = S[jn * kLS];
                cfma_acc<false>(av, pv, sw);
                A[j * kLS] = av;
                sw = cmul(sw, sv);
            }
        }
    }
    // columns min(n2, l-1) - 1 .. 1 with c_j >= 2
    {
        int j = (n2 < l - 1 ? n2 : l - 1) - 1;
        if (j >= 1) {
            double2 pn = P[j * kLS], an = A[j * kLS], wn = PW[j * kLS], fn = FULL[j * kLS];
#pragma unroll 1
            for (; j >= 1; --j) {
                const double2 pv = pn, wv = wn, fv = fn;
                double2 av = an;
                const int jn = j - 1 >= 1 ? j - 1 : j;
                pn = P[jn * kLS];
                an = A[jn * kLS];
                wn = PW[jn * kLS];
                fn = FULL[jn * kLS];
                const double2 q = cmul(pv, sw);
                cfma_acc<false>(av, q, wv);
                A[j * kLS] = av;
                sw = cmul(sw, fv);
            }
        }
    }
    // column 0: Q_0 = c_0 S_0^{c_0 - 1} * prod_{j > 0}
    double2 av = A[0];
    if (n2 > 0) {
        cfma_acc<false>(av, sw, PW[0]);
    } else {
        av.x = __dadd_rn(av.x, sw.x);
        av.y = __dadd_rn(av.y, sw.y);
    }
    A[0] = av;
}

template <class SM>
__device__ void bwd_stage(const BwdArgs& a, const PermDesc& D, const MetaView& mv, SM& sm,
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
        sm.cm[j] = mv.cmul[j];
    for (int i = lane; i < k; i += kWarp) {
        int dg = -1;
        for (int d = 0; d < D.J; ++d)
            if (mv.drow[d] == i)
                dg = d;
        sm.rowdig[i] = dg;
    }
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

__device__ void bwd_combine(const BwdArgs& a, const Task& t, const PermDesc& D, int kl, int lane);

__device__ void bwd_task(const BwdArgs& a, const Task& t, BwdSmem& sm, int& staged, int lane)
{
    const PermDesc D = a.desc[t.perm];
    const MetaView mv = meta_view(a.meta, D);
    const int k = D.k, l = D.l, J = D.J, ndig = D.ndig;
    const int kl = k * l;
    double* slot = a.gpart + 2 * (a.gpart_off[t.perm] + (int64_t)t.part * kl);

    if (!D.trivial) {
        if (staged != t.perm) {
            __syncwarp();
            bwd_stage(a, D, mv, sm, lane);
            staged = t.perm;
        }
        const int64_t chunk0 = (int64_t)t.part * kWarp;
        const bool active = chunk0 + lane < D.nchunks;
        const int64_t chunk = active ? (chunk0 + lane) : 0;
        double2* S = sm.S + lane;
        double2* A = sm.A + lane;
#pragma unroll 1
        for (int j = 0; j < l; ++j) {
            S[j * kLS] = sm.base[j];
            A[j * kLS] = make_double2(0.0, 0.0);
        }
        // the high digits of this lane's chunk: column sums and weight
        uint64_t whigh_u = 1;
        int gpar = 0;
        int64_t c = chunk;
#pragma unroll 1
        for (int d = J; d < ndig; ++d) {
            const int rad = mv.drad[d];
            const int g = (int)(c % rad);
            c /= rad;
            if (g == 0)
                continue;
            const double2* Mr = sm.M + mv.drow[d] * sm.ld;
            const double coef = (double)(-2 * g);
            double2 bn = Mr[0], sn = S[0];
#pragma unroll 1
            for (int j = 0; j < l; ++j) {
                const double2 b = bn;
                double2 sv = sn;
                const int jn = j + 1 < l ? j + 1 : j;
                bn = Mr[jn];
                sn = S[jn * kLS];
                sv.x = __fma_rn(coef, b.x, sv.x);
                sv.y = __fma_rn(coef, b.y, sv.y);
                S[j * kLS] = sv;
            }
            whigh_u *= binom_u64(mv.dtop[d], g);
            gpar += g;
        }
        double whigh = active ? (double)whigh_u : 0.0;
        if (gpar & 1)
            whigh = -whigh;
        sm.wh[lane] = whigh;
        for (int e = 0; e < J * l; ++e) {
            const int d = e / l, j = e - d * l;
            sm.C[(d * sm.ld + j) * kLS + lane] = make_double2(0.0, 0.0);
        }
        int n2 = 0;
        while (n2 < l && sm.cm[n2] >= 2)
            ++n2;

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
        double wlow = 1.0;
        const int64_t L = D.L;
#pragma unroll 1
        for (int64_t s = 0; s < L; ++s) {
            bwd_term(S, sm.P + lane, sm.PW + lane, sm.FULL + lane, A, l, n2, sm.cm,
                     (s & 1) ? -wlow : wlow);
            if (s + 1 < L) {
                int up;
                const int d = low_step(wk, up);
                const int row = sm.lowrow[d];
                const double delta = up > 0 ? -2.0 : 2.0;
                const double2* Mr = sm.M + row * sm.ld;
                double2* Cd = sm.C + d * sm.ld * kLS + lane;
                double2 bn = Mr[0], svn = S[0], avn = A[0], cvn = Cd[0];
#pragma unroll 1
                for (int j = 0; j < l; ++j) {
                    const double2 b = bn, av = avn;
                    double2 sv = svn, cv = cvn;
                    const int jn = j + 1 < l ? j + 1 : j;
                    bn = Mr[jn];
                    svn = S[jn * kLS];
                    avn = A[jn * kLS];
                    cvn = Cd[jn * kLS];
                    sv.x = __fma_rn(delta, b.x, sv.x);
                    sv.y = __fma_rn(delta, b.y, sv.y);
                    S[j * kLS] = sv;
                    cv.x = __fma_rn(delta, av.x, cv.x);
                    cv.y = __fma_rn(delta, av.y, cv.y);
                    Cd[j * kLS] = cv;
                }
                if (((wk.radm1 >> (4 * d)) & 15u) > 1u)
                    wlow = (double)low_weight(wk, J);
            }
        }
        // Contraction G_ij = sum_q wh_q (x_iq A_jq - C_{d(i) j q}) over the 32
        // lanes q in order, as sum_q u_iq A_jq - V_{d(i) j} with u_iq = wh_q x_iq
        // and V_dj = sum_q wh_q C_djq, so that each product is formed once.
        // The walk region (S, P, PW, FULL) is free now and holds u and V.
        // x_i = r_i - 2 g_i: rows without a digit keep r_i, high-digit rows
        // take g from this lane's chunk index, low-digit rows from the walk's
        // final Gray value, which every lane shares.
        __syncwarp();
        {
            const double whl = sm.wh[lane];
            double* X = sm.X + lane;
            for (int i = 0; i < k; ++i)
                X[i * kLS] = whl * (double)mv.rmul[i];
            int64_t cc = chunk;
            for (int d = J; d < ndig; ++d) {
                const int rad = mv.drad[d];
                const int g = (int)(cc % rad);
                cc /= rad;
                const int row = mv.drow[d];
                X[row * kLS] = whl * (double)(mv.rmul[row] - 2 * g);
            }
            for (int d = 0; d < J; ++d) {
                const int g = (int)((wk.g >> (4 * d)) & 15u);
                const int row = sm.lowrow[d];
                X[row * kLS] = whl * (double)(mv.rmul[row] - 2 * g);
            }
        }
        __syncwarp();
        for (int e = lane; e < J * l; e += kWarp) {
            const int d = e / l, j = e - d * l;
            const double2* Cq = sm.C + (d * sm.ld + j) * kLS;
            double vx = 0.0, vy = 0.0;
            for (int q = 0; q < 32; ++q) {
                const double2 cv = Cq[q];
                vx = __fma_rn(sm.wh[q], cv.x, vx);
                vy = __fma_rn(sm.wh[q], cv.y, vy);
            }
            sm.V[d * sm.ld + j] = make_double2(vx, vy);
        }
        __syncwarp();
        for (int e = lane; e < kl; e += kWarp) {
            const int i = e / l, j = e - i * l;
            const int dg = sm.rowdig[i];
            const double2* Aq = sm.A + j * kLS;
            const double* uq = sm.X + i * kLS;
            double gx = 0.0, gy = 0.0;
            for (int q = 0; q < 32; ++q) {
                const double2 av = Aq[q];
                gx = __fma_rn(uq[q], av.x, gx);
                gy = __fma_rn(uq[q], av.y, gy);
            }
            if (dg >= 0) {
                const double2 v = sm.V[dg * sm.ld + j];
                gx = __dsub_rn(gx, v.x);
                gy = __dsub_rn(gy, v.y);
            }
            slot[2 * e] = gx;
            slot[2 * e + 1] = gy;
        }
    }

    bwd_combine(a, t, D, kl, lane);
}

// The tasks of a permanent are summed in task order by the warp that finishes
// last, and the sum is scaled by 2^{1-n} and the upstream gradient.
__device__ void bwd_combine(const BwdArgs& a, const Task& t, const PermDesc& D, int kl, int lane)
{
    int last = 1;
    if (D.ntasks > 1) {
        __threadfence();  // every lane's slot entries, before the count
        __syncwarp();
        if (lane == 0) {
            const int old = atomicAdd(a.counters + 1 + t.perm, 1);
            last = (old == D.ntasks - 1);
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last)
            return;
        __threadfence();
    }
    __syncwarp();
    // upstream gradient: coef = dL/dper (PyTorch convention)
    double2 coef = make_double2(1.0, 0.0);
    if (a.grad_out) {
        coef = a.grad_out[D.out];
    } else if (a.grad_prob) {
        const double2 amp = a.amps[D.out];
        const double gp = a.grad_prob[D.out] * 2.0 * D.norm;
        coef = make_double2(gp * amp.x, gp * amp.y);
    }
    const double* base_slot = a.gpart + 2 * a.gpart_off[t.perm];
    double2* outg = a.grad_local + a.grad_local_off[t.perm];
    for (int e = lane; e < kl; e += kWarp) {
        double gx = 0.0, gy = 0.0;
        for (int q = 0; q < D.ntasks; ++q) {
            gx += __ldcg(base_slot + 2 * ((int64_t)q * kl + e));
            gy += __ldcg(base_slot + 2 * ((int64_t)q * kl + e) + 1);
        }
        gx = scalbn(gx, 1 - D.n);
        gy = scalbn(gy, 1 - D.n);
        // grad_b = coef * conj(G)
        outg[e] = make_double2(coef.x * gx + coef.y * gy, coef.y * gx - coef.x * gy);
    }
}

// The guards of task ti (those of the forward with the class's low-digit
// bound jb, and at most n2 product columns with multiplicity >= 2, for which
// the launch keeps powers per lane; they come first, the columns being
// sorted by non-increasing multiplicity).  Returns 0 or the error code.
__device__ __forceinline__ int32_t bwd_guard(const BwdArgs& a, int64_t ti, int kmax, int ld, int jb,
                                          int n2)
{
    const Task t = a.tasks[ti];
    const int32_t bad = task_guard(t, a.desc, a.nperm, a.nmeta, -1, kmax, ld, jb);
    if (bad)
        return bad;
    const PermDesc D = a.desc[t.perm];
    const int32_t* cm = a.meta + D.meta + 2 * D.k + D.l;  // cmul
    int rep = 0;
    while (rep < D.l && cm[rep] >= 2)
        ++rep;
    return rep > n2 ? kErrDescLayout : 0;
}

// Tasks [t_begin, t_end) of the list; a task whose guards fail is skipped
// and recorded in the error record.
// At least 2 blocks of 256 threads per SM caps the kernel at 128 registers
// per thread (it takes 118 without spilling, the prefetched operands of the
// column loops included): 17 warps per SM, more than the shared-memory
// workspace of every class but the narrowest leaves room for.
__global__ void __launch_bounds__(256, 2) glynn_bwd_kernel(BwdArgs a, int64_t t_begin,
                                                         int64_t t_end, int kmax, int ld, int jb,
                                                         int n2, int queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    BwdSmem sm(smem_raw + warp * bwd_warp_smem_bytes(kmax, ld, jb, n2), kmax, ld, jb, n2);
    int staged = -1;
    if (!queue) {
        const int64_t ti = t_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
        if (ti >= t_end)
            return;
        const int32_t bad = bwd_guard(a, ti, kmax, ld, jb, n2);
        if (bad) {
            if (lane == 0)
                record_error(a.err, bad, ti);
            return;
        }
        bwd_task(a, a.tasks[ti], sm, staged, lane);
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
        const int32_t bad = bwd_guard(a, ti, kmax, ld, jb, n2);
        if (bad) {
            if (lane == 0)
                record_error(a.err, bad, ti);
            continue;
        }
        bwd_task(a, a.tasks[ti], sm, staged, lane);
    }
}

// ---------------------------------------------------------------- register-resident walk
// For product-column bounds NL <= 14 a lane keeps its column sums S, its
// accumulators A and the term's prefixes P in registers: every column loop is
// unrolled over NL and columns j >= l are skipped by warp-uniform tests.  Only
// the correction rows C stay in shared memory, so a warp needs about a third
// of the shared memory of the kernel above and more warps fit on an SM (the
// FP64 pipe of an SM sub-partition with a single warp idles whenever that
// warp waits on a dependent result).
//
// The factor c_j of the repeated columns is applied once, when the task's
// gradient is written: the lanes accumulate A'_j = sum_t w_t Q_j(t) / c_j,
// and everything built from A' (the corrections, the contraction) is linear
// in it.  A column with c_j >= 2 then costs, per term, (c_j - 1) extra
// complex products in the prefix pass and (c_j - 1) in the suffix pass:
// t = sw S_j^{c_j - 1}, A'_j += P_j t, sw = t S_j.
//
// Per-warp shared memory: base matrix M (kmax x ld), base column sums (ld),
// a region that holds the correction rows C (jb x ld x kLS) during the walk
// and, at the end of a task, the accumulators A' (ld x kLS) and the row
// multipliers X (kmax x kLS doubles), then the correction sums V (jb x ld),
// the weights wh (32) and small integer arrays.
__host__ __device__ inline long bwdr_region_bytes(int kmax, int ld, int jb)
{
    const long walk = 16L * kLS * jb * ld;
    const long end = 16L * kLS * ld + ((8L * kLS * kmax + 15) & ~15L);
    return walk > end ? walk : end;
}

__host__ __device__ inline int bwdr_warp_smem_bytes(int kmax, int ld, int jb)
{
    const long bytes = 16L * (kmax * ld + ld) + bwdr_region_bytes(kmax, ld, jb) + 16L * jb * ld +
                       8L * 32 + 4L * (16 + ld + kmax);
    return (int)((bytes + 15) & ~15L);
}

struct BwdRegSmem {
    double2* M;       // kmax x ld
    double2* base;    // ld
    double2* C;       // jb x ld x kLS    -- region, during the walk
    double2* A;       // ld x kLS         -- region, at the end of a task
    double* X;        // kmax x kLS       -- region, at the end of a task
    double2* V;       // jb x ld
    double* wh;       // 32
    int32_t* lowrow;  // 16
    int32_t* cm;      // ld
    int32_t* rowdig;  // kmax
    int ld;
    __device__ BwdRegSmem(unsigned char* raw, int kmax, int ld_, int jb)
    {
        ld = ld_;
        M = reinterpret_cast<double2*>(raw);
        base = M + kmax * ld;
        C = base + ld;
        A = C;
        X = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(C) + 16L * kLS * ld);
        V = reinterpret_cast<double2*>(reinterpret_cast<unsigned char*>(C) +
                                       bwdr_region_bytes(kmax, ld, jb));
        wh = reinterpret_cast<double*>(V + jb * ld);
        lowrow = reinterpret_cast<int32_t*>(wh + 32);
        cm = lowrow + 16;
        rowdig = cm + ld;
    }
};

// One term: A'_j += ws Q_j / c_j for j < l.  n2 = number of leading columns
// with c_j >= 2 (their multiplicities in cm).
template <int NL>
__device__ __forceinline__ void bwdr_term(const double2 (&S)[NL], double2 (&A)[NL],
                                          const int (&cm)[NL], int l, int n2, double ws)
{
    // prefixes P_j = prod_{j' < j} S_{j'}^{c_{j'}}, j = 1 .. l-1
    double2 P[NL];
    double2 run = S[0];
    if (n2 > 0) {
#pragma unroll 1
        for (int e = 1; e < cm[0]; ++e)
            run = cmul(run, S[0]);
    }
    P[NL > 1 ? 1 : 0] = run;
#pragma unroll
    for (int j = 1; j < NL - 1; ++j) {
        if (j < l - 1) {
            run = cmul(run, S[j]);
            if (j < n2) {
#pragma unroll 1
                for (int e = 1; e < cm[j]; ++e)
                    run = cmul(run, S[j]);
            }
            P[j + 1] = run;
        }
    }
    // suffix pass, last column first; sw = ws prod_{j' > j} S_{j'}^{c_{j'}}
    // (a separate branch for the last column, whose suffix is real, made the
    // compiler keep S, A and P in local memory)
    double2 sw = make_double2(ws, 0.0);
#pragma unroll
    for (int j = NL - 1; j >= 1; --j) {
        if (j < l) {
            double2 t = sw;
            if (j < n2) {
#pragma unroll 1
                for (int e = 1; e < cm[j]; ++e)
                    t = cmul(t, S[j]);
            }
            cfma_acc<false>(A[j], P[j], t);
            sw = cmul(t, S[j]);
        }
    }
    // column 0: S_0^{c_0 - 1} times the suffix (for l = 1 the weight alone)
    double2 t = sw;
    if (n2 > 0) {
#pragma unroll 1
        for (int e = 1; e < cm[0]; ++e)
            t = cmul(t, S[0]);
    }
    A[0].x = __dadd_rn(A[0].x, t.x);
    A[0].y = __dadd_rn(A[0].y, t.y);
}

template <int NL>
__device__ void bwdr_task(const BwdArgs& a, const Task& t, BwdRegSmem& sm, int& staged, int lane)
{
    const PermDesc D = a.desc[t.perm];
    const MetaView mv = meta_view(a.meta, D);
    const int k = D.k, l = D.l, J = D.J, ndig = D.ndig;
    const int kl = k * l;
    double* slot = a.gpart + 2 * (a.gpart_off[t.perm] + (int64_t)t.part * kl);

    if (!D.trivial) {
        __syncwarp();  // the previous task's contraction read the region that C reuses
        if (staged != t.perm) {
            bwd_stage(a, D, mv, sm, lane);
            staged = t.perm;
        }
        const int64_t chunk0 = (int64_t)t.part * kWarp;
        const bool active = chunk0 + lane < D.nchunks;
        const int64_t chunk = active ? (chunk0 + lane) : 0;
        double2 S[NL], A[NL];
        int cm[NL];
#pragma unroll
        for (int j = 0; j < NL; ++j) {
            S[j] = j < l ? sm.base[j] : make_double2(0.0, 0.0);
            A[j] = make_double2(0.0, 0.0);
            cm[j] = j < l ? sm.cm[j] : 1;
        }
        // the high digits of this lane's chunk: column sums and weight
        uint64_t whigh_u = 1;
        int gpar = 0;
        int64_t c = chunk;
#pragma unroll 1
        for (int d = J; d < ndig; ++d) {
            const int rad = mv.drad[d];
            const int g = (int)(c % rad);
            c /= rad;
            if (g == 0)
                continue;
            const double2* Mr = sm.M + mv.drow[d] * NL;
            const double coef = (double)(-2 * g);
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                if (j < l) {
                    const double2 b = Mr[j];
                    S[j].x = __fma_rn(coef, b.x, S[j].x);
                    S[j].y = __fma_rn(coef, b.y, S[j].y);
                }
            }
            whigh_u *= binom_u64(mv.dtop[d], g);
            gpar += g;
        }
        double whigh = active ? (double)whigh_u : 0.0;
        if (gpar & 1)
            whigh = -whigh;
        sm.wh[lane] = whigh;
        for (int e = 0; e < J * l; ++e) {
            const int d = e / l, j = e - d * l;
            sm.C[(d * NL + j) * kLS + lane] = make_double2(0.0, 0.0);
        }
        int n2 = 0;
        while (n2 < l && sm.cm[n2] >= 2)
            ++n2;
        uint32_t lowrows = 0;  // row of low digit d in bits [6d, 6d + 6): rows < 64
        for (int d = 0; d < J; ++d)
            lowrows |= (uint32_t)sm.lowrow[d] << (6 * d);

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
        double wlow = 1.0;
        const int64_t L = D.L;
#pragma unroll 1
        for (int64_t s = 0; s < L; ++s) {
            bwdr_term<NL>(S, A, cm, l, n2, (s & 1) ? -wlow : wlow);
            if (s + 1 < L) {
                int up;
                const int d = low_step(wk, up);
                const int row = (int)((lowrows >> (6 * d)) & 63u);
                const double delta = up > 0 ? -2.0 : 2.0;
                const double2* Mr = sm.M + row * NL;
                double2* Cd = sm.C + d * NL * kLS + lane;
#pragma unroll
                for (int j = 0; j < NL; ++j) {
                    if (j < l) {
                        const double2 b = Mr[j];
                        double2 cv = Cd[j * kLS];
                        S[j].x = __fma_rn(delta, b.x, S[j].x);
                        S[j].y = __fma_rn(delta, b.y, S[j].y);
                        cv.x = __fma_rn(delta, A[j].x, cv.x);
                        cv.y = __fma_rn(delta, A[j].y, cv.y);
                        Cd[j * kLS] = cv;
                    }
                }
                if (((wk.radm1 >> (4 * d)) & 15u) > 1u)
                    wlow = (double)low_weight(wk, J);
            }
        }
        // Contraction, as in the kernel above: V from the corrections first,
        // then the accumulators and row multipliers go to the region that
        // held the corrections.
        __syncwarp();
        for (int e = lane; e < J * l; e += kWarp) {
            const int d = e / l, j = e - d * l;
            const double2* Cq = sm.C + (d * NL + j) * kLS;
            double vx = 0.0, vy = 0.0;
            for (int q = 0; q < 32; ++q) {
                const double2 cv = Cq[q];
                vx = __fma_rn(sm.wh[q], cv.x, vx);
                vy = __fma_rn(sm.wh[q], cv.y, vy);
            }
            sm.V[d * NL + j] = make_double2(vx, vy);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NL; ++j)
            if (j < l)
                sm.A[j * kLS + lane] = A[j];
        {
            const double whl = sm.wh[lane];
            double* X = sm.X + lane;
            for (int i = 0; i < k; ++i)
                X[i * kLS] = whl * (double)mv.rmul[i];
            int64_t cc = chunk;
            for (int d = J; d < ndig; ++d) {
                const int rad = mv.drad[d];
                const int g = (int)(cc % rad);
                cc /= rad;
                const int row = mv.drow[d];
                X[row * kLS] = whl * (double)(mv.rmul[row] - 2 * g);
            }
            for (int d = 0; d < J; ++d) {
                const int g = (int)((wk.g >> (4 * d)) & 15u);
                const int row = sm.lowrow[d];
                X[row * kLS] = whl * (double)(mv.rmul[row] - 2 * g);
            }
        }
        __syncwarp();
        for (int e = lane; e < kl; e += kWarp) {
            const int i = e / l, j = e - i * l;
            const int dg = sm.rowdig[i];
            const double2* Aq = sm.A + j * kLS;
            const double* uq = sm.X + i * kLS;
            double gx = 0.0, gy = 0.0;
            for (int q = 0; q < 32; ++q) {
                const double2 av = Aq[q];
                gx = __fma_rn(uq[q], av.x, gx);
                gy = __fma_rn(uq[q], av.y, gy);
            }
            if (dg >= 0) {
                const double2 v = sm.V[dg * NL + j];
                gx = __dsub_rn(gx, v.x);
                gy = __dsub_rn(gy, v.y);
            }
            const double cj = (double)sm.cm[j];
            slot[2 * e] = cj * gx;
            slot[2 * e + 1] = cj * gy;
        }
    }
    bwd_combine(a, t, D, kl, lane);
}

// The register-resident kernel for product-column bound NL (the launch's
// class bound); the guards are those of the kernel above, without a bound on
// the repeated columns.
template <int NL>
__global__ void __launch_bounds__(256, 1) glynn_bwd_reg_kernel(BwdArgs a, int64_t t_begin,
                                                            int64_t t_end, int kmax, int jb,
                                                            int queue)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    BwdRegSmem sm(smem_raw + warp * bwdr_warp_smem_bytes(kmax, NL, jb), kmax, NL, jb);
    int staged = -1;
    if (!queue) {
        const int64_t ti = t_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
        if (ti >= t_end)
            return;
        const int32_t bad = bwd_guard(a, ti, kmax, NL, jb, NL);
        if (bad) {
            if (lane == 0)
                record_error(a.err, bad, ti);
            return;
        }
        bwdr_task<NL>(a, a.tasks[ti], sm, staged, lane);
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
        const int32_t bad = bwd_guard(a, ti, kmax, NL, jb, NL);
        if (bad) {
            if (lane == 0)
                record_error(a.err, bad, ti);
            continue;
        }
        bwdr_task<NL>(a, a.tasks[ti], sm, staged, lane);
    }
}

// ---------------------------------------------------------------- scatter
// Batch: one block per item; zero the item's block, then write the oriented
// gradient back to the original (row, column) positions.
__global__ void scatter_batch_kernel(const PermDesc* desc, const int32_t* meta,
                                     const double2* gl, const int64_t* gl_off,
                                     const int64_t* mat_off, const int32_t* ik,
                                     const int32_t* il, double2* out)
{
    const int64_t p = blockIdx.x;
    const PermDesc D = desc[p];
    const int k0 = ik[p], l0 = il[p];
    double2* o = out + mat_off[p];
    for (int e = threadIdx.x; e < k0 * l0; e += blockDim.x)
        o[e] = make_double2(0.0, 0.0);
    __syncthreads();
    if (D.trivial)
        return;
    const MetaView mv = meta_view(meta, D);
    const double2* g = gl + gl_off[p];
    for (int e = threadIdx.x; e < D.k * D.l; e += blockDim.x) {
        const int i = e / D.l, j = e - i * D.l;
        // oriented (i, j) -> source offset ridx*si + cidx*sj within the item
        const int64_t off = (int64_t)mv.ridx[i] * D.si + (int64_t)mv.cidx[j] * D.sj;
        o[off] = g[e];
    }
}

// Boson sampling: grad_U[a][c] = sum over patterns of the entry of that
// pattern's gradient that U[a][c] became.  pos[p][2m] maps output mode a and
// input mode c to the oriented (row, column) indices of pattern p's base
// matrix: pos[p][a] = row of a, pos[p][m + c] = column of c, -1 if absent
// (for a pattern whose summed side is its input modes the roles swap in the
// planner, which writes the map accordingly).
//
// One block of kScatterThreads threads per entry (a, c): thread q adds the
// patterns [q B / T, (q + 1) B / T) in order, each warp adds its 32 sums with
// a fixed shuffle tree and the first thread adds the warp sums in warp order,
// so the result is the same on every run and no floating-point atomics are
// needed.  The loads of one pattern (map, descriptor, gradient block) are
// independent of the next pattern's, so a thread keeps several in flight.
constexpr int kScatterThreads = 128;

__global__ void __launch_bounds__(kScatterThreads) scatter_bs_kernel(
    const PermDesc* desc, int64_t nperm, int m, const int32_t* pos, const double2* gl,
    const int64_t* gl_off, double2* gU)
{
    __shared__ double2 wsum[kScatterThreads / kWarp];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t e = blockIdx.x;  // < m * m by the launch
    const int ar = (int)(e / m), ac = (int)(e - (int64_t)ar * m);  // U row (output), column (input)
    const int64_t p0 = nperm * tid / kScatterThreads, p1 = nperm * (tid + 1) / kScatterThreads;
    double gx = 0.0, gy = 0.0;
#pragma unroll 4
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t* pp = pos + p * 2 * (int64_t)m;
        const int io = pp[ar], jo = pp[m + ac];
        if (io < 0 || jo < 0)
            continue;
        const int l = desc[p].l;
        const bool tr = desc[p].si == 1 && m > 1;  // summed side = input modes
        const double2 v = gl[gl_off[p] + (tr ? (int64_t)jo * l + io : (int64_t)io * l + jo)];
        gx += v.x;
        gy += v.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gx += __shfl_down_sync(0xffffffffu, gx, off);
        gy += __shfl_down_sync(0xffffffffu, gy, off);
    }
    if (lane == 0)
        wsum[warp] = make_double2(gx, gy);
    __syncthreads();
    if (tid == 0) {
        double2 t = wsum[0];
        for (int w = 1; w < kScatterThreads / kWarp; ++w) {
            t.x += wsum[w].x;
            t.y += wsum[w].y;
        }
        gU[e] = t;
    }
}

// ---------------------------------------------------------------- host side
int bwd_smem_bytes_for(int kmax, int ld, int jb, int n2)
{
    return bwd_warp_smem_bytes(kmax, ld, jb, n2);
}

int bwd_regs_per_thread(int)
{
    cudaFuncAttributes at{};
    return cudaFuncGetAttributes(&at, glynn_bwd_kernel) == cudaSuccess ? at.numRegs : 255;
}

// Raise (never lower) the kernel's dynamic shared-memory limit.
cudaError_t bwd_prepare(int, int smem_bytes)
{
    cudaFuncAttributes at{};
    cudaError_t e = cudaFuncGetAttributes(&at, glynn_bwd_kernel);
    if (e != cudaSuccess)
        return e;
    if (at.maxDynamicSharedSizeBytes >= smem_bytes)
        return cudaSuccess;
    return cudaFuncSetAttribute(glynn_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem_bytes);
}

cudaError_t bwd_launch_persistent(int ld, const BwdArgs& a, int64_t t_begin, int64_t t_end,
                                  int kmax, int jb, int n2, int blocks, int wpb, cudaStream_t st)
{
    const int smem = wpb * bwd_warp_smem_bytes(kmax, ld, jb, n2);
    glynn_bwd_kernel<<<blocks, 32 * wpb, smem, st>>>(a, t_begin, t_end, kmax, ld, jb, n2, 1);
    return cudaGetLastError();
}

cudaError_t bwd_launch_plain(int ld, const BwdArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                             int jb, int n2, int wpb, cudaStream_t st)
{
    const int smem = wpb * bwd_warp_smem_bytes(kmax, ld, jb, n2);
    const int64_t nt = t_end - t_begin;
    const unsigned grid = (unsigned)((nt + wpb - 1) / wpb);
    glynn_bwd_kernel<<<grid, 32 * wpb, smem, st>>>(a, t_begin, t_end, kmax, ld, jb, n2, 0);
    return cudaGetLastError();
}

// ---- register-resident walk
bool bwdr_supported(int ld) { return ld >= 2 && ld <= kBwdRegMaxLd && ld % 2 == 0; }

int bwdr_smem_bytes_for(int kmax, int ld, int jb) { return bwdr_warp_smem_bytes(kmax, ld, jb); }

static const void* bwdr_kernel_for(int ld)
{
    switch (ld) {
    case 2: return (const void*)glynn_bwd_reg_kernel<2>;
    case 4: return (const void*)glynn_bwd_reg_kernel<4>;
    case 6: return (const void*)glynn_bwd_reg_kernel<6>;
    case 8: return (const void*)glynn_bwd_reg_kernel<8>;
    case 10: return (const void*)glynn_bwd_reg_kernel<10>;
    case 12: return (const void*)glynn_bwd_reg_kernel<12>;
    case 14: return (const void*)glynn_bwd_reg_kernel<14>;
    default: return nullptr;
    }
}

int bwdr_regs_per_thread(int ld)
{
    cudaFuncAttributes at{};
    const void* f = bwdr_kernel_for(ld);
    return (f && cudaFuncGetAttributes(&at, f) == cudaSuccess) ? at.numRegs : 255;
}

// Raise (never lower) the dynamic shared-memory limit of the class's kernel.
cudaError_t bwdr_prepare(int ld, int smem_bytes)
{
    const void* f = bwdr_kernel_for(ld);
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

template <int NL>
static void bwdr_launch_nl(const BwdArgs& a, int64_t t_begin, int64_t t_end, int kmax, int jb,
                           unsigned grid, int wpb, int queue, cudaStream_t st)
{
    glynn_bwd_reg_kernel<NL><<<grid, 32 * wpb, wpb * bwdr_warp_smem_bytes(kmax, NL, jb), st>>>(
        a, t_begin, t_end, kmax, jb, queue);
}

static cudaError_t bwdr_launch(int ld, const BwdArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                               int jb, unsigned grid, int wpb, int queue, cudaStream_t st)
{
    switch (ld) {
    case 2: bwdr_launch_nl<2>(a, t_begin, t_end, kmax, jb, grid, wpb, queue, st); break;
    case 4: bwdr_launch_nl<4>(a, t_begin, t_end, kmax, jb, grid, wpb, queue, st); break;
    case 6: bwdr_launch_nl<6>(a, t_begin, t_end, kmax, jb, grid, wpb, queue, st); break;
    case 8: bwdr_launch_nl<8>(a, t_begin, t_end, kmax, jb, grid, wpb, queue, st); break;
    case 10: bwdr_launch_nl<10>(a, t_begin, t_end, kmax, jb, grid, wpb, queue, st); break;
    case 12: bwdr_launch_nl<12>(a, t_begin, t_end, kmax, jb, grid, wpb, queue, st); break;
    case 14: bwdr_launch_nl<14>(a, t_begin, t_end, kmax, jb, grid, wpb, queue, st); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t bwdr_launch_persistent(int ld, const BwdArgs& a, int64_t t_begin, int64_t t_end,
                                   int kmax, int jb, int blocks, int wpb, cudaStream_t st)
{
    return bwdr_launch(ld, a, t_begin, t_end, kmax, jb, (unsigned)blocks, wpb, 1, st);
}

cudaError_t bwdr_launch_plain(int ld, const BwdArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                              int jb, int wpb, cudaStream_t st)
{
    const int64_t nt = t_end - t_begin;
    return bwdr_launch(ld, a, t_begin, t_end, kmax, jb, (unsigned)((nt + wpb - 1) / wpb), wpb, 0,
                       st);
}

cudaError_t scatter_grad_batch(const PermDesc* desc, const int32_t* meta, int64_t nperm,
                               const double2* grad_local, const int64_t* grad_local_off,
                               const int64_t* item_mat_off, const int32_t* item_l,
                               const int32_t* item_k, double2* grad_mats, int64_t,
                               cudaStream_t st)
{
    if (nperm == 0)
        return cudaSuccess;
    scatter_batch_kernel<<<(unsigned)nperm, 128, 0, st>>>(desc, meta, grad_local, grad_local_off,
                                                          item_mat_off, item_k, item_l, grad_mats);
    return cudaGetLastError();
}

cudaError_t scatter_grad_bs(const PermDesc* desc, const int32_t* pos, int64_t nperm, int32_t m,
                            const double2* grad_local, const int64_t* grad_local_off,
                            double2* grad_U, cudaStream_t st)
{
    if (m <= 0)
        return cudaSuccess;
    scatter_bs_kernel<<<(unsigned)(m * m), kScatterThreads, 0, st>>>(desc, nperm, m, pos,
                                                                     grad_local, grad_local_off,
                                                                     grad_U);
    return cudaGetLastError();
}

}  // namespace pqi
