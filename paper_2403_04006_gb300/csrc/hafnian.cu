// hafnian.cu -- hafnians and loop hafnians of symmetric matrices with
// repeated indices (Sec. 4.1, Eq. (haf_def), Eq. (loop_hafnian), Figs.
// hafnian and loop_hafnian with (2, ..., 2) repetitions), on the same
// warp-uniform mixed-radix Gray walk and double-double accumulation as the
// permanent.
//
// Glynn-type formulas (a reading: the paper names the Glynn-type strategy but
// prints no formula).  For a sign vector d of the N expanded indices, the
// coefficient of d_1 ... d_N in exp(Q(d) + Lin(d)), Q = sum_{p<q} A_pq d_p d_q,
// Lin = sum_p A_pp d_p, counts every matching with loops once, and the mean of
// (prod d) times a polynomial in d is exactly that coefficient.  Without loops
// only Q^n / n! (N = 2n) has degree N.  With base index i repeated r_i times
// and g_i of its copies negative, x_i = r_i - 2 g_i and, B the base matrix and
// gamma the loop weights,
//   q(g) = 1/2 (x^T B x - sum_i r_i B_ii),   l(g) = gamma^T x,
//   haf  = 1 / (n! 2^{N-1}) sum_g s(g) q^n,
//   lhaf = 1 / 2^{N-1} sum_g s(g) sum_{j <= N/2} q^j l^{N-2j} / (j! (N-2j)!),
//   s(g) = (-1)^{sum g} prod_i C(top_i, g_i),
// one copy of the least repeated index keeping a + sign (top = r - 1 there;
// the summand is even under flipping every sign).  A Gray step changes one
// x_r by D = -+2:  q += D y_r + 2 B_rr with y = B x, then y_j += D B_jr and
// l += D gamma_r.  Inside a chunk only the J low digits move, so the walk
// reads y at the J low rows alone and keeps only those (2J DFMA a step
// instead of 2k); y is formed in full once per chunk for the start value of
// q.  q^n is taken by repeated squaring.  The loop polynomial is homogeneous
// of degree N/2 in (q, l^2): sum_j q^j s^{J-j} / (j! (N-2j)!) with s = l^2,
// J = floor(N/2), equals c_J prod_m (q - z_m s) (times l for odd N), where
// z_m = -1 / (2 x_m^2) and x_m runs over the positive roots of the Hermite
// polynomial He_N (substituting z = -1/(2x^2) turns the sum into
// x^{-N} He_N(x) / N!).  The roots are real, found once per N on the host by
// Sturm-count bisection on the Jacobi matrix of He_N, and the kernel
// multiplies the factors in pairs: 2 FP64 operations per unit of N instead
// of Horner's 5.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/pq.h"
#include "pq_device.cuh"
#include "pq_fixsum.cuh"
#include "pq_kernels.h"

namespace pqi {

constexpr int kHafMaxHalf = PQ_MAX_N / 2;  // loop-polynomial factors j = 1 .. N/2

// Per (loop) hafnian: k kept base indices, digits as for the permanent.
struct alignas(16) HafDesc {
    int64_t T, nchunks, L, src_off, gam_off;
    int32_t k, n, N, ld;   // kept indices, N/2, expanded size, source row stride
    int32_t meta;          // ridx[k], rmul[k], drow[nd], drad[nd], dtop[nd]
    int32_t ndig, J, ntasks, slot0;
    int32_t weighted, trivial;  // trivial: result = value (0 for odd N, 1 for N = 0)
    int32_t coef_off;           // loop hafnian: factors of its loop polynomial in loopc
    double value;               // final multiplier (or the trivial result)
};

struct HafArgs {
    const HafDesc* desc;
    const int32_t* meta;
    const Task* tasks;
    int64_t ntasks;
    const double2* src;
    const double2* gamma;  // loop weights (loop hafnian only)
    const double* loopc;   // loop-polynomial factors per distinct N (loop hafnian only)
    double2* out;
    double* partials;
    int32_t* counters;
};

// Shared memory of one warp: M (k x k), y0 = B r (k), gamma (k), y (k x 32,
// lane-major), y at the low rows (J x 32, lane-major), B restricted to the
// low rows (J x J), Horner coefficients, low-digit rows.
__host__ __device__ inline int haf_warp_smem_bytes(int kmax, int jmax)
{
    int bytes = (kmax * kmax + 2 * kmax + 32 * kmax + 32 * jmax + jmax * jmax) * 16 +
                (kHafMaxHalf + 1) * 8 + 16 * 4;
    return (bytes + 15) & ~15;
}

// q^E by the binary method, unrolled at compile time.
template <int E>
__device__ __forceinline__ double2 cpow_c(double2 q)
{
    if constexpr (E == 1) {
        return q;
    } else if constexpr ((E & 1) == 0) {
        const double2 h = cpow_c<E / 2>(q);
        return cmul(h, h);
    } else {
        return cmul(cpow_c<E - 1>(q), q);
    }
}

// q^n for a warp-uniform 1 <= n <= PQ_MAX_N / 2: one uniform branch to
// straight-line code (a runtime bit loop would issue its conditional
// multiplies under false predicates).
__device__ __forceinline__ double2 cpow_n(double2 q, int n)
{
    switch (n) {
#define PQ_POW_CASE(E) \
    case E: return cpow_c<E>(q);
        PQ_POW_CASE(1) PQ_POW_CASE(2) PQ_POW_CASE(3) PQ_POW_CASE(4) PQ_POW_CASE(5)
        PQ_POW_CASE(6) PQ_POW_CASE(7) PQ_POW_CASE(8) PQ_POW_CASE(9) PQ_POW_CASE(10)
        PQ_POW_CASE(11) PQ_POW_CASE(12) PQ_POW_CASE(13) PQ_POW_CASE(14) PQ_POW_CASE(15)
        PQ_POW_CASE(16) PQ_POW_CASE(17) PQ_POW_CASE(18) PQ_POW_CASE(19) PQ_POW_CASE(20)
        PQ_POW_CASE(21) PQ_POW_CASE(22) PQ_POW_CASE(23) PQ_POW_CASE(24)
#undef PQ_POW_CASE
    default: return q;  // not reached: the planner bounds n by PQ_MAX_N / 2
    }
}
static_assert(PQ_MAX_N / 2 == 24, "cpow_n covers exponents up to 24");

// sum_{j=0}^{N/2} q^j l^{N-2j} / (j! (N-2j)!) from the factors cf = [c_J,
// a_0, b_0, a_1, b_1, ..., (z_last)]: each of the P = floor(N/4) pairs of
// roots gives q^2 + a q s + b s^2 (a = -(z1 + z2), b = z1 z2); an odd root
// count J leaves one factor q - z s; odd N one factor l.  JODD and NODD are
// template flags so that no factor is issued under a false predicate.
template <bool JODD, bool NODD>
__device__ __forceinline__ double2 loop_poly(double2 q, double2 l, int P, const double* cf)
{
    const double2 s = cmul(l, l);
    double2 h = make_double2(cf[0], 0.0);
    if (P) {
        const double2 q2 = cmul(q, q), qs = cmul(q, s), s2 = cmul(s, s);
#pragma unroll 1
        for (int p = 0; p < P; ++p) {
            const double a = cf[1 + 2 * p], b = cf[2 + 2 * p];
            double2 t;
            t.x = __fma_rn(b, s2.x, __fma_rn(a, qs.x, q2.x));
            t.y = __fma_rn(b, s2.y, __fma_rn(a, qs.y, q2.y));
            h = cmul(h, t);
        }
    }
    if (JODD) {
        const double z = cf[1 + 2 * P];
        double2 t;
        t.x = __fma_rn(-z, s.x, q.x);
        t.y = __fma_rn(-z, s.y, q.y);
        h = cmul(h, t);
    }
    if (NODD)
        h = cmul(h, l);
    return h;
}

template <bool LOOP>
__device__ void haf_task(const HafArgs& a, const Task& t, unsigned char* raw, int kmax, int jmax,
                         int& staged, int lane)
{
    const HafDesc D = a.desc[t.perm];
    const int k = D.k, J = D.J, nd = D.ndig;
    double2* M = reinterpret_cast<double2*>(raw);
    double2* y0 = M + kmax * kmax;
    double2* gam = y0 + kmax;
    double2* Y = gam + kmax;
    double2* YL = Y + 32 * kmax;
    double2* Bll = YL + 32 * jmax;
    double* cj = reinterpret_cast<double*>(Bll + jmax * jmax);
    int32_t* lowrow = reinterpret_cast<int32_t*>(cj + kHafMaxHalf + 1);
    const int32_t* ridx = a.meta + D.meta;
    const int32_t* rmul = ridx + k;
    const int32_t* drow = rmul + k;
    const int32_t* drad = drow + nd;
    const int32_t* dtop = drad + nd;
    dd2 res = {0.0, 0.0, 0.0, 0.0};

    if (!D.trivial) {
        if (staged != t.perm) {
            __syncwarp();
            for (int e = lane; e < k * k; e += kWarp) {
                const int i = e / k, j = e - i * k;
                M[e] = a.src[D.src_off + (int64_t)ridx[i] * D.ld + ridx[j]];
            }
            for (int d = lane; d < J; d += kWarp)
                lowrow[d] = drow[d];
            if (LOOP) {
                for (int i = lane; i < k; i += kWarp)
                    gam[i] = a.gamma[D.gam_off + ridx[i]];
                for (int j = lane; j <= D.N / 2; j += kWarp)
                    cj[j] = a.loopc[D.coef_off + j];
            }
            __syncwarp();
            for (int e = lane; e < J * J; e += kWarp) {  // B at the low rows
                const int u = e / J, v = e - u * J;
                Bll[e] = M[lowrow[u] * k + lowrow[v]];
            }
            for (int j = lane; j < k; j += kWarp) {  // y0 = B r
                double2 s = make_double2(0.0, 0.0);
                for (int i = 0; i < k; ++i) {
                    const double r = (double)rmul[i];
                    s.x = __fma_rn(r, M[j * k + i].x, s.x);
                    s.y = __fma_rn(r, M[j * k + i].y, s.y);
                }
                y0[j] = s;
            }
            __syncwarp();
            staged = t.perm;
        }
        const int64_t chunk0 = (int64_t)t.part * kWarp;
        const bool active = chunk0 + lane < D.nchunks;
        int64_t c = active ? (chunk0 + lane) : 0;
        const int64_t c_first = c;
        double2* y = Y + lane;
#pragma unroll 1
        for (int j = 0; j < k; ++j)
            y[j * 32] = y0[j];
        // High digits of this lane's chunk: x_row = r_row - 2 g.  y = B x is
        // finished before x^T y is formed in a second pass over the digits.
        uint64_t whigh_u = 1;
        int gpar = 0;
#pragma unroll 1
        for (int d = J; d < nd; ++d) {
            const int rad = drad[d];
            const int g = (int)(c % rad);
            c /= rad;
            if (!g)
                continue;
            const int row = drow[d];
            const double coef = (double)(-2 * g);
#pragma unroll 1
            for (int j = 0; j < k; ++j) {
                const double2 b = M[j * k + row];
                double2 v = y[j * 32];
                v.x = __fma_rn(coef, b.x, v.x);
                v.y = __fma_rn(coef, b.y, v.y);
                y[j * 32] = v;
            }
            whigh_u *= binom_u64(dtop[d], g);
            gpar += g;
        }
        // q = 1/2 (x^T y - sum_i r_i B_ii) and l = gamma^T x, low digits at 0
        double2 q = make_double2(0.0, 0.0), l = make_double2(0.0, 0.0);
#pragma unroll 1
        for (int i = 0; i < k; ++i) {
            const double2 v = y[i * 32];
            const double2 bii = M[i * k + i];
            const double r = (double)rmul[i];
            q.x = __fma_rn(r, __dsub_rn(v.x, bii.x), q.x);
            q.y = __fma_rn(r, __dsub_rn(v.y, bii.y), q.y);
            if (LOOP) {
                l.x = __fma_rn(r, gam[i].x, l.x);
                l.y = __fma_rn(r, gam[i].y, l.y);
            }
        }
        c = c_first;
#pragma unroll 1
        for (int d = J; d < nd; ++d) {
            const int rad = drad[d];
            const int g = (int)(c % rad);
            c /= rad;
            if (!g)
                continue;
            const int row = drow[d];
            const double2 v = y[row * 32];
            const double coef = (double)(-2 * g);
            q.x = __fma_rn(coef, v.x, q.x);
            q.y = __fma_rn(coef, v.y, q.y);
            if (LOOP) {
                l.x = __fma_rn(coef, gam[row].x, l.x);
                l.y = __fma_rn(coef, gam[row].y, l.y);
            }
        }
        q.x *= 0.5;
        q.y *= 0.5;
        double2* yl = YL + lane;
#pragma unroll 1
        for (int e = 0; e < J; ++e)
            yl[e * 32] = y[lowrow[e] * 32];
        double whigh = active ? (double)whigh_u : 0.0;
        if (gpar & 1)
            whigh = -whigh;

        LowWalk wk;
        wk.v = 0;
        wk.g = 0;
        wk.dir = 0;
        wk.radm1 = 0;
        wk.topp = 0;
        for (int d = 0; d < J; ++d) {
            wk.radm1 |= uint64_t(drad[d] - 1) << (4 * d);
            wk.topp |= uint64_t(dtop[d]) << (4 * d);
        }
        const bool weighted = D.weighted != 0;
        const int n = D.n, N = D.N;
        const int form = ((N >> 1) & 1) * 2 + (N & 1), P = N >> 2;
        double wlow = 1.0;
        double2 acc = make_double2(0.0, 0.0);
        double rh = 0.0, rl = 0.0, ih = 0.0, il = 0.0;
        const int64_t L = D.L;
        // The term's polynomial value; the uniform switches pick straight-line
        // code for the exponent or the loop-polynomial shape, so no FP64
        // instruction is issued under a false predicate.
        auto value = [&]() -> double2 {
            if (LOOP) {
                switch (form) {
                case 0: return loop_poly<false, false>(q, l, P, cj);
                case 1: return loop_poly<false, true>(q, l, P, cj);
                case 2: return loop_poly<true, false>(q, l, P, cj);
                default: return loop_poly<true, true>(q, l, P, cj);
                }
            }
            return cpow_n(q, n);
        };
        auto term_pos = [&]() {
            const double2 p = value();
            acc.x = __fma_rn(wlow, p.x, acc.x);
            acc.y = __fma_rn(wlow, p.y, acc.y);
        };
        auto term_neg = [&]() {
            const double2 p = value();
            acc.x = __fma_rn(-wlow, p.x, acc.x);
            acc.y = __fma_rn(-wlow, p.y, acc.y);
        };
        // One Gray step: x_row moves by -+2.
        auto step = [&]() {
            int up;
            const int d = low_step(wk, up);
            const double delta = up > 0 ? -2.0 : 2.0;
            const double2 yr = yl[d * 32];
            const double2* Bd = Bll + d * J;
            const double2 brr = Bd[d];
            q.x = __fma_rn(delta, yr.x, q.x);
            q.y = __fma_rn(delta, yr.y, q.y);
            q.x = __fma_rn(2.0, brr.x, q.x);
            q.y = __fma_rn(2.0, brr.y, q.y);
            if (LOOP) {
                const double2 gr = gam[lowrow[d]];
                l.x = __fma_rn(delta, gr.x, l.x);
                l.y = __fma_rn(delta, gr.y, l.y);
            }
#pragma unroll 1
            for (int e = 0; e < J; ++e) {
                const double2 b = Bd[e];
                double2 v = yl[e * 32];
                v.x = __fma_rn(delta, b.x, v.x);
                v.y = __fma_rn(delta, b.y, v.y);
                yl[e * 32] = v;
            }
            if (weighted && ((wk.radm1 >> (4 * d)) & 15u) > 1u)
                wlow = (double)low_weight(wk, J);
        };
        // Term 0 has sign +; then pairs (odd: -, even: +), folded into the
        // double-double sums every 16 terms by the outer loop.
        term_pos();
        int64_t s = 1;
#pragma unroll 1
        while (s < L) {
            const int npairs = (int)min((L - s) >> 1, (int64_t)8);
#pragma unroll 1
            for (int i = 0; i < npairs; ++i) {
                step();
                term_neg();
                step();
                term_pos();
            }
            s += 2 * npairs;
            if (npairs == 0) {  // one (odd) term left
                step();
                term_neg();
                s += 1;
            }
            dd_acc(rh, rl, acc.x);
            dd_acc(ih, il, acc.y);
            acc = make_double2(0.0, 0.0);
        }
        dd_acc(rh, rl, acc.x);
        dd_acc(ih, il, acc.y);
        fast_two_sum(rh, rl, rh, rl);
        fast_two_sum(ih, il, ih, il);
        dd_mul_d(rh, rl, whigh);
        dd_mul_d(ih, il, whigh);
        // the lanes' sums added exactly in integers (pq_fixsum.cuh)
        warp_fix_sum(rh, rl, res.rh, res.rl);
        warp_fix_sum(ih, il, res.ih, res.il);
    }

    auto finish = [&](dd2 v) {
        double2 o;
        if (D.trivial) {
            o = make_double2(D.value, 0.0);
        } else {
            double h, e;
            fast_two_sum(v.rh, v.rl, h, e);
            o.x = scalbn(h + e, 1 - D.N) * D.value;
            fast_two_sum(v.ih, v.il, h, e);
            o.y = scalbn(h + e, 1 - D.N) * D.value;
        }
        a.out[t.perm] = o;
    };
    if (D.ntasks <= 1) {
        if (lane == 0)
            finish(res);
        return;
    }
    // Several tasks: partials in task order; the last warp to finish sums them
    // in a fixed order (no waiting on other warps).
    int last = 0;
    if (lane == 0) {
        double* pp = a.partials + 4 * (int64_t)(D.slot0 + t.part);
        pp[0] = res.rh;
        pp[1] = res.rl;
        pp[2] = res.ih;
        pp[3] = res.il;
        __threadfence();
        last = (atomicAdd(a.counters + 1 + t.perm, 1) == D.ntasks - 1);
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last)
        return;
    __threadfence();
    dd2 tot = {0.0, 0.0, 0.0, 0.0};
    for (int p = lane; p < D.ntasks; p += kWarp) {
        const double* pp = a.partials + 4 * (int64_t)(D.slot0 + p);
        dd_add(tot.rh, tot.rl, __ldcg(pp + 0), __ldcg(pp + 1));
        dd_add(tot.ih, tot.il, __ldcg(pp + 2), __ldcg(pp + 3));
    }
    warp_fix_sum(tot.rh, tot.rl, tot.rh, tot.rl);
    warp_fix_sum(tot.ih, tot.il, tot.ih, tot.il);
    if (lane == 0)
        finish(tot);
}

// Persistent: every warp takes tasks from a global queue (counters[0]).
template <bool LOOP>
__global__ void __launch_bounds__(256, 1) hafnian_kernel(HafArgs a, int kmax, int jmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* raw = smem_raw + warp * haf_warp_smem_bytes(kmax, jmax);
    int staged = -1;
    for (;;) {
        int q = 0;
        if (lane == 0)
            q = atomicAdd(a.counters, 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= a.ntasks)
            break;
        haf_task<LOOP>(a, a.tasks[q], raw, kmax, jmax, staged, lane);
    }
}

// Positive roots of the Hermite polynomial He_N (He_{k+1} = x He_k - k He_{k-1}),
// ascending: bisection on the number of eigenvalues of its Jacobi matrix
// (zero diagonal, off-diagonal sqrt(k)) below t, counted by the signs of the
// LDL^T pivots of J - t, then Newton steps on He_N.
static std::vector<double> hermite_positive_roots(int N)
{
    auto count_below = [N](double t) {
        int c = 0;
        double d = -t;
        c += d < 0.0;
        for (int k = 1; k < N; ++k) {
            if (d == 0.0)
                d = 1e-300;
            d = -t - (double)k / d;
            c += d < 0.0;
        }
        return c;
    };
    const int J = N / 2;
    const double top = 2.0 * std::sqrt((double)N) + 2.0;  // every root lies below
    std::vector<double> x;
    for (int i = N - J + 1; i <= N; ++i) {  // i-th smallest root
        double lo = 0.0, hi = top;
        for (int it = 0; it < 2000; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi)
                break;
            if (count_below(mid) >= i)
                hi = mid;
            else
                lo = mid;
        }
        double r = 0.5 * (lo + hi);
        for (int it = 0; it < 2; ++it) {
            double p0 = 1.0, p1 = r;  // He_{k-1}, He_k
            for (int k = 1; k < N; ++k) {
                const double p2 = r * p1 - (double)k * p0;
                p0 = p1;
                p1 = p2;
            }
            if (p0 != 0.0)
                r -= p1 / ((double)N * p0);
        }
        x.push_back(r);
    }
    return x;
}

// Factors of the loop polynomial of size N for loop_poly: [c_J, a_0, b_0,
// ..., (z_last)], J + 1 numbers.
static std::vector<double> loop_factors(int N)
{
    const int J = N / 2;
    std::vector<double> cf;
    double cJ = 1.0;
    for (int i = 2; i <= J; ++i)
        cJ /= (double)i;  // 1 / (J! (N - 2J)!), N - 2J <= 1
    cf.push_back(cJ);
    const std::vector<double> x = hermite_positive_roots(N);
    std::vector<double> z;
    for (double v : x)
        z.push_back(-1.0 / (2.0 * v * v));
    int m = 0;
    for (; m + 1 < J; m += 2) {
        cf.push_back(-(z[m] + z[m + 1]));
        cf.push_back(z[m] * z[m + 1]);
    }
    if (m < J)
        cf.push_back(z[m]);
    return cf;
}

static double factorial_h(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i)
        r *= (double)i;
    return r;
}

// Plan, upload, run and synchronise; gamma == nullptr selects the hafnian.
}  // namespace pqi

// A planned batch of (loop) hafnians: host schedule uploaded once, device
// workspace owned by the plan.
struct pq_haf_plan {
    int loop = 0;
    int64_t batch = 0, ntasks = 0;
    int kmax = 1, jmax = 1, wpb = 1, blocks = 1, per_warp = 0;
    pqi::HafDesc* desc_d = nullptr;
    int32_t* meta_d = nullptr;
    pqi::Task* tasks_d = nullptr;
    double* part_d = nullptr;
    int32_t* cnt_d = nullptr;
    double* loopc_d = nullptr;
};

namespace pqi {

static void haf_plan_free(pq_haf_plan* P)
{
    if (!P)
        return;
    dev_free(P->desc_d);
    dev_free(P->meta_d);
    dev_free(P->tasks_d);
    dev_free(P->part_d);
    dev_free(P->cnt_d);
    dev_free(P->loopc_d);
    delete P;
    host_object_freed();
}

// Plan: digits, chunks, tasks (longest first), loop-polynomial factors;
// uploads them and raises the kernel's shared-memory limit.
static int haf_plan_build(const int64_t* mat_off, const int32_t* k, const int32_t* rep,
                          const int64_t* rep_off, int64_t batch, bool loop, pq_haf_plan** out)
{
    *out = nullptr;
    if (batch < 0 || (batch > 0 && (!mat_off || !k || !rep || !rep_off)))
        return report(PQ_ERR_ARG, "null argument or negative batch");
    if (batch > (int64_t(1) << 30))
        return report(PQ_ERR_UNSUPPORTED, "batch above 2^30");
    int dev = 0, sms = 1;
    if (batch > 0 && (cudaGetDevice(&dev) != cudaSuccess ||
                      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                          cudaSuccess))
        return report(PQ_ERR_CUDA, "no CUDA device");
    struct Dg {
        int rad, row, top;
    };
    struct Item {
        std::vector<int32_t> ridx, rm;
        std::vector<Dg> dg;
    };
    std::vector<HafDesc> desc(batch);
    std::vector<Item> items(batch);
    double t_total = 0.0;
    // Pass 1: kept indices, digits and term counts.
    for (int64_t b = 0; b < batch; ++b) {
        HafDesc& D = desc[b];
        Item& it = items[b];
        std::memset(&D, 0, sizeof(D));
        if (k[b] < 0 || k[b] > PQ_MAX_DIM || mat_off[b] < 0 || rep_off[b] < 0)
            return report(PQ_ERR_ARG, "bad size or offset");
        const int32_t* r = rep + rep_off[b];
        int N = 0;
        for (int i = 0; i < k[b]; ++i) {
            if (r[i] < 0)
                return report(PQ_ERR_ARG, "negative repetition");
            if (r[i] > PQ_MAX_N)
                return report(PQ_ERR_UNSUPPORTED, "expanded size above PQ_MAX_N");
            if (r[i] > 0) {
                it.ridx.push_back(i);
                it.rm.push_back(r[i]);
                N += r[i];
            }
        }
        if (N > PQ_MAX_N)
            return report(PQ_ERR_UNSUPPORTED, "expanded size above PQ_MAX_N");
        D.src_off = mat_off[b];
        D.gam_off = rep_off[b];
        D.ld = k[b];
        D.N = N;
        D.n = N / 2;
        if (N == 0 || (!loop && (N & 1))) {
            D.trivial = 1;
            D.value = (N == 0) ? 1.0 : 0.0;
            continue;
        }
        const int kk = (int)it.ridx.size();
        D.k = kk;
        D.value = loop ? 1.0 : 1.0 / factorial_h(N / 2);
        // Digits: one copy of the least repeated index fixed (radix r_f), the
        // others radix r_i + 1; ascending radix so that small ones walk inside
        // a chunk.
        const int f = (int)(std::min_element(it.rm.begin(), it.rm.end()) - it.rm.begin());
        int64_t T = 1;
        for (int i = 0; i < kk; ++i) {
            const int rad = (i == f) ? it.rm[i] : it.rm[i] + 1;
            if (rad < 2)
                continue;
            it.dg.push_back({rad, i, (i == f) ? it.rm[i] - 1 : it.rm[i]});
            if (T > (int64_t(1) << 62) / rad)
                return report(PQ_ERR_UNSUPPORTED, "term count above 2^62");
            T *= rad;
        }
        std::stable_sort(it.dg.begin(), it.dg.end(),
                         [](const Dg& x, const Dg& y) { return x.rad < y.rad; });
        D.T = T;
        D.ndig = (int)it.dg.size();
        t_total += (double)T;
    }
    // Pass 2: chunks and tasks.  Every item gets a share of about 64 warp
    // tasks per SM in proportion to its terms, so that one large hafnian still
    // fills the GPU.
    const double want_tasks = 64.0 * sms;
    std::vector<int32_t> meta;
    std::vector<Task> tasks;
    std::vector<double> cost;
    std::vector<double> loopc;
    std::vector<int32_t> coef_at(PQ_MAX_N + 1, -1);
    int kmax = 1, jmax = 1;
    int32_t slot = 0;
    for (int64_t b = 0; b < batch; ++b) {
        HafDesc& D = desc[b];
        Item& it = items[b];
        D.slot0 = slot;
        if (D.trivial) {
            D.ntasks = 1;
            tasks.push_back(Task{(int32_t)b, 0});
            cost.push_back(0.0);
            slot += 1;
            continue;
        }
        const int kk = D.k, N = D.N;
        const int64_t T = D.T;
        kmax = std::max(kmax, kk);
        if (loop) {
            if (coef_at[N] < 0) {
                coef_at[N] = (int32_t)loopc.size();
                const std::vector<double> cf = loop_factors(N);
                loopc.insert(loopc.end(), cf.begin(), cf.end());
            }
            D.coef_off = coef_at[N];
        }
        // Chunk length L = product of the J low radices, at most 4096 terms,
        // at most T / (32 x the item's task share), and J minimising the FP64
        // work per term: 2J + 8 for the walk plus 2k(ndig - J) + 4k + 64 per
        // chunk for the start value.
        const double share = std::max(1.0, std::ceil(want_tasks * (double)T / t_total));
        const int64_t cap = std::max<int64_t>(
            1, std::min<int64_t>(4096, (int64_t)((double)T / (kWarp * share))));
        int J = 0;
        int64_t L = 1;
        {
            double best = 1e300;
            int64_t Lc = 1;
            for (int j = 0;; ++j) {
                const double c = 2.0 * j + 8.0 + (2.0 * kk * (D.ndig - j) + 4.0 * kk + 64.0) / Lc;
                if (c < best) {
                    best = c;
                    J = j;
                    L = Lc;
                }
                if (j >= D.ndig || j >= kMaxLowDigits || it.dg[j].rad > kMaxLowRadix ||
                    Lc * it.dg[j].rad > cap)
                    break;
                Lc *= it.dg[j].rad;
            }
        }
        jmax = std::max(jmax, J);
        D.J = J;
        D.L = L;
        D.nchunks = T / L;
        for (int d = 0; d < J; ++d)
            if (it.dg[d].rad > 2)
                D.weighted = 1;
        const int64_t nt = (D.nchunks + kWarp - 1) / kWarp;
        if (nt + slot > (int64_t(1) << 30))
            return report(PQ_ERR_UNSUPPORTED, "too many tasks");
        D.ntasks = (int32_t)nt;
        D.meta = (int32_t)meta.size();
        meta.insert(meta.end(), it.ridx.begin(), it.ridx.end());
        meta.insert(meta.end(), it.rm.begin(), it.rm.end());
        for (const Dg& d : it.dg)
            meta.push_back(d.row);
        for (const Dg& d : it.dg)
            meta.push_back(d.rad);
        for (const Dg& d : it.dg)
            meta.push_back(d.top);
        const double per_term = loop ? (2.0 * J + 10.0 * (N / 2) + 12.0) : (2.0 * J + 24.0);
        for (int64_t q = 0; q < nt; ++q) {
            tasks.push_back(Task{(int32_t)b, (int32_t)q});
            cost.push_back((double)L * per_term);
        }
        slot += (int32_t)nt;
    }
    if (!host_object_alloc_ok())
        return report(PQ_ERR_NOMEM, "host allocation failed");
    pq_haf_plan* P = new (std::nothrow) pq_haf_plan();
    if (!P) {
        host_object_freed();
        return report(PQ_ERR_NOMEM, "host allocation failed");
    }
    P->loop = loop ? 1 : 0;
    P->batch = batch;
    if (batch == 0) {
        *out = P;
        return PQ_OK;
    }
    // longest task first
    std::vector<int64_t> order(tasks.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t x, int64_t y) { return cost[x] > cost[y]; });
    std::vector<Task> sorted(tasks.size());
    for (size_t q = 0; q < order.size(); ++q)
        sorted[q] = tasks[order[q]];
    P->ntasks = (int64_t)sorted.size();
    P->kmax = kmax;
    P->jmax = jmax;
    int rc = PQ_OK;
    if (dev_alloc((void**)&P->loopc_d, sizeof(double) * std::max<size_t>(loopc.size(), 1)) !=
            cudaSuccess ||
        dev_alloc((void**)&P->desc_d, sizeof(HafDesc) * batch) != cudaSuccess ||
        dev_alloc((void**)&P->meta_d, sizeof(int32_t) * std::max<size_t>(meta.size(), 1)) !=
            cudaSuccess ||
        dev_alloc((void**)&P->tasks_d, sizeof(Task) * sorted.size()) != cudaSuccess ||
        dev_alloc((void**)&P->part_d, sizeof(double) * 4 * std::max<int32_t>(slot, 1)) !=
            cudaSuccess ||
        dev_alloc((void**)&P->cnt_d, sizeof(int32_t) * (batch + 1)) != cudaSuccess)
        rc = report(PQ_ERR_NOMEM, "hafnian workspace allocation failed");
    if (rc == PQ_OK &&
        (cudaMemcpy(P->desc_d, desc.data(), sizeof(HafDesc) * batch, cudaMemcpyHostToDevice) !=
             cudaSuccess ||
         (!meta.empty() && cudaMemcpy(P->meta_d, meta.data(), sizeof(int32_t) * meta.size(),
                                      cudaMemcpyHostToDevice) != cudaSuccess) ||
         cudaMemcpy(P->tasks_d, sorted.data(), sizeof(Task) * sorted.size(),
                    cudaMemcpyHostToDevice) != cudaSuccess ||
         (!loopc.empty() && cudaMemcpy(P->loopc_d, loopc.data(), sizeof(double) * loopc.size(),
                                       cudaMemcpyHostToDevice) != cudaSuccess)))
        rc = report(PQ_ERR_CUDA, "hafnian upload failed");
    if (rc == PQ_OK) {
        P->per_warp = haf_warp_smem_bytes(kmax, jmax);
        int wpb = 8;
        while (wpb > 1 && wpb * P->per_warp > 227 * 1024)
            --wpb;
        const int bps = std::max(1, std::min(2, (227 * 1024) / (wpb * P->per_warp)));
        P->wpb = wpb;
        const int64_t want_blocks = (P->ntasks + wpb - 1) / wpb;
        P->blocks = (int)std::max<int64_t>(1, std::min<int64_t>(sms * bps, want_blocks));
        // raise (never lower) the dynamic shared-memory limit of the kernel
        cudaFuncAttributes at{};
        cudaError_t e = loop ? cudaFuncGetAttributes(&at, hafnian_kernel<true>)
                             : cudaFuncGetAttributes(&at, hafnian_kernel<false>);
        const int need = wpb * P->per_warp;
        if (e == cudaSuccess && at.maxDynamicSharedSizeBytes < need)
            e = loop ? cudaFuncSetAttribute(hafnian_kernel<true>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, need)
                     : cudaFuncSetAttribute(hafnian_kernel<false>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        if (e != cudaSuccess)
            rc = report(PQ_ERR_CUDA, "hafnian kernel attribute setup failed");
    }
    if (rc != PQ_OK) {
        haf_plan_free(P);
        return rc;
    }
    *out = P;
    return PQ_OK;
}

// Execution: clear the counters and launch; allocates nothing, no sync.
static int haf_plan_launch(pq_haf_plan* P, const pq_c128* mats, const pq_c128* gamma,
                           pq_c128* out, cudaStream_t st)
{
    if (P->batch == 0)
        return PQ_OK;
    if (cudaMemsetAsync(P->cnt_d, 0, sizeof(int32_t) * (P->batch + 1), st) != cudaSuccess)
        return report(PQ_ERR_CUDA, "hafnian counter reset failed");
    HafArgs a;
    a.desc = P->desc_d;
    a.meta = P->meta_d;
    a.tasks = P->tasks_d;
    a.ntasks = P->ntasks;
    a.src = reinterpret_cast<const double2*>(mats);
    a.gamma = reinterpret_cast<const double2*>(gamma);
    a.loopc = P->loopc_d;
    a.out = reinterpret_cast<double2*>(out);
    a.partials = P->part_d;
    a.counters = P->cnt_d;
    const int smem = P->wpb * P->per_warp;
    if (P->loop)
        hafnian_kernel<true><<<P->blocks, 32 * P->wpb, smem, st>>>(a, P->kmax, P->jmax);
    else
        hafnian_kernel<false><<<P->blocks, 32 * P->wpb, smem, st>>>(a, P->kmax, P->jmax);
    if (cudaGetLastError() != cudaSuccess)
        return report(PQ_ERR_CUDA, "hafnian kernel launch failed");
    return PQ_OK;
}

// The one-shot calls: plan, run, synchronise, free.
static int run_hafnians(const pq_c128* mats, const int64_t* mat_off, const int32_t* k,
                        const int32_t* rep, const int64_t* rep_off, const pq_c128* gamma,
                        int64_t batch, pq_c128* out, void* stream)
{
    if (batch > 0 && (!mats || !out))
        return report(PQ_ERR_ARG, "null argument");
    pq_haf_plan* P = nullptr;
    int rc = haf_plan_build(mat_off, k, rep, rep_off, batch, gamma != nullptr, &P);
    if (rc != PQ_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = haf_plan_launch(P, mats, gamma, out, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == PQ_OK)
        rc = report(PQ_ERR_CUDA, "hafnian kernel failed");
    haf_plan_free(P);
    return rc;
}

}  // namespace pqi

extern "C" int pq_hafnian_repeated(const pq_c128* mats, const int64_t* mat_off, const int32_t* k,
                                   const int32_t* rep, const int64_t* rep_off, int64_t batch,
                                   pq_c128* out, void* stream)
{
    return pqi::run_hafnians(mats, mat_off, k, rep, rep_off, nullptr, batch, out, stream);
}

extern "C" int pq_loop_hafnian_repeated(const pq_c128* mats, const pq_c128* gamma,
                                        const int64_t* mat_off, const int32_t* k,
                                        const int32_t* rep, const int64_t* rep_off, int64_t batch,
                                        pq_c128* out, void* stream)
{
    if (batch > 0 && !gamma)
        return pqi::report(PQ_ERR_ARG, "null gamma");
    return pqi::run_hafnians(mats, mat_off, k, rep, rep_off, gamma, batch, out, stream);
}

extern "C" int pq_loop_poly_factors(int32_t N, double* out)
{
    if (N < 0 || N > PQ_MAX_N || !out)
        return pqi::report(PQ_ERR_ARG, "N outside [0, PQ_MAX_N] or null output");
    const std::vector<double> cf = pqi::loop_factors(N);
    for (size_t i = 0; i < cf.size(); ++i)
        out[i] = cf[i];
    return PQ_OK;
}

extern "C" int pq_hafnian_plan_create(const int64_t* mat_off, const int32_t* k, const int32_t* rep,
                                      const int64_t* rep_off, int64_t batch, int32_t loop,
                                      pq_haf_plan** out)
{
    if (!out)
        return pqi::report(PQ_ERR_ARG, "null output");
    return pqi::haf_plan_build(mat_off, k, rep, rep_off, batch, loop != 0, out);
}

extern "C" int pq_hafnian_plan_run(pq_haf_plan* plan, const pq_c128* mats, const pq_c128* gamma,
                                   pq_c128* out, void* stream)
{
    if (!plan)
        return pqi::report(PQ_ERR_ARG, "null plan");
    if (plan->batch > 0 && (!mats || !out || (plan->loop && !gamma)))
        return pqi::report(PQ_ERR_ARG, "null argument");
    return pqi::haf_plan_launch(plan, mats, plan->loop ? gamma : nullptr, out,
                                (cudaStream_t)stream);
}

extern "C" int pq_hafnian_plan_destroy(pq_haf_plan* plan)
{
    if (plan) {
        cudaDeviceSynchronize();
        pqi::haf_plan_free(plan);
    }
    return PQ_OK;
}
