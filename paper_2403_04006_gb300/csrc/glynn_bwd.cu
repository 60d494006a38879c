// glynn_bwd.cu -- gradient of the permanent with respect to the base matrix,
// in the same Gray-code pass as the permanent itself.
//
// With per = 2^{-(n-1)} sum_t w_t prod_j S_j(t)^{c_j} and
// S_j = sum_i x_i b_ij, x_i = r_i - 2 g_i, the derivative is
//   G_ij = d per / d b_ij = 2^{-(n-1)} sum_t w_t x_i(t) Q_j(t),
//   Q_j  = c_j S_j^{c_j - 1} prod_{j' != j} S_{j'}^{c_{j'}},
// which counts every copy of b_ij in the expanded matrix.  Q_j comes from
// prefix and suffix products of the column sums (no division, so S_j = 0 is
// harmless).
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
#include <cuda_runtime.h>

#include "pq_device.cuh"
#include "pq_kernels.h"

namespace pqi {

__host__ __device__ inline int bwd_warp_smem_bytes(int kmax, int lmax, int jb)
{
    long bytes = 16L * (kmax * lmax + lmax + 64L * lmax + 32L * jb * lmax) + 8L * 32 +
                 4L * (32L * kmax + 16 + lmax + kmax);
    return (int)((bytes + 15) & ~15L);
}

template <int LMAX>
struct BwdSmem {
    double2* M;       // kmax x LMAX
    double2* base;    // LMAX
    double2* A;       // LMAX x 32 (lane-major)
    double2* P;       // LMAX x 32
    double2* C;       // JB x LMAX x 32
    double* wh;       // 32
    int32_t* x;       // kmax x 32
    int32_t* lowrow;  // 16
    int32_t* cm;      // LMAX
    int32_t* rowdig;  // kmax: low digit of each row, or -1
    __device__ BwdSmem(unsigned char* raw, int kmax, int jb)
    {
        M = reinterpret_cast<double2*>(raw);
        base = M + kmax * LMAX;
        A = base + LMAX;
        P = A + LMAX * 32;
        C = P + LMAX * 32;
        wh = reinterpret_cast<double*>(C + jb * LMAX * 32);
        x = reinterpret_cast<int32_t*>(wh + 32);
        lowrow = x + kmax * 32;
        cm = lowrow + 16;
        rowdig = cm + LMAX;
    }
};

// A_j +-= w Q_j for the current column sums (prefix products kept in P).
template <int LMAX, bool NEG>
__device__ __forceinline__ void bwd_term(const double2 (&S)[LMAX], int l, int n,
                                         const int32_t* cm, double w, double2* P, double2* A,
                                         int lane)
{
    const double ws = NEG ? -w : w;
    if (n == 1) {  // per = b: dper/db = 1
        double2 a = A[lane];
        a.x = __dadd_rn(a.x, ws);
        A[lane] = a;
        return;
    }
    // prefix: P_j = prod_{j' < j} S_{j'}^{c_{j'}}
    double2 run = make_double2(1.0, 0.0);
#pragma unroll
    for (int j = 0; j < LMAX; ++j) {
        if (j < l) {
            if (j > 0)
                P[j * 32 + lane] = run;
            const int c = cm[j];
            int e0 = 0;
            if (j == 0) {
                run = S[0];
                e0 = 1;
            }
            for (int e = e0; e < c; ++e)
                run = cmul(run, S[j]);
        }
    }
    // suffix pass: Q_j = c_j S_j^{c_j-1} P_j Sf_j, Sf_j = prod_{j' > j} S_{j'}^{c_{j'}}
    double2 sf = make_double2(1.0, 0.0);
    bool sf_one = true;
#pragma unroll
    for (int j = LMAX - 1; j >= 0; --j) {
        if (j < l) {
            const int c = cm[j];
            double2 q;
            bool q_one;
            if (j == 0) {
                q = sf;
                q_one = sf_one;
            } else {
                q = P[j * 32 + lane];
                q_one = false;
                if (!sf_one)
                    q = cmul(q, sf);
            }
            for (int e = 1; e < c; ++e) {
                if (q_one) {
                    q = S[j];
                    q_one = false;
                } else {
                    q = cmul(q, S[j]);
                }
            }
            double2 a = A[j * 32 + lane];
            const double wc = (c > 1) ? ws * (double)c : ws;
            if (q_one) {
                a.x = __dadd_rn(a.x, wc);
            } else {
                a.x = __fma_rn(wc, q.x, a.x);
                a.y = __fma_rn(wc, q.y, a.y);
            }
            A[j * 32 + lane] = a;
            if (j > 0) {
                for (int e = 0; e < c; ++e) {
                    if (sf_one) {
                        sf = S[j];
                        sf_one = false;
                    } else {
                        sf = cmul(sf, S[j]);
                    }
                }
            }
        }
    }
}

template <int LMAX>
__device__ void bwd_stage(const BwdArgs& a, const PermDesc& D, const MetaView& mv,
                          BwdSmem<LMAX>& sm, int lane)
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
            double r = (double)mv.rmul[i];
            double2 b = sm.M[i * LMAX + j];
            s.x = __fma_rn(r, b.x, s.x);
            s.y = __fma_rn(r, b.y, s.y);
        }
        sm.base[j] = s;
    }
    __syncwarp();
}

template <int LMAX>
__device__ void bwd_task(const BwdArgs& a, const Task& t, BwdSmem<LMAX>& sm, int& staged,
                         int lane, int jb)
{
    const PermDesc D = a.desc[t.perm];
    const MetaView mv = meta_view(a.meta, D);
    const int k = D.k, l = D.l, n = D.n, J = D.J, ndig = D.ndig;
    const int kl = k * l;
    double* slot = a.gpart + 2 * (a.gpart_off[t.perm] + (int64_t)t.part * kl);

    if (D.trivial) {
        // nothing depends on the matrix: zero gradient
        for (int e = lane; e < kl; e += kWarp) {
            slot[2 * e] = 0.0;
            slot[2 * e + 1] = 0.0;
        }
    } else {
        if (staged != t.perm) {
            __syncwarp();
            bwd_stage<LMAX>(a, D, mv, sm, lane);
            staged = t.perm;
        }
        const int64_t chunk0 = (int64_t)t.part * kWarp;
        const bool active = chunk0 + lane < D.nchunks;
        int64_t c = active ? (chunk0 + lane) : 0;
        double2 S[LMAX];
#pragma unroll
        for (int j = 0; j < LMAX; ++j)
            S[j] = (j < l) ? sm.base[j] : make_double2(0.0, 0.0);
        for (int i = 0; i < k; ++i)
            sm.x[i * 32 + lane] = mv.rmul[i];
        uint64_t whigh_u = 1;
        int gpar = 0;
        for (int d = J; d < ndig; ++d) {
            int rad = mv.drad[d];
            int g = (int)(c % rad);
            c /= rad;
            const int row = mv.drow[d];
            const double2* Mr = sm.M + row * LMAX;
            const double coef = -2.0 * (double)g;
#pragma unroll
            for (int j = 0; j < LMAX; ++j) {
                if (j < l) {
                    double2 b = Mr[j];
                    S[j].x = __fma_rn(coef, b.x, S[j].x);
                    S[j].y = __fma_rn(coef, b.y, S[j].y);
                }
            }
            sm.x[row * 32 + lane] = mv.rmul[row] - 2 * g;
            if (g) {
                whigh_u *= binom_u64(mv.dtop[d], g);
                gpar += g;
            }
        }
        double whigh = active ? (double)whigh_u : 0.0;
        if (gpar & 1)
            whigh = -whigh;
        sm.wh[lane] = whigh;
        for (int j = 0; j < l; ++j)
            sm.A[j * 32 + lane] = make_double2(0.0, 0.0);
        for (int e = 0; e < J * l; ++e) {
            const int d = e / l, j = e - d * l;
            sm.C[(d * LMAX + j) * 32 + lane] = make_double2(0.0, 0.0);
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
        double wlow = 1.0;
        const int64_t L = D.L;
        for (int64_t s = 0; s < L; ++s) {
            if (s & 1)
                bwd_term<LMAX, true>(S, l, n, sm.cm, wlow, sm.P, sm.A, lane);
            else
                bwd_term<LMAX, false>(S, l, n, sm.cm, wlow, sm.P, sm.A, lane);
            if (s + 1 < L) {
                int up;
                const int d = low_step(wk, up);
                const int row = sm.lowrow[d];
                const double delta = up > 0 ? -2.0 : 2.0;
                const double2* Mr = sm.M + row * LMAX;
                double2* Cd = sm.C + d * LMAX * 32;
#pragma unroll
                for (int j = 0; j < LMAX; ++j) {
                    if (j < l) {
                        double2 b = Mr[j];
                        S[j].x = __fma_rn(delta, b.x, S[j].x);
                        S[j].y = __fma_rn(delta, b.y, S[j].y);
                        double2 av = sm.A[j * 32 + lane];
                        double2 cv = Cd[j * 32 + lane];
                        cv.x = __fma_rn(delta, av.x, cv.x);
                        cv.y = __fma_rn(delta, av.y, cv.y);
                        Cd[j * 32 + lane] = cv;
                    }
                }
                sm.x[row * 32 + lane] += (up > 0 ? -2 : 2);
                if (((wk.radm1 >> (4 * d)) & 15u) > 1u)
                    wlow = (double)low_weight(wk, J);
            }
        }
        __syncwarp();
        // lane-parallel contraction: entry e = (i, j) summed over the 32 lanes in order
        for (int e = lane; e < kl; e += kWarp) {
            const int i = e / l, j = e - i * l;
            const int dg = sm.rowdig[i];
            double gx = 0.0, gy = 0.0;
            for (int q = 0; q < 32; ++q) {
                const double2 av = sm.A[j * 32 + q];
                const double xv = (double)sm.x[i * 32 + q];
                double tx = xv * av.x, ty = xv * av.y;
                if (dg >= 0) {
                    const double2 cv = sm.C[(dg * LMAX + j) * 32 + q];
                    tx -= cv.x;
                    ty -= cv.y;
                }
                gx = __fma_rn(sm.wh[q], tx, gx);
                gy = __fma_rn(sm.wh[q], ty, gy);
            }
            slot[2 * e] = gx;
            slot[2 * e + 1] = gy;
        }
    }

    // ---- combine the tasks of this permanent
    int last = 1;
    if (D.ntasks > 1) {
        __threadfence();  // every lane's slot entries, before the count
        __syncwarp();
        if (lane == 0) {
            int old = atomicAdd(a.counters + 1 + t.perm, 1);
            last = (old == D.ntasks - 1);
        }
        __syncwarp();
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
        if (!D.trivial) {
            gx = scalbn(gx, 1 - n);
            gy = scalbn(gy, 1 - n);
        }
        // grad_b = coef * conj(G)
        outg[e] = make_double2(coef.x * gx + coef.y * gy, coef.y * gx - coef.x * gy);
    }
}

template <int LMAX>
__global__ void __launch_bounds__(256) glynn_bwd_persistent(BwdArgs a, int kmax, int jb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    BwdSmem<LMAX> sm(smem_raw + warp * bwd_warp_smem_bytes(kmax, LMAX, jb), kmax, jb);
    int staged = -1;
    for (;;) {
        int ti = 0;
        if (lane == 0)
            ti = atomicAdd(a.counters, 1);
        ti = __shfl_sync(0xffffffffu, ti, 0);
        if (ti >= a.ntasks)
            break;
        Task t = a.tasks[ti];
        bwd_task<LMAX>(a, t, sm, staged, lane, jb);
    }
}

template <int LMAX>
__global__ void __launch_bounds__(256) glynn_bwd_plain(BwdArgs a, int64_t t_begin, int64_t t_end,
                                                       int kmax, int jb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    BwdSmem<LMAX> sm(smem_raw + warp * bwd_warp_smem_bytes(kmax, LMAX, jb), kmax, jb);
    int staged = -1;
    int64_t ti = t_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (ti >= t_end)
        return;
    Task t = a.tasks[ti];
    bwd_task<LMAX>(a, t, sm, staged, lane, jb);
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

// Boson sampling: grad_U[a][c] = sum over patterns (in order) of the entry of
// that pattern's gradient that U[a][c] became.
__global__ void scatter_bs_kernel(const PermDesc* desc, const int32_t* meta, int64_t nperm, int m,
                                  const double2* gl, const int64_t* gl_off, double2* gU)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
        const int ar = e / m, ac = e - ar * m;  // U row (output mode), column (input mode)
        double gx = 0.0, gy = 0.0;
        for (int64_t p = 0; p < nperm; ++p) {
            const PermDesc D = desc[p];
            if (D.trivial)
                continue;
            const MetaView mv = meta_view(meta, D);
            // source element (ar, ac) sits at ar * m + ac = ridx*si + cidx*sj
            int io = -1, jo = -1;
            const int want_i = (D.si == 1) ? ac : ar;  // transposed: summed side is columns
            const int want_j = (D.si == 1) ? ar : ac;
            for (int i = 0; i < D.k; ++i)
                if (mv.ridx[i] == want_i)
                    io = i;
            if (io < 0)
                continue;
            for (int j = 0; j < D.l; ++j)
                if (mv.cidx[j] == want_j)
                    jo = j;
            if (jo < 0)
                continue;
            const double2 v = gl[gl_off[p] + io * D.l + jo];
            gx += v.x;
            gy += v.y;
        }
        gU[e] = make_double2(gx, gy);
    }
}

// ---------------------------------------------------------------- host side
int bwd_smem_per_warp(int kmax, int lmax) { return bwd_warp_smem_bytes(kmax, lmax, kMaxLowDigits); }

static const int g_bwd_jb = kBwdMaxLowDigits;

template <int LMAX>
static cudaError_t bwd_attrs(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(glynn_bwd_persistent<LMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(glynn_bwd_plain<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                bytes);
}

cudaError_t bwd_prepare(int lmax, int smem_bytes)
{
    switch (lmax) {
    case 8: return bwd_attrs<8>(smem_bytes);
    case 16: return bwd_attrs<16>(smem_bytes);
    case 24: return bwd_attrs<24>(smem_bytes);
    case 32: return bwd_attrs<32>(smem_bytes);
    case 40: return bwd_attrs<40>(smem_bytes);
    default: return cudaErrorInvalidValue;
    }
}

int bwd_smem_bytes_for(int kmax, int lmax, int jb) { return bwd_warp_smem_bytes(kmax, lmax, jb); }

cudaError_t bwd_launch_persistent(int lmax, const BwdArgs& a, int kmax, int blocks, int wpb,
                                  cudaStream_t st)
{
    const int jb = g_bwd_jb;
    const int smem = wpb * bwd_warp_smem_bytes(kmax, lmax, jb);
    const dim3 grid(blocks), block(32 * wpb);
    switch (lmax) {
    case 8: glynn_bwd_persistent<8><<<grid, block, smem, st>>>(a, kmax, jb); break;
    case 16: glynn_bwd_persistent<16><<<grid, block, smem, st>>>(a, kmax, jb); break;
    case 24: glynn_bwd_persistent<24><<<grid, block, smem, st>>>(a, kmax, jb); break;
    case 32: glynn_bwd_persistent<32><<<grid, block, smem, st>>>(a, kmax, jb); break;
    case 40: glynn_bwd_persistent<40><<<grid, block, smem, st>>>(a, kmax, jb); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t bwd_launch_plain(int lmax, const BwdArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                             int wpb, cudaStream_t st)
{
    const int jb = g_bwd_jb;
    const int smem = wpb * bwd_warp_smem_bytes(kmax, lmax, jb);
    const int64_t nt = t_end - t_begin;
    const dim3 grid((unsigned)((nt + wpb - 1) / wpb)), block(32 * wpb);
    switch (lmax) {
    case 8: glynn_bwd_plain<8><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax, jb); break;
    case 16: glynn_bwd_plain<16><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax, jb); break;
    case 24: glynn_bwd_plain<24><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax, jb); break;
    case 32: glynn_bwd_plain<32><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax, jb); break;
    case 40: glynn_bwd_plain<40><<<grid, block, smem, st>>>(a, t_begin, t_end, kmax, jb); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t scatter_grad_batch(const PermDesc* desc, const int32_t* meta, int64_t nperm,
                               const double2* grad_local, const int64_t* grad_local_off,
                               const int64_t* item_mat_off, const int32_t* item_l,
                               const int32_t* item_k, double2* grad_mats, int64_t total_elems,
                               cudaStream_t st)
{
    (void)total_elems;
    if (nperm == 0)
        return cudaSuccess;
    scatter_batch_kernel<<<(unsigned)nperm, 128, 0, st>>>(desc, meta, grad_local, grad_local_off,
                                                          item_mat_off, item_k, item_l, grad_mats);
    return cudaGetLastError();
}

cudaError_t scatter_grad_bs(const PermDesc* desc, const int32_t* meta, int64_t nperm, int32_t m,
                            const double2* grad_local, const int64_t* grad_local_off,
                            double2* grad_U, cudaStream_t st)
{
    const int threads = 128;
    const int blocks = (m * m + threads - 1) / threads;
    scatter_bs_kernel<<<blocks, threads, 0, st>>>(desc, meta, nperm, m, grad_local, grad_local_off,
                                                  grad_U);
    return cudaGetLastError();
}

}  // namespace pqi
