// clements.cu -- beamsplitter mesh U(theta, phi) and its adjoint.
//
// Beamsplitter k acts on modes (j, j+1) with the block [[t, -conj(r)], [r, t]],
// t = cos theta_k, r = exp(i phi_k) sin theta_k (paper Appendix A,
// "Beamsplitter gate").  Mesh: m layers, layer q on pairs j = q mod 2,
// q mod 2 + 2, ...; numbering layer by layer, j ascending; U = T_{L-1}..T_0.
//
// Forward: U starts as the identity in shared memory; each layer updates the
// two rows of every pair (pairs of one layer are disjoint, so a layer is one
// parallel step).  Both kernels first take sin and cos of every angle once
// into shared memory: a beamsplitter's block is used for every row or column
// it touches, and FP64 sincos is dear on this GPU.
//
// Adjoint: with G = dL/dRe U + i dL/dIm U and W = G U^H,
//   dL/dtheta_k = Re sum_{a,b in pair} conj((W_k T_k)_ab) (dT_k/dtheta)_ab,
//   W_{k-1} = T_k^H W_k T_k,
// walking the layers backwards.  Beamsplitters of one layer act on disjoint
// modes, so their 2 x 2 blocks of W are unaffected by each other and a whole
// layer is handled in one step.
#include <cuda_runtime.h>

#include "pq_kernels.h"

namespace pqi {

__device__ __forceinline__ int layer_count(int q, int m) { return (q & 1) ? (m - 1) / 2 : m / 2; }

__device__ __forceinline__ double2 c_mul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_conj(double2 a) { return make_double2(a.x, -a.y); }

struct Blk {
    double2 a00, a01, a10, a11;
};

// cos theta_k, sin theta_k, cos phi_k, sin phi_k of every beamsplitter, at
// trig[4k .. 4k+3].
__device__ void load_trig(const double* theta, const double* phi, int L, double* trig)
{
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        double s, c, sp, cp;
        sincos(theta[k], &s, &c);
        sincos(phi[k], &sp, &cp);
        trig[4 * k + 0] = c;
        trig[4 * k + 1] = s;
        trig[4 * k + 2] = cp;
        trig[4 * k + 3] = sp;
    }
}

__device__ __forceinline__ Blk bs_block(const double* trig, int k)
{
    const double c = trig[4 * k], s = trig[4 * k + 1], cp = trig[4 * k + 2], sp = trig[4 * k + 3];
    Blk b;
    b.a00 = make_double2(c, 0.0);
    b.a01 = make_double2(-cp * s, sp * s);  // -conj(e^{i phi} sin)
    b.a10 = make_double2(cp * s, sp * s);   // e^{i phi} sin
    b.a11 = make_double2(c, 0.0);
    return b;
}

__global__ void __launch_bounds__(256) clements_fwd_kernel(const double* theta, const double* phi,
                                                           int m, double2* U)
{
    extern __shared__ double2 sh[];  // m x m, then the angles' sin and cos
    double* trig = reinterpret_cast<double*>(sh + m * m);
    load_trig(theta, phi, m * (m - 1) / 2, trig);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x)
        sh[e] = make_double2((e / m == e % m) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    int kbase = 0;
    for (int q = 0; q < m; ++q) {
        const int np = layer_count(q, m);
        for (int w = threadIdx.x; w < np * m; w += blockDim.x) {
            const int pi = w / m, col = w - pi * m;
            const int j = (q & 1) + 2 * pi;
            const Blk b = bs_block(trig, kbase + pi);
            const double2 u0 = sh[j * m + col], u1 = sh[(j + 1) * m + col];
            sh[j * m + col] = c_add(c_mul(b.a00, u0), c_mul(b.a01, u1));
            sh[(j + 1) * m + col] = c_add(c_mul(b.a10, u0), c_mul(b.a11, u1));
        }
        kbase += np;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x)
        U[e] = sh[e];
}

__global__ void __launch_bounds__(256) clements_adj_kernel(const double* theta, const double* phi,
                                                           int m, const double2* U,
                                                           const double2* G, double* gtheta,
                                                           double* gphi)
{
    extern __shared__ double2 W[];  // m x m, then the angles' sin and cos
    double* trig = reinterpret_cast<double*>(W + m * m);
    load_trig(theta, phi, m * (m - 1) / 2, trig);
    // W = G U^H
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int a = e / m, b = e - a * m;
        double2 s = make_double2(0.0, 0.0);
        for (int c = 0; c < m; ++c)
            s = c_add(s, c_mul(G[a * m + c], c_conj(U[b * m + c])));
        W[e] = s;
    }
    __syncthreads();
    int kend = m * (m - 1) / 2;
    for (int q = m - 1; q >= 0; --q) {
        const int np = layer_count(q, m);
        const int kbase = kend - np;
        // gradients of this layer from the 2 x 2 blocks of W T
        for (int pi = threadIdx.x; pi < np; pi += blockDim.x) {
            const int j = (q & 1) + 2 * pi;
            const Blk b = bs_block(trig, kbase + pi);
            const double2 w00 = W[j * m + j], w01 = W[j * m + j + 1];
            const double2 w10 = W[(j + 1) * m + j], w11 = W[(j + 1) * m + j + 1];
            // M = Wblk * Blk
            const double2 m00 = c_add(c_mul(w00, b.a00), c_mul(w01, b.a10));
            const double2 m01 = c_add(c_mul(w00, b.a01), c_mul(w01, b.a11));
            const double2 m10 = c_add(c_mul(w10, b.a00), c_mul(w11, b.a10));
            const double2 m11 = c_add(c_mul(w10, b.a01), c_mul(w11, b.a11));
            const double c = trig[4 * (kbase + pi)], s = trig[4 * (kbase + pi) + 1];
            const double cp = trig[4 * (kbase + pi) + 2], sp = trig[4 * (kbase + pi) + 3];
            // dT/dtheta = [[-s, -e^{-i phi} c], [e^{i phi} c, -s]]
            const double2 t00 = make_double2(-s, 0.0), t01 = make_double2(-cp * c, sp * c);
            const double2 t10 = make_double2(cp * c, sp * c), t11 = make_double2(-s, 0.0);
            // dT/dphi = [[0, i e^{-i phi} s], [i e^{i phi} s, 0]]
            const double2 p01 = make_double2(sp * s, cp * s), p10 = make_double2(-sp * s, cp * s);
            double gt = c_mul(c_conj(m00), t00).x + c_mul(c_conj(m01), t01).x +
                        c_mul(c_conj(m10), t10).x + c_mul(c_conj(m11), t11).x;
            double gp = c_mul(c_conj(m01), p01).x + c_mul(c_conj(m10), p10).x;
            gtheta[kbase + pi] = gt;
            gphi[kbase + pi] = gp;
        }
        __syncthreads();
        // W <- W T (columns j, j+1 of every row)
        for (int w = threadIdx.x; w < np * m; w += blockDim.x) {
            const int pi = w / m, row = w - pi * m;
            const int j = (q & 1) + 2 * pi;
            const Blk b = bs_block(trig, kbase + pi);
            const double2 x0 = W[row * m + j], x1 = W[row * m + j + 1];
            W[row * m + j] = c_add(c_mul(x0, b.a00), c_mul(x1, b.a10));
            W[row * m + j + 1] = c_add(c_mul(x0, b.a01), c_mul(x1, b.a11));
        }
        __syncthreads();
        // W <- T^H W (rows j, j+1 of every column)
        for (int w = threadIdx.x; w < np * m; w += blockDim.x) {
            const int pi = w / m, col = w - pi * m;
            const int j = (q & 1) + 2 * pi;
            const Blk b = bs_block(trig, kbase + pi);
            const double2 y0 = W[j * m + col], y1 = W[(j + 1) * m + col];
            // (T^H)_{00} = conj(a00), (T^H)_{01} = conj(a10), (T^H)_{10} = conj(a01), (T^H)_{11} = conj(a11)
            W[j * m + col] = c_add(c_mul(c_conj(b.a00), y0), c_mul(c_conj(b.a10), y1));
            W[(j + 1) * m + col] = c_add(c_mul(c_conj(b.a01), y0), c_mul(c_conj(b.a11), y1));
        }
        __syncthreads();
        kend = kbase;
    }
}

static bool g_attr_set = false;

static cudaError_t ensure_attrs()
{
    if (g_attr_set)
        return cudaSuccess;
    const int bytes = 64 * 64 * 16 + 32 * (64 * 63 / 2);  // m <= 64: U or W, and the angles
    cudaError_t e = cudaFuncSetAttribute(clements_fwd_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(clements_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 bytes);
    if (e == cudaSuccess)
        g_attr_set = true;
    return e;
}

cudaError_t clements_forward(const double* theta, const double* phi, int m, double2* U,
                             cudaStream_t st)
{
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess)
        return e;
    clements_fwd_kernel<<<1, 256, m * m * 16 + 32 * (m * (m - 1) / 2), st>>>(theta, phi, m, U);
    return cudaGetLastError();
}

cudaError_t clements_backward(const double* theta, const double* phi, int m, const double2* U,
                              const double2* gU, double* gtheta, double* gphi, cudaStream_t st)
{
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess)
        return e;
    clements_adj_kernel<<<1, 256, m * m * 16 + 32 * (m * (m - 1) / 2), st>>>(theta, phi, m, U, gU,
                                                                          gtheta, gphi);
    return cudaGetLastError();
}

}  // namespace pqi
