// pq_sampler.cu -- boson sampling by Clifford and Clifford's "Algorithm A",
// the sampler the paper uses with its permanent (Sec. 4.2, "Boson
// Sampling"), on top of the batched permanent kernel.
//
// For an input occupation s with n photons, let A be the m x n matrix of the
// columns of U of the occupied input modes (column j repeated s_j times),
// with its columns in a uniformly random order.  The sample is built one
// photon at a time: at step k (k = 1 .. n), with r_1 .. r_{k-1} already drawn,
//   w_i = |per(A[{r_1 .. r_{k-1}, i}, 1 .. k])|^2,   i = 0 .. m-1,
// and r_k is drawn with probability w_i / sum w.  The multiset {r_1 .. r_n}
// is a sample of Eq. (BS_prob).  Rows r may repeat, so every step is a batch
// of permanents with repeated rows (and repeated columns when s_j > 1): one
// persistent launch per step for all samples at once.
//
// Random numbers are inputs (column orders and one uniform per photon), so
// a caller can reproduce a run exactly.  Selection rule: with the weights
// summed in mode order, r_k is the first mode whose running sum exceeds
// u * total (the last mode with a positive weight if rounding leaves none).
#include <cuda_runtime.h>

#include <vector>

#include "../../include/pq.h"
#include "pq_kernels.h"
#include "pq_plan.h"

namespace pqi {

__global__ void sample_select_kernel(const double* w, int64_t B, int m, const double* u,
                                     int32_t* chosen)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        const double* wb = w + b * m;
        double tot = 0.0;
        for (int i = 0; i < m; ++i)
            tot += wb[i];
        const double thr = u[b] * tot;
        double run = 0.0;
        int pick = -1, last = -1;
        for (int i = 0; i < m; ++i) {
            if (wb[i] > 0.0)
                last = i;
            run += wb[i];
            if (pick < 0 && run > thr)
                pick = i;
        }
        chosen[b] = pick >= 0 ? pick : last;
    }
}

}  // namespace pqi

using namespace pqi;

extern "C" int pq_bs_sample(const pq_c128* U, int32_t m, const int32_t* input_occ,
                            int64_t nsamples, const int32_t* col_order, const double* uniforms,
                            int32_t* samples, void* stream)
{
    if (!U || !input_occ || (nsamples > 0 && (!col_order || !uniforms || !samples)))
        return report(PQ_ERR_ARG, "null argument");
    if (m <= 0 || m > PQ_MAX_DIM || nsamples < 0)
        return report(PQ_ERR_ARG, "bad sizes");
    int n = 0;
    std::vector<int32_t> cols;  // input mode of each photon column
    for (int j = 0; j < m; ++j) {
        if (input_occ[j] < 0)
            return report(PQ_ERR_ARG, "negative input occupation");
        for (int q = 0; q < input_occ[j]; ++q)
            cols.push_back(j);
        n += input_occ[j];
    }
    if (n > PQ_MAX_N)
        return report(PQ_ERR_UNSUPPORTED, "too many photons");
    for (int64_t b = 0; b < nsamples; ++b) {  // every column order is a permutation
        std::vector<char> seen(n, 0);
        for (int q = 0; q < n; ++q) {
            const int32_t c = col_order[b * n + q];
            if (c < 0 || c >= n || seen[c])
                return report(PQ_ERR_ARG, "col_order row is not a permutation of 0 .. n-1");
            seen[c] = 1;
        }
    }
    for (int64_t b = 0; b < nsamples * n; ++b)
        if (!(uniforms[b] >= 0.0 && uniforms[b] < 1.0))
            return report(PQ_ERR_ARG, "uniforms must lie in [0, 1)");
    std::vector<int32_t> occ((size_t)nsamples * m, 0);
    if (nsamples == 0 || n == 0) {
        for (size_t e = 0; e < occ.size(); ++e)
            samples[e] = 0;
        return PQ_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t B = nsamples * m;
    double *w_d = nullptr, *u_d = nullptr;
    int32_t* pick_d = nullptr;
    if (cudaMalloc((void**)&w_d, B * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&u_d, nsamples * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&pick_d, nsamples * sizeof(int32_t)) != cudaSuccess) {
        cudaFree(w_d);
        cudaFree(u_d);
        cudaFree(pick_d);
        return report(PQ_ERR_NOMEM, "sampler workspace allocation failed");
    }
    std::vector<int32_t> t((size_t)B * m), s((size_t)B * m), pick(nsamples);
    std::vector<double> u(nsamples);
    int rc = PQ_OK;
    for (int k = 1; k <= n && rc == PQ_OK; ++k) {
        // item (b, i): rows = drawn photons of sample b plus mode i; columns =
        // the input modes of sample b's first k photon columns
        for (int64_t b = 0; b < nsamples; ++b) {
            std::vector<int32_t> sc(m, 0);
            for (int q = 0; q < k; ++q)
                sc[cols[col_order[b * n + q]]] += 1;
            for (int i = 0; i < m; ++i) {
                int32_t* tb = t.data() + (size_t)(b * m + i) * m;
                int32_t* sb = s.data() + (size_t)(b * m + i) * m;
                for (int a = 0; a < m; ++a) {
                    tb[a] = occ[(size_t)b * m + a];
                    sb[a] = sc[a];
                }
                tb[i] += 1;
            }
            u[b] = uniforms[b * n + (k - 1)];
        }
        pq_plan* P = nullptr;
        rc = plan_create_occupations(m, t, s, B, &P);
        if (rc != PQ_OK)
            break;
        rc = plan_run_forward(P, U, nullptr, w_d, st);
        if (rc == PQ_OK) {
            if (cudaMemcpyAsync(u_d, u.data(), nsamples * sizeof(double), cudaMemcpyHostToDevice,
                                st) != cudaSuccess)
                rc = report(PQ_ERR_CUDA, "uniform upload failed");
        }
        if (rc == PQ_OK) {
            const unsigned blocks = (unsigned)((nsamples + 127) / 128 < 1024 ? (nsamples + 127) / 128 : 1024);
            sample_select_kernel<<<blocks, 128, 0, st>>>(w_d, nsamples, m, u_d, pick_d);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(pick.data(), pick_d, nsamples * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                rc = report(PQ_ERR_CUDA, "sampling step failed");
        }
        pq_plan_destroy(P);
        for (int64_t b = 0; b < nsamples && rc == PQ_OK; ++b) {
            if (pick[b] < 0) {
                rc = report(PQ_ERR_ARG, "all weights of a sampling step are zero");
                break;
            }
            occ[(size_t)b * m + pick[b]] += 1;
        }
    }
    cudaFree(w_d);
    cudaFree(u_d);
    cudaFree(pick_d);
    if (rc == PQ_OK)
        for (size_t e = 0; e < occ.size(); ++e)
            samples[e] = occ[e];
    return rc;
}
