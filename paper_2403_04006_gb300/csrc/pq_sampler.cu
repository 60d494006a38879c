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
// is a sample of Eq. (BS_prob).
//
// Expanding each permanent along its last row,
//   per(A[{r, i}, 1 .. k]) = sum_{j <= k} A[i, j] per(M_j),
//   M_j = A[{r_1 .. r_{k-1}}, {1 .. k} \ {j}],
// so a step needs k permanents of size k - 1 per sample, not m of size k.
// Every step runs on the device without the host: a gather kernel builds the
// minors from the rows drawn so far (repeated rows stay separate rows, so
// all minors of a step have one shape and the step's plan is made once,
// before the first step), one persistent launch evaluates them, a kernel
// forms the m weights of every sample and draws its photon.  The host reads
// the drawn modes back once, after the last step.
//
// Random numbers are inputs (column orders and one uniform per photon), so
// a caller can reproduce a run exactly.  Selection rule: with the weights
// summed in mode order, r_k is the first mode whose running sum exceeds
// u * total (the last mode with a positive weight if rounding leaves none).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pq.h"
#include "pq_kernels.h"
#include "pq_plan.h"

namespace pqi {

// Minors of step k: item (b, j) is A_b[{r_1 .. r_{k-1}}, {c_0 .. c_{k-1}} \ {c_j}],
// (k-1) x (k-1) row-major at (b k + j) (k-1)^2.  cols[b n + q] is the input
// mode of sample b's q-th photon column, drawn[b n + p] its p-th drawn mode.
__global__ void sampler_gather_kernel(const double2* U, int m, int n, int k, int64_t nsamples,
                                      const int32_t* cols, const int32_t* drawn, double2* mats)
{
    const int d = k - 1;
    const int64_t total = nsamples * k * d * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t item = e / (d * d);
        const int rem = (int)(e - item * d * d);
        const int p = rem / d, q = rem - p * d;
        const int64_t b = item / k;
        const int j = (int)(item - b * k);
        const int qq = q < j ? q : q + 1;
        const int row = drawn[b * n + p];
        const int col = cols[b * n + qq];
        mats[e] = U[(int64_t)row * m + col];
    }
}

// Weights of step k, w_i = |sum_j U[i, c_j] per_j|^2 (per_j = 1 for k = 1),
// and the draw: the first mode whose running weight sum exceeds u * total,
// else the last mode with a positive weight; a sample whose weights are all
// zero records an error and draws mode 0 so that later steps stay in bounds.
__global__ void sampler_step_kernel(const double2* U, int m, int n, int k, int64_t nsamples,
                                    const int32_t* cols, const double2* per, const double* uniforms,
                                    double* w, int32_t* drawn, int32_t* err)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nsamples;
         b += (int64_t)gridDim.x * blockDim.x) {
        double* wb = w + b * m;
        double tot = 0.0;
        for (int i = 0; i < m; ++i) {
            double2 z = make_double2(0.0, 0.0);
            for (int j = 0; j < k; ++j) {
                const double2 a = U[(int64_t)i * m + cols[b * n + j]];
                const double2 pj = (k == 1) ? make_double2(1.0, 0.0) : per[b * k + j];
                z.x = __fma_rn(a.x, pj.x, z.x);
                z.x = __fma_rn(-a.y, pj.y, z.x);
                z.y = __fma_rn(a.x, pj.y, z.y);
                z.y = __fma_rn(a.y, pj.x, z.y);
            }
            const double wi = z.x * z.x + z.y * z.y;
            wb[i] = wi;
            tot += wi;
        }
        const double thr = uniforms[b * n + (k - 1)] * tot;
        double run = 0.0;
        int pick = -1, last = -1;
        for (int i = 0; i < m; ++i) {
            if (wb[i] > 0.0)
                last = i;
            run += wb[i];
            if (pick < 0 && run > thr)
                pick = i;
        }
        if (pick < 0)
            pick = last;
        if (pick < 0) {
            atomicExch(err, 1);
            pick = 0;
        }
        drawn[b * n + (k - 1)] = pick;
    }
}

}  // namespace pqi

// A planned sampler: the plan of every step's minors (made once, by host
// threads side by side), the photon columns' input modes and the device
// workspace.  A run uploads the draws, runs the steps and reads the samples.
struct pq_sampler_plan {
    int32_t m = 0, n = 0;
    int64_t nsamples = 0;
    std::vector<int32_t> modes;   // input mode of each photon column
    std::vector<pq_plan*> plans;  // index k = 2 .. n
    double2 *mats_d = nullptr, *per_d = nullptr;
    double *w_d = nullptr, *u_d = nullptr;
    int32_t *cols_d = nullptr, *drawn_d = nullptr, *err_d = nullptr;
    std::vector<int32_t> cols_h, drawn_h;  // host staging of one run
};

namespace pqi {

static void sampler_plan_free(pq_sampler_plan* S)
{
    if (!S)
        return;
    for (pq_plan* P : S->plans)
        if (P)
            pq_plan_destroy(P);
    dev_free(S->mats_d);
    dev_free(S->per_d);
    dev_free(S->w_d);
    dev_free(S->u_d);
    dev_free(S->cols_d);
    dev_free(S->drawn_d);
    dev_free(S->err_d);
    delete S;
    host_object_freed();
}

static int sampler_plan_build(int32_t m, const int32_t* input_occ, int64_t nsamples,
                              pq_sampler_plan** out)
{
    *out = nullptr;
    if (!input_occ)
        return report(PQ_ERR_ARG, "null argument");
    if (m <= 0 || m > PQ_MAX_DIM || nsamples < 0)
        return report(PQ_ERR_ARG, "bad sizes");
    int n = 0;
    std::vector<int32_t> modes;
    for (int j = 0; j < m; ++j) {
        if (input_occ[j] < 0)
            return report(PQ_ERR_ARG, "negative input occupation");
        for (int q = 0; q < input_occ[j]; ++q)
            modes.push_back(j);
        n += input_occ[j];
    }
    if (n > PQ_MAX_N)
        return report(PQ_ERR_UNSUPPORTED, "too many photons");
    if (n > 0 && nsamples > (int64_t(1) << 40) / ((int64_t)n * n * n + m))
        return report(PQ_ERR_UNSUPPORTED, "sampler workspace too large");
    if (!host_object_alloc_ok())
        return report(PQ_ERR_NOMEM, "host allocation failed");
    pq_sampler_plan* S = new (std::nothrow) pq_sampler_plan();
    if (!S) {
        host_object_freed();
        return report(PQ_ERR_NOMEM, "host allocation failed");
    }
    S->m = m;
    S->n = n;
    S->nsamples = nsamples;
    S->modes = modes;
    S->plans.assign(n + 1, nullptr);
    if (nsamples == 0 || n == 0) {
        *out = S;
        return PQ_OK;
    }

    // one plan per step k >= 2: nsamples * k minors of size k - 1, every
    // multiplicity one, item (b, j) at element offset (b k + j) (k-1)^2.  The
    // plans are independent, so host threads build them side by side.
    std::vector<int> prc(n + 1, PQ_OK);
    std::vector<std::string> perr(n + 1);
    std::atomic<int> next_k(2);
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        sampler_plan_free(S);
        return report(PQ_ERR_CUDA, "no current CUDA device");
    }
    auto worker = [&]() {
        cudaSetDevice(device);  // a new host thread starts on device 0
        for (int k = next_k++; k <= n; k = next_k++) {
            const int d = k - 1;
            const int64_t B = nsamples * k;
            std::vector<int64_t> mat_off(B), zero_off(B, 0);
            std::vector<int32_t> dim(B, d), ones(d, 1);
            for (int64_t q = 0; q < B; ++q)
                mat_off[q] = q * d * d;
            pq_batch_sizes sz;
            sz.batch = B;
            sz.mat_off = mat_off.data();
            sz.k = dim.data();
            sz.l = dim.data();
            sz.row_mult = ones.data();
            sz.row_off = zero_off.data();
            sz.col_mult = ones.data();
            sz.col_off = zero_off.data();
            prc[k] = pq_plan_create(&sz, nullptr, &S->plans[k]);
            if (prc[k] != PQ_OK)
                perr[k] = pq_last_error();
        }
    };
    {
        const int nthreads = std::max(1, std::min(n - 1, 16));
        std::vector<std::thread> pool;
        for (int q = 1; q < nthreads; ++q)
            pool.emplace_back(worker);
        worker();
        for (std::thread& th : pool)
            th.join();
    }
    int rc = PQ_OK;
    for (int k = 2; k <= n && rc == PQ_OK; ++k)
        if (prc[k] != PQ_OK)
            rc = report(prc[k], perr[k].c_str());
    // Plans made side by side may have raised the kernel's shared-memory
    // limit out of order: raise it once more for each, in turn.
    for (int k = 2; k <= n && rc == PQ_OK; ++k)
        if (plan_prepare_forward(S->plans[k]) != PQ_OK)
            rc = report(PQ_ERR_CUDA, "kernel attribute setup failed");
    const int64_t Bmax = nsamples * n;
    const int64_t mat_elems = std::max<int64_t>(1, nsamples * n * (int64_t)(n - 1) * (n - 1));
    if (rc == PQ_OK &&
        (dev_alloc((void**)&S->mats_d, mat_elems * sizeof(double2)) != cudaSuccess ||
         dev_alloc((void**)&S->per_d, Bmax * sizeof(double2)) != cudaSuccess ||
         dev_alloc((void**)&S->w_d, nsamples * m * sizeof(double)) != cudaSuccess ||
         dev_alloc((void**)&S->u_d, nsamples * n * sizeof(double)) != cudaSuccess ||
         dev_alloc((void**)&S->cols_d, nsamples * n * sizeof(int32_t)) != cudaSuccess ||
         dev_alloc((void**)&S->drawn_d, nsamples * n * sizeof(int32_t)) != cudaSuccess ||
         dev_alloc((void**)&S->err_d, sizeof(int32_t)) != cudaSuccess))
        rc = report(PQ_ERR_NOMEM, "sampler workspace allocation failed");
    if (rc != PQ_OK) {
        sampler_plan_free(S);
        return rc;
    }
    S->cols_h.resize((size_t)nsamples * n);
    S->drawn_h.resize((size_t)nsamples * n);
    *out = S;
    return PQ_OK;
}

// One run: check and upload the draws, the steps, read the drawn modes back
// (synchronises `st`) and count them into samples.
static int sampler_plan_launch(pq_sampler_plan* S, const pq_c128* U, const int32_t* col_order,
                               const double* uniforms, int32_t* samples, cudaStream_t st)
{
    const int m = S->m, n = S->n;
    const int64_t nsamples = S->nsamples;
    if (!U || (nsamples > 0 && (!col_order || !uniforms || !samples)))
        return report(PQ_ERR_ARG, "null argument");
    for (int64_t b = 0; b < nsamples; ++b) {  // every column order is a permutation
        std::vector<char> seen(n, 0);
        for (int q = 0; q < n; ++q) {
            const int32_t c = col_order[b * n + q];
            if (c < 0 || c >= n || seen[c])
                return report(PQ_ERR_ARG, "col_order row is not a permutation of 0 .. n-1");
            seen[c] = 1;
            S->cols_h[(size_t)b * n + q] = S->modes[c];
        }
    }
    for (int64_t b = 0; b < nsamples * n; ++b)
        if (!(uniforms[b] >= 0.0 && uniforms[b] < 1.0))
            return report(PQ_ERR_ARG, "uniforms must lie in [0, 1)");
    for (int64_t e = 0; e < nsamples * m; ++e)
        samples[e] = 0;
    if (nsamples == 0 || n == 0)
        return PQ_OK;
    int rc = PQ_OK;
    if (cudaMemcpyAsync(S->u_d, uniforms, nsamples * n * sizeof(double), cudaMemcpyHostToDevice,
                        st) != cudaSuccess ||
        cudaMemcpyAsync(S->cols_d, S->cols_h.data(), nsamples * n * sizeof(int32_t),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(S->drawn_d, 0, nsamples * n * sizeof(int32_t), st) != cudaSuccess ||
        cudaMemsetAsync(S->err_d, 0, sizeof(int32_t), st) != cudaSuccess)
        rc = report(PQ_ERR_CUDA, "sampler upload failed");
    const unsigned sblocks = (unsigned)std::min<int64_t>((nsamples + 127) / 128, 4096);
    for (int k = 1; k <= n && rc == PQ_OK; ++k) {
        if (k >= 2) {
            const int64_t total = nsamples * k * (int64_t)(k - 1) * (k - 1);
            const unsigned gblocks = (unsigned)std::min<int64_t>((total + 255) / 256, 65536);
            sampler_gather_kernel<<<gblocks, 256, 0, st>>>(reinterpret_cast<const double2*>(U), m,
                                                           n, k, nsamples, S->cols_d, S->drawn_d,
                                                           S->mats_d);
            if (cudaGetLastError() != cudaSuccess) {
                rc = report(PQ_ERR_CUDA, "minor gather failed");
                break;
            }
            rc = plan_run_forward(S->plans[k], S->mats_d, S->per_d, nullptr, st);
            if (rc != PQ_OK)
                break;
        }
        sampler_step_kernel<<<sblocks, 128, 0, st>>>(reinterpret_cast<const double2*>(U), m, n, k,
                                                     nsamples, S->cols_d, S->per_d, S->u_d, S->w_d,
                                                     S->drawn_d, S->err_d);
        if (cudaGetLastError() != cudaSuccess)
            rc = report(PQ_ERR_CUDA, "sampling step failed");
    }
    int32_t err = 0;
    if (rc == PQ_OK &&
        (cudaMemcpyAsync(S->drawn_h.data(), S->drawn_d, nsamples * n * sizeof(int32_t),
                         cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaMemcpyAsync(&err, S->err_d, sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
             cudaSuccess ||
         cudaStreamSynchronize(st) != cudaSuccess))
        rc = report(PQ_ERR_CUDA, "sampler read-back failed");
    if (rc == PQ_OK && err)
        rc = report(PQ_ERR_ARG, "all weights of a sampling step are zero");
    if (rc != PQ_OK) {
        cudaStreamSynchronize(st);
        return rc;
    }
    for (int64_t b = 0; b < nsamples; ++b)
        for (int q = 0; q < n; ++q)
            samples[b * m + S->drawn_h[(size_t)b * n + q]] += 1;
    return PQ_OK;
}

}  // namespace pqi

using namespace pqi;

extern "C" int pq_sampler_plan_create(int32_t m, const int32_t* input_occ, int64_t nsamples,
                                      pq_sampler_plan** out)
{
    if (!out)
        return report(PQ_ERR_ARG, "null argument");
    return sampler_plan_build(m, input_occ, nsamples, out);
}

extern "C" int pq_sampler_plan_run(pq_sampler_plan* plan, const pq_c128* U,
                                   const int32_t* col_order, const double* uniforms,
                                   int32_t* samples, void* stream)
{
    if (!plan)
        return report(PQ_ERR_ARG, "null plan");
    return sampler_plan_launch(plan, U, col_order, uniforms, samples, (cudaStream_t)stream);
}

extern "C" int pq_sampler_plan_destroy(pq_sampler_plan* plan)
{
    if (plan) {
        cudaDeviceSynchronize();
        sampler_plan_free(plan);
    }
    return PQ_OK;
}

extern "C" int pq_bs_sample(const pq_c128* U, int32_t m, const int32_t* input_occ,
                            int64_t nsamples, const int32_t* col_order, const double* uniforms,
                            int32_t* samples, void* stream)
{
    if (!U || !input_occ || (nsamples > 0 && (!col_order || !uniforms || !samples)))
        return report(PQ_ERR_ARG, "null argument");
    pq_sampler_plan* S = nullptr;
    int rc = sampler_plan_build(m, input_occ, nsamples, &S);
    if (rc != PQ_OK)
        return rc;
    rc = sampler_plan_launch(S, U, col_order, uniforms, samples, (cudaStream_t)stream);
    sampler_plan_free(S);
    return rc;
}
