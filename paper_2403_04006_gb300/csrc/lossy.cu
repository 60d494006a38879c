// lossy.cu -- boson sampling with losses (paper Sec. 3.2.4, Figs. BS_Setup and
// BS_LossModel).
//
// The lossy interferometer is A = V diag(sqrt(eta)) W with V, W unitary and
// transmissions eta_i in [0, 1].  Following the paper's loss model, mode i
// meets its own inaccessible mode m + i at a beamsplitter with transmission
// amplitude sqrt(eta_i) and reflection sqrt(1 - eta_i).  The 2m-mode
// interferometer (V + I) L(eta) (W + I) is unitary and its input-mode columns
// are
//   M = [ V diag(sqrt(eta)) W ]   (system outputs)
//       [ diag(sqrt(1 - eta)) W ] (lost photons),
// so the probability of detecting t on the m system modes is the marginal of
// the lossless 2m-mode distribution, Eq. (BS_prob), over every occupation u of
// the loss modes holding the n - |t| missing photons:
//   p(t) = sum_u |per(M_{s, (t, u)})|^2 / (prod t! prod u! prod s!).
// One batched launch evaluates all (t, u) permanents; a second kernel adds
// the u terms of each t in a fixed order.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/pq.h"
#include "pq_kernels.h"
#include "pq_plan.h"

namespace pqi {

// Ubig (2m x 2m, row-major, U[out][in]): columns 0..m-1 hold M, columns
// m..2m-1 are zero (no photon enters a loss mode).
__global__ void lossy_dilation_kernel(const double2* V, const double* eta, const double2* W, int m,
                                      double2* Ubig)
{
    const int M2 = 2 * m;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M2 * M2; e += gridDim.x * blockDim.x) {
        const int r = e / M2, c = e - r * M2;
        double2 v = make_double2(0.0, 0.0);
        if (c < m) {
            if (r < m) {  // sum_q V[r][q] sqrt(eta_q) W[q][c]
                for (int q = 0; q < m; ++q) {
                    const double a = sqrt(eta[q]);
                    const double2 x = V[r * m + q], y = W[q * m + c];
                    v.x += a * (x.x * y.x - x.y * y.y);
                    v.y += a * (x.x * y.y + x.y * y.x);
                }
            } else {  // sqrt(1 - eta_i) W[i][c]
                const int i = r - m;
                const double a = sqrt(1.0 - eta[i]);
                v = make_double2(a * W[i * m + c].x, a * W[i * m + c].y);
            }
        }
        Ubig[e] = v;
    }
}

// probs[t] = sum of pbig over that t's consecutive range of loss patterns.
__global__ void lossy_marginal_kernel(const double* pbig, const int64_t* first, int64_t B,
                                      double* probs)
{
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
         b += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t q = first[b]; q < first[b + 1]; ++q)
            s += pbig[q];
        probs[b] = s;
    }
}

// All occupations u of m modes with sum k, lexicographic.
static void compositions(int k, int m, std::vector<int32_t>& cur, int pos,
                         std::vector<std::vector<int32_t>>& out)
{
    if (pos == m - 1) {
        cur[pos] = k;
        out.push_back(cur);
        return;
    }
    for (int v = 0; v <= k; ++v) {
        cur[pos] = v;
        compositions(k - v, m, cur, pos + 1, out);
    }
}

}  // namespace pqi

// A planned lossy batch: the 2m-mode boson-sampling plan of every (t, u)
// pattern, the pattern offsets of each t and the device workspace.
struct pq_lossy_plan {
    int32_t m = 0;
    int64_t B = 0, NB = 0;
    pq_plan* P = nullptr;
    double2* Ubig = nullptr;     // 2m x 2m
    double* pbig = nullptr;      // NB probabilities of the (t, u) patterns
    int64_t* first_d = nullptr;  // B + 1 offsets of each t's patterns
};

namespace pqi {

static void lossy_plan_free(pq_lossy_plan* L)
{
    if (!L)
        return;
    if (L->P)
        pq_plan_destroy(L->P);
    dev_free(L->Ubig);
    dev_free(L->pbig);
    dev_free(L->first_d);
    delete L;
    host_object_freed();
}

// Host planning: expand every output pattern t into its loss patterns u,
// plan the permanents, allocate and upload.  Synchronous.
static int lossy_plan_build(int32_t m, const int32_t* input_occ, const int32_t* output_occ,
                            int64_t B, pq_lossy_plan** out)
{
    *out = nullptr;
    if (!input_occ || (B > 0 && !output_occ))
        return report(PQ_ERR_ARG, "null argument");
    if (m <= 0 || 2 * m > PQ_MAX_DIM || B < 0)
        return report(m <= 0 || B < 0 ? PQ_ERR_ARG : PQ_ERR_UNSUPPORTED,
                      "need 1 <= m and 2m <= PQ_MAX_DIM");
    int n = 0;
    for (int j = 0; j < m; ++j) {
        if (input_occ[j] < 0)
            return report(PQ_ERR_ARG, "negative input occupation");
        n += input_occ[j];
    }
    // (t, u) patterns on 2m modes, grouped by t
    std::vector<int32_t> big_t;
    std::vector<int64_t> first(B + 1, 0);
    std::vector<int32_t> cur(m, 0);
    for (int64_t b = 0; b < B; ++b) {
        int nt = 0;
        for (int i = 0; i < m; ++i) {
            if (output_occ[b * m + i] < 0)
                return report(PQ_ERR_ARG, "negative output occupation");
            nt += output_occ[b * m + i];
        }
        if (nt > n)
            return report(PQ_ERR_ARG, "an output pattern holds more photons than the input");
        std::vector<std::vector<int32_t>> us;
        compositions(n - nt, m, cur, 0, us);
        for (const auto& u : us) {
            big_t.insert(big_t.end(), output_occ + b * m, output_occ + (b + 1) * m);
            big_t.insert(big_t.end(), u.begin(), u.end());
        }
        first[b + 1] = first[b] + (int64_t)us.size();
        if (first[b + 1] > (int64_t(1) << 28))
            return report(PQ_ERR_UNSUPPORTED, "too many loss patterns");
    }
    if (!host_object_alloc_ok())
        return report(PQ_ERR_NOMEM, "host allocation failed");
    pq_lossy_plan* L = new (std::nothrow) pq_lossy_plan();
    if (!L) {
        host_object_freed();
        return report(PQ_ERR_NOMEM, "host allocation failed");
    }
    L->m = m;
    L->B = B;
    L->NB = first[B];
    if (B == 0) {
        *out = L;
        return PQ_OK;
    }
    std::vector<int32_t> sbig(2 * m, 0);
    for (int j = 0; j < m; ++j)
        sbig[j] = input_occ[j];
    int rc = pq_plan_create_bs(2 * m, sbig.data(), big_t.data(), L->NB, nullptr, &L->P);
    if (rc == PQ_OK &&
        (dev_alloc((void**)&L->Ubig, sizeof(double2) * 4 * m * m) != cudaSuccess ||
         dev_alloc((void**)&L->pbig, sizeof(double) * L->NB) != cudaSuccess ||
         dev_alloc((void**)&L->first_d, sizeof(int64_t) * (B + 1)) != cudaSuccess))
        rc = report(PQ_ERR_NOMEM, "lossy workspace allocation failed");
    if (rc == PQ_OK && cudaMemcpy(L->first_d, first.data(), sizeof(int64_t) * (B + 1),
                                  cudaMemcpyHostToDevice) != cudaSuccess)
        rc = report(PQ_ERR_CUDA, "pattern offsets upload failed");
    if (rc != PQ_OK) {
        lossy_plan_free(L);
        return rc;
    }
    *out = L;
    return PQ_OK;
}

// The dilation, the permanents of every (t, u) and the marginals, on stream;
// no allocation, no host access, no synchronisation.
static int lossy_plan_launch(pq_lossy_plan* L, const pq_c128* V, const double* eta,
                             const pq_c128* W, double* probs, cudaStream_t st)
{
    if (!V || !eta || !W || (L->B > 0 && !probs))
        return report(PQ_ERR_ARG, "null argument");
    if (L->B == 0)
        return PQ_OK;
    const int m = L->m;
    lossy_dilation_kernel<<<(4 * m * m + 255) / 256, 256, 0, st>>>(
        reinterpret_cast<const double2*>(V), eta, reinterpret_cast<const double2*>(W), m, L->Ubig);
    if (cudaGetLastError() != cudaSuccess)
        return report(PQ_ERR_CUDA, "dilation kernel failed");
    int rc = plan_run_forward(L->P, L->Ubig, nullptr, L->pbig, st);
    if (rc != PQ_OK)
        return rc;
    const unsigned blocks = (unsigned)((L->B + 127) / 128 < 4096 ? (L->B + 127) / 128 : 4096);
    lossy_marginal_kernel<<<blocks, 128, 0, st>>>(L->pbig, L->first_d, L->B, probs);
    if (cudaGetLastError() != cudaSuccess)
        return report(PQ_ERR_CUDA, "lossy marginal failed");
    return PQ_OK;
}

}  // namespace pqi

using namespace pqi;

extern "C" int pq_lossy_plan_create(int32_t m, const int32_t* input_occ, const int32_t* output_occ,
                                    int64_t B, pq_lossy_plan** out)
{
    if (!out)
        return report(PQ_ERR_ARG, "null argument");
    return lossy_plan_build(m, input_occ, output_occ, B, out);
}

extern "C" int pq_lossy_plan_run(pq_lossy_plan* plan, const pq_c128* V, const double* eta,
                                 const pq_c128* W, double* probs, void* stream)
{
    if (!plan)
        return report(PQ_ERR_ARG, "null plan");
    return lossy_plan_launch(plan, V, eta, W, probs, (cudaStream_t)stream);
}

extern "C" int pq_lossy_plan_destroy(pq_lossy_plan* plan)
{
    if (plan) {
        cudaDeviceSynchronize();
        lossy_plan_free(plan);
    }
    return PQ_OK;
}

extern "C" int pq_bs_probs_lossy(const pq_c128* V, const double* eta, const pq_c128* W, int32_t m,
                                 const int32_t* input_occ, const int32_t* output_occ, int64_t B,
                                 double* probs, void* stream)
{
    if (!V || !eta || !W || !input_occ || (B > 0 && (!output_occ || !probs)))
        return report(PQ_ERR_ARG, "null argument");
    pq_lossy_plan* L = nullptr;
    int rc = lossy_plan_build(m, input_occ, output_occ, B, &L);
    if (rc != PQ_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = lossy_plan_launch(L, V, eta, W, probs, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == PQ_OK)
        rc = report(PQ_ERR_CUDA, "lossy probabilities failed");
    lossy_plan_free(L);
    return rc;
}
