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

using namespace pqi;

extern "C" int pq_bs_probs_lossy(const pq_c128* V, const double* eta, const pq_c128* W, int32_t m,
                                 const int32_t* input_occ, const int32_t* output_occ, int64_t B,
                                 double* probs, void* stream)
{
    if (!V || !eta || !W || !input_occ || (B > 0 && (!output_occ || !probs)))
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
    const int64_t NB = first[B];
    std::vector<int32_t> sbig(2 * m, 0);
    for (int j = 0; j < m; ++j)
        sbig[j] = input_occ[j];
    if (B == 0)
        return PQ_OK;
    pq_plan* P = nullptr;
    int rc = pq_plan_create_bs(2 * m, sbig.data(), big_t.data(), NB, nullptr, &P);
    if (rc != PQ_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double2* Ubig = nullptr;
    double* pbig = nullptr;
    int64_t* first_d = nullptr;
    if (dev_alloc((void**)&Ubig, sizeof(double2) * 4 * m * m) != cudaSuccess ||
        dev_alloc((void**)&pbig, sizeof(double) * NB) != cudaSuccess ||
        dev_alloc((void**)&first_d, sizeof(int64_t) * (B + 1)) != cudaSuccess) {
        rc = report(PQ_ERR_NOMEM, "lossy workspace allocation failed");
    }
    if (rc == PQ_OK &&
        cudaMemcpyAsync(first_d, first.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice,
                        st) != cudaSuccess)
        rc = report(PQ_ERR_CUDA, "pattern offsets upload failed");
    if (rc == PQ_OK) {
        lossy_dilation_kernel<<<(4 * m * m + 255) / 256, 256, 0, st>>>(
            reinterpret_cast<const double2*>(V), eta, reinterpret_cast<const double2*>(W), m,
            Ubig);
        if (cudaGetLastError() != cudaSuccess)
            rc = report(PQ_ERR_CUDA, "dilation kernel failed");
    }
    if (rc == PQ_OK)
        rc = plan_run_forward(P, Ubig, nullptr, pbig, st);
    if (rc == PQ_OK) {
        const unsigned blocks = (unsigned)((B + 127) / 128 < 4096 ? (B + 127) / 128 : 4096);
        lossy_marginal_kernel<<<blocks, 128, 0, st>>>(pbig, first_d, B, probs);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
            rc = report(PQ_ERR_CUDA, "lossy marginal failed");
    }
    dev_free(Ubig);
    dev_free(pbig);
    dev_free(first_d);
    pq_plan_destroy(P);
    return rc;
}
