// pq_kernels.h -- host-side entry points of the kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "pq_internal.h"

namespace pqi {

// ---- forward (glynn_fwd.cu)
int fwd_smem_per_warp(int kmax, int lmax);
int fwd_regs_per_thread(int lmax);
int bwd_regs_per_thread(int lmax);

// Warps per block and resident blocks per SM that registers and shared
// memory allow (65536 registers per SM, allocated per warp in units of 256;
// up to 227 KB of shared memory per SM for all resident blocks).
inline void launch_geometry(int regs_per_thread, int smem_per_warp, int want_wpb,
                            int want_bps, int& wpb, int& bps)
{
    const int regs_warp = ((regs_per_thread * 32 + 255) / 256) * 256;
    int max_warps = 65536 / regs_warp;
    if (max_warps < 1)
        max_warps = 1;
    wpb = want_wpb < max_warps ? want_wpb : max_warps;
    while (wpb > 1 && wpb * smem_per_warp > 220 * 1024)
        --wpb;
    int by_regs = max_warps / wpb;
    int by_smem = smem_per_warp > 0 ? (227 * 1024) / (wpb * smem_per_warp) : 32;
    int cap = by_regs < by_smem ? by_regs : by_smem;
    if (cap < 1)
        cap = 1;
    bps = want_bps < cap ? want_bps : cap;
}
// The (warps per block, blocks per SM) with the most resident warps, at most
// want_wpb warps per block: registers as above; dynamic shared memory at most
// 227 KB per block and 228 KB per SM including 1 KB the system reserves per
// block.
inline void launch_geometry_max(int regs_per_thread, int smem_per_warp, int want_wpb, int& wpb,
                                int& bps)
{
    const int regs_warp = ((regs_per_thread * 32 + 255) / 256) * 256;
    const int max_warps = 65536 / regs_warp > 0 ? 65536 / regs_warp : 1;
    wpb = 1;
    bps = 1;
    int best = 0;
    for (int w = 1; w <= want_wpb && w <= max_warps; ++w) {
        const long block = (long)w * smem_per_warp;
        if (block > 232448L)
            break;
        int b = (int)(233472L / (block + 1024L));
        b = b < max_warps / w ? b : max_warps / w;
        if (b < 1)
            continue;
        if (w * b >= best) {
            best = w * b;
            wpb = w;
            bps = b;
        }
    }
}
cudaError_t fwd_prepare(int lmax, int smem_bytes);
cudaError_t fwd_launch_persistent(int lmax, const ExecArgs& a, int kmax, int blocks, int wpb,
                                  cudaStream_t st);
cudaError_t fwd_launch_plain(int lmax, const ExecArgs& a, int64_t t_begin, int64_t t_end,
                             int kmax, int wpb, cudaStream_t st);
// The register-resident forward walk (glynn_fwd_reg_kernel<NL>) for product
// sides of at most kFwdRegMaxLd columns: one instantiation per even column
// bound NL = 4 .. 20 (fwd_reg_class_of(l)), launched per class.
constexpr int kFwdRegMaxLd = 20;
int fwd_reg_class_of(int l);
int fwd_reg_smem_per_warp(int kmax, int ld);
int fwd_reg_regs_per_thread(int nl);
cudaError_t fwd_reg_prepare(int nl, int smem_bytes);
cudaError_t fwd_reg_launch(int nl, const ExecArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                           int ld, unsigned grid, int wpb, int queue, cudaStream_t st);
int fwd_reg_mixed_regs_per_thread();
cudaError_t fwd_reg_mixed_prepare(int smem_bytes);
cudaError_t fwd_reg_mixed_launch(const ExecArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                                 int ld, unsigned grid, int wpb, int queue, cudaStream_t st);

// ---- backward (glynn_bwd.cu)
struct BwdArgs {
    const PermDesc* desc;
    const int32_t* meta;
    const Task* tasks;
    int64_t ntasks;
    const double2* src;
    const double2* grad_out;   // per permanent: dL/dper (PyTorch convention), nullable
    const double2* amps;       // boson sampling: per values, used with grad_prob
    const double* grad_prob;   // boson sampling: dL/dp, nullable
    double* gpart;             // per task slot: k*l complex (oriented), 2 doubles each
    int64_t* gpart_off;        // per permanent: offset (in complex entries) of slot 0
    double2* grad_local;       // per permanent: oriented k x l gradient (complex)
    int64_t* grad_local_off;   // per permanent: offset of its block
    int32_t* counters;
    int32_t* err;             // device error record (pq_internal.h)
    int64_t nperm;            // permanents (bound of Task::perm)
    int64_t nmeta;            // entries of the metadata pool
};
int bwd_smem_bytes_for(int kmax, int lmax, int jb, int n2);
constexpr int kBwdMaxLowDigits = 4;  // low digits the backward workspace holds
constexpr int kBwdChunkLog2 = 7;     // backward chunks of at most 2^7 terms
cudaError_t bwd_prepare(int lmax, int smem_bytes);
cudaError_t bwd_launch_persistent(int ld, const BwdArgs& a, int64_t t_begin, int64_t t_end,
                                  int kmax, int jb, int n2, int blocks, int wpb, cudaStream_t st);
cudaError_t bwd_launch_plain(int lmax, const BwdArgs& a, int64_t t_begin, int64_t t_end,
                             int kmax, int jb, int n2, int wpb, cudaStream_t st);
// The register-resident walk (column sums, accumulators and prefixes in
// registers) for even product-column bounds up to kBwdRegMaxLd.
constexpr int kBwdRegMaxLd = 14;
bool bwdr_supported(int ld);
int bwdr_smem_bytes_for(int kmax, int ld, int jb);
int bwdr_regs_per_thread(int ld);
cudaError_t bwdr_prepare(int ld, int smem_bytes);
cudaError_t bwdr_launch_persistent(int ld, const BwdArgs& a, int64_t t_begin, int64_t t_end,
                                   int kmax, int jb, int blocks, int wpb, cudaStream_t st);
cudaError_t bwdr_launch_plain(int ld, const BwdArgs& a, int64_t t_begin, int64_t t_end, int kmax,
                              int jb, int wpb, cudaStream_t st);

// Scatter of oriented per-permanent gradients into the caller's layouts.
cudaError_t scatter_grad_batch(const PermDesc* desc, const int32_t* meta, int64_t nperm,
                               const double2* grad_local, const int64_t* grad_local_off,
                               const int64_t* item_mat_off, const int32_t* item_l,
                               const int32_t* item_k, double2* grad_mats, int64_t total_elems,
                               cudaStream_t st);
cudaError_t scatter_grad_bs(const PermDesc* desc, const int32_t* pos, int64_t nperm, int32_t m,
                            const double2* grad_local, const int64_t* grad_local_off,
                            double2* grad_U, cudaStream_t st);

// ---- Clements mesh (clements.cu)
cudaError_t clements_forward(const double* theta, const double* phi, int m, double2* U,
                             cudaStream_t st);
cudaError_t clements_backward(const double* theta, const double* phi, int m, const double2* U,
                              const double2* gU, double* gtheta, double* gphi, cudaStream_t st);

// ---- runtime services (pq_runtime.cu)
// Every device buffer of the library comes from dev_alloc and goes back
// through dev_free, which count the live buffers; the test hook of
// pq_debug_fail_allocation makes one allocation report failure.
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
// The same hook and count for the host objects the library creates (plans).
bool host_object_alloc_ok();
void host_object_freed();
// Process-wide chunk length (log2) per photon number; 0 = default.
int tune_get(int n);
void tune_set(int n, int v);

// ---- error message of the calling thread, read by pq_last_error (pq_api.cu)
void set_last_error(const char* msg);
int report(int code, const char* msg);  // set the message, return code

// ---- FP64 probe (fp64_probe.cu)
cudaError_t fp64_probe(int64_t iters, double* flops_per_s, double* ms, cudaStream_t st);

}  // namespace pqi
