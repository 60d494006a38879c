// pq_plan.h -- host-side plan structure (internal).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/pq.h"
#include "pq_internal.h"

namespace pqi {

// Host copy of one permanent before upload.
struct ItemPlan {
    int64_t src_off = 0;
    int32_t k = 0, l = 0, n = 0, si = 0, sj = 0;
    bool transposed = false;
    std::vector<int32_t> ridx, cidx, rmul, cmul;  // oriented
    std::vector<int32_t> drow, drad, dtop;        // digits, ascending radix
    std::vector<int32_t> ecnt;                    // extra prefix factors per product column
    int32_t jf = -1;                              // first column with an extra (-1: unit)
    int32_t J = 0;
    int64_t T = 0, L = 1, nchunks = 0;
    bool weighted = false;
    bool trivial = false;
    double norm = 1.0;
};

// One backward launch: the permanents whose product side fits ld columns,
// with the shared-memory layout sized for them.
struct BwdClass {
    int ld = 1, kmax = 1, jb = 0, n2 = 0, wpb = 1, blocks = 1;
    int reg = 0;  // 1: the register-resident walk (glynn_bwd_reg_kernel)
    int64_t t_begin = 0, t_end = 0;  // range in the batched backward task list
};

struct DeviceBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace pqi

struct pq_plan {
    int kind = 0;  // 0: permanent batch, 1: boson sampling
    pq_plan_options opts{};
    int device = 0;
    int num_sms = 0;
    int64_t nperm = 0;
    int64_t nslots = 0;  // partial-sum slots of the forward
    int lmax = 8;
    int kmax = 1;
    int wpb = 8;
    int blocks = 0;
    int bwd_wpb = 4;
    int bwd_blocks = 0;
    int bwd_jb = 0;  // low digits per backward chunk, at most
    int bwd_n2 = 0;  // repeated product columns, at most
    int bwd_kmax = 1;
    // boson sampling inputs
    int32_t m = 0;
    std::vector<int32_t> in_occ, out_occ;
    // ragged batch sizes (for gradient scatter)
    std::vector<int64_t> item_mat_off;
    std::vector<int32_t> item_k, item_l;
    int64_t total_mat_elems = 0;
    // host schedule
    std::vector<pqi::ItemPlan> items;
    std::vector<pqi::PermDesc> desc_h;
    std::vector<int32_t> meta_h;
    std::vector<pqi::Task> tasks_batched_h, tasks_plain_h;
    std::vector<int64_t> plain_first;  // first plain task of each permanent (+ end)
    std::vector<int32_t> class_log2;   // chunk log2 per photon number (index n)
    // device
    pqi::PermDesc* desc_d = nullptr;
    int32_t* meta_d = nullptr;
    int32_t* meta_bwd_d = nullptr;  // the metadata pool with the backward's digit order
    pqi::Task* tasks_batched_d = nullptr;
    pqi::Task* tasks_plain_d = nullptr;
    double* partials_d = nullptr;
    int32_t* counters_d = nullptr;
    int32_t* err_d = nullptr;
    // backward schedule and workspace (built on the first backward call)
    bool bwd_ready = false;
    // where the forward walk keeps its column sums: 0 shared memory; NL > 0
    // registers, every permanent in column class NL (glynn_fwd_reg_kernel<NL>);
    // -1 registers, several classes (glynn_fwd_reg_mixed_kernel)
    int fwd_nl = 0;
    // columns of a row of the forward walk's shared-memory layout: lmax for
    // shared memory; the class bound of the widest permanent for registers
    // (a row of class NL holds NL columns, at least 4, so it can be wider
    // than lmax)
    int fwd_ld = 0;
    bool uploaded = false;  // device data matches the host schedule (a failed re-plan clears it)
    std::vector<pqi::PermDesc> desc_bwd_h;
    std::vector<pqi::Task> tasks_bwd_plain_h, tasks_bwd_batched_h;
    std::vector<int64_t> plain_first_bwd;
    std::vector<pqi::BwdClass> bwd_classes;
    std::vector<int32_t> bwd_class_of;  // class of each permanent
    pqi::PermDesc* desc_bwd_d = nullptr;
    pqi::Task* tasks_bwd_plain_d = nullptr;
    pqi::Task* tasks_bwd_batched_d = nullptr;
    double* gpart_d = nullptr;
    int64_t* gpart_off_d = nullptr;
    double2* grad_local_d = nullptr;
    int64_t* grad_local_off_d = nullptr;
    int64_t* item_mat_off_d = nullptr;
    int32_t* item_k_d = nullptr;
    int32_t* item_l_d = nullptr;
    double2* grad_out_tmp_d = nullptr;
    int32_t* bs_pos_d = nullptr;  // boson sampling: mode -> oriented index, 2m per pattern
    size_t gpart_elems = 0, grad_local_elems = 0;
    // graph of the batched forward
    cudaGraphExec_t graph = nullptr;
    const void* graph_key[4] = {nullptr, nullptr, nullptr, nullptr};
    void* graph_stream = nullptr;
    // statistics
    pq_plan_stats stats{};
};

namespace pqi {
// Plans over one m x m matrix with per-item row occupations t[b] and column
// occupations s[b] (host, B x m each), no normalisation; and a forward run.
int plan_create_occupations(int32_t m, const std::vector<int32_t>& t, const std::vector<int32_t>& s,
                            int64_t B, pq_plan** out);
int plan_run_forward(pq_plan* P, const void* src, void* amps, double* probs, cudaStream_t st);
// Raise the forward kernel's shared-memory limit to what plan P launches with.
int plan_prepare_forward(pq_plan* P);
}  // namespace pqi
