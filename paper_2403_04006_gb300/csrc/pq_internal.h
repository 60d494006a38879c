// pq_internal.h -- structures shared by the host planner and the kernels.
//
// A permanent is evaluated by the BB/FG (Glynn) formula extended to row and
// column multiplicities with a mixed-radix Gray code (paper Sec. 4.2, "Boson
// Sampling").  For a base matrix B (k x l) with row multiplicities r and column
// multiplicities c, sum r = sum c = n, one row f ("fixed") keeps one copy's
// sign at +1 and the remaining sign choices are grouped per row:
//
//   per = 2^{-(n-1)} sum_g prod_d (-1)^{g_d} C(top_d, g_d)
//                          prod_j ( sum_i (r_i - 2 g_i) b_ij )^{c_j}
//
// g_i in [0, r_i] counts the copies of row i that carry a minus sign
// (top = r_i), except for the fixed row, whose g_f in [0, r_f - 1]
// (top = r_f - 1); rows whose digit has a single value drop out of the code.
// The digits d (one per remaining row) form the "n-ary Gray code" of the
// paper; T = prod_d radix_d terms.
//
// Parallel split (a design of this library, not the paper's): the lowest J
// digits form a chunk of L = prod_{d<J} radix_d terms that one thread walks
// in reflected mixed-radix Gray order starting from all-zero low digits; the
// high digits are constant within a chunk and are decoded from the chunk
// index.  Because every chunk starts its walk from the same state, all lanes
// of a warp change the same row by the same amount at every step, so the
// Gray-code bookkeeping and the row read are warp-uniform.  A warp task is up
// to 32 consecutive chunks of one permanent (one per lane).
#pragma once
#include <stdint.h>

namespace pqi {

constexpr int kMaxLowDigits = 15;  // digits packed 4 bits each in a 64-bit word
constexpr int kMaxLowRadix = 15;   // radix of a low digit fits 4 bits
constexpr int kWarp = 32;

// One permanent, oriented so that its rows are the summed (Gray-code) side.
struct alignas(16) PermDesc {
    int64_t T;        // Gray-code terms
    int64_t nchunks;  // T / L
    int64_t src_off;  // element offset of this item's source matrix
    int32_t k, l, n;  // summed rows, product columns, photons
    int32_t si, sj;   // element (i, j) = src[src_off + ridx[i] * si + cidx[j] * sj]
    int32_t meta;     // offset of this item's integer metadata in the pool
    int32_t ndig, J;  // Gray digits; low digits walked inside a chunk
    int32_t weighted; // 1 if some digit has radix > 2 (|weight| not always 1)
    int32_t slot0;    // first partial-sum slot (one per task of this permanent)
    int32_t ntasks;   // warp tasks of this permanent
    int32_t out;      // output index
    int32_t trivial;  // 1: n == 0, per = 1
    int32_t jf;       // first product column whose prefix is an extra factor (-1: none)
    int64_t L;        // chunk length
    double norm;      // 1 / (prod t! prod s!) for boson sampling, else 1
    int32_t part0;    // first task part of this plan's shard (0 unless sharded)
    int32_t pad2;
};

// Integer metadata of one permanent, at pool + PermDesc::meta:
//   ridx[k]  source index of each summed row
//   cidx[l]  source index of each product column
//   rmul[k]  row multiplicities (summed side)
//   cmul[l]  column multiplicities (product side)
//   drow[ndig] row of digit d; drad[ndig] radix of digit d; dtop[ndig] binomial top
//   ecnt[l]  extra factors at product column j (see below)
// Product columns are sorted by non-increasing multiplicity c_0 >= c_1 >= ...
// Then prod_j S_j^{c_j} = prod_{m >= 1} P(n_m), with P(q) = S_0 ... S_{q-1} and
// n_m the number of columns with c_j >= m, so a term needs l - 1 products for
// P(l) plus one product per extra prefix: ecnt[j] = c_j - max(c_{j+1}, 1)
// (c_l = 0) extra copies of P(j + 1).
__host__ __device__ inline int meta_size(int k, int l, int ndig) { return 2 * k + 3 * l + 3 * ndig; }

struct alignas(8) Task {
    int32_t perm;  // permanent
    int32_t part;  // index of this task among its permanent's tasks; it covers
                   // chunks [32 part, min(32 part + 32, nchunks)); a sharded
                   // plan holds the parts [part0, part0 + ntasks) of each
};

// Arguments of one kernel execution (device pointers).
struct ExecArgs {
    const PermDesc* desc;
    const int32_t* meta;
    const Task* tasks;
    int64_t ntasks;
    const double2* src;   // matrices (batch) or U (boson sampling)
    double2* out_amp;     // permanents, nullable
    double* out_prob;     // |per|^2 * norm, nullable
    double* out_partial;  // sharded plans: unscaled double-double sum, 4 doubles per
                          // permanent (re hi, re lo, im hi, im lo); nullable
    double* partials;     // 4 doubles per task slot
    int32_t* counters;    // [0] task queue head, [1 + p] finished tasks of p
    int32_t* err;         // device error record, see below
    int64_t nperm;        // permanents of the plan (bound of Task::perm and PermDesc::out)
    int64_t nmeta;        // entries of the metadata pool
    int64_t nslots;       // task slots of `partials`
};

// Device error record (two int32 words, zero = no error): the kernels check
// every task and the descriptor it names against the launch before using
// them, skip a task that fails and keep the first failure: err[0] = one of
// the codes below, err[1] = the index of the task in the task list.
constexpr int32_t kErrTaskPerm = 1;     // task names a permanent outside the batch
constexpr int32_t kErrTaskPart = 2;     // task part outside its permanent's range
constexpr int32_t kErrDescLayout = 3;   // k or l beyond the launch's shared-memory layout
constexpr int32_t kErrDescDigits = 4;   // digit counts beyond the walk's limits
constexpr int32_t kErrDescIndex = 5;    // metadata, partial slots or output outside the plan's arrays

}  // namespace pqi
