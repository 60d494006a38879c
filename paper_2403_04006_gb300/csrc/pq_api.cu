// pq_api.cu -- the C ABI (include/pq.h): argument checks, planning, launches.
//
// Planning (host): for every permanent, drop zero-multiplicity rows/columns,
// pick the side whose Gray code has fewer terms ("column or row
// multiplicities", Sec. 4.2), fix one copy of the least repeated row, order
// the digits by radix, cut the code into chunks of the low digits and the
// chunks into warp tasks.  Execution (device) then needs no host reads and no
// allocation, so it can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

#include "../../include/pq.h"
#include "pq_kernels.h"
#include "pq_plan.h"

using namespace pqi;

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define PQ_ALLOC(pp, bytes)                                                             \
    do {                                                                                \
        cudaError_t e_ = dev_alloc((void**)(pp), (bytes));                              \
        if (e_ != cudaSuccess)                                                          \
            return fail(PQ_ERR_NOMEM, "device allocation of %zu bytes failed: %s",      \
                        (size_t)(bytes), cudaGetErrorString(e_));                       \
    } while (0)

#define PQ_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(PQ_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

extern "C" const char* pq_last_error(void) { return g_err.c_str(); }

namespace pqi {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace pqi
extern "C" const char* pq_version(void) { return "pq-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------- planning
static const int64_t kMaxTerms = int64_t(1) << 62;

// Terms of the Gray code when the given side is summed: the least repeated
// line keeps one copy fixed (radix m_f = mult_f), every other line has radix
// mult + 1.  Returns -1 on overflow.
static int64_t side_terms(const std::vector<int32_t>& mult)
{
    if (mult.empty())
        return 1;
    size_t f = std::min_element(mult.begin(), mult.end()) - mult.begin();
    int64_t T = 1;
    for (size_t i = 0; i < mult.size(); ++i) {
        int64_t rad = (i == f) ? mult[i] : mult[i] + 1;
        if (rad <= 0)
            rad = 1;
        if (T > kMaxTerms / rad)
            return -1;
        T *= rad;
    }
    return T;
}

// Build the oriented item for base (k0 x l0) with multiplicities r, c whose
// element (i, j) sits at src_off + i * ld0 + j.
static int build_item(const int32_t* r, const int32_t* c, int k0, int l0, int64_t src_off,
                      int64_t ld0, ItemPlan& it)
{
    if (k0 < 0 || l0 < 0 || k0 > PQ_MAX_DIM || l0 > PQ_MAX_DIM)
        return fail(k0 < 0 || l0 < 0 ? PQ_ERR_ARG : PQ_ERR_UNSUPPORTED,
                    "base matrix %d x %d outside [0, %d]", k0, l0, PQ_MAX_DIM);
    std::vector<int32_t> rs, cs, rm, cm;
    int nr = 0, nc = 0;
    for (int i = 0; i < k0; ++i) {
        if (r[i] < 0)
            return fail(PQ_ERR_ARG, "negative row multiplicity");
        if (r[i] > 0) {
            rs.push_back(i);
            rm.push_back(r[i]);
            nr += r[i];
        }
    }
    for (int j = 0; j < l0; ++j) {
        if (c[j] < 0)
            return fail(PQ_ERR_ARG, "negative column multiplicity");
        if (c[j] > 0) {
            cs.push_back(j);
            cm.push_back(c[j]);
            nc += c[j];
        }
    }
    if (nr != nc)
        return fail(PQ_ERR_ARG, "sum of row multiplicities (%d) != sum of column multiplicities (%d)",
                    nr, nc);
    if (nr > PQ_MAX_N)
        return fail(PQ_ERR_UNSUPPORTED, "n = %d above PQ_MAX_N = %d", nr, PQ_MAX_N);
    it = ItemPlan();
    it.n = nr;
    it.src_off = src_off;
    if (nr == 0) {
        it.trivial = true;
        it.T = 0;
        return PQ_OK;
    }
    int64_t Tr = side_terms(rm), Tc = side_terms(cm);
    if (Tr < 0 && Tc < 0)
        return fail(PQ_ERR_UNSUPPORTED, "term count above 2^62");
    bool transpose = (Tr < 0) || (Tc >= 0 && Tc < Tr);
    if (transpose) {
        it.transposed = true;
        it.ridx = cs;
        it.rmul = cm;
        it.cidx = rs;
        it.cmul = rm;
        it.si = 1;
        it.sj = (int32_t)ld0;
        it.T = Tc;
    } else {
        it.ridx = rs;
        it.rmul = rm;
        it.cidx = cs;
        it.cmul = cm;
        it.si = (int32_t)ld0;
        it.sj = 1;
        it.T = Tr;
    }
    it.k = (int32_t)it.ridx.size();
    it.l = (int32_t)it.cidx.size();
    if (it.l > PQ_MAX_PRODUCT_COLS)
        return fail(PQ_ERR_UNSUPPORTED, "%d product-side columns above %d", it.l,
                    PQ_MAX_PRODUCT_COLS);
    // product columns by non-increasing multiplicity; extra prefix factors:
    // prod_j S_j^{c_j} = prod_{m>=1} P(n_m), n_m = #{j : c_j >= m}, and P(j+1)
    // appears c_j - max(c_{j+1}, 1) extra times (c_l = 0)
    {
        std::vector<int> ord(it.l);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return it.cmul[a] > it.cmul[b]; });
        std::vector<int32_t> ci(it.l), cm2(it.l);
        for (int j = 0; j < it.l; ++j) {
            ci[j] = it.cidx[ord[j]];
            cm2[j] = it.cmul[ord[j]];
        }
        it.cidx = ci;
        it.cmul = cm2;
        it.ecnt.assign(it.l, 0);
        it.jf = -1;
        for (int j = 0; j < it.l; ++j) {
            const int next = (j + 1 < it.l) ? it.cmul[j + 1] : 0;
            it.ecnt[j] = std::max(0, it.cmul[j] - std::max(next, 1));
            if (it.ecnt[j] > 0 && it.jf < 0)
                it.jf = j;
        }
    }
    // digits: fixed copy on the least repeated row, ascending radix
    int f = (int)(std::min_element(it.rmul.begin(), it.rmul.end()) - it.rmul.begin());
    struct Dg {
        int rad, row, top;
    };
    std::vector<Dg> dg;
    for (int i = 0; i < it.k; ++i) {
        if (i == f) {
            if (it.rmul[i] >= 2)
                dg.push_back({it.rmul[i], i, it.rmul[i] - 1});
        } else {
            dg.push_back({it.rmul[i] + 1, i, it.rmul[i]});
        }
    }
    std::stable_sort(dg.begin(), dg.end(), [](const Dg& a, const Dg& b) { return a.rad < b.rad; });
    for (const Dg& d : dg) {
        it.drow.push_back(d.row);
        it.drad.push_back(d.rad);
        it.dtop.push_back(d.top);
    }
    return PQ_OK;
}

// Share of the Gray steps of a chunk (the lowest j digits, ascending radix)
// after which the low-digit weight prod_d C(top_d, g_d) changes: only digits
// of radix > 2 change it, and the a leading radix-2 digits take all but
// 2^-a of the steps.  Zero when every low digit has radix 2.
static double weight_change_rate(const std::vector<int32_t>& drad, int j)
{
    int a = 0;
    while (a < j && drad[a] == 2)
        ++a;
    return a == j ? 0.0 : std::ldexp(1.0, -a);
}

// Put the digits of the given low multiset first (ascending radix, ties in
// row order), then the others in the same order.  low_count[v]: how many
// digits of radix v go low.  The walk takes any digits as its low ones: the
// Gray code over all digits is the same set of codes in another order.
static void order_digits(ItemPlan& it, const std::vector<int>& low_count)
{
    const int nd = (int)it.drad.size();
    std::vector<int> idx(nd), taken(low_count.size(), 0), lo, hi;
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return it.drad[a] != it.drad[b] ? it.drad[a] < it.drad[b] : it.drow[a] < it.drow[b];
    });
    for (int d : idx) {
        const int v = it.drad[d];
        if (v < (int)low_count.size() && taken[v] < low_count[v]) {
            ++taken[v];
            lo.push_back(d);
        } else {
            hi.push_back(d);
        }
    }
    lo.insert(lo.end(), hi.begin(), hi.end());
    std::vector<int32_t> r(nd), rad(nd), top(nd);
    for (int q = 0; q < nd; ++q) {
        r[q] = it.drow[lo[q]];
        rad[q] = it.drad[lo[q]];
        top[q] = it.dtop[lo[q]];
    }
    it.drow = r;
    it.drad = rad;
    it.dtop = top;
}

// FP64 warp instructions of a cut, the quantity the batched cut minimises:
// per task, L terms of per_term (plus per_weight times the rate at which the
// low-digit weight changes), per_high per high digit for the chunk start,
// per_task_low per low digit and per_task once; per_task_weighted more when
// the low-digit weight is not constant (a low radix above 2) and
// per_task_whigh more when a high digit can carry a weight above 1 (a high
// radix above 2).
struct CutCost {
    double per_term = 0.0, per_weight = 0.0, per_high = 0.0, per_task = 0.0, per_task_low = 0.0;
    double per_task_weighted = 0.0, per_task_whigh = 0.0;
};

// The forward kernel's costs: Gray step 2l, the products 4 each, the fused
// accumulation 4, the double-double fold 10 every 32 terms; 2 DFMA per weight
// change; a chunk start 2l + 2 per high digit; per lane and task the chunk's
// last fold (8), the weighted run's (4), the high-digit weight's double-double
// product (14, when some high digit has radix > 2; the lane sum itself is
// integer work) and the staging (2k).
static CutCost forward_cut_cost(const ItemPlan& it)
{
    int cmax = 1;
    for (int c : it.cmul)
        cmax = std::max(cmax, c);
    const double products = (cmax == 1) ? (it.l - 2) : (it.l + cmax - 3);
    CutCost cc;
    cc.per_term = 2.0 * it.l + 4.0 * std::max(products, 0.0) + 4.0 + 10.0 / 32.0;
    cc.per_weight = 2.0;
    cc.per_high = 2.0 * it.l + 2.0;
    cc.per_task = 8.0 + 2.0 * it.k;
    cc.per_task_weighted = 4.0;
    cc.per_task_whigh = 14.0;
    return cc;
}

// Cut the item's code into chunks of the lowest digits: the longest prefix of
// digits whose radix product stays within the target length.  With reorder
// (batched plans), the low digits may be any sub-multiset of the digits, not
// only a prefix of the ascending list; see below.  cc: the kernel's costs
// (default: the forward's).
static void choose_chunks(ItemPlan& it, int log2_cap, int jmax = kMaxLowDigits,
                          int64_t min_chunks = kWarp, bool reorder = false,
                          const CutCost* cc = nullptr)
{
    if (it.trivial) {
        it.J = 0;
        it.L = 1;
        it.nchunks = 0;
        return;
    }
    if (reorder)  // start from the ascending order, whatever an earlier cut chose
        order_digits(it, {});
    int64_t target = it.T / min_chunks;  // aim for at least min_chunks chunks
    int64_t cap = int64_t(1) << std::max(0, std::min(log2_cap, 30));
    if (target > cap)
        target = cap;
    if (target < 1)
        target = 1;
    int J = 0;
    int64_t L = 1;
    while (J < (int)it.drad.size() && J < jmax && it.drad[J] <= kMaxLowRadix &&
           L * it.drad[J] <= target) {
        L *= it.drad[J];
        ++J;
    }
    if (min_chunks == kWarp) {
        // Batched method: among the neighbouring cuts (one digit longer, up
        // to two shorter) take the one with the fewest FP64 warp instructions:
        // every lane of a task executes L terms whether or not it has a chunk,
        // and every task pays its chunk start-up and reductions.
        const CutCost k = cc ? *cc : forward_cut_cost(it);
        const int nd = (int)it.drad.size();
        auto cost_rate = [&](int j, int64_t lj, double wrate, bool whigh) {
            const double ppt = k.per_term + k.per_weight * wrate;
            const double ovh = (nd - j) * k.per_high + k.per_task + j * k.per_task_low +
                               (wrate > 0.0 ? k.per_task_weighted : 0.0) +
                               (whigh ? k.per_task_whigh : 0.0);
            const int64_t tasks = (it.T / lj + kWarp - 1) / kWarp;
            return tasks * ((double)lj * ppt + ovh);
        };
        auto cost_of = [&](int j, int64_t lj) {
            bool whigh = false;
            for (int d = j; d < nd; ++d)
                whigh = whigh || it.drad[d] > 2;
            return cost_rate(j, lj, weight_change_rate(it.drad, j), whigh);
        };
        int bestJ = J;
        int64_t bestL = L;
        double best = cost_of(J, L);
        int64_t lj = 1;
        for (int j = 0; j <= J + 1 && j <= nd && j <= jmax; ++j) {
            if (j > 0) {
                if (it.drad[j - 1] > kMaxLowRadix)
                    break;
                lj *= it.drad[j - 1];
            }
            if (j < J - 2 || (j == J + 1 && lj > cap))
                continue;
            const double c = cost_of(j, lj);
            if (c < best * 0.999) {
                best = c;
                bestJ = j;
                bestL = lj;
            }
        }
        J = bestJ;
        L = bestL;
        if (reorder) {
            // Any sub-multiset of the digits can be the low ones.  The number
            // of chunks is the product of the high radices, and a task is 32
            // of them, so the prefix cuts often leave most lanes of a
            // permanent's last task without a chunk (36 chunks: two tasks, 28
            // idle lanes); choosing which radices go low finds chunk counts
            // that fill the tasks (ragged batch: 3.9% fewer FP64 instructions
            // by this model).  Depth-first over the counts of each distinct
            // radix, products within the cap, at most 4096 cuts evaluated;
            // a cut replaces the prefix cut only if 0.1% cheaper.
            std::vector<int> vals, cnt;
            for (int v : it.drad) {
                if (v > kMaxLowRadix)
                    break;  // ascending: no larger radix can go low
                if (vals.empty() || vals.back() != v) {
                    vals.push_back(v);
                    cnt.push_back(0);
                }
                ++cnt.back();
            }
            std::vector<int> cur(vals.size(), 0), bestc;
            int budget = 4096;
            std::function<void(size_t, int, int64_t)> dfs = [&](size_t i, int j, int64_t lj) {
                if (budget <= 0)
                    return;
                if (i == vals.size()) {
                    --budget;
                    const int a2 = (!vals.empty() && vals[0] == 2) ? cur[0] : 0;
                    const double wr = (a2 == j) ? 0.0 : std::ldexp(1.0, -a2);
                    bool whigh = !it.drad.empty() && it.drad.back() > kMaxLowRadix;
                    for (size_t q = 0; q < vals.size(); ++q)
                        whigh = whigh || (vals[q] > 2 && cur[q] < cnt[q]);
                    const double c = cost_rate(j, lj, wr, whigh);
                    if (c < best * 0.999) {
                        best = c;
                        bestc = cur;
                    }
                    return;
                }
                int64_t p = lj;
                for (int a = 0; a <= cnt[i] && j + a <= jmax; ++a) {
                    if (a > 0) {
                        if (p > cap / vals[i])
                            break;
                        p *= vals[i];
                    }
                    cur[i] = a;
                    dfs(i + 1, j + a, p);
                }
                cur[i] = 0;
            };
            dfs(0, 0, 1);
            if (!bestc.empty()) {
                std::vector<int> low_count(kMaxLowRadix + 1, 0);
                J = 0;
                L = 1;
                for (size_t i = 0; i < vals.size(); ++i) {
                    low_count[vals[i]] = bestc[i];
                    J += bestc[i];
                    for (int a = 0; a < bestc[i]; ++a)
                        L *= vals[i];
                }
                order_digits(it, low_count);
            }
        }
    }
    it.J = J;
    it.L = L;
    it.nchunks = it.T / L;
    it.weighted = false;
    for (int d = 0; d < J; ++d)
        if (it.drad[d] > 2)
            it.weighted = true;
}

static double fwd_flops_per_term(const ItemPlan& it)
{
    // column update 2l, n-1 complex products at 6, accumulate 2, weight 2
    return 2.0 * it.l + 6.0 * (it.n - 1) + 2.0 + (it.weighted ? 2.0 : 0.0);
}

// FP64 instructions of one term in glynn_fwd.cu: Gray step 2l; products of
// P(l) and the extra prefixes, 4 each; fused accumulation 4; 2 DFMA per
// change of the low-digit weight; the double-double fold, 10 every 32 terms.
static double fwd_instr_per_term(const ItemPlan& it)
{
    if (it.n == 1)
        return 2.0;
    int cmax = 1;
    for (int c : it.cmul)
        cmax = std::max(cmax, c);
    const double products = (cmax == 1) ? (it.l - 2) : (it.l + cmax - 3);
    return 2.0 * it.l + 4.0 * products + 4.0 + 2.0 * weight_change_rate(it.drad, it.J) +
           10.0 / 32.0;
}

static double bwd_flops_per_term(const ItemPlan& it)
{
    return fwd_flops_per_term(it) + 18.0 * it.l + 8.0 * it.k * it.l;
}

// FP64 instructions of one backward term in glynn_bwd.cu: column-sum and
// correction updates 4l; prefixes 4(l - 2); per middle column the fused
// accumulation of prefix times weighted suffix and the suffix update, 8; the
// end columns and the weighted suffix's start 6; per repeated column its
// powers, the scaled derivative and one more product, 4(c - 1) + 6.
static double bwd_instr_per_term(const ItemPlan& it, bool reg)
{
    if (it.n == 1)
        return 2.0;
    const int l = it.l;
    if (reg) {
        // register-resident walk: the step 4l, column 0's add 2; prefix
        // products c_j for columns 1 .. l-2 and c_0 - 1 for column 0; per
        // suffix column j >= 1 its c_j - 1 powers, the accumulation and the
        // suffix update, 4(c_j - 1) + 8; column 0's c_0 - 1 powers
        const std::vector<int32_t>& c = it.cmul;
        double v = 4.0 * l + 2.0 + 8.0 * (c[0] - 1);
        for (int j = 1; j < l - 1; ++j)
            v += 4.0 * c[j];
        for (int j = 1; j < l; ++j)
            v += 4.0 * (c[j] - 1) + 8.0;
        return v;
    }
    double rep = 0.0;
    for (int c : it.cmul)
        if (c >= 2)
            rep += 4.0 * (c - 1) + 6.0;
    return 4.0 * l + 4.0 * std::max(l - 2, 0) + 8.0 * std::max(l - 2, 0) + 6.0 + rep;
}

// The chunk log2 that the caller fixed for this permanent (plan option,
// autotuned class, process-wide table), or 0 if none did.
static int explicit_log2_for(const pq_plan* P, const ItemPlan& it)
{
    if (P->opts.chunk_log2 > 0)
        return P->opts.chunk_log2;
    // The shards of a permanent must cut its Gray code identically: a sharded
    // plan reads only the process-wide table, which every shard must share
    // (pq_tune_table_set / pq_tune_cache_load).
    if (P->opts.shard_count == 0 && it.n >= 0 && it.n < (int)P->class_log2.size() &&
        P->class_log2[it.n] > 0)
        return P->class_log2[it.n];
    return tune_get(it.n);
}

static int default_log2_for(const pq_plan* P, const ItemPlan& it)
{
    const int e = explicit_log2_for(P, it);
    return e > 0 ? e : 10;
}

template <typename T>
static int dev_upload(T** dst, const std::vector<T>& src)
{
    if (*dst) {
        dev_free(*dst);
        *dst = nullptr;
    }
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    cudaError_t e = dev_alloc((void**)dst, bytes);
    if (e != cudaSuccess)
        return fail(PQ_ERR_NOMEM, "device allocation of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    if (!src.empty()) {
        e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return fail(PQ_ERR_CUDA, "cudaMemcpy failed: %s", cudaGetErrorString(e));
    }
    return PQ_OK;
}

static void free_plan_device(pq_plan* P)
{
    void* ptrs[] = {P->desc_d,        P->meta_d,           P->tasks_batched_d, P->tasks_plain_d,
                    P->partials_d,    P->counters_d,       P->err_d,           P->gpart_d,
                    P->gpart_off_d,   P->grad_local_d,     P->grad_local_off_d, P->item_mat_off_d,
                    P->item_k_d,      P->item_l_d,         P->grad_out_tmp_d, P->bs_pos_d};
    for (void* p : ptrs)
        dev_free(p);
    void* bptrs[] = {P->desc_bwd_d, P->tasks_bwd_plain_d, P->tasks_bwd_batched_d,
                     P->meta_bwd_d};
    for (void* p : bptrs)
        dev_free(p);
    P->desc_bwd_d = nullptr;
    P->meta_bwd_d = nullptr;
    P->tasks_bwd_plain_d = P->tasks_bwd_batched_d = nullptr;
    P->bwd_ready = false;
    P->desc_d = nullptr;
    P->meta_d = nullptr;
    P->tasks_batched_d = P->tasks_plain_d = nullptr;
    P->partials_d = nullptr;
    P->counters_d = P->err_d = nullptr;
    P->gpart_d = nullptr;
    P->gpart_off_d = nullptr;
    P->grad_local_d = nullptr;
    P->grad_local_off_d = nullptr;
    P->item_mat_off_d = nullptr;
    P->item_k_d = P->item_l_d = nullptr;
    P->grad_out_tmp_d = nullptr;
    P->bs_pos_d = nullptr;
    if (P->graph) {
        cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
    }
}

// Chunks, tasks, descriptors, device upload.
// Raise the dynamic shared-memory limit of the plan's forward kernel.
static cudaError_t forward_prepare(const pq_plan* P)
{
    if (P->fwd_nl > 0)
        return fwd_reg_prepare(P->fwd_nl, P->wpb * fwd_reg_smem_per_warp(P->kmax, P->fwd_ld));
    if (P->fwd_nl < 0)
        return fwd_reg_mixed_prepare(P->wpb * fwd_reg_smem_per_warp(P->kmax, P->fwd_ld));
    return fwd_prepare(P->lmax, P->wpb * fwd_smem_per_warp(P->kmax, P->lmax));
}

static int schedule_and_upload(pq_plan* P)
{
    P->uploaded = false;
    if (P->graph) {  // it holds the old buffers' addresses
        cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
    }
    const int64_t np = (int64_t)P->items.size();
    P->nperm = np;
    int lmax_needed = 1, kmax = 1;
    for (const ItemPlan& it : P->items) {
        lmax_needed = std::max(lmax_needed, it.l);
        kmax = std::max(kmax, it.k);
    }
    P->lmax = lmax_needed;
    P->kmax = kmax;
    // The plain method runs one permanent per launch, so each permanent is cut
    // finely enough to occupy the whole GPU: at least 4 warps per SM, and for
    // a large permanent up to two waves of 16 resident warps per SM (chunks of
    // at least 64 terms, so that each chunk's start stays cheap; eight waves
    // measured slower at 2.9e7 terms).
    // The batched method keeps a warp's worth of chunks per permanent and
    // fills the GPU with many permanents at once.
    const int64_t plain_min = (int64_t)P->num_sms * 4 * kWarp;
    const int64_t plain_max = (int64_t)P->num_sms * 16 * 2 * kWarp;

    // Where the walk keeps its column sums.  Registers pay when every
    // permanent falls in one column class (m = 24 boson sampling, 4096
    // patterns of 12 photons: 0.92 ms against 1.08 ms in shared memory); a
    // batch that mixes classes runs one instantiation per class in one kernel,
    // whose register count is that of the widest (226: 8 warps per SM), and
    // was slower than shared memory (ragged batch: 24.6 ms against 22.7 ms),
    // so the planner takes registers for a single class only, and a caller
    // may ask for them (PQ_SUMS_REGISTERS) or for shared memory.
    {
        int cls = 0;
        bool one = true;
        for (const ItemPlan& it : P->items) {
            if (it.trivial)
                continue;
            const int c = fwd_reg_class_of(it.l);
            if (cls == 0)
                cls = c;
            else if (c != cls)
                one = false;
        }
        const bool want = P->opts.column_sums == PQ_SUMS_REGISTERS ||
                          (P->opts.column_sums == PQ_SUMS_AUTO && one);
        P->fwd_nl = (want && P->lmax <= kFwdRegMaxLd) ? (one ? std::max(cls, 4) : -1) : 0;
        P->fwd_ld = P->fwd_nl > 0   ? P->fwd_nl
                    : P->fwd_nl < 0 ? fwd_reg_class_of(P->lmax)
                                    : P->lmax;
    }
    // launch geometry (it fixes the resident warps the batched cut is balanced for)
    const int per_warp = P->fwd_nl != 0 ? fwd_reg_smem_per_warp(P->kmax, P->fwd_ld)
                                        : fwd_smem_per_warp(P->kmax, P->lmax);
    if (per_warp > 200 * 1024)
        return fail(PQ_ERR_UNSUPPORTED, "shared memory per warp %d too large", per_warp);
    int wpb = 0, bps = 0;
    launch_geometry(P->fwd_nl > 0   ? fwd_reg_regs_per_thread(P->fwd_nl)
                    : P->fwd_nl < 0 ? fwd_reg_mixed_regs_per_thread()
                                    : fwd_regs_per_thread(P->lmax),
                    per_warp,
                    P->opts.warps_per_block > 0 ? P->opts.warps_per_block : 8,
                    P->opts.blocks_per_sm > 0 ? P->opts.blocks_per_sm : 8, wpb, bps);
    P->wpb = wpb;
    P->blocks = std::max(1, P->num_sms * bps);

    if (P->opts.method == PQ_METHOD_PLAIN) {
        for (ItemPlan& it : P->items) {
            const int64_t plain_chunks = std::max(plain_min, std::min(plain_max, it.T / 64));
            choose_chunks(it, default_log2_for(P, it), kMaxLowDigits,
                          P->opts.chunk_log2 == 0 ? plain_chunks : kWarp);
        }
    } else {
        // The batched method cuts each permanent into at least a warp's worth
        // of chunks.  A small batch then has too few, too long tasks for the
        // GPU: the last ones leave SMs idle (4096 permanents of the ragged
        // recipe took 4.0 ms with chunks of up to 2^10 terms, 1.5 ms with 2^6).
        // So the chunk cap is lowered, for the whole batch, until the longest
        // warp task is at most half of a resident warp's average share of the
        // work; large batches keep their caps (65536 permanents: the longest
        // task is a quarter of a share).  Chunk lengths that the caller fixed
        // are kept as they are.
        const double warps = (double)P->blocks * P->wpb;
        auto cut_all = [&](int gcap) {
            double total = 0.0, longest = 0.0;
            for (ItemPlan& it : P->items) {
                const int e = explicit_log2_for(P, it);
                choose_chunks(it, e > 0 ? e : std::min(10, gcap), kMaxLowDigits, kWarp, true);
                if (it.trivial)
                    continue;
                const double cost = (double)it.L * fwd_flops_per_term(it) +
                                    2.0 * (double)((int)it.drow.size() - it.J) * it.l + 2.0 * it.l;
                total += cost * (double)((it.nchunks + kWarp - 1) / kWarp);
                longest = std::max(longest, cost);
            }
            return total > 0.0 ? longest / (total / warps) : 0.0;
        };
        int gcap = 30;
        double ratio = cut_all(gcap);
        if (P->opts.chunk_log2 == 0 && P->opts.shard_count == 0) {
            for (int c = 12; c >= 4 && ratio > 0.5; --c) {
                gcap = c;
                ratio = cut_all(gcap);
            }
        }
    }

    P->desc_h.assign(np, PermDesc{});
    P->meta_h.clear();
    P->tasks_plain_h.clear();
    P->plain_first.assign(np + 1, 0);
    std::vector<double> task_cost;
    int32_t slot = 0;
    double flops_f = 0.0, flops_b = 0.0, instr_f = 0.0, instr_fx = 0.0;
    int64_t terms = 0;
    for (int64_t p = 0; p < np; ++p) {
        ItemPlan& it = P->items[p];
        PermDesc& D = P->desc_h[p];
        D.T = it.T;
        D.nchunks = it.nchunks;
        D.src_off = it.src_off;
        D.k = it.k;
        D.l = it.l;
        D.n = it.n;
        D.si = it.si;
        D.sj = it.sj;
        D.meta = (int32_t)P->meta_h.size();
        D.ndig = (int32_t)it.drow.size();
        D.J = it.J;
        D.weighted = it.weighted ? 1 : 0;
        D.out = (int32_t)p;
        D.trivial = it.trivial ? 1 : 0;
        D.jf = it.jf;
        D.L = it.L;
        D.norm = it.norm;
        auto app = [&](const std::vector<int32_t>& v) {
            P->meta_h.insert(P->meta_h.end(), v.begin(), v.end());
        };
        app(it.ridx);
        app(it.cidx);
        app(it.rmul);
        app(it.cmul);
        app(it.drow);
        app(it.drad);
        app(it.dtop);
        app(it.ecnt);
        const int64_t nt_all = it.trivial ? 1 : (it.nchunks + kWarp - 1) / kWarp;
        if (nt_all > (int64_t(1) << 30))
            return fail(PQ_ERR_UNSUPPORTED, "too many tasks for one permanent");
        // A sharded plan keeps one contiguous part range of every permanent.
        // The ranges are cut in R equal pieces, and permanent p gives piece
        // (shard_index + p) mod R to this shard: a permanent with fewer tasks
        // than shards then lands on a different shard for each p, instead of
        // always on the last one.
        int64_t q0 = 0, q1 = nt_all;
        if (P->opts.shard_count > 1) {
            const int64_t R = P->opts.shard_count;
            const int64_t piece = (P->opts.shard_index + p) % R;
            q0 = nt_all * piece / R;
            q1 = nt_all * (piece + 1) / R;
        }
        const int64_t nt = q1 - q0;
        D.ntasks = (int32_t)nt;
        D.part0 = (int32_t)q0;
        D.slot0 = slot;
        slot += (int32_t)nt;
        P->plain_first[p] = (int64_t)P->tasks_plain_h.size();
        const double fpt = it.trivial ? 0.0 : fwd_flops_per_term(it);
        const double init = 2.0 * (it.drow.size() - it.J) * it.l + 2.0 * it.l;
        for (int64_t q = q0; q < q1; ++q) {
            Task t;
            t.perm = (int32_t)p;
            t.part = (int32_t)q;
            P->tasks_plain_h.push_back(t);
            task_cost.push_back((double)it.L * fpt + init);
        }
        if (!it.trivial && nt > 0) {
            // terms of this plan's chunks (all of them unless sharded)
            const int64_t c1 = std::min<int64_t>(it.nchunks, q1 * kWarp);
            const int64_t tt = (c1 - q0 * kWarp) * it.L;
            terms += tt;
            flops_f += (double)tt * fpt;
            instr_f += (double)tt * fwd_instr_per_term(it);
            flops_b += (double)tt * bwd_flops_per_term(it);
            // per task, every lane: L terms, the chunk start ((ndig - J) row
            // updates of 2l), the chunk's last folds (8, 12 when weighted) and
            // the high-digit weight's product (14, when a high radix is above
            // 2); the lane sum is integer work.  Per permanent with several
            // tasks, the partials' double-double sum (14 per 32 tasks and lane)
            bool whigh = false;
            for (size_t d = it.J; d < it.drad.size(); ++d)
                whigh = whigh || it.drad[d] > 2;
            const double lane = (double)it.L * fwd_instr_per_term(it) +
                                2.0 * it.l * (double)((int)it.drow.size() - it.J) +
                                (it.weighted ? 12.0 : 8.0) + (whigh ? 14.0 : 0.0);
            instr_fx += (double)nt * 32.0 * lane;
            if (nt > 1)
                instr_fx += 32.0 * 14.0 * (double)((nt + kWarp - 1) / kWarp);
        }
        if (slot < 0)
            return fail(PQ_ERR_UNSUPPORTED, "too many tasks");
    }
    P->plain_first[np] = (int64_t)P->tasks_plain_h.size();
    // batched order: longest task first (LPT), ties by permanent then part
    std::vector<int64_t> order(P->tasks_plain_h.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return task_cost[a] > task_cost[b]; });
    P->tasks_batched_h.resize(order.size());
    for (size_t q = 0; q < order.size(); ++q)
        P->tasks_batched_h[q] = P->tasks_plain_h[order[q]];

    P->stats.permanents = np;
    P->stats.terms = terms;
    P->stats.flops_forward = flops_f;
    P->stats.flops_backward = flops_b;
    P->stats.fp64_instr_forward = instr_f;
    P->stats.fp64_instr_forward_executed = instr_fx;
    P->stats.tasks = (int64_t)P->tasks_plain_h.size();
    P->stats.launches_forward = (P->opts.method == PQ_METHOD_PLAIN) ? np : 1;
    P->stats.launches_backward = (P->opts.method == PQ_METHOD_PLAIN) ? np + 1 : 2;
    P->stats.lmax = P->lmax;
    P->stats.column_sums = P->fwd_nl != 0 ? PQ_SUMS_REGISTERS : PQ_SUMS_SHARED;

    // upload
    int rc;
    if ((rc = dev_upload(&P->desc_d, P->desc_h)) != PQ_OK)
        return rc;
    if ((rc = dev_upload(&P->meta_d, P->meta_h)) != PQ_OK)
        return rc;
    if ((rc = dev_upload(&P->tasks_plain_d, P->tasks_plain_h)) != PQ_OK)
        return rc;
    if ((rc = dev_upload(&P->tasks_batched_d, P->tasks_batched_h)) != PQ_OK)
        return rc;
    dev_free(P->partials_d);
    P->partials_d = nullptr;
    P->nslots = slot;
    PQ_ALLOC(&P->partials_d, std::max<size_t>(slot, 1) * 4 * sizeof(double));
    dev_free(P->counters_d);
    P->counters_d = nullptr;
    PQ_ALLOC(&P->counters_d, (size_t)(np + 1) * sizeof(int32_t));
    if (!P->err_d) {
        PQ_ALLOC(&P->err_d, 2 * sizeof(int32_t));
        PQ_CUDA(cudaMemset(P->err_d, 0, 2 * sizeof(int32_t)));
    }
    cudaError_t e = forward_prepare(P);
    if (e != cudaSuccess)
        return fail(PQ_ERR_CUDA, "kernel attribute setup failed: %s", cudaGetErrorString(e));
    P->uploaded = true;
    return PQ_OK;
}

// Plan objects are counted like device buffers (pq_debug_live_allocations),
// and the allocation-failure test hook applies to them as well.
static pq_plan* plan_new()
{
    if (!host_object_alloc_ok())
        return nullptr;
    pq_plan* P = new (std::nothrow) pq_plan();
    if (!P)
        host_object_freed();
    return P;
}

static void plan_delete(pq_plan* P)
{
    if (!P)
        return;
    delete P;
    host_object_freed();
}

static int plan_common_init(pq_plan* P, const pq_plan_options* opts)
{
    if (opts)
        P->opts = *opts;
    if (P->opts.method != PQ_METHOD_BATCHED && P->opts.method != PQ_METHOD_PLAIN)
        return fail(PQ_ERR_ARG, "unknown method %d", P->opts.method);
    if (P->opts.chunk_log2 < 0 || P->opts.chunk_log2 > 30)
        return fail(PQ_ERR_ARG, "chunk_log2 %d outside [0, 30]", P->opts.chunk_log2);
    if (P->opts.warps_per_block < 0 || P->opts.warps_per_block > 16)
        return fail(PQ_ERR_ARG, "warps_per_block %d outside [0, 16]", P->opts.warps_per_block);
    if (P->opts.blocks_per_sm < 0 || P->opts.blocks_per_sm > 32)
        return fail(PQ_ERR_ARG, "blocks_per_sm %d outside [0, 32]", P->opts.blocks_per_sm);
    if (P->opts.column_sums < PQ_SUMS_AUTO || P->opts.column_sums > PQ_SUMS_REGISTERS)
        return fail(PQ_ERR_ARG, "column_sums %d is not a PQ_SUMS_* value", P->opts.column_sums);
    if (P->opts.shard_count < 0 || P->opts.shard_count > 65536 || P->opts.shard_index < 0 ||
        (P->opts.shard_count > 0 && P->opts.shard_index >= P->opts.shard_count) ||
        (P->opts.shard_count == 0 && P->opts.shard_index != 0))
        return fail(PQ_ERR_ARG, "shard %d of %d", P->opts.shard_index, P->opts.shard_count);
    PQ_CUDA(cudaGetDevice(&P->device));
    PQ_CUDA(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device));
    return PQ_OK;
}

// The size arrays a batch needs: all of them for a non-empty batch, except
// that the multiplicity arrays may be null when every item has no rows
// (row_mult) or no columns (col_mult), as a batch of n = 0 items has.
static bool sizes_present(const pq_batch_sizes* sz, bool need_mat_off)
{
    if (sz->batch <= 0)
        return true;
    if (!sz->k || !sz->l || !sz->row_off || !sz->col_off || (need_mat_off && !sz->mat_off))
        return false;
    bool rows = false, cols = false;
    for (int64_t b = 0; b < sz->batch; ++b) {
        rows = rows || sz->k[b] > 0;
        cols = cols || sz->l[b] > 0;
    }
    return (!rows || sz->row_mult) && (!cols || sz->col_mult);
}

extern "C" int pq_plan_create(const pq_batch_sizes* sz, const pq_plan_options* opts,
                              pq_plan** out)
{
    if (!sz || !out)
        return fail(PQ_ERR_ARG, "null argument");
    *out = nullptr;
    if (sz->batch < 0)
        return fail(PQ_ERR_ARG, "negative batch");
    if (!sizes_present(sz, true))
        return fail(PQ_ERR_ARG, "null size array");
    if (sz->batch > (int64_t(1) << 30))
        return fail(PQ_ERR_UNSUPPORTED, "batch above 2^30");
    pq_plan* P = plan_new();
    if (!P)
        return fail(PQ_ERR_NOMEM, "host allocation failed");
    int rc = plan_common_init(P, opts);
    if (rc != PQ_OK) {
        plan_delete(P);
        return rc;
    }
    P->kind = 0;
    P->items.resize(sz->batch);
    P->item_mat_off.resize(sz->batch);
    P->item_k.resize(sz->batch);
    P->item_l.resize(sz->batch);
    int64_t off = 0;
    for (int64_t b = 0; b < sz->batch; ++b) {
        if (sz->row_off[b] < 0 || sz->col_off[b] < 0 || sz->mat_off[b] < 0) {
            plan_delete(P);
            return fail(PQ_ERR_ARG, "negative offset at item %lld", (long long)b);
        }
        rc = build_item(sz->row_mult + sz->row_off[b], sz->col_mult + sz->col_off[b], sz->k[b],
                        sz->l[b], sz->mat_off[b], sz->l[b], P->items[b]);
        if (rc != PQ_OK) {
            plan_delete(P);
            return fail(rc, "item %lld: %s", (long long)b, g_err.c_str());
        }
        P->item_mat_off[b] = sz->mat_off[b];
        P->item_k[b] = sz->k[b];
        P->item_l[b] = sz->l[b];
        off += (int64_t)sz->k[b] * sz->l[b];
    }
    P->total_mat_elems = off;
    P->class_log2.assign(PQ_MAX_N + 1, 0);
    rc = schedule_and_upload(P);
    if (rc != PQ_OK) {
        free_plan_device(P);
        plan_delete(P);
        return rc;
    }
    *out = P;
    return PQ_OK;
}

static double factorial_d(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i)
        r *= (double)i;
    return r;
}

extern "C" int pq_plan_create_bs(int32_t m, const int32_t* in_occ, const int32_t* out_occ,
                                 int64_t B, const pq_plan_options* opts, pq_plan** out)
{
    if (!out || !in_occ || (B > 0 && !out_occ))
        return fail(PQ_ERR_ARG, "null argument");
    *out = nullptr;
    if (m <= 0 || m > PQ_MAX_DIM)
        return fail(m <= 0 ? PQ_ERR_ARG : PQ_ERR_UNSUPPORTED, "m = %d outside [1, %d]", m,
                    PQ_MAX_DIM);
    if (B < 0)
        return fail(PQ_ERR_ARG, "negative pattern count");
    if (B > (int64_t(1) << 30))
        return fail(PQ_ERR_UNSUPPORTED, "more than 2^30 patterns");
    int ns = 0;
    double fs = 1.0;
    for (int i = 0; i < m; ++i) {
        if (in_occ[i] < 0)
            return fail(PQ_ERR_ARG, "negative input occupation");
        ns += in_occ[i];
        fs *= factorial_d(in_occ[i]);
    }
    if (opts && opts->shard_count > 1)
        return fail(PQ_ERR_UNSUPPORTED, "boson-sampling plans are not sharded");
    pq_plan* P = plan_new();
    if (!P)
        return fail(PQ_ERR_NOMEM, "host allocation failed");
    int rc = plan_common_init(P, opts);
    if (rc != PQ_OK) {
        plan_delete(P);
        return rc;
    }
    P->kind = 1;
    P->m = m;
    P->in_occ.assign(in_occ, in_occ + m);
    P->out_occ.assign(out_occ, out_occ + B * m);
    P->items.resize(B);
    for (int64_t b = 0; b < B; ++b) {
        const int32_t* t = out_occ + b * m;
        int nt = 0;
        double ft = 1.0;
        for (int i = 0; i < m; ++i) {
            if (t[i] < 0) {
                plan_delete(P);
                return fail(PQ_ERR_ARG, "negative output occupation in pattern %lld",
                            (long long)b);
            }
            nt += t[i];
            ft *= factorial_d(t[i]);
        }
        if (nt != ns) {
            plan_delete(P);
            return fail(PQ_ERR_ARG, "pattern %lld has %d photons, input has %d", (long long)b, nt,
                        ns);
        }
        // rows = output modes (t), columns = input modes (s); U[out][in]
        rc = build_item(t, in_occ, m, m, 0, m, P->items[b]);
        if (rc != PQ_OK) {
            plan_delete(P);
            return fail(rc, "pattern %lld: %s", (long long)b, g_err.c_str());
        }
        P->items[b].norm = 1.0 / (ft * fs);
    }
    P->class_log2.assign(PQ_MAX_N + 1, 0);
    rc = schedule_and_upload(P);
    if (rc != PQ_OK) {
        free_plan_device(P);
        plan_delete(P);
        return rc;
    }
    *out = P;
    return PQ_OK;
}

extern "C" int pq_plan_destroy(pq_plan* P)
{
    if (!P)
        return PQ_OK;
    cudaDeviceSynchronize();
    free_plan_device(P);
    plan_delete(P);
    return PQ_OK;
}

extern "C" int pq_plan_get_stats(const pq_plan* P, pq_plan_stats* out)
{
    if (!P || !out)
        return fail(PQ_ERR_ARG, "null argument");
    *out = P->stats;
    return PQ_OK;
}

// ---------------------------------------------------------------- execution
static ExecArgs exec_args(pq_plan* P, const void* src, void* amps, double* probs, bool batched,
                          double* partial = nullptr)
{
    ExecArgs a;
    a.out_partial = partial;
    a.desc = P->desc_d;
    a.meta = P->meta_d;
    a.tasks = batched ? P->tasks_batched_d : P->tasks_plain_d;
    a.ntasks = (int64_t)P->tasks_plain_h.size();
    a.src = reinterpret_cast<const double2*>(src);
    a.out_amp = reinterpret_cast<double2*>(amps);
    a.out_prob = probs;
    a.partials = P->partials_d;
    a.counters = P->counters_d;
    a.err = P->err_d;
    a.nperm = P->nperm;
    a.nmeta = (int64_t)P->meta_h.size();
    a.nslots = P->nslots;
    return a;
}

static int run_forward_raw(pq_plan* P, const void* src, void* amps, double* probs,
                           cudaStream_t st, double* partial = nullptr)
{
    if (!P->uploaded)
        return fail(PQ_ERR_STATE, "the plan lost its device data in a failed re-planning");
    PQ_CUDA(cudaMemsetAsync(P->counters_d, 0, (size_t)(P->nperm + 1) * sizeof(int32_t), st));
    if (P->nperm == 0)
        return PQ_OK;
    if (P->opts.method == PQ_METHOD_PLAIN) {
        ExecArgs a = exec_args(P, src, amps, probs, false, partial);
        for (int64_t p = 0; p < P->nperm; ++p) {
            const int64_t tb = P->plain_first[p], te = P->plain_first[p + 1];
            const unsigned grid = (unsigned)((te - tb + P->wpb - 1) / P->wpb);
            cudaError_t e =
                P->fwd_nl > 0 ? fwd_reg_launch(P->fwd_nl, a, tb, te, P->kmax, P->fwd_ld, grid,
                                               P->wpb, 0, st)
                : P->fwd_nl < 0
                    ? fwd_reg_mixed_launch(a, tb, te, P->kmax, P->fwd_ld, grid, P->wpb, 0, st)
                    : fwd_launch_plain(P->lmax, a, tb, te, P->kmax, P->wpb, st);
            if (e != cudaSuccess)
                return fail(PQ_ERR_CUDA, "plain launch failed: %s", cudaGetErrorString(e));
        }
        return PQ_OK;
    }
    ExecArgs a = exec_args(P, src, amps, probs, true, partial);
    if (P->fwd_nl != 0) {
        cudaError_t e =
            P->fwd_nl > 0 ? fwd_reg_launch(P->fwd_nl, a, 0, a.ntasks, P->kmax, P->fwd_ld,
                                           (unsigned)P->blocks, P->wpb, 1, st)
                          : fwd_reg_mixed_launch(a, 0, a.ntasks, P->kmax, P->fwd_ld,
                                                 (unsigned)P->blocks, P->wpb, 1, st);
        if (e != cudaSuccess)
            return fail(PQ_ERR_CUDA, "persistent launch failed: %s", cudaGetErrorString(e));
        return PQ_OK;
    }
    cudaError_t e = fwd_launch_persistent(P->lmax, a, P->kmax, P->blocks, P->wpb, st);
    if (e != cudaSuccess)
        return fail(PQ_ERR_CUDA, "persistent launch failed: %s", cudaGetErrorString(e));
    return PQ_OK;
}

static int run_forward(pq_plan* P, const void* src, void* amps, double* probs, cudaStream_t st)
{
    bool graph = P->opts.use_graph && P->opts.method == PQ_METHOD_BATCHED && st != nullptr;
    if (graph) {
        // Inside a caller's stream capture the launch is simply recorded into
        // the caller's graph (a capture cannot begin on a capturing stream).
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        PQ_CUDA(cudaStreamIsCapturing(st, &cs));
        graph = (cs == cudaStreamCaptureStatusNone);
    }
    if (!graph)
        return run_forward_raw(P, src, amps, probs, st);
    const void* key[4] = {src, amps, probs, st};
    if (P->graph && std::memcmp(key, P->graph_key, sizeof(key)) != 0) {
        cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
    }
    if (!P->graph) {
        cudaGraph_t g = nullptr;
        PQ_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = run_forward_raw(P, src, amps, probs, st);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (rc != PQ_OK) {
            if (g)
                cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess)
            return fail(PQ_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&P->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            P->graph = nullptr;
            return fail(PQ_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
        }
        std::memcpy(P->graph_key, key, sizeof(key));
    }
    PQ_CUDA(cudaGraphLaunch(P->graph, st));
    return PQ_OK;
}

// Read (and optionally clear) the plan's device error record; synchronous.
static int read_device_error(pq_plan* P, int32_t* code, int64_t* task, bool clear)
{
    int32_t rec[2] = {0, 0};
    *code = 0;
    *task = 0;
    if (!P->err_d)
        return PQ_OK;
    PQ_CUDA(cudaMemcpy(rec, P->err_d, sizeof(rec), cudaMemcpyDeviceToHost));
    if (clear && (rec[0] || rec[1]))
        PQ_CUDA(cudaMemset(P->err_d, 0, sizeof(rec)));
    *code = rec[0];
    *task = rec[1];
    return PQ_OK;
}

// After the synchronous convenience path: fail loudly if a guard tripped.
static int check_device_error(pq_plan* P)
{
    int32_t code = 0;
    int64_t task = 0;
    int rc = read_device_error(P, &code, &task, false);
    if (rc != PQ_OK)
        return rc;
    if (code)
        return fail(PQ_ERR_STATE, "kernel guard %d tripped at task %lld", code, (long long)task);
    return PQ_OK;
}

extern "C" int pq_plan_device_error(pq_plan* P, int32_t* code, int64_t* task, int32_t clear)
{
    if (!P || !code || !task)
        return fail(PQ_ERR_ARG, "null argument");
    return read_device_error(P, code, task, clear != 0);
}

extern "C" int pq_debug_corrupt_plan(pq_plan* P, int32_t what)
{
    if (!P)
        return fail(PQ_ERR_ARG, "null plan");
    if (P->nperm == 0)
        return fail(PQ_ERR_ARG, "empty plan");
    if (what == 1) {
        Task t = P->tasks_batched_h[0];
        t.perm = (int32_t)(P->nperm + 5);
        PQ_CUDA(cudaMemcpy(P->tasks_batched_d, &t, sizeof(t), cudaMemcpyHostToDevice));
        t = P->tasks_plain_h[0];
        t.perm = (int32_t)(P->nperm + 5);
        PQ_CUDA(cudaMemcpy(P->tasks_plain_d, &t, sizeof(t), cudaMemcpyHostToDevice));
        return PQ_OK;
    }
    if (what == 2) {
        PermDesc D = P->desc_h[0];
        D.l = P->lmax + 7;
        PQ_CUDA(cudaMemcpy(P->desc_d, &D, sizeof(D), cudaMemcpyHostToDevice));
        return PQ_OK;
    }
    return fail(PQ_ERR_ARG, "unknown corruption %d", what);
}

// Sizes of a device batch descriptor copied to the host (convenience path).
struct HostSizes {
    std::vector<int32_t> k, l, rm, cm;
    std::vector<int64_t> ro, co, mo;
    pq_batch_sizes view() const
    {
        pq_batch_sizes s;
        s.batch = (int64_t)k.size();
        s.mat_off = mo.data();
        s.k = k.data();
        s.l = l.data();
        s.row_mult = rm.data();
        s.row_off = ro.data();
        s.col_mult = cm.data();
        s.col_off = co.data();
        return s;
    }
};

static int fetch_sizes(const pq_batch* b, HostSizes& h)
{
    const int64_t n = b->batch;
    h.k.resize(n);
    h.l.resize(n);
    h.ro.resize(n);
    h.co.resize(n);
    h.mo.resize(n);
    if (n == 0)
        return PQ_OK;
    if (!b->k || !b->l || !b->row_off || !b->col_off || !b->row_mult || !b->col_mult ||
        !b->mat_off)
        return fail(PQ_ERR_ARG, "null pointer in batch descriptor");
    PQ_CUDA(cudaMemcpy(h.k.data(), b->k, n * 4, cudaMemcpyDeviceToHost));
    PQ_CUDA(cudaMemcpy(h.l.data(), b->l, n * 4, cudaMemcpyDeviceToHost));
    PQ_CUDA(cudaMemcpy(h.ro.data(), b->row_off, n * 8, cudaMemcpyDeviceToHost));
    PQ_CUDA(cudaMemcpy(h.co.data(), b->col_off, n * 8, cudaMemcpyDeviceToHost));
    PQ_CUDA(cudaMemcpy(h.mo.data(), b->mat_off, n * 8, cudaMemcpyDeviceToHost));
    int64_t nr = 0, nc = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (h.k[i] < 0 || h.l[i] < 0 || h.ro[i] < 0 || h.co[i] < 0)
            return fail(PQ_ERR_ARG, "negative size or offset at item %lld", (long long)i);
        nr = std::max(nr, h.ro[i] + h.k[i]);
        nc = std::max(nc, h.co[i] + h.l[i]);
    }
    h.rm.resize(nr);
    h.cm.resize(nc);
    if (nr)
        PQ_CUDA(cudaMemcpy(h.rm.data(), b->row_mult, nr * 4, cudaMemcpyDeviceToHost));
    if (nc)
        PQ_CUDA(cudaMemcpy(h.cm.data(), b->col_mult, nc * 4, cudaMemcpyDeviceToHost));
    return PQ_OK;
}

static int check_batch_plan(const pq_plan* P, const pq_batch* b, bool sharded = false)
{
    if (P->kind != 0)
        return fail(PQ_ERR_STATE, "plan was made for boson sampling, not a permanent batch");
    if (sharded != (P->opts.shard_count > 0))
        return fail(PQ_ERR_STATE, sharded ? "plan is not sharded: use pq_permanent_batched"
                                          : "sharded plan: use pq_permanent_partials");
    if (b->batch != P->nperm)
        return fail(PQ_ERR_STATE, "plan made for %lld items, batch has %lld",
                    (long long)P->nperm, (long long)b->batch);
    return PQ_OK;
}

extern "C" int pq_permanent_batched(const pq_batch* b, pq_c128* out, pq_plan* plan, void* stream)
{
    if (!b || (b->batch > 0 && (!out || !b->mats)))
        return fail(PQ_ERR_ARG, "null argument");
    if (b->batch < 0)
        return fail(PQ_ERR_ARG, "negative batch");
    cudaStream_t st = (cudaStream_t)stream;
    if (plan) {
        int rc = check_batch_plan(plan, b);
        if (rc != PQ_OK)
            return rc;
        return run_forward(plan, b->mats, out, nullptr, st);
    }
    HostSizes h;
    int rc = fetch_sizes(b, h);
    if (rc != PQ_OK)
        return rc;
    pq_batch_sizes sz = h.view();
    pq_plan* P = nullptr;
    rc = pq_plan_create(&sz, nullptr, &P);
    if (rc != PQ_OK)
        return rc;
    rc = run_forward_raw(P, b->mats, out, nullptr, st);
    if (rc == PQ_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess)
            rc = fail(PQ_ERR_CUDA, "stream synchronize failed: %s", cudaGetErrorString(e));
    }
    if (rc == PQ_OK)
        rc = check_device_error(P);
    pq_plan_destroy(P);
    return rc;
}

extern "C" int pq_permanent_partials(const pq_batch* b, double* partials, pq_plan* plan,
                                     void* stream)
{
    if (!b || !plan || (b->batch > 0 && (!partials || !b->mats)))
        return fail(PQ_ERR_ARG, "null argument");
    int rc = check_batch_plan(plan, b, true);
    if (rc != PQ_OK)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (b->batch == 0)
        return PQ_OK;
    // permanents none of whose tasks fall in this shard contribute zero
    PQ_CUDA(cudaMemsetAsync(partials, 0, (size_t)b->batch * 4 * sizeof(double), st));
    return run_forward_raw(plan, b->mats, nullptr, nullptr, st, partials);
}

extern "C" int pq_bs_probs(const pq_c128* U, int32_t m, const int32_t* in_occ,
                           const int32_t* out_occ, int64_t B, double* probs, pq_c128* amps,
                           pq_plan* plan, void* stream)
{
    if (!U || !in_occ || (B > 0 && (!out_occ || !probs)))
        return fail(PQ_ERR_ARG, "null argument");
    if (m <= 0 || m > PQ_MAX_DIM || B < 0)
        return fail(PQ_ERR_ARG, "bad sizes m = %d, B = %lld", m, (long long)B);
    cudaStream_t st = (cudaStream_t)stream;
    if (plan) {
        if (plan->kind != 1 || plan->m != m || plan->nperm != B)
            return fail(PQ_ERR_STATE, "plan was made for different occupations");
        return run_forward(plan, U, amps, probs, st);
    }
    std::vector<int32_t> s(m), t((size_t)B * m);
    PQ_CUDA(cudaMemcpy(s.data(), in_occ, m * 4, cudaMemcpyDeviceToHost));
    if (B)
        PQ_CUDA(cudaMemcpy(t.data(), out_occ, (size_t)B * m * 4, cudaMemcpyDeviceToHost));
    pq_plan* P = nullptr;
    int rc = pq_plan_create_bs(m, s.data(), t.data(), B, nullptr, &P);
    if (rc != PQ_OK)
        return rc;
    rc = run_forward_raw(P, U, amps, probs, st);
    if (rc == PQ_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess)
            rc = fail(PQ_ERR_CUDA, "stream synchronize failed: %s", cudaGetErrorString(e));
    }
    if (rc == PQ_OK)
        rc = check_device_error(P);
    pq_plan_destroy(P);
    return rc;
}

// ---------------------------------------------------------------- probe
extern "C" int pq_probe_fp64_peak(int64_t iters, double* flops_per_s, double* ms, void* stream)
{
    if (!flops_per_s || !ms || iters <= 0)
        return fail(PQ_ERR_ARG, "bad argument");
    cudaError_t e = fp64_probe(iters, flops_per_s, ms, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return fail(PQ_ERR_CUDA, "fp64 probe failed: %s", cudaGetErrorString(e));
    return PQ_OK;
}

// ---------------------------------------------------------------- backward
// The backward pass keeps one row of per-lane corrections for each low digit
// in shared memory, so it uses its own chunks: at most kBwdMaxLowDigits low
// digits and 2^kBwdChunkLog2 terms (radices 3 and 4 among the chunk's digits
// make chunks longer than 2^J; on the ragged batch caps of 2^4 .. 2^8 terms
// took 78.2, 73.2, 71.1, 70.6 and 71.7 ms: fewer chunk starts, each of which
// costs 2l per high digit).
// Product-column bounds of the backward launch classes: every permanent runs
// in the launch of the smallest bound that holds its l, so its per-lane
// workspace (column sums, accumulators, prefixes, corrections) is sized for
// permanents like it rather than for the largest in the batch.
static const int kBwdClassLd[] = {2, 4, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32, 40};

static int ensure_backward(pq_plan* P)
{
    if (P->bwd_ready)
        return PQ_OK;
    const int64_t np = P->nperm;
    std::vector<ItemPlan> items = P->items;
    P->desc_bwd_h = P->desc_h;
    P->tasks_bwd_plain_h.clear();
    P->plain_first_bwd.assign(np + 1, 0);
    P->bwd_class_of.assign(np, 0);
    const int ncls = (int)(sizeof(kBwdClassLd) / sizeof(kBwdClassLd[0]));
    std::vector<BwdClass> cls(ncls);
    std::vector<int> cls_used(ncls, 0);
    std::vector<double> cls_terms(ncls, 0.0), cls_nterms(ncls, 0.0);
    for (int c = 0; c < ncls; ++c)
        cls[c].ld = kBwdClassLd[c];
    for (int64_t p = 0; p < np; ++p) {
        const ItemPlan& it = items[p];
        int c = 0;
        while (c + 1 < ncls && kBwdClassLd[c] < it.l)
            ++c;
        P->bwd_class_of[p] = c;
        cls_used[c] = 1;
        cls[c].kmax = std::max(cls[c].kmax, it.k);
        int c2 = 0;
        for (int cm : it.cmul)
            c2 += (cm >= 2) ? 1 : 0;
        cls[c].n2 = std::max(cls[c].n2, c2);
        if (!it.trivial) {
            cls_terms[c] += (double)it.T;
            cls_nterms[c] += (double)it.T * it.n;
        }
    }
    // Low digits per chunk for each class: each digit costs every lane one row
    // of corrections; fewer digits mean shorter chunks whose start-up (column
    // sums from the high digits, about 2l(n - J) operations) is paid more
    // often.  Take the J that maximises (share of 8 warps per SM) x (share of
    // the work that is per-term work): four warps saturate a plain FP64 loop,
    // but the backward's prefix and suffix chains wait on their own results,
    // and a second warp per SMSP hides that (ragged batch: 121 ms with the
    // share taken of 4 warps, 114 ms of 6 or 8).
    for (int c = 0; c < ncls; ++c) {
        if (!cls_used[c])
            continue;
        BwdClass& C = cls[c];
        C.reg = bwdr_supported(C.ld) ? 1 : 0;
        const int regs = C.reg ? bwdr_regs_per_thread(C.ld) : bwd_regs_per_thread(C.ld);
        const double nbar = cls_terms[c] > 0 ? cls_nterms[c] / cls_terms[c] : 1.0;
        double best = -1.0;
        for (int J = kBwdMaxLowDigits; J >= 1; --J) {
            const int per_warp = C.reg ? bwdr_smem_bytes_for(C.kmax, C.ld, J)
                                       : bwd_smem_bytes_for(C.kmax, C.ld, J, C.n2);
            if (per_warp > 200 * 1024)
                continue;
            int wpb = 0, bps = 0;
            launch_geometry_max(regs, per_warp, 8, wpb, bps);
            const double warps = std::min(8.0, (double)(wpb * bps)) / 8.0;
            const double per_term = 16.0 * C.ld - 10.0;
            const double start = std::max(0.0, nbar - J) * 2.0 * C.ld / (double)(1 << J);
            const double score = warps * per_term / (per_term + start);
            if (score > best) {
                best = score;
                C.jb = J;
                C.wpb = wpb;
                C.blocks = std::max(1, P->num_sms * bps);
            }
        }
        if (best < 0)
            return fail(PQ_ERR_UNSUPPORTED, "backward shared memory for l <= %d too large", C.ld);
    }
    std::vector<double> cost;
    std::vector<int64_t> gpart_off(np), gl_off(np);
    int64_t gpart = 0, gl = 0;
    double instr_b = 0.0;
    // The backward cuts each permanent with its own costs and its own choice
    // of low digits (any sub-multiset, as the forward), so its digit order
    // can differ from the forward's: the backward reads a copy of the
    // metadata pool whose digit sections follow its order.
    std::vector<int32_t> meta_bwd = P->meta_h;
    // per term as glynn_bwd.cu counts it; a chunk start 2l per high digit;
    // per task the staging (k), the lane contraction (2l per low digit, about
    // 2kl) and the gradient write
    auto bwd_cut_cost = [&](const ItemPlan& it, const BwdClass& C) {
        CutCost bc;
        bc.per_term = bwd_instr_per_term(it, C.reg != 0);
        bc.per_high = 2.0 * it.l;
        bc.per_task = it.k + 66.0 * it.k * it.l / 32.0;
        bc.per_task_low = 2.0 * it.l;
        return bc;
    };
    // Chunk cap of each class.  Long chunks start less often, but a class
    // with few permanents then has too few, too long warp tasks for its
    // launch (4096 permanents of the ragged recipe: 5.5 ms with caps of 2^4
    // terms, 7.4 ms with 2^7): as for the forward, the cap is lowered from
    // 2^kBwdChunkLog2 towards 2^4 until the longest task is at most half of a
    // resident warp's average share of the class's work.
    // The plain method launches one permanent at a time and needs its many
    // short chunks to fill the GPU: it keeps caps of 2^4 terms (the ragged
    // batch's plain backward took 5.9 s with them, 17.7 s with 2^7).
    const int cap0 = P->opts.method == PQ_METHOD_PLAIN ? 4 : kBwdChunkLog2;
    std::vector<int> cls_cap(ncls, cap0);
    for (int c = 0; c < ncls && cap0 > 4; ++c) {
        if (!cls_used[c])
            continue;
        const BwdClass& C = cls[c];
        const double warps = (double)C.blocks * C.wpb;
        for (int cap = cap0; cap >= 4; --cap) {
            double total = 0.0, longest = 0.0;
            for (int64_t p = 0; p < np; ++p) {
                if (P->bwd_class_of[p] != c || items[p].trivial)
                    continue;
                ItemPlan it = items[p];
                const CutCost bc = bwd_cut_cost(it, C);
                choose_chunks(it, cap, std::max(C.jb, 1), kWarp, true, &bc);
                const double task = (double)it.L * bc.per_term +
                                    ((int)it.drad.size() - it.J) * bc.per_high + bc.per_task +
                                    it.J * bc.per_task_low;
                total += task * (double)((it.nchunks + kWarp - 1) / kWarp);
                longest = std::max(longest, task);
            }
            cls_cap[c] = cap;
            if (total <= 0.0 || longest <= 0.5 * total / warps)
                break;
        }
    }
    for (int64_t p = 0; p < np; ++p) {
        ItemPlan& it = items[p];
        const BwdClass& C = cls[P->bwd_class_of[p]];
        if (!it.trivial) {
            const CutCost bc = bwd_cut_cost(it, C);
            choose_chunks(it, cls_cap[P->bwd_class_of[p]], std::max(C.jb, 1), kWarp, true, &bc);
            const PermDesc& Df = P->desc_h[p];
            const int nd = (int)it.drow.size();
            int32_t* dig = meta_bwd.data() + Df.meta + 2 * Df.k + 2 * Df.l;
            for (int d = 0; d < nd; ++d) {
                dig[d] = it.drow[d];
                dig[nd + d] = it.drad[d];
                dig[2 * nd + d] = it.dtop[d];
            }
        } else {
            choose_chunks(it, kBwdChunkLog2, std::max(C.jb, 1));
        }
        PermDesc& D = P->desc_bwd_h[p];
        D.J = it.J;
        D.L = it.L;
        D.nchunks = it.nchunks;
        D.weighted = it.weighted ? 1 : 0;
        const int64_t nt = it.trivial ? 1 : (it.nchunks + kWarp - 1) / kWarp;
        D.ntasks = (int32_t)nt;
        D.slot0 = 0;
        D.part0 = 0;
        P->plain_first_bwd[p] = (int64_t)P->tasks_bwd_plain_h.size();
        const int64_t kl = (int64_t)it.k * it.l;
        gpart_off[p] = gpart;
        gl_off[p] = gl;
        gpart += nt * kl;
        gl += kl;
        const double fpt = it.trivial ? 0.0 : bwd_flops_per_term(it);
        for (int64_t q = 0; q < nt; ++q) {
            Task t;
            t.perm = (int32_t)p;
            t.part = (int32_t)q;
            P->tasks_bwd_plain_h.push_back(t);
            cost.push_back((double)it.L * fpt + 4.0 * kl);
        }
        if (!it.trivial) {
            // every lane of a task walks L terms and starts its chunk from the
            // high digits; the task ends with the lane contraction
            const double lane = (double)it.L * bwd_instr_per_term(it, C.reg != 0) +
                                2.0 * it.l * (double)((int)it.drad.size() - it.J);
            instr_b += (double)nt * (32.0 * lane + 32.0 * it.k + 64.0 * it.J * it.l + 66.0 * kl);
        }
    }
    P->plain_first_bwd[np] = (int64_t)P->tasks_bwd_plain_h.size();
    // batched order: class by class, longest task first within a class
    std::vector<int64_t> order(P->tasks_bwd_plain_h.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        const int ca = P->bwd_class_of[P->tasks_bwd_plain_h[a].perm];
        const int cb = P->bwd_class_of[P->tasks_bwd_plain_h[b].perm];
        if (ca != cb)
            return ca < cb;
        return cost[a] > cost[b];
    });
    P->tasks_bwd_batched_h.resize(order.size());
    for (size_t q = 0; q < order.size(); ++q)
        P->tasks_bwd_batched_h[q] = P->tasks_bwd_plain_h[order[q]];
    P->bwd_classes.clear();
    {
        std::vector<int32_t> compact(ncls, -1);
        int64_t q = 0;
        const int64_t nt = (int64_t)order.size();
        for (int c = 0; c < ncls; ++c) {
            if (!cls_used[c])
                continue;
            BwdClass C = cls[c];
            C.t_begin = q;
            while (q < nt && P->bwd_class_of[P->tasks_bwd_batched_h[q].perm] == c)
                ++q;
            C.t_end = q;
            compact[c] = (int32_t)P->bwd_classes.size();
            P->bwd_classes.push_back(C);
        }
        for (int64_t p = 0; p < np; ++p)
            P->bwd_class_of[p] = compact[P->bwd_class_of[p]];
    }

    int rc;
    if ((rc = dev_upload(&P->desc_bwd_d, P->desc_bwd_h)) != PQ_OK)
        return rc;
    if ((rc = dev_upload(&P->meta_bwd_d, meta_bwd)) != PQ_OK)
        return rc;
    if ((rc = dev_upload(&P->tasks_bwd_plain_d, P->tasks_bwd_plain_h)) != PQ_OK)
        return rc;
    if ((rc = dev_upload(&P->tasks_bwd_batched_d, P->tasks_bwd_batched_h)) != PQ_OK)
        return rc;
    if ((rc = dev_upload(&P->gpart_off_d, gpart_off)) != PQ_OK)
        return rc;
    if ((rc = dev_upload(&P->grad_local_off_d, gl_off)) != PQ_OK)
        return rc;
    dev_free(P->gpart_d);
    dev_free(P->grad_local_d);
    P->gpart_d = nullptr;
    P->grad_local_d = nullptr;
    PQ_ALLOC(&P->gpart_d, std::max<int64_t>(gpart, 1) * 2 * sizeof(double));
    PQ_ALLOC(&P->grad_local_d, std::max<int64_t>(gl, 1) * sizeof(double2));
    P->gpart_elems = (size_t)gpart;
    P->grad_local_elems = (size_t)gl;
    if (P->kind == 0) {
        if ((rc = dev_upload(&P->item_mat_off_d, P->item_mat_off)) != PQ_OK)
            return rc;
        if ((rc = dev_upload(&P->item_k_d, P->item_k)) != PQ_OK)
            return rc;
        if ((rc = dev_upload(&P->item_l_d, P->item_l)) != PQ_OK)
            return rc;
    } else {
        // mode -> oriented index maps for the dL/dU scatter: pos[p][a] for the
        // output mode a, pos[p][m + c] for the input mode c (-1 if empty)
        const int m = P->m;
        std::vector<int32_t> pos((size_t)np * 2 * m, -1);
        for (int64_t p = 0; p < np; ++p) {
            const ItemPlan& it = P->items[p];
            int32_t* pp = pos.data() + (size_t)p * 2 * m;
            const std::vector<int32_t>& outs = it.transposed ? it.cidx : it.ridx;
            const std::vector<int32_t>& ins = it.transposed ? it.ridx : it.cidx;
            for (size_t q = 0; q < outs.size(); ++q)
                pp[outs[q]] = (int32_t)q;
            for (size_t q = 0; q < ins.size(); ++q)
                pp[m + ins[q]] = (int32_t)q;
        }
        if ((rc = dev_upload(&P->bs_pos_d, pos)) != PQ_OK)
            return rc;
    }
    int max_smem = 0, jb = 0, n2 = 0;
    for (const BwdClass& C : P->bwd_classes) {
        if (C.reg) {
            cudaError_t e = bwdr_prepare(C.ld, C.wpb * bwdr_smem_bytes_for(C.kmax, C.ld, C.jb));
            if (e != cudaSuccess)
                return fail(PQ_ERR_CUDA, "backward attribute setup failed: %s",
                            cudaGetErrorString(e));
        } else {
            max_smem = std::max(max_smem, C.wpb * bwd_smem_bytes_for(C.kmax, C.ld, C.jb, C.n2));
        }
        jb = std::max(jb, C.jb);
        n2 = std::max(n2, C.n2);
    }
    P->bwd_jb = jb;
    P->bwd_n2 = n2;
    cudaError_t e = bwd_prepare(P->lmax, max_smem);
    if (e != cudaSuccess)
        return fail(PQ_ERR_CUDA, "backward attribute setup failed: %s", cudaGetErrorString(e));
    P->stats.launches_backward = (P->opts.method == PQ_METHOD_PLAIN)
                                     ? np + 1
                                     : (int64_t)P->bwd_classes.size() + 1;
    P->stats.fp64_instr_backward = instr_b;
    P->bwd_ready = true;
    return PQ_OK;
}

static int run_backward(pq_plan* P, const void* src, const pq_c128* grad_out, const double* grad_prob,
                        const pq_c128* amps, cudaStream_t st)
{
    if (P->opts.shard_count > 0)
        return fail(PQ_ERR_UNSUPPORTED, "the backward does not run on a sharded plan");
    if (!P->uploaded)
        return fail(PQ_ERR_STATE, "the plan lost its device data in a failed re-planning");
    int rc = ensure_backward(P);
    if (rc != PQ_OK)
        return rc;
    PQ_CUDA(cudaMemsetAsync(P->counters_d, 0, (size_t)(P->nperm + 1) * sizeof(int32_t), st));
    if (P->nperm == 0)
        return PQ_OK;
    BwdArgs a;
    a.desc = P->desc_bwd_d;
    a.meta = P->meta_bwd_d;
    a.ntasks = (int64_t)P->tasks_bwd_plain_h.size();
    a.src = reinterpret_cast<const double2*>(src);
    a.grad_out = reinterpret_cast<const double2*>(grad_out);
    a.amps = reinterpret_cast<const double2*>(amps);
    a.grad_prob = grad_prob;
    a.gpart = P->gpart_d;
    a.gpart_off = P->gpart_off_d;
    a.grad_local = P->grad_local_d;
    a.grad_local_off = P->grad_local_off_d;
    a.counters = P->counters_d;
    a.err = P->err_d;
    a.nperm = P->nperm;
    a.nmeta = (int64_t)P->meta_h.size();
    cudaError_t e;
    if (P->opts.method == PQ_METHOD_PLAIN) {
        a.tasks = P->tasks_bwd_plain_d;
        for (int64_t p = 0; p < P->nperm; ++p) {
            const BwdClass& C = P->bwd_classes[P->bwd_class_of[p]];
            e = C.reg ? bwdr_launch_plain(C.ld, a, P->plain_first_bwd[p],
                                          P->plain_first_bwd[p + 1], C.kmax, C.jb, C.wpb, st)
                      : bwd_launch_plain(C.ld, a, P->plain_first_bwd[p], P->plain_first_bwd[p + 1],
                                         C.kmax, C.jb, C.n2, C.wpb, st);
            if (e != cudaSuccess)
                return fail(PQ_ERR_CUDA, "plain backward launch failed: %s", cudaGetErrorString(e));
        }
    } else {
        // one persistent launch per class; the task queue counter restarts at
        // zero for each (the per-permanent counters were cleared above)
        a.tasks = P->tasks_bwd_batched_d;
        for (size_t c = 0; c < P->bwd_classes.size(); ++c) {
            const BwdClass& C = P->bwd_classes[c];
            if (c > 0)
                PQ_CUDA(cudaMemsetAsync(P->counters_d, 0, sizeof(int32_t), st));
            e = C.reg ? bwdr_launch_persistent(C.ld, a, C.t_begin, C.t_end, C.kmax, C.jb,
                                               C.blocks, C.wpb, st)
                      : bwd_launch_persistent(C.ld, a, C.t_begin, C.t_end, C.kmax, C.jb, C.n2,
                                              C.blocks, C.wpb, st);
            if (e != cudaSuccess)
                return fail(PQ_ERR_CUDA, "backward launch failed: %s", cudaGetErrorString(e));
        }
    }
    return PQ_OK;
}

extern "C" int pq_permanent_backward(const pq_batch* b, const pq_c128* grad_out, pq_c128* grad_mats,
                                     pq_plan* plan, void* stream)
{
    if (!b || (b->batch > 0 && (!grad_out || !grad_mats || !b->mats)))
        return fail(PQ_ERR_ARG, "null argument");
    if (b->batch < 0)
        return fail(PQ_ERR_ARG, "negative batch");
    cudaStream_t st = (cudaStream_t)stream;
    pq_plan* P = plan;
    HostSizes h;
    if (!P) {
        int rc = fetch_sizes(b, h);
        if (rc != PQ_OK)
            return rc;
        pq_batch_sizes sz = h.view();
        rc = pq_plan_create(&sz, nullptr, &P);
        if (rc != PQ_OK)
            return rc;
    } else {
        int rc = check_batch_plan(P, b);
        if (rc != PQ_OK)
            return rc;
    }
    int rc = run_backward(P, b->mats, grad_out, nullptr, nullptr, st);
    if (rc == PQ_OK && P->nperm > 0) {
        cudaError_t e = scatter_grad_batch(P->desc_bwd_d, P->meta_bwd_d, P->nperm, P->grad_local_d,
                                           P->grad_local_off_d, P->item_mat_off_d, P->item_l_d,
                                           P->item_k_d, reinterpret_cast<double2*>(grad_mats),
                                           P->total_mat_elems, st);
        if (e != cudaSuccess)
            rc = fail(PQ_ERR_CUDA, "gradient scatter failed: %s", cudaGetErrorString(e));
    }
    if (!plan) {
        if (rc == PQ_OK) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess)
                rc = fail(PQ_ERR_CUDA, "stream synchronize failed: %s", cudaGetErrorString(e));
        }
        if (rc == PQ_OK)
            rc = check_device_error(P);
        pq_plan_destroy(P);
    }
    return rc;
}

extern "C" int pq_bs_probs_backward(const pq_c128* U, int32_t m, const int32_t* in_occ,
                                    const int32_t* out_occ, int64_t B, const double* grad_probs,
                                    const pq_c128* amps, pq_c128* grad_U, pq_plan* plan,
                                    void* stream)
{
    if (!U || !in_occ || !grad_U || (B > 0 && (!out_occ || !grad_probs || !amps)))
        return fail(PQ_ERR_ARG, "null argument");
    if (m <= 0 || m > PQ_MAX_DIM || B < 0)
        return fail(PQ_ERR_ARG, "bad sizes m = %d, B = %lld", m, (long long)B);
    cudaStream_t st = (cudaStream_t)stream;
    pq_plan* P = plan;
    if (!P) {
        std::vector<int32_t> s(m), t((size_t)B * m);
        PQ_CUDA(cudaMemcpy(s.data(), in_occ, m * 4, cudaMemcpyDeviceToHost));
        if (B)
            PQ_CUDA(cudaMemcpy(t.data(), out_occ, (size_t)B * m * 4, cudaMemcpyDeviceToHost));
        int rc = pq_plan_create_bs(m, s.data(), t.data(), B, nullptr, &P);
        if (rc != PQ_OK)
            return rc;
    } else if (P->kind != 1 || P->m != m || P->nperm != B) {
        return fail(PQ_ERR_STATE, "plan was made for different occupations");
    }
    int rc = run_backward(P, U, nullptr, grad_probs, amps, st);
    if (rc == PQ_OK) {
        cudaError_t e = scatter_grad_bs(P->desc_bwd_d, P->bs_pos_d, P->nperm, m, P->grad_local_d,
                                        P->grad_local_off_d, reinterpret_cast<double2*>(grad_U),
                                        st);
        if (e != cudaSuccess)
            rc = fail(PQ_ERR_CUDA, "gradient scatter failed: %s", cudaGetErrorString(e));
    }
    if (!plan) {
        if (rc == PQ_OK) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess)
                rc = fail(PQ_ERR_CUDA, "stream synchronize failed: %s", cudaGetErrorString(e));
        }
        if (rc == PQ_OK)
            rc = check_device_error(P);
        pq_plan_destroy(P);
    }
    return rc;
}

// ---------------------------------------------------------------- Clements mesh
extern "C" int pq_clements_forward(const double* theta, const double* phi, int32_t m, pq_c128* U,
                                   void* stream)
{
    if (!theta || !phi || !U)
        return fail(PQ_ERR_ARG, "null argument");
    if (m < 1 || m > PQ_MAX_DIM)
        return fail(m < 1 ? PQ_ERR_ARG : PQ_ERR_UNSUPPORTED, "m = %d outside [1, %d]", m,
                    PQ_MAX_DIM);
    cudaError_t e = clements_forward(theta, phi, m, reinterpret_cast<double2*>(U),
                                     (cudaStream_t)stream);
    if (e != cudaSuccess)
        return fail(PQ_ERR_CUDA, "clements forward failed: %s", cudaGetErrorString(e));
    return PQ_OK;
}

extern "C" int pq_clements_backward(const double* theta, const double* phi, int32_t m,
                                    const pq_c128* U, const pq_c128* grad_U, double* grad_theta,
                                    double* grad_phi, void* stream)
{
    if (!theta || !phi || !U || !grad_U || !grad_theta || !grad_phi)
        return fail(PQ_ERR_ARG, "null argument");
    if (m < 1 || m > PQ_MAX_DIM)
        return fail(m < 1 ? PQ_ERR_ARG : PQ_ERR_UNSUPPORTED, "m = %d outside [1, %d]", m,
                    PQ_MAX_DIM);
    cudaError_t e = clements_backward(theta, phi, m, reinterpret_cast<const double2*>(U),
                                      reinterpret_cast<const double2*>(grad_U), grad_theta,
                                      grad_phi, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return fail(PQ_ERR_CUDA, "clements backward failed: %s", cudaGetErrorString(e));
    return PQ_OK;
}

// ---------------------------------------------------------------- autotuning
// For every photon number present (a size class), time the class's own
// permanents -- a temporary plan of just those items, reading the same matrix
// data -- with the current chunk cap (the incumbent) and with caps of 2^4 ..
// 2^14 terms, and keep a candidate only if it is at least 1% faster than the
// incumbent.  Timing each class on its own matters: a small class changes
// the whole batch's time by less than the timing noise, and a choice made
// from whole-batch times can then only be noise.  The picks are then checked
// once on the whole batch against the plan's previous chunking.
extern "C" int pq_autotune(pq_plan* P, const pq_batch* b, const pq_c128* U, void* stream)
{
    if (!P)
        return fail(PQ_ERR_ARG, "null plan");
    if (P->opts.shard_count > 0)
        return fail(PQ_ERR_STATE, "a sharded plan keeps the fixed chunking all shards share");
    const void* src = nullptr;
    if (P->kind == 0) {
        if (!b)
            return fail(PQ_ERR_ARG, "permanent plan needs the batch descriptor");
        int rc = check_batch_plan(P, b);
        if (rc != PQ_OK)
            return rc;
        src = b->mats;
    } else {
        if (!U)
            return fail(PQ_ERR_ARG, "boson-sampling plan needs U");
        src = U;
    }
    if (P->nperm == 0)
        return PQ_OK;
    cudaStream_t st = (cudaStream_t)stream;
    double2* amps = nullptr;
    PQ_ALLOC(&amps, (size_t)P->nperm * sizeof(double2));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<std::vector<ItemPlan>> by_n(PQ_MAX_N + 1);
    for (const ItemPlan& it : P->items)
        if (!it.trivial)
            by_n[it.n].push_back(it);
    int rc = PQ_OK;
    // time one execution of plan T (best of 5 after a warm-up)
    auto time_plan = [&](pq_plan* T, float& ms) -> int {
        float best = 1e30f;
        for (int rep = 0; rep < 6; ++rep) {
            cudaEventRecord(e0, st);
            int r = run_forward_raw(T, src, amps, nullptr, st);
            if (r != PQ_OK)
                return r;
            cudaEventRecord(e1, st);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess)
                return fail(PQ_ERR_CUDA, "autotune timing failed: %s", cudaGetErrorString(e));
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0)
                best = std::min(best, t);
        }
        ms = best;
        return PQ_OK;
    };
    const int cands[] = {4, 6, 8, 10, 12, 14};
    const std::vector<int32_t> saved_class = P->class_log2;
    for (int n = 0; n <= PQ_MAX_N && rc == PQ_OK; ++n) {
        if (by_n[n].empty())
            continue;
        int incumbent = P->class_log2[n] > 0 ? P->class_log2[n] : tune_get(n);
        if (incumbent <= 0)
            incumbent = 10;
        pq_plan* T = plan_new();
        if (!T) {
            rc = fail(PQ_ERR_NOMEM, "host allocation failed");
            break;
        }
        T->kind = P->kind;
        T->opts = P->opts;
        T->opts.method = PQ_METHOD_BATCHED;
        // time the class with the walk the whole plan runs
        T->opts.column_sums = P->fwd_nl == 0 ? PQ_SUMS_SHARED : PQ_SUMS_REGISTERS;
        T->opts.use_graph = 0;
        T->opts.chunk_log2 = 0;
        T->device = P->device;
        T->num_sms = P->num_sms;
        T->items = by_n[n];
        T->class_log2.assign(PQ_MAX_N + 1, 0);
        int best_c = incumbent;
        float best_t = 1e30f;
        T->class_log2[n] = incumbent;
        rc = schedule_and_upload(T);
        if (rc == PQ_OK)
            rc = time_plan(T, best_t);
        for (int cnd : cands) {
            if (rc != PQ_OK || cnd == incumbent)
                continue;
            T->class_log2[n] = cnd;
            float t = 0.0f;
            rc = schedule_and_upload(T);
            if (rc == PQ_OK)
                rc = time_plan(T, t);
            if (rc == PQ_OK && t < best_t * 0.99f) {
                best_t = t;
                best_c = cnd;
            }
        }
        cudaStreamSynchronize(st);
        free_plan_device(T);
        plan_delete(T);
        if (rc != PQ_OK)
            break;
        P->class_log2[n] = best_c;
    }
    // The classes were timed alone.  In the whole batch the chunking the plan
    // had before (for a small batch, caps lowered so that the warp tasks
    // balance over the GPU) can be the faster one: time the batch both ways
    // and keep the per-class choice only if it is at least 1% faster.
    if (rc == PQ_OK) {
        const std::vector<int32_t> picks = P->class_log2;
        float t_picks = 0.0f, t_before = 0.0f;
        rc = schedule_and_upload(P);
        if (rc == PQ_OK)
            rc = time_plan(P, t_picks);
        if (rc == PQ_OK) {
            P->class_log2 = saved_class;
            rc = schedule_and_upload(P);
            if (rc == PQ_OK)
                rc = time_plan(P, t_before);
        }
        if (rc == PQ_OK && t_picks < 0.99f * t_before) {
            P->class_log2 = picks;
            for (int n = 0; n <= PQ_MAX_N; ++n)
                if (!by_n[n].empty())
                    tune_set(n, picks[n]);
            rc = schedule_and_upload(P);
        }
    }
    // Where the walk keeps its column sums.  For a batch of one column class
    // the planner takes registers, which measured from 10% slower (4096
    // collision-free permanents of n = 16) to 11% faster (m = 24 boson
    // sampling, 4096 patterns) than shared memory, with its chunking: time
    // the whole plan both ways and keep shared memory only if it is at least
    // 1% faster.  The choice is the plan's (its options), not the process's.
    const int32_t saved_sums = P->opts.column_sums;
    if (rc == PQ_OK && P->opts.column_sums == PQ_SUMS_AUTO && P->fwd_nl > 0) {
        float t_reg = 0.0f, t_sh = 0.0f;
        rc = time_plan(P, t_reg);
        if (rc == PQ_OK) {
            P->opts.column_sums = PQ_SUMS_SHARED;
            rc = schedule_and_upload(P);
            if (rc == PQ_OK)
                rc = time_plan(P, t_sh);
            if (rc == PQ_OK && !(t_sh < 0.99f * t_reg)) {
                P->opts.column_sums = saved_sums;
                rc = schedule_and_upload(P);
            }
        }
    }
    if (rc != PQ_OK && !P->uploaded) {  // try to leave the plan as it was
        P->class_log2 = saved_class;
        P->opts.column_sums = saved_sums;
        schedule_and_upload(P);
    }
    P->bwd_ready = false;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(amps);
    return rc;
}

// ---------------------------------------------------------------- diagnostics
extern "C" int pq_plan_item_info(int32_t k, int32_t l, const int32_t* row_mult,
                                 const int32_t* col_mult, int32_t chunk_log2, pq_item_info* out)
{
    if (!out || (k > 0 && !row_mult) || (l > 0 && !col_mult))
        return fail(PQ_ERR_ARG, "null argument");
    if (chunk_log2 < 0 || chunk_log2 > 30)
        return fail(PQ_ERR_ARG, "chunk_log2 outside [0, 30]");
    ItemPlan it;
    int rc = build_item(row_mult, col_mult, k, l, 0, l, it);
    if (rc != PQ_OK)
        return rc;
    choose_chunks(it, chunk_log2 > 0 ? chunk_log2 : 10, kMaxLowDigits, kWarp, true);
    std::memset(out, 0, sizeof(*out));
    out->n = it.n;
    out->k = it.k;
    out->l = it.l;
    out->transposed = it.transposed ? 1 : 0;
    out->ndig = (int32_t)it.drow.size();
    out->J = it.J;
    out->terms = it.T;
    out->chunk_len = it.L;
    out->chunks = it.nchunks;
    for (size_t d = 0; d < it.drow.size() && d < (size_t)PQ_MAX_N; ++d) {
        out->radix[d] = it.drad[d];
        out->row_of_digit[d] = it.drow[d];
    }
    return PQ_OK;
}

// ---------------------------------------------------------------- batch partition
// Largest work first, each to the rank with the least work so far (ties: the
// lower rank); work = Gray-code terms x algorithmic flops per term, the
// quantity the forward kernel's time follows.  Host only.
extern "C" int pq_partition_batch(const pq_batch_sizes* sz, int32_t ranks, int32_t* rank_of_item,
                                  int64_t* terms_per_rank)
{
    if (!sz || !terms_per_rank || (sz->batch > 0 && !rank_of_item))
        return fail(PQ_ERR_ARG, "null argument");
    if (ranks < 1 || ranks > 65536)
        return fail(PQ_ERR_ARG, "ranks %d outside [1, 65536]", ranks);
    if (sz->batch < 0)
        return fail(PQ_ERR_ARG, "negative batch");
    if (!sizes_present(sz, false))
        return fail(PQ_ERR_ARG, "null size array");
    if (sz->batch > (int64_t(1) << 30))
        return fail(PQ_ERR_UNSUPPORTED, "batch above 2^30");
    const int64_t nb = sz->batch;
    std::vector<double> work(nb);
    std::vector<int64_t> terms(nb);
    for (int64_t b = 0; b < nb; ++b) {
        if (sz->row_off[b] < 0 || sz->col_off[b] < 0)
            return fail(PQ_ERR_ARG, "negative offset at item %lld", (long long)b);
        ItemPlan it;
        const int rc = build_item(sz->row_mult + sz->row_off[b], sz->col_mult + sz->col_off[b],
                                  sz->k[b], sz->l[b], 0, sz->l[b], it);
        if (rc != PQ_OK)
            return fail(rc, "item %lld: %s", (long long)b, g_err.c_str());
        terms[b] = it.trivial ? 0 : it.T;
        work[b] = it.trivial ? 1.0 : (double)it.T * fwd_flops_per_term(it);
    }
    std::vector<int64_t> order(nb);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t a, int64_t b) { return work[a] > work[b]; });
    // min-heap of (work so far, rank)
    using Load = std::pair<double, int32_t>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int32_t r = 0; r < ranks; ++r) {
        heap.push({0.0, r});
        terms_per_rank[r] = 0;
    }
    for (int64_t q = 0; q < nb; ++q) {
        const int64_t b = order[q];
        Load top = heap.top();
        heap.pop();
        rank_of_item[b] = top.second;
        terms_per_rank[top.second] += terms[b];
        top.first += work[b];
        heap.push(top);
    }
    return PQ_OK;
}

// ---------------------------------------------------------------- internal: occupation plans
namespace pqi {

// A plan over one m x m matrix whose item b is the submatrix with row
// occupations t[b] and column occupations s[b] (each length m, host); no
// normalisation (norm = 1), so probs receive |per|^2.
int plan_create_occupations(int32_t m, const std::vector<int32_t>& t, const std::vector<int32_t>& s,
                            int64_t B, pq_plan** out)
{
    *out = nullptr;
    pq_plan* P = plan_new();
    if (!P)
        return fail(PQ_ERR_NOMEM, "host allocation failed");
    int rc = plan_common_init(P, nullptr);
    if (rc != PQ_OK) {
        plan_delete(P);
        return rc;
    }
    P->kind = 2;
    P->m = m;
    P->items.resize(B);
    for (int64_t b = 0; b < B; ++b) {
        rc = build_item(t.data() + b * m, s.data() + b * m, m, m, 0, m, P->items[b]);
        if (rc != PQ_OK) {
            plan_delete(P);
            return rc;
        }
        P->items[b].norm = 1.0;
    }
    P->class_log2.assign(PQ_MAX_N + 1, 0);
    rc = schedule_and_upload(P);
    if (rc != PQ_OK) {
        free_plan_device(P);
        plan_delete(P);
        return rc;
    }
    *out = P;
    return PQ_OK;
}

int plan_run_forward(pq_plan* P, const void* src, void* amps, double* probs, cudaStream_t st)
{
    return run_forward_raw(P, src, amps, probs, st);
}

int plan_prepare_forward(pq_plan* P)
{
    const cudaError_t e = forward_prepare(P);
    return e == cudaSuccess ? PQ_OK : fail(PQ_ERR_CUDA, "kernel attribute setup failed: %s",
                                            cudaGetErrorString(e));
}

int report(int code, const char* msg) { return fail(code, "%s", msg); }

}  // namespace pqi
