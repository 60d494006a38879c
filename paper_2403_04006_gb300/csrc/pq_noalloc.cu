// pq_noalloc.cu -- permanent of one base matrix without any memory allocation.
//
// Some callers cannot call cudaMalloc: code embedded in a framework whose
// caching allocator owns the device memory (a cudaMalloc of its own can fail
// or fragment that pool), processes that run under a fixed device-memory
// budget, and latency-critical paths that cannot afford the implicit device
// synchronisation an allocation may bring.  pq_permanent_noalloc serves them:
// it runs the same forward kernel as pq_permanent_batched, but every piece of
// workspace it needs (the permanent's descriptor and integer metadata, its
// warp-task list, the per-task partial sums and the task counters) lives in
// one file-scope static device array that is part of the loaded library.
//
// The host plans the permanent into a fixed-size structure and passes it by
// value, as a kernel argument, to a set-up kernel that writes it into the
// array, clears the counters and fills the task list; so no host buffer has
// to outlive the call.  The array is shared by every call on a device and
// keeps the contents of the last call.  Calls whose GPU work overlaps (two
// streams, or two host threads) race on the array, so issue them in one
// stream or serialise them.  The device address of the array is looked up
// once per device, on the first call with that device current; make that
// first call before any stream capture.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/pq.h"
#include "pq_device.cuh"
#include "pq_kernels.h"

namespace pqi {

// Workspace: [0, 8 KB) descriptor, metadata and counters; then the task list
// (8 bytes per task) and the partial sums (32 bytes per task).
constexpr size_t kNoAllocBytes = size_t(PQ_NOALLOC_SCRATCH_BYTES);
constexpr size_t kNoAllocHead = 8192;
constexpr int64_t kNoAllocMaxTasks = (int64_t)((kNoAllocBytes - kNoAllocHead) / 40);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The workspace head: descriptor, then integer metadata.  Built on the host
// and handed to noalloc_setup by value.
struct NoAllocHead {
    PermDesc desc;
    int32_t meta[2 * PQ_MAX_DIM + 3 * PQ_MAX_DIM + 3 * PQ_MAX_DIM];
};
static_assert(sizeof(NoAllocHead) + 64 <= kNoAllocHead, "workspace head too small");
static_assert(sizeof(NoAllocHead) % 4 == 0, "head copied as 32-bit words");
static_assert(sizeof(NoAllocHead) <= 4000, "head must fit the kernel-parameter space");

// Copy the head into the workspace, clear the counters and fill the task
// list (task q is part q of permanent 0).  Block 0 writes the head and the
// counters; every block fills its share of the tasks.
__global__ void noalloc_setup(const NoAllocHead h, unsigned char* base, int32_t* counters,
                              Task* tasks, int64_t ntasks)
{
    if (blockIdx.x == 0) {
        const int32_t* src = reinterpret_cast<const int32_t*>(&h);
        int32_t* dst = reinterpret_cast<int32_t*>(base);
        for (int w = threadIdx.x; w < (int)(sizeof(NoAllocHead) / 4); w += blockDim.x)
            dst[w] = src[w];
        if (threadIdx.x < 16)
            counters[threadIdx.x] = 0;
    }
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < ntasks;
         q += (int64_t)gridDim.x * blockDim.x) {
        tasks[q].perm = 0;
        tasks[q].part = (int32_t)q;
    }
}

static int noalloc_fail(int code, const char* msg)
{
    set_last_error(msg);  // readable through pq_last_error()
    return code;
}

// Plan one permanent with fixed-size arrays only: drop empty rows/columns,
// sum the side with fewer Gray-code terms, sort product columns by
// non-increasing multiplicity, put the fixed copy on the least repeated row,
// order digits by radix, and cut the code into chunks of the low digits so
// that the tasks fit the workspace.
static int noalloc_plan(int k0, int l0, const int32_t* r, const int32_t* c, NoAllocHead& h,
                        int64_t& ntasks)
{
    int rs[PQ_MAX_DIM], cs[PQ_MAX_DIM], rm[PQ_MAX_DIM], cm[PQ_MAX_DIM];
    int kr = 0, kc = 0, nr = 0, nc = 0;
    for (int i = 0; i < k0; ++i) {
        if (r[i] < 0)
            return noalloc_fail(PQ_ERR_ARG, "negative row multiplicity");
        if (r[i] > 0) {
            rs[kr] = i;
            rm[kr++] = r[i];
            nr += r[i];
        }
    }
    for (int j = 0; j < l0; ++j) {
        if (c[j] < 0)
            return noalloc_fail(PQ_ERR_ARG, "negative column multiplicity");
        if (c[j] > 0) {
            cs[kc] = j;
            cm[kc++] = c[j];
            nc += c[j];
        }
    }
    if (nr != nc)
        return noalloc_fail(PQ_ERR_ARG, "sum of row multiplicities != sum of column multiplicities");
    if (nr > PQ_MAX_N)
        return noalloc_fail(PQ_ERR_UNSUPPORTED, "n above PQ_MAX_N");
    std::memset(&h, 0, sizeof(h));
    PermDesc& D = h.desc;
    D.n = nr;
    D.out = 0;
    D.norm = 1.0;
    D.jf = -1;
    if (nr == 0) {
        D.trivial = 1;
        D.ntasks = 1;
        ntasks = 1;
        return PQ_OK;
    }
    auto terms = [](const int* m, int cnt) -> int64_t {
        int f = 0;
        for (int i = 1; i < cnt; ++i)
            if (m[i] < m[f])
                f = i;
        int64_t T = 1;
        for (int i = 0; i < cnt; ++i) {
            const int64_t rad = (i == f) ? m[i] : m[i] + 1;
            if (T > (int64_t(1) << 62) / rad)
                return -1;
            T *= rad;
        }
        return T;
    };
    const int64_t Tr = terms(rm, kr), Tc = terms(cm, kc);
    if (Tr < 0 && Tc < 0)
        return noalloc_fail(PQ_ERR_UNSUPPORTED, "term count above 2^62");
    const bool tr = (Tr < 0) || (Tc >= 0 && Tc < Tr);
    int *ri = tr ? cs : rs, *rmul = tr ? cm : rm, *ci = tr ? rs : cs, *cmul = tr ? rm : cm;
    const int k = tr ? kc : kr, l = tr ? kr : kc;
    if (l > PQ_MAX_PRODUCT_COLS)
        return noalloc_fail(PQ_ERR_UNSUPPORTED, "too many product-side columns");
    D.T = tr ? Tc : Tr;
    D.k = k;
    D.l = l;
    D.si = tr ? 1 : l0;
    D.sj = tr ? l0 : 1;
    // product columns by non-increasing multiplicity (stable insertion sort)
    int co[PQ_MAX_DIM], cmo[PQ_MAX_DIM];
    for (int j = 0; j < l; ++j) {
        int p = j;
        while (p > 0 && cmo[p - 1] < cmul[j]) {
            co[p] = co[p - 1];
            cmo[p] = cmo[p - 1];
            --p;
        }
        co[p] = ci[j];
        cmo[p] = cmul[j];
    }
    int ecnt[PQ_MAX_DIM];
    for (int j = 0; j < l; ++j) {
        const int next = (j + 1 < l) ? cmo[j + 1] : 0;
        const int e = cmo[j] - (next > 1 ? next : 1);
        ecnt[j] = e > 0 ? e : 0;
        if (ecnt[j] > 0 && D.jf < 0)
            D.jf = j;
    }
    // digits: fixed copy on the least repeated row, ascending radix (stable)
    int f = 0;
    for (int i = 1; i < k; ++i)
        if (rmul[i] < rmul[f])
            f = i;
    int drow[PQ_MAX_DIM], drad[PQ_MAX_DIM], dtop[PQ_MAX_DIM], nd = 0;
    for (int i = 0; i < k; ++i) {
        int rad, top;
        if (i == f) {
            if (rmul[i] < 2)
                continue;
            rad = rmul[i];
            top = rmul[i] - 1;
        } else {
            rad = rmul[i] + 1;
            top = rmul[i];
        }
        int p = nd++;
        while (p > 0 && drad[p - 1] > rad) {
            drow[p] = drow[p - 1];
            drad[p] = drad[p - 1];
            dtop[p] = dtop[p - 1];
            --p;
        }
        drow[p] = i;
        drad[p] = rad;
        dtop[p] = top;
    }
    D.ndig = nd;
    // chunks: about 2^10 terms (at least one warp of chunks), longer if the
    // task list would not fit the workspace
    int J = 0;
    int64_t L = 1;
    int64_t target = D.T / kWarp;
    if (target > 1024)
        target = 1024;
    while (J < nd && J < kMaxLowDigits && drad[J] <= kMaxLowRadix &&
           (L * drad[J] <= target || (D.T / L + kWarp - 1) / kWarp > kNoAllocMaxTasks)) {
        L *= drad[J];
        ++J;
    }
    D.J = J;
    D.L = L;
    D.nchunks = D.T / L;
    ntasks = (D.nchunks + kWarp - 1) / kWarp;
    if (ntasks > kNoAllocMaxTasks)
        return noalloc_fail(PQ_ERR_UNSUPPORTED,
                            "permanent needs more warp tasks than the static workspace holds");
    D.ntasks = (int32_t)ntasks;
    D.slot0 = 0;
    D.weighted = 0;
    for (int d = 0; d < J; ++d)
        if (drad[d] > 2)
            D.weighted = 1;
    // metadata: ridx, cidx, rmul, cmul, drow, drad, dtop, ecnt
    int32_t* m = h.meta;
    D.meta = 0;
    for (int i = 0; i < k; ++i)
        *m++ = ri[i];
    for (int j = 0; j < l; ++j)
        *m++ = co[j];
    for (int i = 0; i < k; ++i)
        *m++ = rmul[i];
    for (int j = 0; j < l; ++j)
        *m++ = cmo[j];
    for (int d = 0; d < nd; ++d)
        *m++ = drow[d];
    for (int d = 0; d < nd; ++d)
        *m++ = drad[d];
    for (int d = 0; d < nd; ++d)
        *m++ = dtop[d];
    for (int j = 0; j < l; ++j)
        *m++ = ecnt[j];
    return PQ_OK;
}

static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_addr[64] = {nullptr};

}  // namespace pqi

using namespace pqi;

extern "C" int pq_permanent_noalloc(const pq_c128* B, int32_t k, int32_t l,
                                    const int32_t* row_mult, const int32_t* col_mult,
                                    pq_c128* out, void* stream)
{
    if (!out || (k > 0 && !row_mult) || (l > 0 && !col_mult) || (k > 0 && l > 0 && !B))
        return noalloc_fail(PQ_ERR_ARG, "null argument");
    if (k < 0 || l < 0)
        return noalloc_fail(PQ_ERR_ARG, "negative size");
    if (k > PQ_MAX_DIM || l > PQ_MAX_DIM)
        return noalloc_fail(PQ_ERR_UNSUPPORTED, "base matrix larger than PQ_MAX_DIM");
    NoAllocHead h;
    int64_t ntasks = 0;
    int rc = noalloc_plan(k, l, row_mult, col_mult, h, ntasks);
    if (rc != PQ_OK)
        return rc;

    // device address of the static workspace, looked up once per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return noalloc_fail(PQ_ERR_CUDA, "cudaGetDevice failed");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return noalloc_fail(PQ_ERR_CUDA, "cudaGetSymbolAddress of the workspace failed");
            g_noalloc_addr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_noalloc_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    PermDesc* desc_d = reinterpret_cast<PermDesc*>(base);
    int32_t* meta_d = reinterpret_cast<int32_t*>(base + offsetof(NoAllocHead, meta));
    int32_t* counters_d = reinterpret_cast<int32_t*>(base + kNoAllocHead - 64);
    Task* tasks_d = reinterpret_cast<Task*>(base + kNoAllocHead);
    double* partials_d = reinterpret_cast<double*>(base + kNoAllocHead + 8 * (size_t)ntasks);

    const unsigned fill_blocks = (unsigned)((ntasks + 255) / 256 < 1024 ? (ntasks + 255) / 256 : 1024);
    noalloc_setup<<<fill_blocks, 256, 0, st>>>(h, base, counters_d, tasks_d, ntasks);
    if (cudaGetLastError() != cudaSuccess)
        return noalloc_fail(PQ_ERR_CUDA, "workspace set-up launch failed");

    const int ld = h.desc.l > 0 ? h.desc.l : 1;
    const int kmax = h.desc.k > 0 ? h.desc.k : 1;
    const int per_warp = fwd_smem_per_warp(kmax, ld);
    int wpb = 0, bps = 0, sms = 0;
    launch_geometry(fwd_regs_per_thread(ld), per_warp, 8, 8, wpb, bps);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        fwd_prepare(ld, wpb * per_warp) != cudaSuccess)
        return noalloc_fail(PQ_ERR_CUDA, "kernel set-up failed");
    ExecArgs a;
    a.desc = desc_d;
    a.meta = meta_d;
    a.tasks = tasks_d;
    a.ntasks = ntasks;
    a.src = reinterpret_cast<const double2*>(B);
    a.out_amp = reinterpret_cast<double2*>(out);
    a.out_prob = nullptr;
    a.out_partial = nullptr;
    a.partials = partials_d;
    a.counters = counters_d;
    a.err = counters_d + 8;
    a.nperm = 1;
    a.nmeta = (int64_t)(sizeof(h.meta) / sizeof(h.meta[0]));
    a.nslots = ntasks;
    int64_t want = (ntasks + wpb - 1) / wpb;
    int blocks = sms * bps;
    if (want < blocks)
        blocks = (int)(want > 0 ? want : 1);
    if (fwd_launch_persistent(ld, a, kmax, blocks, wpb, st) != cudaSuccess)
        return noalloc_fail(PQ_ERR_CUDA, "forward launch failed");
    return PQ_OK;
}
