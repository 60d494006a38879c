/*
 * pq.h -- C ABI of the GB300 (sm_103a) permanent library.
 *
 * The library evaluates permanents of matrices with repeated rows and columns
 * and the boson-sampling output probabilities built on them, with their
 * gradients, on one GPU.  Paper: "Piquasso: A Photonic Quantum Computer
 * Simulation Software Platform", arXiv 2403.04006.
 *
 *   per(A) = sum_{sigma in S_n} prod_i A[sigma(i)][i]            Eq. (per_def)
 *   p(s,t) = |per(U_{s,t})|^2 / (prod_i t_i! prod_i s_i!)        Eq. (BS_prob)
 *
 * A is given by a k x l base matrix B and multiplicities r (rows), c (columns)
 * with sum r = sum c = n: A repeats base row i r_i times and base column j c_j
 * times ("row or column multiplicities", Sec. 4.2 "Boson Sampling").  The GPU
 * evaluates the Balasubramanian-Bax-Franklin-Glynn (BB/FG) formula extended to
 * multiplicities with a mixed-radix ("n-ary") Gray code whose digit for row i
 * runs over the number of sign flips among its r_i copies (Sec. 4.2).
 *
 * Conventions shared by every call:
 *  - Complex numbers are pq_c128 = {re, im}, 16 bytes, interleaved; the layout
 *    of torch.complex128 / std::complex<double>.
 *  - Matrices are dense row-major.  In the boson-sampling calls U is m x m and
 *    indexed U[out][in]: U_{s,t} takes the rows of the output modes (repeated
 *    t_i times) and the columns of the input modes (repeated s_j times).
 *    |per|^2 does not change under transposition, so probabilities do not
 *    depend on this choice; gradient layouts do.
 *  - Pointers documented "device" must point to device memory of the current
 *    CUDA device; "host" pointers to host memory.  The caller owns every buffer
 *    it passes; the library never frees caller memory and keeps no pointer to
 *    it after the call returns (except inside a plan, see below).
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls are asynchronous with respect to the host unless stated.
 *  - Return value: PQ_OK (0) or a negative PQ_ERR_* code; pq_last_error()
 *    gives a message for the calling thread.  Nothing aborts and nothing
 *    throws across this boundary.  Argument errors are detected on the host
 *    before any launch.
 *  - Gradients follow PyTorch's convention for complex tensors: for a real
 *    loss L, grad_z = dL/dRe z + i dL/dIm z; for a holomorphic f,
 *    grad_in = grad_out * conj(df/dz).
 *  - Limits: n <= PQ_MAX_N photons, base dimensions k, l <= PQ_MAX_DIM, and on
 *    the side that is not summed at most PQ_MAX_PRODUCT_COLS distinct columns;
 *    term counts below 2^62.  Larger inputs return PQ_ERR_UNSUPPORTED.
 */
#ifndef PQ_GB300_H
#define PQ_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PQ_OK 0
#define PQ_ERR_ARG (-1)         /* null pointer, negative size, sum r != sum c, ... */
#define PQ_ERR_UNSUPPORTED (-2) /* beyond the limits below                          */
#define PQ_ERR_CUDA (-3)        /* a CUDA runtime call failed                       */
#define PQ_ERR_TIMEOUT (-4)     /* a bounded device wait gave up                    */
#define PQ_ERR_NOMEM (-5)       /* host or device allocation failed                 */
#define PQ_ERR_STATE (-6)       /* plan used with data it was not made for          */

#define PQ_MAX_N 48
#define PQ_MAX_DIM 64
#define PQ_MAX_PRODUCT_COLS 40

typedef struct { double re, im; } pq_c128;

/* Ragged batch of base matrices; every pointer is a DEVICE pointer.
 * Item b: base matrix at mats + mat_off[b] (k[b] x l[b], row-major), row
 * multiplicities row_mult[row_off[b] .. row_off[b]+k[b]-1], column
 * multiplicities col_mult[col_off[b] .. col_off[b]+l[b]-1].  Offsets count
 * elements.  Multiplicities are >= 0; zero drops that row or column. */
typedef struct {
    int64_t batch;
    const pq_c128* mats;
    const int64_t* mat_off;
    const int32_t* k;
    const int32_t* l;
    const int32_t* row_mult;
    const int64_t* row_off;
    const int32_t* col_mult;
    const int64_t* col_off;
} pq_batch;

/* The same ragged layout with HOST pointers to the offsets, sizes and
 * multiplicities only (no matrix values): what planning needs.  Same meaning
 * as the fields of pq_batch. */
typedef struct {
    int64_t batch;
    const int64_t* mat_off;
    const int32_t* k;
    const int32_t* l;
    const int32_t* row_mult;
    const int64_t* row_off;
    const int32_t* col_mult;
    const int64_t* col_off;
} pq_batch_sizes;

/* Execution method of a plan. */
#define PQ_METHOD_BATCHED 0 /* one persistent launch for the whole batch (default)   */
#define PQ_METHOD_PLAIN 1   /* one launch per permanent, issued back to back          */

/* Where a lane keeps its column sums in the forward walk. */
#define PQ_SUMS_AUTO 0      /* the planner's choice (default)                            */
#define PQ_SUMS_SHARED 1    /* shared memory, lane-major: any product side               */
#define PQ_SUMS_REGISTERS 2 /* registers: product sides of at most 20 columns (the plan
                               falls back to shared memory for wider ones)              */

/* Plan options; zero-initialise and set what you need. */
typedef struct {
    int32_t method;          /* PQ_METHOD_*                                              */
    int32_t use_graph;       /* 1: capture the batched launch in a CUDA graph and replay */
    int32_t chunk_log2;      /* 0: per size class from the tuning table; else Gray-code
                                chunk of about 2^chunk_log2 terms for every permanent     */
    int32_t warps_per_block; /* 0: default (8)                                            */
    int32_t blocks_per_sm;   /* 0: default (1)                                            */
    int32_t shard_index;     /* with shard_count > 1: this plan covers shard shard_index  */
    int32_t shard_count;     /* of the warp tasks of every permanent (see
                                pq_permanent_partials); 0 or 1: no sharding              */
    int32_t column_sums;     /* PQ_SUMS_*                                                 */
} pq_plan_options;

/* Opaque plan: the host-side schedule of one batch shape (which side of each
 * permanent is summed, how its Gray-code range is cut into chunks, the order
 * in which warps take them) plus the device workspace it needs.  Creating a
 * plan is the only place the library allocates; executing it allocates
 * nothing, reads no host memory and does not synchronise, so it can run
 * inside stream capture.  A plan may be used by one stream at a time. */
typedef struct pq_plan pq_plan;

/* Plan a ragged permanent batch.  `sizes` is host memory and is copied; the
 * matrix values are only read at execution.  opts may be NULL (defaults).
 * Allocates device memory on the current device.
 * Errors: PQ_ERR_ARG, PQ_ERR_UNSUPPORTED, PQ_ERR_NOMEM, PQ_ERR_CUDA. */
int pq_plan_create(const pq_batch_sizes* sizes, const pq_plan_options* opts, pq_plan** out);

/* Plan the boson-sampling batch of pq_bs_probs: m modes, input occupation
 * input_occ[m] and output occupations output_occ[B*m] (row-major), both HOST
 * memory and copied.  Every output pattern must hold as many photons as the
 * input (PQ_ERR_ARG otherwise).  The plan also keeps the factorial
 * normalisation 1/(prod t! prod s!) of every pattern. */
int pq_plan_create_bs(int32_t m, const int32_t* input_occ, const int32_t* output_occ, int64_t B,
                      const pq_plan_options* opts, pq_plan** out);

/* Frees the plan and its device workspace (synchronises the device first). */
int pq_plan_destroy(pq_plan* plan);

/* Per(A_b) for every item of the batch (Eq. (per_def) with the multiplicities
 * of Sec. 4.2), evaluated by the multiplicity-extended BB/FG formula over a
 * mixed-radix Gray code in FP64 with double-double accumulation.
 * b: device descriptor; out: device, batch entries.  plan: made by
 * pq_plan_create for the same sizes, or NULL, in which case the call copies
 * the sizes to the host, plans, runs the batched method and synchronises
 * `stream` before returning (convenience path; it allocates). */
int pq_permanent_batched(const pq_batch* b, pq_c128* out, pq_plan* plan, void* stream);

/* Partial sums of a sharded permanent batch: the warp tasks of every
 * permanent (runs of 32 Gray-code chunks) are cut into shard_count contiguous
 * ranges, and a plan made with shard_index = r covers range r.  One rank (or
 * one GPU) per shard runs this call; partials[4p .. 4p+3] receives its
 * double-double sum (re hi, re lo, im hi, im lo) of the Glynn terms of
 * permanent p, WITHOUT the factor 2^{-(n-1)}.  Adding the shards' partials
 * (in double-double, in shard order) and scaling by 2^{-(n-1)} gives per; a
 * permanent with n = 0 contributes 1 on exactly one shard and 0 on the
 * others.  This is the exchange step of one permanent split across GPUs.
 * b: device descriptor as for pq_permanent_batched; partials: device,
 * 4 * batch doubles; plan: made by pq_plan_create for the same sizes with
 * shard_count >= 1 (required).  Allocates nothing, does not synchronise.
 * Errors: PQ_ERR_ARG (null), PQ_ERR_STATE (plan not sharded, or made for
 * other sizes), PQ_ERR_CUDA. */
int pq_permanent_partials(const pq_batch* b, double* partials, pq_plan* plan, void* stream);

/* The exchange step of a permanent batch split over ranks: combines the
 * shards' partial sums written by pq_permanent_partials into permanents,
 * out[p] = 2^{-(n[p]-1)} * sum over shards r = 0 .. nshards-1, in that order,
 * of parts[r][p] (double-double additions: TwoSum of the high parts, errors
 * and low parts gathered into the low part; no scaling for n[p] = 0).  This
 * is the normalisation of the BB/FG formula (Sec. 4.2) applied once to the
 * whole sum.  parts: nshards x batch x 4 doubles (re hi, re lo, im hi, im
 * lo), shard-major, as an all-gather of each shard's partials lays them out;
 * n: photons of each permanent (int32, batch); out: batch complex.
 * pq_combine_partials takes DEVICE pointers and runs one kernel on `stream`
 * (asynchronous, allocates nothing); pq_combine_partials_host takes HOST
 * pointers, needs no GPU and gives the same bits.  Errors: PQ_ERR_ARG (null
 * pointer with batch > 0, batch < 0, nshards < 1; on the host also n outside
 * [0, PQ_MAX_N]), PQ_ERR_CUDA. */
int pq_combine_partials(const double* parts, int32_t nshards, int64_t batch, const int32_t* n,
                        pq_c128* out, void* stream);
int pq_combine_partials_host(const double* parts, int32_t nshards, int64_t batch,
                             const int32_t* n, pq_c128* out);

/* A batch split over ranks by whole permanents (independent problems need no
 * exchange step; each rank evaluates its items with an ordinary plan and the
 * outputs are gathered).  Items are taken largest first and each goes to the
 * rank with the least work so far, ties to the lower rank; an item's work is
 * its Gray-code term count times the algorithmic flops per term of the
 * forward pass (2l + 6(n-1) + 2, +2 for weighted codes), which the forward
 * kernel's time follows.  sz: the batch's sizes (host, as for
 * pq_plan_create; mat_off is not read).  rank_of_item: host, batch entries,
 * written with each item's rank in [0, ranks).  terms_per_rank: host, ranks
 * entries, written with the Gray-code terms each rank sums.  The result
 * depends only on the sizes, so every rank computes the same partition.
 * Host only, no GPU.  Errors: PQ_ERR_ARG (null, ranks outside [1, 65536],
 * negative sizes or offsets), PQ_ERR_UNSUPPORTED (as pq_plan_create). */
int pq_partition_batch(const pq_batch_sizes* sizes, int32_t ranks, int32_t* rank_of_item,
                       int64_t* terms_per_rank);

/* Boson-sampling probabilities, Eq. (BS_prob).  U: device, m x m, U[out][in];
 * input_occ: device, m; output_occ: device, B x m; probs: device, B doubles;
 * amps: device, B complex, nullable -- receives per(U_{s,t}) (needed by the
 * backward call).  plan: from pq_plan_create_bs for the same occupations, or
 * NULL (the call then copies the occupations to the host, plans, runs and
 * synchronises `stream`). */
int pq_bs_probs(const pq_c128* U, int32_t m, const int32_t* input_occ,
                const int32_t* output_occ, int64_t B, double* probs, pq_c128* amps,
                pq_plan* plan, void* stream);

/* Backward of pq_permanent_batched: grad_mats[b][i][j] = grad_out[b] *
 * conj(d per(A_b) / d B_b[i][j]), where d per / d b_ij counts every one of the
 * r_i c_j copies of b_ij (equal to r_i c_j per(B; r - e_i, c - e_j)).  Computed
 * in the same Gray-code pass as the permanent, with prefix and suffix products
 * of the column sums.  grad_out: device, batch; grad_mats: device, laid out
 * like b->mats (entries of zero-multiplicity rows/columns are set to zero).
 * plan: same rules as pq_permanent_batched. */
int pq_permanent_backward(const pq_batch* b, const pq_c128* grad_out, pq_c128* grad_mats,
                          pq_plan* plan, void* stream);

/* Backward of pq_bs_probs for L with dL/dp_b = grad_probs[b]:
 * grad_U (device, m x m) = sum_b 2 grad_probs[b] / (prod t! prod s!) *
 * amps[b] * conj(d per(U_{s,t_b}) / dU), summed over patterns in a fixed
 * order (no floating-point atomics, so the result is deterministic).
 * amps: device, the amplitudes from the forward call.  grad_U is overwritten.
 * plan: from pq_plan_create_bs for the same occupations, or NULL. */
int pq_bs_probs_backward(const pq_c128* U, int32_t m, const int32_t* input_occ,
                         const int32_t* output_occ, int64_t B, const double* grad_probs,
                         const pq_c128* amps, pq_c128* grad_U, pq_plan* plan, void* stream);

/* Clements mesh of m(m-1)/2 beamsplitters.  Beamsplitter k acts on modes
 * (j_k, j_k + 1) with the 2 x 2 block [[t, -conj(r)], [r, t]], t = cos theta_k,
 * r = exp(i phi_k) sin theta_k (Appendix A, "Beamsplitter gate").  Layout:
 * m layers; layer q holds the pairs j = q mod 2, q mod 2 + 2, ... (j + 1 < m),
 * numbered layer by layer with j ascending; U = T_{L-1} ... T_1 T_0.
 * theta, phi: device, L doubles; U: device, m x m, written (U[out][in]).
 * m <= PQ_MAX_DIM. */
int pq_clements_forward(const double* theta, const double* phi, int32_t m, pq_c128* U,
                        void* stream);

/* Adjoint of pq_clements_forward: given grad_U (device, m x m, PyTorch
 * convention) writes grad_theta and grad_phi (device, L doubles each).
 * Uses the recurrence W <- T_k^H W T_k from W = grad_U U^H, so U (device, the
 * forward output) is read rather than recomputed. */
int pq_clements_backward(const double* theta, const double* phi, int32_t m, const pq_c128* U,
                         const pq_c128* grad_U, double* grad_theta, double* grad_phi,
                         void* stream);

/* Boson-sampling probabilities with losses (Sec. 3.2.4, Fig. BS_LossModel):
 * the interferometer A = V diag(sqrt(eta)) W (V, W unitary, eta_i in [0, 1]
 * the transmission of mode i) loses photons to one inaccessible mode per
 * mode through a beamsplitter, and p(t) is the probability that the m system
 * detectors see t (|t| <= n; the rest were lost): the marginal of Eq.
 * (BS_prob) on the 2m-mode unitary dilation over every occupation of the loss
 * modes.  V, W: device, m x m (U[out][in] convention, A = V diag W); eta:
 * device, m doubles; input_occ: host, m; output_occ: host, B x m; probs:
 * device, B doubles.  2m <= PQ_MAX_DIM.  Allocates its workspace and
 * synchronises `stream`.  Errors: PQ_ERR_ARG (null, negative, |t| > n),
 * PQ_ERR_UNSUPPORTED (sizes), PQ_ERR_NOMEM, PQ_ERR_CUDA. */
int pq_bs_probs_lossy(const pq_c128* V, const double* eta, const pq_c128* W, int32_t m,
                      const int32_t* input_occ, const int32_t* output_occ, int64_t B,
                      double* probs, void* stream);

/* Planned lossy probabilities, for callers that evaluate the same patterns
 * for many interferometers: pq_lossy_plan_create does the host work of
 * pq_bs_probs_lossy once for input_occ (host, m) and output_occ (host, B x m)
 * -- every loss pattern of every output, the permanents' plan, the device
 * workspace -- and pq_lossy_plan_run evaluates probs (device, B doubles) for
 * V, eta, W (device, as for pq_bs_probs_lossy) with three launches on
 * `stream`: no host work, no allocation, no synchronisation.  One plan serves
 * one stream at a time; pq_lossy_plan_destroy synchronises the device and
 * frees it.  Errors as for pq_bs_probs_lossy; PQ_ERR_ARG for a null plan. */
typedef struct pq_lossy_plan pq_lossy_plan;
int pq_lossy_plan_create(int32_t m, const int32_t* input_occ, const int32_t* output_occ, int64_t B,
                         pq_lossy_plan** out);
int pq_lossy_plan_run(pq_lossy_plan* plan, const pq_c128* V, const double* eta, const pq_c128* W,
                      double* probs, void* stream);
int pq_lossy_plan_destroy(pq_lossy_plan* plan);

/* Boson sampling by Clifford and Clifford's "Algorithm A", the sampler the
 * paper uses with its permanents (Sec. 4.2): photons are drawn one at a time;
 * at step k every candidate output mode i is weighted by
 * |per(A[{r_1..r_{k-1}, i}, 1..k])|^2, A = the columns of U of the occupied
 * input modes (mode j repeated s_j times) in a random order.  Each step is
 * one batched launch over all samples and candidates.
 * U: device, m x m, U[out][in].  input_occ: host, m.  col_order: host,
 * nsamples x n, row b a permutation of 0 .. n-1 (the random column order of
 * sample b).  uniforms: host, nsamples x n, in [0, 1): the draw of photon k of
 * sample b picks the first mode whose running weight sum (modes in order)
 * exceeds uniforms[b][k-1] times the total.  samples: host, nsamples x m
 * output occupations.  Synchronises `stream`; allocates its workspace.
 * Errors: PQ_ERR_ARG (null, sizes, not a permutation, uniform outside
 * [0, 1), all weights zero), PQ_ERR_UNSUPPORTED, PQ_ERR_NOMEM, PQ_ERR_CUDA. */
int pq_bs_sample(const pq_c128* U, int32_t m, const int32_t* input_occ, int64_t nsamples,
                 const int32_t* col_order, const double* uniforms, int32_t* samples, void* stream);

/* Planned sampler, for callers that draw batch after batch from interferometers
 * with the same input occupation: pq_sampler_plan_create does the host work of
 * pq_bs_sample once for m, input_occ (host, m) and nsamples -- the plans of the
 * n - 1 steps' minors (nsamples x k minors of size k - 1 at step k) and the
 * device workspace -- and pq_sampler_plan_run draws nsamples samples for U
 * (device) with col_order, uniforms and samples as for pq_bs_sample: it uploads
 * the draws, launches the steps on `stream`, reads the drawn modes back and
 * synchronises `stream`; it allocates nothing.  The same U, orders and
 * uniforms give the samples of pq_bs_sample.  One plan serves one stream at a
 * time; pq_sampler_plan_destroy synchronises the device and frees it.  Errors
 * as for pq_bs_sample; PQ_ERR_ARG for a null plan. */
typedef struct pq_sampler_plan pq_sampler_plan;
int pq_sampler_plan_create(int32_t m, const int32_t* input_occ, int64_t nsamples,
                           pq_sampler_plan** out);
int pq_sampler_plan_run(pq_sampler_plan* plan, const pq_c128* U, const int32_t* col_order,
                        const double* uniforms, int32_t* samples, void* stream);
int pq_sampler_plan_destroy(pq_sampler_plan* plan);

/* Hafnians with repeated indices (Sec. 4.1, Eq. (haf_def); the paper's
 * hafnian benchmark repeats every index twice).  Item b is the hafnian of the
 * N x N matrix that repeats base index i of the symmetric k[b] x k[b] base
 * matrix rep[rep_off[b] + i] times in both rows and columns, N = sum of the
 * repetitions.  Evaluated by the sign-vector (Glynn-type) formula
 *   haf = 1/(n! 2^{N-1}) sum_g (-1)^{|g|} prod_i C(top_i, g_i) q(g)^n,
 *   q(g) = 1/2 (x^T B x - sum_i r_i B_ii),  x_i = r_i - 2 g_i,  n = N/2,
 * one copy of the least repeated index fixed to +, over a mixed-radix Gray
 * code with O(k) work per term and double-double accumulation.  Odd N gives
 * 0, N = 0 gives 1.
 * mats: device, packed row-major complex bases at element offsets
 * mat_off[b] (host, int64); k, rep, rep_off: host; only the upper triangle
 * and diagonal matter for a symmetric base (the kernel reads both halves, so
 * pass a symmetric matrix).  out: device, batch complex.  N <= PQ_MAX_N,
 * k <= PQ_MAX_DIM.  Allocates its workspace and synchronises `stream`.
 * Errors: PQ_ERR_ARG (null, negative sizes or repetitions),
 * PQ_ERR_UNSUPPORTED (N or term count too large), PQ_ERR_NOMEM, PQ_ERR_CUDA. */
int pq_hafnian_repeated(const pq_c128* mats, const int64_t* mat_off, const int32_t* k,
                        const int32_t* rep, const int64_t* rep_off, int64_t batch, pq_c128* out,
                        void* stream);

/* Planned (loop) hafnians, for callers that evaluate the same shapes many
 * times: pq_hafnian_plan_create does the host planning of pq_hafnian_repeated
 * (loop = 0) or pq_loop_hafnian_repeated (loop = 1) once for the sizes and
 * repetitions given (host arrays, copied; same layout and limits as those
 * calls), uploads the schedule and allocates the device workspace.
 * pq_hafnian_plan_run then evaluates the batch for the matrix values at mats
 * (and loop weights at gamma when loop = 1; device, same layout as those
 * calls) into out (device, batch complex): it allocates nothing, reads no
 * host memory and does not synchronise `stream`.  One plan serves one stream
 * at a time.  pq_hafnian_plan_destroy synchronises the device and frees the
 * plan.  Errors as for pq_hafnian_repeated; PQ_ERR_ARG for a null plan, or a
 * null gamma on a loop plan. */
typedef struct pq_haf_plan pq_haf_plan;
int pq_hafnian_plan_create(const int64_t* mat_off, const int32_t* k, const int32_t* rep,
                           const int64_t* rep_off, int64_t batch, int32_t loop, pq_haf_plan** out);
int pq_hafnian_plan_run(pq_haf_plan* plan, const pq_c128* mats, const pq_c128* gamma, pq_c128* out,
                        void* stream);
int pq_hafnian_plan_destroy(pq_haf_plan* plan);

/* Loop hafnians with repeated indices (Eq. (loop_hafnian), with the filldiag
 * of the displaced Gaussian detection probability in Appendix A: every copy
 * of base index i gets the loop weight gamma_i on the diagonal).  Item b is
 * lhaf(filldiag(A_r, gamma_r)), A_r repeating index i of the k[b] x k[b] base
 * rep[rep_off[b] + i] times.  Glynn-type formula
 *   lhaf = 1/2^{N-1} sum_g (-1)^{|g|} prod_i C(top_i, g_i)
 *          sum_{j <= N/2} q(g)^j l(g)^{N-2j} / (j! (N-2j)!),   l(g) = gamma^T x,
 * q, x, the digits and the Gray walk as for pq_hafnian_repeated; any N >= 0
 * (N = 0 gives 1).  gamma: device, complex, packed like rep (element
 * rep_off[b] + i is the loop weight of base index i of item b); the base
 * diagonal B_ii is still the weight of a pair of two copies of index i.
 * Other arguments, allocation, synchronisation and errors as for
 * pq_hafnian_repeated (PQ_ERR_ARG also for gamma == NULL with batch > 0). */
int pq_loop_hafnian_repeated(const pq_c128* mats, const pq_c128* gamma, const int64_t* mat_off,
                             const int32_t* k, const int32_t* rep, const int64_t* rep_off,
                             int64_t batch, pq_c128* out, void* stream);

/* Times trial launches of the plan's batched kernel for each size class on
 * the given data and picks the fastest chunk length per class; then times the
 * whole batch with those picks and with the chunking the plan had, and keeps
 * the picks -- in the plan and in the process-wide tuning table used by later
 * plans -- only if they are at least 1% faster.  Otherwise the plan and the
 * table stay as they were.  A plan whose column sums the planner put in
 * registers (column_sums PQ_SUMS_AUTO, one column class) is then timed with
 * them in shared memory as well, and keeps shared memory if that is at least
 * 1% faster (pq_plan_get_stats reports the choice).  Synchronises `stream`.
 * b is the batch the plan
 * was made for (device descriptor); for a boson-sampling plan pass b = NULL
 * and U (device) instead.  If re-planning fails (PQ_ERR_NOMEM, PQ_ERR_CUDA)
 * and the plan cannot be restored, later runs of it return PQ_ERR_STATE. */
int pq_autotune(pq_plan* plan, const pq_batch* b, const pq_c128* U, void* stream);

/* The process-wide tuning table: entry n (n = 0 .. PQ_MAX_N) is the Gray-code
 * chunk length, as log2 of the number of terms, that later plans use for
 * permanents of n photons (0: the built-in default); pq_autotune fills it.
 * host arrays of PQ_MAX_N + 1 int32; set rejects entries outside [0, 30]
 * (PQ_ERR_ARG).  Every shard of a split permanent batch (pq_plan_options
 * shard_count > 1) must be planned under the same table: planning reads it,
 * so shards planned under different tables cut the Gray code differently
 * and their partials do not add up.  No GPU needed. */
int pq_tune_table_get(int32_t* log2);
int pq_tune_table_set(const int32_t* log2);

/* Tuning cache on disk: a JSON file {"format": ..., "tables": {"<device
 * key>": [PQ_MAX_N + 1 ints], ...}} holding one tuning table per GPU model.
 * pq_tune_cache_save writes the current table under device_key (NULL: the
 * current device's name and SM count, which needs a GPU), keeping the other
 * keys of an existing file; the file is replaced atomically.
 * pq_tune_cache_load sets the table from the entry of device_key (same
 * default) and reports in *found whether the file had one (a missing file is
 * not an error: *found = 0).  Planning itself never touches the file.
 * Errors: PQ_ERR_ARG (null, unreadable or malformed file, bad table),
 * PQ_ERR_CUDA (no device to name the key). */
int pq_tune_cache_save(const char* path, const char* device_key);
int pq_tune_cache_load(const char* path, const char* device_key, int32_t* found);

/* Device error record of a plan.  Before using a warp task, the forward and
 * backward kernels check it and the descriptor it names against the launch:
 * the permanent index, the task's part, the base sizes against the launch's
 * shared-memory layout, the digit counts against the Gray walk's limits, and
 * the descriptor's indices into the plan's metadata, partial sums and
 * outputs.  A task that fails is skipped (its permanent's output is left
 * unwritten) and the first failure is kept.  This call reads the record
 * (it synchronises the device): *code receives 0 or a PQ_DEVERR_* code,
 * *task the index of the failing task in the launch's task list; clear != 0
 * resets the record.  The synchronous calls (plan == NULL) read it
 * themselves and return PQ_ERR_STATE when it is set.  No device wait exists
 * in the library, so PQ_ERR_TIMEOUT is never returned. */
#define PQ_DEVERR_TASK_PERM 1   /* task names a permanent outside the batch          */
#define PQ_DEVERR_TASK_PART 2   /* task part outside its permanent's range             */
#define PQ_DEVERR_LAYOUT 3      /* base sizes beyond the launch's shared-memory layout */
#define PQ_DEVERR_DIGITS 4      /* digit counts beyond the walk's limits               */
#define PQ_DEVERR_INDEX 5       /* metadata, partial-sum or output index out of range  */
int pq_plan_device_error(pq_plan* plan, int32_t* code, int64_t* task, int32_t clear);

/* Statistics of a plan, host memory: number of permanents, total Gray-code
 * terms, algorithmic FP64 flops of one forward execution (FMA = 2; the count
 * of a straightforward Glynn evaluation: 2l + 6(n-1) + 2 per term, +2 for a
 * non-unit weight), FP64 instructions the forward kernel needs for its terms
 * (Gray step, products, fused accumulation, weights, double-double fold;
 * each DADD, DMUL or DFMA counts one), number of warp tasks and of kernel
 * launches one execution makes.  flops_backward is the algorithmic count of
 * a backward that forms the k x l rank-1 update of every term (2l + 6(n-1)
 * + 2 + 18l + 8kl); the kernel's correction scheme avoids that update, so
 * fp64_instr_backward (per term: column and correction updates, prefix and
 * suffix products, accumulation; per chunk: the start from the high digits;
 * per task: the lane contraction) is the count to compare with the FP64
 * pipe.  fp64_instr_backward is filled in by the first backward call (zero
 * before it), which also settles launches_backward.
 * fp64_instr_forward_executed adds what the forward executes besides the
 * terms, counted per lane: the lanes of a task without a chunk (they walk
 * with the others), each chunk's start from its high digits, the fold and
 * scaling of each chunk's sum, the per-task lane reduction and the
 * per-permanent combination of task partials. */
typedef struct {
    int64_t permanents;
    int64_t terms;
    double flops_forward;
    double flops_backward;
    int64_t tasks;
    int64_t launches_forward;
    int64_t launches_backward;
    int32_t lmax;
    int32_t column_sums; /* where the forward walk keeps them: PQ_SUMS_SHARED or
                            PQ_SUMS_REGISTERS (the planner's choice under AUTO)    */
    double fp64_instr_forward;
    double fp64_instr_backward;
    double fp64_instr_forward_executed;
} pq_plan_stats;
int pq_plan_get_stats(const pq_plan* plan, pq_plan_stats* out);

/* FP64 throughput probe: runs independent DFMA chains on every SM for about
 * `iters` iterations and returns the measured rate in FLOP/s (FMA = 2) and
 * the elapsed milliseconds.  Synchronises `stream`.  Measures the chip, not
 * the paper's method; it provides the roofline denominator. */
int pq_probe_fp64_peak(int64_t iters, double* flops_per_s, double* ms, void* stream);

/* FP64 pipe sweep: op 0 = DFMA, 1 = DADD, 2 = DMUL; `warps_per_sm` resident
 * warps on every SM (1 .. 64), each thread running `chains` (1, 2, 4 or 8)
 * independent dependency chains of that instruction for 4 x iters steps.
 * Writes the measured lane operations per second per SM (divide by the SM
 * clock for operations per clock).  Synchronises `stream`.  Measures the
 * chip: how many warps saturate the FP64 pipe and whether dependency
 * latency matters, which fixes the layout of the kernels. */
int pq_probe_fp64_sweep(int32_t op, int32_t warps_per_sm, int32_t chains, int64_t iters,
                        double* lane_ops_per_sm_per_s, void* stream);

/* ---- Permanent without allocation ---------------------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: code inside a framework whose caching
 * allocator owns the device memory (an allocation of its own can fail or
 * fragment that pool), processes held to a fixed device-memory budget, and
 * latency-critical paths that cannot pay for the device synchronisation an
 * allocation may cause.
 *
 * Computes per(A) of ONE base matrix exactly like pq_permanent_batched (same
 * kernel, same method) but allocates nothing: the descriptor, the task list,
 * the partial sums and the counters live in a static device array of
 * PQ_NOALLOC_SCRATCH_BYTES that every GPU holds from the moment it loads the
 * library until the process exits.  The call plans on the host into a
 * fixed-size structure and hands it to a set-up kernel by value, so nothing
 * the host passes has to outlive the call.
 *   B: device, k x l row-major complex; row_mult[k], col_mult[l]: HOST
 *   (read during the call); out: device, one complex.  Asynchronous on stream.
 * Errors: PQ_ERR_ARG (null, negative, sum r != sum c); PQ_ERR_UNSUPPORTED
 * beyond the limits of pq.h or when the permanent needs more warp tasks
 * than the array holds (about 26,000 tasks: every collision-free permanent up
 * to n = 35 fits);
 * PQ_ERR_CUDA.
 * The first call on a device looks up the array's device address with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture, and do not use the call after
 * cudaDeviceReset on that device.  Every call reuses the same array (the
 * counters are cleared at the start of each call), so calls whose GPU work
 * overlaps -- on two streams or from two host threads -- race with each
 * other: serialise them. */
#define PQ_NOALLOC_SCRATCH_BYTES (1 << 20)
int pq_permanent_noalloc(const pq_c128* B, int32_t k, int32_t l, const int32_t* row_mult,
                         const int32_t* col_mult, pq_c128* out, void* stream);

/* ---- Test hooks ----------------------------------------------------------
 * pq_debug_fail_allocation(after): the allocation that follows `after`
 * successful ones -- device buffers and the host plan objects the library
 * creates -- reports failure (PQ_ERR_NOMEM from the call that made it), once;
 * after < 0 disarms the hook.  pq_debug_live_allocations: the device buffers
 * and plan objects the library currently holds (a call that fails must leave
 * both where they were).  pq_debug_corrupt_plan(plan, what) overwrites the
 * plan's device-side schedule so that the kernels' guards have something to
 * catch: what = 1, the first task of each task list names permanent
 * batch + 5; what = 2, permanent 0's descriptor gets more product columns
 * than the launch's layout holds.  The host copy is left alone; destroy the
 * plan afterwards.  The hooks need no GPU except pq_debug_corrupt_plan. */
int pq_debug_fail_allocation(int64_t after);
int pq_debug_live_allocations(int64_t* device_buffers, int64_t* host_objects);
int pq_debug_corrupt_plan(pq_plan* plan, int32_t what);

/* ---- Diagnostics (host only; no GPU needed) ---------------------------- */

/* How the planner treats one permanent in a batched forward plan: the side it
 * sums, the digits of the mixed-radix Gray code (digit d belongs to summed
 * row row_of_digit[d]; the J low digits walked inside a chunk come first, then
 * the others, each group in ascending radix) and how the code is cut into
 * chunks. */
typedef struct {
    int32_t n, k, l;     /* photons; summed rows and product columns after orientation */
    int32_t transposed;  /* 1 if the input's columns became the summed side         */
    int32_t ndig, J;     /* Gray digits; low digits walked inside one chunk          */
    int64_t terms;       /* Gray-code terms T = prod radix                            */
    int64_t chunk_len;   /* L = prod of the J low radices                             */
    int64_t chunks;      /* T / L                                                     */
    int32_t radix[PQ_MAX_N];
    int32_t row_of_digit[PQ_MAX_N];
} pq_item_info;

/* Plan one permanent of a k x l base with multiplicities row_mult[k],
 * col_mult[l] (host memory) for the given chunk_log2 (0 = default) and
 * describe it.  Errors as pq_plan_create. */
int pq_plan_item_info(int32_t k, int32_t l, const int32_t* row_mult, const int32_t* col_mult,
                      int32_t chunk_log2, pq_item_info* out);

/* The exact warp sum of the forward kernels' lane reduction, run on the host:
 * out[0] + out[1] = sum_q (hi[q] + lo[q]) over n <= 32 finite pairs (host
 * arrays), exact except for bits below 2^-64 of the last significand bit of
 * the largest input, truncated; out[0] holds the leading 53 bits, out[1] the
 * leading 53 bits of the rest.  PQ_ERR_ARG: n outside [0, 32], a null
 * pointer or a value that is not finite. */
int pq_fixsum_host(const double* hi, const double* lo, int32_t n, double* out);

/* The same warp sum run by one warp on the device (a test of the device
 * code): hi[n], lo[n] device arrays, n <= 32; out: device array of 64
 * doubles, lane q's copy of the sum in out[2q], out[2q + 1].  Asynchronous
 * on stream.  A non-finite input makes the warp add in plain FP64 (the
 * result is then not finite).  PQ_ERR_ARG: n outside [0, 32] or a null
 * pointer; PQ_ERR_CUDA: the launch failed. */
int pq_fixsum_device(const double* hi, const double* lo, int32_t n, double* out, void* stream);

/* Run the kernels' warp-uniform Gray walk on the host: ndig <= 15 digits with
 * radix[d] in [2, 15]; for `steps` steps writes the digit that changes and
 * its direction (+1 / -1) to host arrays digit[steps], dir[steps]. */
int pq_gray_walk(const int32_t* radix, int32_t ndig, int64_t steps, int32_t* digit, int32_t* dir);

/* The factors the loop-hafnian kernel evaluates its degree-N polynomial
 * sum_{j <= N/2} q^j l^{N-2j} / (j! (N-2j)!) with (host only; no GPU needed):
 * out[0] = 1 / J!, J = floor(N/2); then for each pair of the real roots
 * z_m = -1/(2 x_m^2) (x_m the positive roots of the Hermite polynomial He_N,
 * ascending) a = -(z_1 + z_2) and b = z_1 z_2; then, if J is odd, the last
 * root.  The polynomial is out[0] prod_pairs (q^2 + a q s + b s^2)
 * [(q - z s)] [l], s = l^2.  out: host, J + 1 doubles.
 * Errors: PQ_ERR_ARG (N outside [0, PQ_MAX_N], null out). */
int pq_loop_poly_factors(int32_t N, double* out);

/* Message of the last error on the calling thread ("" if none). */
const char* pq_last_error(void);

/* Library version string. */
const char* pq_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PQ_GB300_H */
