/*
 * pq_oracle.c -- CPU oracle for permanents with repeated rows/columns and for
 * boson-sampling probabilities.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path in
 * paper_2403_04006_gb300/csrc; the two meet only through seeded inputs.
 *
 * What it computes (paper: "Piquasso", arXiv 2403.04006):
 *   - per(A) = sum over permutations s of prod_i A[s(i)][i]
 *       (Appendix A, "Particle number measurement", Eq. (per_def)),
 *     by brute force over all n! permutations                 -> oracle_perm_bruteforce
 *   - per of the n x n matrix A obtained from a k x l base matrix B by
 *     repeating row i r_i times and column j c_j times (the "row or column
 *     multiplicities" of Sec. 4.2, "Boson Sampling"), by Ryser's
 *     inclusion-exclusion formula (the Ryser variant the paper compares
 *     against in Sec. 4.2) with the repetitions grouped:
 *       per(A) = (-1)^n sum_{0<=k_i<=r_i} (-1)^{sum k} prod_i C(r_i,k_i)
 *                        prod_j ( sum_i k_i b_ij )^{c_j}             -> oracle_perm_ryser
 *     Choosing k_i of the r_i copies of base row i can be done C(r_i,k_i)
 *     ways and every such choice gives the same column sums, which is all
 *     the grouping does.
 *   - p(s,t) = |per(U_{s,t})|^2 / (prod t_i! prod s_i!)  (Eq. (BS_prob))
 *                                                              -> oracle_bs_probs
 *   - d per / d b_ij = r_i c_j per(B; r - e_i, c - e_j): b_ij sits in r_i c_j
 *     entries of A and d per(A)/d A_pq is the permanent of A without row p and
 *     column q (Laplace expansion of Eq. (per_def)).             -> oracle_perm_grad
 *
 * Arithmetic.  "fast" mode: column sums and products in IEEE binary64, every
 * term added into a double-double (hi, lo) accumulator with Knuth's TwoSum.
 * "gold" mode: column sums, products and accumulation all in double-double
 * (TwoProd via a single fma).  Column sums are recomputed from scratch every
 * 1024 enumeration steps so that incremental updates cannot drift.  Build with
 * -ffp-contract=off so every operation rounds as written.
 *
 * Every result also carries sum_terms |term| and an a-posteriori error bound
 * gamma = sum|term| * (2n+4) * u (u = 2^-53 fast, 2^-104 gold, plus the final
 * double rounding), so a test can tell when a tolerance is beyond what the
 * oracle can vouch for.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_TOO_LARGE (-2)
#define ORC_ERR_NOMEM (-3)

/* ------------------------------------------------------------------------ */
/* double-double arithmetic                                                  */
/* ------------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd_t;
typedef struct { dd_t re, im; } cdd_t;
typedef struct { double re, im; } cd_t;

/* Knuth's TwoSum: s + e == a + b exactly. */
static dd_t two_sum(double a, double b)
{
    double s = a + b;
    double bv = s - a;
    double av = s - bv;
    dd_t r;
    r.hi = s;
    r.lo = (a - av) + (b - bv);
    return r;
}

/* Dekker's Fast2Sum; exact when |a| >= |b| (or a == 0). */
static dd_t fast_two_sum(double a, double b)
{
    double s = a + b;
    dd_t r;
    r.hi = s;
    r.lo = b - (s - a);
    return r;
}

static dd_t dd_from(double a)
{
    dd_t r = { a, 0.0 };
    return r;
}

/* Accurate double-double addition (two TwoSums, two renormalisations). */
static dd_t dd_add(dd_t a, dd_t b)
{
    dd_t s = two_sum(a.hi, b.hi);
    dd_t t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

static dd_t dd_neg(dd_t a)
{
    dd_t r = { -a.hi, -a.lo };
    return r;
}

/* Double-double product; the exact error of hi*hi comes from one fma. */
static dd_t dd_mul(dd_t a, dd_t b)
{
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);
    e += a.hi * b.lo;
    e += a.lo * b.hi;
    return fast_two_sum(p, e);
}

static cdd_t cdd_add(cdd_t a, cdd_t b)
{
    cdd_t r;
    r.re = dd_add(a.re, b.re);
    r.im = dd_add(a.im, b.im);
    return r;
}

static cdd_t cdd_mul(cdd_t a, cdd_t b)
{
    cdd_t r;
    r.re = dd_add(dd_mul(a.re, b.re), dd_neg(dd_mul(a.im, b.im)));
    r.im = dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re));
    return r;
}

static cd_t cd_mul(cd_t a, cd_t b)
{
    cd_t r;
    r.re = a.re * b.re - a.im * b.im;
    r.im = a.re * b.im + a.im * b.re;
    return r;
}

/* ------------------------------------------------------------------------ */
/* binomials                                                                 */
/* ------------------------------------------------------------------------ */
static double binom(int n, int k)
{
    double r = 1.0;
    int i;
    if (k < 0 || k > n)
        return 0.0;
    for (i = 1; i <= k; i++)
        r = r * (double)(n - k + i) / (double)i; /* exact while < 2^53 */
    return r;
}

static double factorial(int n)
{
    double r = 1.0;
    int i;
    for (i = 2; i <= n; i++)
        r *= (double)i;
    return r;
}

/* ------------------------------------------------------------------------ */
/* brute force over permutations, Eq. (per_def)                              */
/* ------------------------------------------------------------------------ */

/* a: n x n complex, row-major, interleaved (re, im).  out[0..1] = per(a),
 * out[2] = sum |term|.  Permutations are visited in lexicographic order. */
int oracle_perm_bruteforce(const double *a, int n, double *out)
{
    int perm[16];
    int i, j;
    cdd_t acc;
    double sumabs = 0.0;
    if (n < 0 || n > 12 || (n > 0 && a == NULL) || out == NULL)
        return ORC_ERR_ARG;
    acc.re = dd_from(n == 0 ? 1.0 : 0.0);
    acc.im = dd_from(0.0);
    if (n == 0) {
        out[0] = 1.0;
        out[1] = 0.0;
        out[2] = 1.0;
        return ORC_OK;
    }
    for (i = 0; i < n; i++)
        perm[i] = i;
    for (;;) {
        /* term = prod_i A[sigma(i)][i] */
        cd_t t;
        t.re = a[2 * (perm[0] * n + 0)];
        t.im = a[2 * (perm[0] * n + 0) + 1];
        for (i = 1; i < n; i++) {
            cd_t x;
            x.re = a[2 * (perm[i] * n + i)];
            x.im = a[2 * (perm[i] * n + i) + 1];
            t = cd_mul(t, x);
        }
        acc.re = dd_add(acc.re, dd_from(t.re));
        acc.im = dd_add(acc.im, dd_from(t.im));
        sumabs += hypot(t.re, t.im);
        /* next permutation in lexicographic order */
        i = n - 2;
        while (i >= 0 && perm[i] > perm[i + 1])
            i--;
        if (i < 0)
            break;
        j = n - 1;
        while (perm[j] < perm[i])
            j--;
        {
            int tmp = perm[i];
            perm[i] = perm[j];
            perm[j] = tmp;
        }
        {
            /* reverse the tail perm[i+1 .. n-1] */
            int lo = i + 1, hi = n - 1;
            while (lo < hi) {
                int tmp = perm[lo];
                perm[lo] = perm[hi];
                perm[hi] = tmp;
                lo++;
                hi--;
            }
        }
    }
    out[0] = acc.re.hi + acc.re.lo;
    out[1] = acc.im.hi + acc.im.lo;
    out[2] = sumabs;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Ryser's formula with repeated rows and columns                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    const double *b; /* k x l complex, row-major, interleaved */
    int k, l, n;
    const int *r, *c;
    int gold;
    int64_t lo, hi;   /* odometer ranks [lo, hi) handled by this worker */
    cdd_t acc;        /* partial sum of the signed, weighted terms        */
    double sumabs;    /* sum of |term|                                    */
} ryser_job;

#define RESYNC_STEPS 1024

/* column sums S_j = sum_i k_i b_ij from scratch */
static void colsums_fast(const ryser_job *jb, const int *kd, cd_t *S)
{
    int i, j;
    for (j = 0; j < jb->l; j++) {
        S[j].re = 0.0;
        S[j].im = 0.0;
    }
    for (i = 0; i < jb->k; i++) {
        if (kd[i] == 0)
            continue;
        for (j = 0; j < jb->l; j++) {
            S[j].re += (double)kd[i] * jb->b[2 * (i * jb->l + j)];
            S[j].im += (double)kd[i] * jb->b[2 * (i * jb->l + j) + 1];
        }
    }
}

static void colsums_gold(const ryser_job *jb, const int *kd, cdd_t *S)
{
    int i, j;
    for (j = 0; j < jb->l; j++) {
        S[j].re = dd_from(0.0);
        S[j].im = dd_from(0.0);
    }
    for (i = 0; i < jb->k; i++) {
        dd_t ki = dd_from((double)kd[i]);
        if (kd[i] == 0)
            continue;
        for (j = 0; j < jb->l; j++) {
            S[j].re = dd_add(S[j].re, dd_mul(ki, dd_from(jb->b[2 * (i * jb->l + j)])));
            S[j].im = dd_add(S[j].im, dd_mul(ki, dd_from(jb->b[2 * (i * jb->l + j) + 1])));
        }
    }
}

/* One worker: enumerate the mixed-radix counter k (digit i in [0, r_i],
 * digit 0 least significant) from rank lo to hi-1. */
static void *ryser_worker(void *arg)
{
    ryser_job *jb = (ryser_job *)arg;
    int K = jb->k, L = jb->l;
    int kd[64];
    cd_t Sf[64];
    cdd_t Sg[64];
    int64_t rank, rem;
    int i, j, steps = 0;
    jb->acc.re = dd_from(0.0);
    jb->acc.im = dd_from(0.0);
    jb->sumabs = 0.0;
    if (jb->lo >= jb->hi)
        return NULL;
    /* decode the starting rank */
    rem = jb->lo;
    for (i = 0; i < K; i++) {
        kd[i] = (int)(rem % (jb->r[i] + 1));
        rem /= (jb->r[i] + 1);
    }
    if (jb->gold)
        colsums_gold(jb, kd, Sg);
    else
        colsums_fast(jb, kd, Sf);
    for (rank = jb->lo; rank < jb->hi; rank++) {
        /* weight (-1)^{sum k} prod_i C(r_i, k_i) */
        int ksum = 0;
        double w = 1.0;
        for (i = 0; i < K; i++) {
            ksum += kd[i];
            w *= binom(jb->r[i], kd[i]);
        }
        if (ksum & 1)
            w = -w;
        if (jb->gold) {
            cdd_t p;
            dd_t wd = dd_from(w);
            p.re = dd_from(1.0);
            p.im = dd_from(0.0);
            for (j = 0; j < L; j++) {
                int e;
                for (e = 0; e < jb->c[j]; e++)
                    p = cdd_mul(p, Sg[j]);
            }
            p.re = dd_mul(p.re, wd);
            p.im = dd_mul(p.im, wd);
            jb->acc = cdd_add(jb->acc, p);
            jb->sumabs += hypot(p.re.hi, p.im.hi);
        } else {
            cd_t p = { 1.0, 0.0 };
            for (j = 0; j < L; j++) {
                int e;
                for (e = 0; e < jb->c[j]; e++)
                    p = cd_mul(p, Sf[j]);
            }
            p.re *= w;
            p.im *= w;
            jb->acc.re = dd_add(jb->acc.re, dd_from(p.re));
            jb->acc.im = dd_add(jb->acc.im, dd_from(p.im));
            jb->sumabs += hypot(p.re, p.im);
        }
        if (rank + 1 >= jb->hi)
            break;
        /* advance the odometer, updating the column sums incrementally */
        for (i = 0; i < K; i++) {
            if (kd[i] < jb->r[i]) {
                kd[i] += 1;
                for (j = 0; j < L; j++) {
                    double bre = jb->b[2 * (i * L + j)], bim = jb->b[2 * (i * L + j) + 1];
                    if (jb->gold) {
                        Sg[j].re = dd_add(Sg[j].re, dd_from(bre));
                        Sg[j].im = dd_add(Sg[j].im, dd_from(bim));
                    } else {
                        Sf[j].re += bre;
                        Sf[j].im += bim;
                    }
                }
                break;
            }
            /* digit wraps from r_i back to 0: remove r_i copies of row i */
            if (jb->r[i] > 0) {
                for (j = 0; j < L; j++) {
                    double bre = jb->b[2 * (i * L + j)], bim = jb->b[2 * (i * L + j) + 1];
                    if (jb->gold) {
                        dd_t ri = dd_from((double)jb->r[i]);
                        Sg[j].re = dd_add(Sg[j].re, dd_neg(dd_mul(ri, dd_from(bre))));
                        Sg[j].im = dd_add(Sg[j].im, dd_neg(dd_mul(ri, dd_from(bim))));
                    } else {
                        Sf[j].re -= (double)jb->r[i] * bre;
                        Sf[j].im -= (double)jb->r[i] * bim;
                    }
                }
            }
            kd[i] = 0;
        }
        if (++steps == RESYNC_STEPS) {
            steps = 0;
            if (jb->gold)
                colsums_gold(jb, kd, Sg);
            else
                colsums_fast(jb, kd, Sf);
        }
    }
    return NULL;
}

/* Permanent of the expanded matrix given by base b (k x l complex, row-major,
 * interleaved) with row multiplicities r[k] and column multiplicities c[l].
 * gold = 0: binary64 products, double-double accumulation; gold = 1:
 * double-double throughout.  nthreads >= 1 splits the rank range into that
 * many contiguous pieces whose partials are added in piece order, so the
 * result does not depend on scheduling.
 * out[0..1] = per, out[2] = sum |term|, out[3] = error bound gamma. */
int oracle_perm_ryser(const double *b, int k, int l, const int *r, const int *c, int gold,
                      int nthreads, double *out)
{
    int i, n = 0, nc = 0;
    int64_t T = 1;
    ryser_job jobs[256];
    pthread_t th[256];
    cdd_t acc;
    double sumabs = 0.0, u;
    if (k < 0 || l < 0 || k > 64 || l > 64 || out == NULL || (k > 0 && (r == NULL)) ||
        (l > 0 && c == NULL) || (k > 0 && l > 0 && b == NULL))
        return ORC_ERR_ARG;
    for (i = 0; i < k; i++) {
        if (r[i] < 0)
            return ORC_ERR_ARG;
        n += r[i];
    }
    for (i = 0; i < l; i++) {
        if (c[i] < 0)
            return ORC_ERR_ARG;
        nc += c[i];
    }
    if (n != nc)
        return ORC_ERR_ARG;
    if (n > 62)
        return ORC_ERR_TOO_LARGE;
    for (i = 0; i < k; i++) {
        if (T > ((int64_t)1 << 62) / (r[i] + 1))
            return ORC_ERR_TOO_LARGE;
        T *= (r[i] + 1);
    }
    if (n == 0) {
        out[0] = 1.0;
        out[1] = 0.0;
        out[2] = 1.0;
        out[3] = 0.0;
        return ORC_OK;
    }
    memset(jobs, 0, sizeof(jobs));
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    if ((int64_t)nthreads > T)
        nthreads = (int)T;
    for (i = 0; i < nthreads; i++) {
        jobs[i].b = b;
        jobs[i].k = k;
        jobs[i].l = l;
        jobs[i].n = n;
        jobs[i].r = r;
        jobs[i].c = c;
        jobs[i].gold = gold;
        jobs[i].lo = T * i / nthreads;
        jobs[i].hi = T * (i + 1) / nthreads;
    }
    if (nthreads == 1) {
        ryser_worker(&jobs[0]);
    } else {
        int started = 0;
        for (i = 0; i < nthreads; i++) {
            if (pthread_create(&th[i], NULL, ryser_worker, &jobs[i]) != 0)
                break;
            started++;
        }
        for (i = started; i < nthreads; i++) /* fall back to this thread */
            ryser_worker(&jobs[i]);
        for (i = 0; i < started; i++)
            pthread_join(th[i], NULL);
    }
    acc = jobs[0].acc;
    sumabs = jobs[0].sumabs;
    for (i = 1; i < nthreads; i++) {
        acc = cdd_add(acc, jobs[i].acc);
        sumabs += jobs[i].sumabs;
    }
    if (n & 1) {
        acc.re = dd_neg(acc.re);
        acc.im = dd_neg(acc.im);
    }
    out[0] = acc.re.hi + acc.re.lo;
    out[1] = acc.im.hi + acc.im.lo;
    out[2] = sumabs;
    u = gold ? ldexp(1.0, -104) : ldexp(1.0, -53);
    out[3] = sumabs * (2.0 * n + 4.0) * u + ldexp(hypot(out[0], out[1]), -52);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* gradient through Laplace minors                                           */
/* ------------------------------------------------------------------------ */

/* grad[i][j] = d per / d b_ij = r_i c_j per(B; r - e_i, c - e_j), k x l complex. */
int oracle_perm_grad(const double *b, int k, int l, const int *r, const int *c, int gold,
                     int nthreads, double *grad)
{
    int i, j, rc;
    int rr[64], cc[64];
    double o[4];
    if (k < 0 || l < 0 || k > 64 || l > 64 || grad == NULL)
        return ORC_ERR_ARG;
    for (i = 0; i < k; i++)
        rr[i] = r[i];
    for (j = 0; j < l; j++)
        cc[j] = c[j];
    for (i = 0; i < k; i++) {
        for (j = 0; j < l; j++) {
            grad[2 * (i * l + j)] = 0.0;
            grad[2 * (i * l + j) + 1] = 0.0;
            if (r[i] == 0 || c[j] == 0)
                continue;
            rr[i] -= 1;
            cc[j] -= 1;
            rc = oracle_perm_ryser(b, k, l, rr, cc, gold, nthreads, o);
            rr[i] += 1;
            cc[j] += 1;
            if (rc != ORC_OK)
                return rc;
            grad[2 * (i * l + j)] = (double)r[i] * (double)c[j] * o[0];
            grad[2 * (i * l + j) + 1] = (double)r[i] * (double)c[j] * o[1];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* batches (one worker thread per slice of items; items are independent)     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t batch;
    const double *mats;
    const int64_t *mat_off;
    const int *k, *l, *rm, *cm;
    const int64_t *roff, *coff;
    int gold;
    int64_t lo, hi, stride;
    double *out;
    int rc;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *jb = (batch_job *)arg;
    int64_t it;
    jb->rc = ORC_OK;
    for (it = jb->lo; it < jb->batch; it += jb->stride) {
        double o[4];
        int rc = oracle_perm_ryser(jb->mats + 2 * jb->mat_off[it], jb->k[it], jb->l[it],
                                   jb->rm + jb->roff[it], jb->cm + jb->coff[it], jb->gold, 1, o);
        if (rc != ORC_OK) {
            jb->rc = rc;
            return NULL;
        }
        jb->out[4 * it + 0] = o[0];
        jb->out[4 * it + 1] = o[1];
        jb->out[4 * it + 2] = o[2];
        jb->out[4 * it + 3] = o[3];
    }
    return NULL;
}

/* Ragged batch: item it has base matrix mats[2*mat_off[it] ...] (k[it] x l[it]
 * complex, row-major), row multiplicities rm[roff[it] ...] and column
 * multiplicities cm[coff[it] ...].  out is batch x 4 doubles
 * (re, im, sum|term|, bound).  Items are dealt to threads round-robin. */
int oracle_perm_batch(int64_t batch, const double *mats, const int64_t *mat_off, const int *k,
                      const int *l, const int *rm, const int64_t *roff, const int *cm,
                      const int64_t *coff, int gold, int nthreads, double *out)
{
    batch_job jobs[256];
    pthread_t th[256];
    int i, started = 0;
    if (batch < 0 || out == NULL)
        return ORC_ERR_ARG;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    for (i = 0; i < nthreads; i++) {
        jobs[i].batch = batch;
        jobs[i].mats = mats;
        jobs[i].mat_off = mat_off;
        jobs[i].k = k;
        jobs[i].l = l;
        jobs[i].rm = rm;
        jobs[i].cm = cm;
        jobs[i].roff = roff;
        jobs[i].coff = coff;
        jobs[i].gold = gold;
        jobs[i].lo = i;
        jobs[i].stride = nthreads;
        jobs[i].out = out;
    }
    for (i = 0; i < nthreads; i++) {
        if (pthread_create(&th[i], NULL, batch_worker, &jobs[i]) != 0)
            break;
        started++;
    }
    for (i = started; i < nthreads; i++)
        batch_worker(&jobs[i]);
    for (i = 0; i < started; i++)
        pthread_join(th[i], NULL);
    for (i = 0; i < nthreads; i++)
        if (jobs[i].rc != ORC_OK)
            return jobs[i].rc;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* boson sampling, Eq. (BS_prob)                                             */
/* ------------------------------------------------------------------------ */

/* Submatrix U_{s,t}: rows are the output modes i with t_i > 0 (row i of U is
 * output mode i, U[out][in]), repeated t_i times; columns are the input modes
 * j with s_j > 0, repeated s_j times.  Returns the number of base rows/cols. */
static void bs_gather(const double *U, int m, const int *s, const int *t, double *B, int *r,
                      int *c, int *kk, int *ll)
{
    int i, j, k = 0, l = 0;
    int cols[64];
    for (j = 0; j < m; j++)
        if (s[j] > 0) {
            cols[l] = j;
            c[l] = s[j];
            l++;
        }
    for (i = 0; i < m; i++) {
        if (t[i] <= 0)
            continue;
        r[k] = t[i];
        for (j = 0; j < l; j++) {
            B[2 * (k * l + j)] = U[2 * (i * m + cols[j])];
            B[2 * (k * l + j) + 1] = U[2 * (i * m + cols[j]) + 1];
        }
        k++;
    }
    *kk = k;
    *ll = l;
}

typedef struct {
    const double *U;
    int m;
    const int *s, *t;
    int64_t B;
    int gold;
    int64_t lo, stride;
    double *probs, *amps;
    int rc;
} bs_job;

static void *bs_worker(void *arg)
{
    bs_job *jb = (bs_job *)arg;
    int64_t b;
    double *Bm = (double *)malloc(sizeof(double) * 2 * 64 * 64);
    jb->rc = ORC_OK;
    if (Bm == NULL) {
        jb->rc = ORC_ERR_NOMEM;
        return NULL;
    }
    for (b = jb->lo; b < jb->B; b += jb->stride) {
        int r[64], c[64], k, l, i, rc;
        double o[4], norm = 1.0;
        const int *t = jb->t + b * jb->m;
        bs_gather(jb->U, jb->m, jb->s, t, Bm, r, c, &k, &l);
        rc = oracle_perm_ryser(Bm, k, l, r, c, jb->gold, 1, o);
        if (rc != ORC_OK) {
            jb->rc = rc;
            break;
        }
        for (i = 0; i < jb->m; i++)
            norm *= factorial(t[i]) * factorial(jb->s[i]);
        jb->probs[b] = (o[0] * o[0] + o[1] * o[1]) / norm;
        if (jb->amps) {
            jb->amps[2 * b] = o[0];
            jb->amps[2 * b + 1] = o[1];
        }
    }
    free(Bm);
    return NULL;
}

/* U: m x m complex (row-major, U[out][in]); s: m input occupations;
 * t: B x m output occupations.  probs[B]; amps (nullable) B complex = per(U_{s,t}). */
int oracle_bs_probs(const double *U, int m, const int *s, const int *t, int64_t B, int gold,
                    int nthreads, double *probs, double *amps)
{
    bs_job jobs[256];
    pthread_t th[256];
    int i, started = 0, ns = 0;
    int64_t b;
    if (U == NULL || s == NULL || (B > 0 && t == NULL) || probs == NULL || m <= 0 || m > 64 ||
        B < 0)
        return ORC_ERR_ARG;
    for (i = 0; i < m; i++) {
        if (s[i] < 0)
            return ORC_ERR_ARG;
        ns += s[i];
    }
    for (b = 0; b < B; b++) {
        int nt = 0;
        for (i = 0; i < m; i++) {
            if (t[b * m + i] < 0)
                return ORC_ERR_ARG;
            nt += t[b * m + i];
        }
        if (nt != ns)
            return ORC_ERR_ARG;
    }
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > 256)
        nthreads = 256;
    for (i = 0; i < nthreads; i++) {
        jobs[i].U = U;
        jobs[i].m = m;
        jobs[i].s = s;
        jobs[i].t = t;
        jobs[i].B = B;
        jobs[i].gold = gold;
        jobs[i].lo = i;
        jobs[i].stride = nthreads;
        jobs[i].probs = probs;
        jobs[i].amps = amps;
    }
    for (i = 0; i < nthreads; i++) {
        if (pthread_create(&th[i], NULL, bs_worker, &jobs[i]) != 0)
            break;
        started++;
    }
    for (i = started; i < nthreads; i++)
        bs_worker(&jobs[i]);
    for (i = 0; i < started; i++)
        pthread_join(th[i], NULL);
    for (i = 0; i < nthreads; i++)
        if (jobs[i].rc != ORC_OK)
            return jobs[i].rc;
    return ORC_OK;
}

/* Gradient of L = sum_b g_b p_b with respect to U, in the convention
 * grad = dL/dRe U + i dL/dIm U.  With P_b = per(U_{s,t_b}) and
 * N_b = prod t! prod s!:  dL/dP_b (same convention) = g_b * 2 P_b / N_b, and
 * for the holomorphic P_b, grad_U[a][c] = sum_b dL/dP_b * conj(dP_b/dU_ac),
 * where dP_b/dU_ac is the Laplace-minor derivative of the base entry that U_ac
 * becomes (zero if mode a is empty in t_b or mode c is empty in s).
 * Patterns are added in index order. */
int oracle_bs_grad_U(const double *U, int m, const int *s, const int *t, int64_t B,
                     const double *grad_probs, int gold, double *grad_U)
{
    int64_t b;
    int i, j;
    double *Bm, *G;
    if (U == NULL || s == NULL || t == NULL || grad_probs == NULL || grad_U == NULL || m <= 0 ||
        m > 64)
        return ORC_ERR_ARG;
    Bm = (double *)malloc(sizeof(double) * 2 * 64 * 64);
    G = (double *)malloc(sizeof(double) * 2 * 64 * 64);
    if (Bm == NULL || G == NULL) {
        free(Bm);
        free(G);
        return ORC_ERR_NOMEM;
    }
    for (i = 0; i < 2 * m * m; i++)
        grad_U[i] = 0.0;
    for (b = 0; b < B; b++) {
        int r[64], c[64], rows[64], cols[64], k = 0, l = 0, rc;
        double o[4], norm = 1.0, gre, gim;
        const int *tb = t + b * m;
        bs_gather(U, m, s, tb, Bm, r, c, &k, &l);
        k = 0;
        for (i = 0; i < m; i++)
            if (tb[i] > 0)
                rows[k++] = i;
        l = 0;
        for (j = 0; j < m; j++)
            if (s[j] > 0)
                cols[l++] = j;
        rc = oracle_perm_ryser(Bm, k, l, r, c, gold, 1, o);
        if (rc != ORC_OK) {
            free(Bm);
            free(G);
            return rc;
        }
        rc = oracle_perm_grad(Bm, k, l, r, c, gold, 1, G);
        if (rc != ORC_OK) {
            free(Bm);
            free(G);
            return rc;
        }
        for (i = 0; i < m; i++)
            norm *= factorial(tb[i]) * factorial(s[i]);
        /* dL/dP = g * 2 P / N */
        gre = grad_probs[b] * 2.0 * o[0] / norm;
        gim = grad_probs[b] * 2.0 * o[1] / norm;
        for (i = 0; i < k; i++) {
            for (j = 0; j < l; j++) {
                double dre = G[2 * (i * l + j)], dim = G[2 * (i * l + j) + 1];
                /* (gre + i gim) * conj(dre + i dim) */
                grad_U[2 * (rows[i] * m + cols[j])] += gre * dre + gim * dim;
                grad_U[2 * (rows[i] * m + cols[j]) + 1] += gim * dre - gre * dim;
            }
        }
    }
    free(Bm);
    free(G);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* hafnian, Eq. (haf_def)                                                    */
/* ------------------------------------------------------------------------ */

/* Sum over perfect matchings: the lowest unmatched index is paired with every
 * later unmatched one in turn (each matching is visited once). */
static void haf_rec(const double *a, int N, int *used, cd_t prod, dd_t *acc_re, dd_t *acc_im,
                    double *sumabs)
{
    int p = 0, q;
    while (p < N && used[p])
        p++;
    if (p == N) {
        *acc_re = dd_add(*acc_re, dd_from(prod.re));
        *acc_im = dd_add(*acc_im, dd_from(prod.im));
        *sumabs += hypot(prod.re, prod.im);
        return;
    }
    used[p] = 1;
    for (q = p + 1; q < N; q++) {
        cd_t x, np;
        if (used[q])
            continue;
        used[q] = 1;
        x.re = a[2 * (p * N + q)];
        x.im = a[2 * (p * N + q) + 1];
        np = cd_mul(prod, x);
        haf_rec(a, N, used, np, acc_re, acc_im, sumabs);
        used[q] = 0;
    }
    used[p] = 0;
}

/* a: N x N complex symmetric (only the upper triangle is read), N even,
 * N <= 16.  out[0..1] = haf(a), out[2] = sum |term|.  haf of size 0 is 1. */
int oracle_haf_bruteforce(const double *a, int N, double *out)
{
    int used[16] = {0};
    dd_t re = dd_from(0.0), im = dd_from(0.0);
    double sumabs = 0.0;
    cd_t one = {1.0, 0.0};
    if (N < 0 || N > 16 || (N & 1) || out == NULL || (N > 0 && a == NULL))
        return ORC_ERR_ARG;
    haf_rec(a, N, used, one, &re, &im, &sumabs);
    out[0] = re.hi + re.lo;
    out[1] = im.hi + im.lo;
    out[2] = sumabs;
    return ORC_OK;
}

/* Hafnian of the matrix that repeats base index i r_i times (rows and
 * columns), N = sum r even, by the grouped sign-vector formula
 *   haf = 1 / (n! 2^{N-1}) sum_g (-1)^{sum g} C(r_f - 1, g_f) prod_{i != f} C(r_i, g_i) q(g)^n,
 *   q(g) = 1/2 (x^T B x - sum_i r_i B_ii),  x_i = r_i - 2 g_i,  n = N / 2,
 * with g_f in [0, r_f - 1] for the first index f with r_f > 0 (one copy's sign
 * fixed), every q evaluated from scratch in double-double, every term added
 * in double-double.  It follows from Eq. (haf_def): the mean over all sign
 * vectors d of (prod d) (sum_{p<q} A_pq d_p d_q)^n is n! haf(A), and the
 * vectors that put g_i minus signs on the copies of index i all give the same
 * x.  b: k x k complex symmetric.  out[0..1] = haf, out[2] = sum |term| / (n! 2^{N-1}). */
int oracle_haf_grouped(const double *b, int k, const int *r, double *out)
{
    int i, j, N = 0, f = -1, kd[64];
    int64_t T = 1, rank;
    dd_t acc_re = dd_from(0.0), acc_im = dd_from(0.0);
    double sumabs = 0.0, scale;
    cd_t dsum;
    if (k < 0 || k > 64 || out == NULL || (k > 0 && (b == NULL || r == NULL)))
        return ORC_ERR_ARG;
    for (i = 0; i < k; i++) {
        if (r[i] < 0)
            return ORC_ERR_ARG;
        N += r[i];
        if (f < 0 && r[i] > 0)
            f = i;
    }
    if (N & 1) {
        out[0] = out[1] = out[2] = 0.0;
        return ORC_OK;
    }
    if (N == 0) {
        out[0] = 1.0;
        out[1] = 0.0;
        out[2] = 1.0;
        return ORC_OK;
    }
    if (N > 62)
        return ORC_ERR_TOO_LARGE;
    for (i = 0; i < k; i++) {
        int64_t rad = (i == f) ? r[i] : r[i] + 1;
        if (T > ((int64_t)1 << 62) / rad)
            return ORC_ERR_TOO_LARGE;
        T *= rad;
    }
    /* sum_i r_i B_ii */
    dsum.re = 0.0;
    dsum.im = 0.0;
    for (i = 0; i < k; i++) {
        dsum.re += r[i] * b[2 * (i * k + i)];
        dsum.im += r[i] * b[2 * (i * k + i) + 1];
    }
    for (rank = 0; rank < T; rank++) {
        int64_t rem = rank;
        int gsum = 0;
        double w = 1.0;
        cdd_t xbx, q, p;
        for (i = 0; i < k; i++) {
            int rad = (i == f) ? r[i] : r[i] + 1;
            kd[i] = (int)(rem % rad);
            rem /= rad;
            gsum += kd[i];
            w *= (i == f) ? binom(r[i] - 1, kd[i]) : binom(r[i], kd[i]);
        }
        if (gsum & 1)
            w = -w;
        /* x^T B x in double-double */
        xbx.re = dd_from(0.0);
        xbx.im = dd_from(0.0);
        for (i = 0; i < k; i++) {
            double xi = (double)(r[i] - 2 * kd[i]);
            for (j = 0; j < k; j++) {
                dd_t c = dd_from(xi * (double)(r[j] - 2 * kd[j])); /* exact small integer */
                xbx.re = dd_add(xbx.re, dd_mul(c, dd_from(b[2 * (i * k + j)])));
                xbx.im = dd_add(xbx.im, dd_mul(c, dd_from(b[2 * (i * k + j) + 1])));
            }
        }
        q.re = dd_mul(dd_add(xbx.re, dd_from(-dsum.re)), dd_from(0.5));
        q.im = dd_mul(dd_add(xbx.im, dd_from(-dsum.im)), dd_from(0.5));
        /* q^n by repeated multiplication */
        p = q;
        for (j = 1; j < N / 2; j++)
            p = cdd_mul(p, q);
        p.re = dd_mul(p.re, dd_from(w));
        p.im = dd_mul(p.im, dd_from(w));
        acc_re = dd_add(acc_re, p.re);
        acc_im = dd_add(acc_im, p.im);
        sumabs += hypot(p.re.hi, p.im.hi);
    }
    scale = ldexp(1.0, -(N - 1)) / factorial(N / 2);
    out[0] = (acc_re.hi + acc_re.lo) * scale;
    out[1] = (acc_im.hi + acc_im.lo) * scale;
    out[2] = sumabs * scale;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* loop hafnian, Eq. (loop_hafnian)                                          */
/* ------------------------------------------------------------------------ */

/* Sum over matchings with loops: the lowest unused index either takes its
 * loop (weight a_pp) or is paired with every later unused index in turn. */
static void lhaf_rec(const double *a, int N, int *used, cd_t prod, dd_t *acc_re, dd_t *acc_im,
                     double *sumabs)
{
    int p = 0, q;
    cd_t x, np;
    while (p < N && used[p])
        p++;
    if (p == N) {
        *acc_re = dd_add(*acc_re, dd_from(prod.re));
        *acc_im = dd_add(*acc_im, dd_from(prod.im));
        *sumabs += hypot(prod.re, prod.im);
        return;
    }
    used[p] = 1;
    x.re = a[2 * (p * N + p)];
    x.im = a[2 * (p * N + p) + 1];
    np = cd_mul(prod, x);
    lhaf_rec(a, N, used, np, acc_re, acc_im, sumabs);
    for (q = p + 1; q < N; q++) {
        if (used[q])
            continue;
        used[q] = 1;
        x.re = a[2 * (p * N + q)];
        x.im = a[2 * (p * N + q) + 1];
        np = cd_mul(prod, x);
        lhaf_rec(a, N, used, np, acc_re, acc_im, sumabs);
        used[q] = 0;
    }
    used[p] = 0;
}

/* a: N x N complex symmetric (upper triangle and diagonal read), N <= 14, any
 * parity.  out[0..1] = lhaf(a), out[2] = sum |term|.  Size 0 gives 1. */
int oracle_lhaf_bruteforce(const double *a, int N, double *out)
{
    int used[16] = {0};
    dd_t re = dd_from(0.0), im = dd_from(0.0);
    double sumabs = 0.0;
    cd_t one = {1.0, 0.0};
    if (N < 0 || N > 14 || out == NULL || (N > 0 && a == NULL))
        return ORC_ERR_ARG;
    lhaf_rec(a, N, used, one, &re, &im, &sumabs);
    out[0] = re.hi + re.lo;
    out[1] = im.hi + im.lo;
    out[2] = sumabs;
    return ORC_OK;
}

/* Loop hafnian of filldiag(A_r, gamma_r): base index i repeated r_i times in
 * rows and columns of the k x k symmetric b, the loop weight of every copy of
 * i being gamma_i (Eq. (loop_hafnian) with the filldiag of the displaced
 * detection probability).  Grouped sign-vector formula
 *   lhaf = 1 / 2^{N-1} sum_g (-1)^{sum g} C(r_f - 1, g_f) prod_{i != f} C(r_i, g_i)
 *            sum_{j=0}^{N/2} q(g)^j l(g)^{N-2j} / (j! (N-2j)!),
 *   q(g) = 1/2 (x^T b x - sum_i r_i b_ii),  l(g) = gamma^T x,  x_i = r_i - 2 g_i:
 * the coefficient of the product of all N signs in exp(q + l) counts every
 * matching with loops once, the mean over sign vectors extracts it, and the
 * summand is even under flipping every sign, so one copy's sign is fixed.
 * Every q, l and term from scratch in double-double.
 * out[0..1] = lhaf, out[2] = sum |term| / 2^{N-1}. */
int oracle_lhaf_grouped(const double *b, const double *gamma, int k, const int *r, double *out)
{
    int i, j, N = 0, f = -1, kd[64];
    int64_t T = 1, rank;
    dd_t acc_re = dd_from(0.0), acc_im = dd_from(0.0);
    double sumabs = 0.0, scale;
    cd_t dsum;
    if (k < 0 || k > 64 || out == NULL || (k > 0 && (b == NULL || r == NULL || gamma == NULL)))
        return ORC_ERR_ARG;
    for (i = 0; i < k; i++) {
        if (r[i] < 0)
            return ORC_ERR_ARG;
        N += r[i];
        if (f < 0 && r[i] > 0)
            f = i;
    }
    if (N == 0) {
        out[0] = 1.0;
        out[1] = 0.0;
        out[2] = 1.0;
        return ORC_OK;
    }
    if (N > 62)
        return ORC_ERR_TOO_LARGE;
    for (i = 0; i < k; i++) {
        int64_t rad = (i == f) ? r[i] : r[i] + 1;
        if (rad < 1)
            rad = 1;
        if (T > ((int64_t)1 << 62) / rad)
            return ORC_ERR_TOO_LARGE;
        T *= rad;
    }
    dsum.re = 0.0;
    dsum.im = 0.0;
    for (i = 0; i < k; i++) {
        dsum.re += r[i] * b[2 * (i * k + i)];
        dsum.im += r[i] * b[2 * (i * k + i) + 1];
    }
    for (rank = 0; rank < T; rank++) {
        int64_t rem = rank;
        int gsum = 0;
        double w = 1.0;
        cdd_t xbx, q, l, term, qp;
        for (i = 0; i < k; i++) {
            int rad = (i == f) ? r[i] : r[i] + 1;
            if (rad < 1)
                rad = 1;
            kd[i] = (int)(rem % rad);
            rem /= rad;
            gsum += kd[i];
            w *= (i == f) ? binom(r[i] - 1, kd[i]) : binom(r[i], kd[i]);
        }
        if (gsum & 1)
            w = -w;
        xbx.re = dd_from(0.0);
        xbx.im = dd_from(0.0);
        l.re = dd_from(0.0);
        l.im = dd_from(0.0);
        for (i = 0; i < k; i++) {
            double xi = (double)(r[i] - 2 * kd[i]);
            l.re = dd_add(l.re, dd_mul(dd_from(xi), dd_from(gamma[2 * i])));
            l.im = dd_add(l.im, dd_mul(dd_from(xi), dd_from(gamma[2 * i + 1])));
            for (j = 0; j < k; j++) {
                dd_t c = dd_from(xi * (double)(r[j] - 2 * kd[j]));
                xbx.re = dd_add(xbx.re, dd_mul(c, dd_from(b[2 * (i * k + j)])));
                xbx.im = dd_add(xbx.im, dd_mul(c, dd_from(b[2 * (i * k + j) + 1])));
            }
        }
        q.re = dd_mul(dd_add(xbx.re, dd_from(-dsum.re)), dd_from(0.5));
        q.im = dd_mul(dd_add(xbx.im, dd_from(-dsum.im)), dd_from(0.5));
        /* sum_j q^j l^{N-2j} / (j! (N-2j)!) */
        term.re = dd_from(0.0);
        term.im = dd_from(0.0);
        qp.re = dd_from(1.0);
        qp.im = dd_from(0.0);
        for (j = 0; 2 * j <= N; j++) {
            cdd_t lp, t;
            int e;
            lp.re = dd_from(1.0);
            lp.im = dd_from(0.0);
            for (e = 0; e < N - 2 * j; e++)
                lp = cdd_mul(lp, l);
            t = cdd_mul(qp, lp);
            t.re = dd_mul(t.re, dd_from(1.0 / (factorial(j) * factorial(N - 2 * j))));
            t.im = dd_mul(t.im, dd_from(1.0 / (factorial(j) * factorial(N - 2 * j))));
            term.re = dd_add(term.re, t.re);
            term.im = dd_add(term.im, t.im);
            qp = cdd_mul(qp, q);
        }
        term.re = dd_mul(term.re, dd_from(w));
        term.im = dd_mul(term.im, dd_from(w));
        acc_re = dd_add(acc_re, term.re);
        acc_im = dd_add(acc_im, term.im);
        sumabs += hypot(term.re.hi, term.im.hi);
    }
    scale = ldexp(1.0, -(N - 1));
    out[0] = (acc_re.hi + acc_re.lo) * scale;
    out[1] = (acc_im.hi + acc_im.lo) * scale;
    out[2] = sumabs * scale;
    return ORC_OK;
}
