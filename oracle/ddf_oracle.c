/*
 * DDF oracle: a plain, sequential, FP64 CPU implementation of what the GPU
 * path computes.  TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and
 * the benchmark's CPU-baseline / reference arm may load this library.  It
 * shares no code with the CUDA path.  Compiled with -O2 -ffp-contract=off so
 * that every product and sum is rounded separately, in CSR order.
 *
 * Contents (paper: "Vectorizing Sparse Matrix Codes with Dependency Driven
 * Trace Analysis", Cetinic, Cheshmi, Dehnavi):
 *   ora_spmv_csr        y = A x in CSR order            (Fig. 1a; Sec. V baseline)
 *   ora_spmv_csr_par    the same rows split over host threads (each row
 *                       still summed in CSR order, so y is bit-identical)
 *   ora_sptrsv_csr      forward substitution L x = b     (Sec. V baseline)
 *   ora_levels          longest-path levels of G         (Sec. IV-A, findDependencies)
 *   ora_level_order     rows ordered by (level, row)     (Sec. IV-A, partitionIterationSpace)
 *   ora_coarse_order    coarsened partitions: (block of R rows, level)  (Sec. IV-A, LBC; R14)
 *   ora_check_schedule  every dependency in an earlier partition (Sec. IV-A)
 *   ora_inspect         Algorithm 1 (DDF inspector)      (Sec. IV-A, Alg. 1, Sec. III-C/D)
 *   ora_check_plan      plan expansion == CSR trace       (Sec. III-A definitions)
 *   ora_codelet_cost    Eq. 1 with weights               (Sec. III-C, Eq. 1)
 *
 * Readings of the paper that this file follows (each is listed with its
 * justification in the design notes):
 *   R1  A codelet covers whole rows: rows q0..q0+m-1 of one partition's
 *       sequence (i0 = row inside the codelet, i1 = position inside the row).
 *   R2  f(i0) is the row (y / x index), g(i0,i1) the value offset, h(i0,i1)
 *       the column (x index).  A function is strided when all its first order
 *       partial differences along i0 are equal and all along i1 are equal
 *       (Sec. III-D); runs of one row have no i0 differences.
 *   R3  Types by form: BLAS = f,g,h strided; PSC I = f,g strided and
 *       h(i0,i1) = h0 + delta*i0 + s[i1] with one offset array s for all rows
 *       (the form of the paper's PSC I example, Sec. III-C); PSC II = any
 *       other run, executed with a per-nonzero offset array for h.
 *   R4  Eq. 1 as c = w_op*|p| + w_cl + w_idx*(|s_f|+|s_g|+|s_h|) with
 *       |s_d| = 0 for a strided function, m rows for a non-strided f or g,
 *       n for PSC I's h and |p| for PSC II's h.  Weights (1,3,1) give the
 *       paper's form (m = 3 access functions).
 *   R5  SpMV has no dependencies: one partition holding every row.  SpTRSV
 *       partitions are the level sets of G, rows in increasing order inside a
 *       level; its iteration points are the off-diagonal entries (the
 *       diagonal, stored last in each row, is the divide after the codelet),
 *       and g addresses a copy of the off-diagonal values laid out in that
 *       level order.
 *   R6  Regions are windows of t consecutive positions of a partition.
 *   R14 Coarsened partitions (the paper partitions SpTRSV with LBC, Sec. IV-A):
 *       rows are cut into blocks of R consecutive rows; the partitions are the
 *       non-empty (block, level) pairs in increasing block then level order,
 *       rows increasing inside one.  R = 0 gives the plain level sets (R5).
 *   R7  Strategies: BLAS_first takes maximal BLAS runs from every row whose
 *       own columns are evenly spaced, then maximal PSC I runs of >= 2 rows in
 *       the gaps, then PSC II runs of what is left; PSCI_first takes maximal
 *       runs of >= 2 rows with f,g strided and a shared s (typed BLAS when h is
 *       also strided), then PSC II runs; PSCII_first makes the region one
 *       PSC II codelet.  min_cost keeps the cheapest; ties prefer BLAS_first,
 *       then PSCI_first.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORA_OK = 0, ORA_ERR_ARG = 1, ORA_ERR_NOT_LOWER = 5, ORA_ERR_MISSING_DIAG = 6,
       ORA_ERR_ZERO_DIAG = 7, ORA_ERR_OOM = 9 };
enum { ORA_SPMV = 1, ORA_SPTRSV = 2 };
enum { T_BLAS = 0, T_PSC1 = 1, T_PSC2 = 2 };
enum { ALLOW_BLAS = 1, ALLOW_PSC1 = 2, ALLOW_PSC2 = 4 };

/* Canonical codelet record (12 x int64), the same layout the GPU plan export
 * uses: part, type, q0, m, n, f_str, rho, g_str, gamma, h0, delta, sigma. */
#define NF 12

/* ------------------------------------------------------------------------ */
/* Executors' definitions                                                     */
/* ------------------------------------------------------------------------ */

/* y_i = sum_{k=Ap[i]}^{Ap[i+1]-1} Ax[k] * x[Ai[k]]  (Fig. 1a) */
int ora_spmv_csr(int32_t n, const int32_t* Ap, const int32_t* Ai, const double* Ax,
                 const double* x, double* y) {
    for (int32_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = Ap[i]; k < Ap[i + 1]; ++k) s += Ax[k] * x[Ai[k]];
        y[i] = s;
    }
    return ORA_OK;
}

/* Row-parallel SpMV: thread t takes the rows whose entries start in the t-th
 * of T equal shares of the nonzeros, and computes each of them exactly as
 * ora_spmv_csr does.  The multi-core CPU baseline; y equals the sequential
 * result bit for bit. */
typedef struct {
    int32_t r0, r1;
    const int32_t *Ap, *Ai;
    const double *Ax, *x;
    double* y;
} spmv_job;

static void* spmv_rows(void* arg) {
    const spmv_job* j = (const spmv_job*)arg;
    for (int32_t i = j->r0; i < j->r1; ++i) {
        double s = 0.0;
        for (int32_t k = j->Ap[i]; k < j->Ap[i + 1]; ++k) s += j->Ax[k] * j->x[j->Ai[k]];
        j->y[i] = s;
    }
    return NULL;
}

/* first row i in [0, n] with Ap[i] >= target */
static int32_t first_row_at(int32_t n, const int32_t* Ap, int64_t target) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if ((int64_t)Ap[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

int ora_spmv_csr_par(int32_t n, const int32_t* Ap, const int32_t* Ai, const double* Ax,
                     const double* x, double* y, int32_t nthreads) {
    if (nthreads < 1 || nthreads > 1024) return ORA_ERR_ARG;
    spmv_job* jobs = (spmv_job*)malloc(sizeof(spmv_job) * (size_t)nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return ORA_ERR_OOM;
    }
    const int64_t nnz = n > 0 ? Ap[n] : 0;
    for (int32_t t = 0; t < nthreads; ++t) {
        jobs[t].r0 = t == 0 ? 0 : first_row_at(n, Ap, nnz * t / nthreads);
        jobs[t].r1 = t == nthreads - 1 ? n : first_row_at(n, Ap, nnz * (t + 1) / nthreads);
        jobs[t].Ap = Ap;
        jobs[t].Ai = Ai;
        jobs[t].Ax = Ax;
        jobs[t].x = x;
        jobs[t].y = y;
    }
    int32_t started = 0;
    for (int32_t t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, spmv_rows, &jobs[t]) != 0) break;
        started = t;
    }
    spmv_rows(&jobs[0]);
    /* threads that could not be started run here, in order */
    for (int32_t t = started + 1; t < nthreads; ++t) spmv_rows(&jobs[t]);
    for (int32_t t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
    return ORA_OK;
}

/* Forward substitution on a lower triangle with the diagonal:
 * x_i = (b_i - sum_{j<i} L_ij x_j) / L_ii. */
int ora_sptrsv_csr(int32_t n, const int32_t* Lp, const int32_t* Li, const double* Lx,
                   const double* b, double* x) {
    for (int32_t i = 0; i < n; ++i) {
        double s = b[i], d = 0.0;
        int found = 0;
        for (int32_t k = Lp[i]; k < Lp[i + 1]; ++k) {
            int32_t j = Li[k];
            if (j < i) s -= Lx[k] * x[j];
            else if (j == i) { d = Lx[k]; found = 1; }
            else return ORA_ERR_NOT_LOWER;
        }
        if (!found) return ORA_ERR_MISSING_DIAG;
        if (d == 0.0) return ORA_ERR_ZERO_DIAG;
        x[i] = s / d;
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* findDependencies / partitionIterationSpace for SpTRSV                      */
/* ------------------------------------------------------------------------ */

/* Vertices are rows; an edge j -> i exists when L_ij != 0 with j < i.  The
 * level of i is the length of the longest path ending at i (0 without
 * incoming edges).  Returns the depth (number of levels), or -1 on a column
 * above the diagonal. */
int32_t ora_levels(int32_t n, const int32_t* Lp, const int32_t* Li, int32_t* lev) {
    int32_t depth = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t l = 0;
        for (int32_t k = Lp[i]; k < Lp[i + 1]; ++k) {
            int32_t j = Li[k];
            if (j > i) return -1;
            if (j < i && lev[j] + 1 > l) l = lev[j] + 1;
        }
        lev[i] = l;
        if (l + 1 > depth) depth = l + 1;
    }
    return depth;
}

/* Rows ordered by (level, row): level_ptr[l] = first position of level l. */
int ora_level_order(int32_t n, const int32_t* lev, int32_t depth, int32_t* level_ptr,
                    int32_t* perm) {
    for (int32_t l = 0; l <= depth; ++l) level_ptr[l] = 0;
    for (int32_t i = 0; i < n; ++i) level_ptr[lev[i] + 1]++;
    for (int32_t l = 0; l < depth; ++l) level_ptr[l + 1] += level_ptr[l];
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(depth > 0 ? depth : 1));
    if (!fill) return ORA_ERR_OOM;
    for (int32_t l = 0; l < depth; ++l) fill[l] = level_ptr[l];
    for (int32_t i = 0; i < n; ++i) perm[fill[lev[i]]++] = i;
    free(fill);
    return ORA_OK;
}

/* Coarsened order (R14): rows sorted by (row / R, level, row); a partition
 * starts wherever the block or the level changes.  part_ptr needs n + 1
 * entries; the number of partitions is stored in *nparts. */
int ora_coarse_order(int32_t n, const int32_t* lev, int32_t depth, int32_t R, int32_t* part_ptr,
                     int32_t* perm, int32_t* nparts) {
    if (R < 1) return ORA_ERR_ARG;
    int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(depth + 1));
    if (!cnt) return ORA_ERR_OOM;
    int32_t np = 0, q = 0;
    for (int64_t b0 = 0; b0 < n; b0 += R) {             /* each block, in order */
        int32_t b1 = (int32_t)(b0 + R < n ? b0 + R : n);
        for (int32_t l = 0; l <= depth; ++l) cnt[l] = 0;
        for (int32_t i = (int32_t)b0; i < b1; ++i) cnt[lev[i] + 1]++;
        for (int32_t l = 0; l < depth; ++l) cnt[l + 1] += cnt[l];
        for (int32_t l = 0; l < depth; ++l)              /* non-empty levels of the block */
            if (cnt[l + 1] > cnt[l]) part_ptr[np++] = q + cnt[l];
        for (int32_t i = (int32_t)b0; i < b1; ++i) perm[q + cnt[lev[i]]++] = i;
        q = b1;
    }
    part_ptr[np] = n;
    *nparts = np;
    free(cnt);
    return ORA_OK;
}

/* Schedule check: every off-diagonal dependency j of row i (L_ij != 0, j < i)
 * sits in a partition strictly before the partition of i.  Returns 0, or 1
 * with the offending row in *bad, or 2 when perm / part_ptr are malformed. */
int ora_check_schedule(int32_t n, const int32_t* Lp, const int32_t* Li, const int32_t* perm,
                       const int32_t* part_ptr, int32_t nparts, int32_t* bad) {
    *bad = -1;
    int32_t* part = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!part) return 99;
    for (int32_t i = 0; i < n; ++i) part[i] = -1;
    int rc = 0;
    if (nparts < 0 || part_ptr[0] != 0 || part_ptr[nparts] != n) rc = 2;
    for (int32_t p = 0; p < nparts && !rc; ++p) {
        if (part_ptr[p + 1] <= part_ptr[p]) { rc = 2; break; }
        for (int32_t q = part_ptr[p]; q < part_ptr[p + 1]; ++q) {
            int32_t r = perm[q];
            if (r < 0 || r >= n || part[r] >= 0) { rc = 2; break; }
            part[r] = p;
        }
    }
    for (int32_t i = 0; i < n && !rc; ++i)
        for (int32_t k = Lp[i]; k < Lp[i + 1]; ++k) {
            int32_t j = Li[k];
            if (j < i && part[j] >= part[i]) { rc = 1; *bad = i; break; }
        }
    free(part);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1                                                                       */
/* ------------------------------------------------------------------------ */

/* c_l = w_op*|p| + w_cl + w_idx * sum_d |s_d|   (R4) */
int64_t ora_codelet_cost(int64_t p, int64_t s_f, int64_t s_g, int64_t s_h, int64_t w_op,
                         int64_t w_cl, int64_t w_idx) {
    return w_op * p + w_cl + w_idx * (s_f + s_g + s_h);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                                 */
/* ------------------------------------------------------------------------ */

/* The access functions of one position q of the partition sequence:
 *   f(q)      = seq[q]                         (row)
 *   g(q, i1)  = gs[q] + i1                     (value offset)
 *   h(q, i1)  = Ai[cs[q] + i1], 0 <= i1 < len[q]  (column)            */
typedef struct {
    int32_t nseq;
    const int32_t* seq;
    const int64_t* gs;
    const int64_t* cs;
    const int32_t* len;
    const int32_t* Ai;
} afun;

/* First order partial differences (Sec. III-D) kept per position:
 *   hstr[q], sigma[q]  all Delta_i1 h of row q equal (value sigma)
 *   dF[q]              Delta_i0 f between q-1 and q
 *   dG[q], eqlen[q]    Delta_i0 g and whether the rows have equal length
 *   trans[q], dH[q]    all Delta_i0 h between q-1 and q equal (value dH)  */
typedef struct {
    uint8_t *hstr, *eqlen, *trans;
    int64_t *sigma, *dF, *dG, *dH;
} fopd;

static void compute_fopd(const afun* a, int32_t q_begin, int32_t q_end, fopd* d) {
    for (int32_t q = q_begin; q < q_end; ++q) {
        int32_t L = a->len[q];
        const int32_t* h = a->Ai + a->cs[q];
        int ok = 1;
        int64_t s = 0;
        if (L >= 2) {
            s = (int64_t)h[1] - h[0];
            for (int32_t i1 = 1; i1 + 1 < L; ++i1)
                if ((int64_t)h[i1 + 1] - h[i1] != s) { ok = 0; break; }
        }
        d->hstr[q] = (uint8_t)ok;
        d->sigma[q] = s;
        if (q == q_begin) {
            d->dF[q] = d->dG[q] = d->dH[q] = 0;
            d->eqlen[q] = d->trans[q] = 0;
            continue;
        }
        d->dF[q] = (int64_t)a->seq[q] - a->seq[q - 1];
        d->dG[q] = a->gs[q] - a->gs[q - 1];
        d->eqlen[q] = (uint8_t)(L == a->len[q - 1]);
        d->trans[q] = 0;
        d->dH[q] = 0;
        if (L == a->len[q - 1]) {
            const int32_t* hp = a->Ai + a->cs[q - 1];
            int t = 1;
            int64_t dh = (L > 0) ? (int64_t)h[0] - hp[0] : 0;
            for (int32_t i1 = 1; i1 < L; ++i1)
                if ((int64_t)h[i1] - hp[i1] != dh) { t = 0; break; }
            d->trans[q] = (uint8_t)t;
            d->dH[q] = t ? dh : 0;
        }
    }
}

/* Does the run [q0, q1) keep f strided / g strided / h = h0 + delta*i0 + s[i1]? */
static int run_F(const fopd* d, int32_t q0, int32_t q1) {
    for (int32_t q = q0 + 2; q < q1; ++q) if (d->dF[q] != d->dF[q0 + 1]) return 0;
    return 1;
}
static int run_G(const fopd* d, int32_t q0, int32_t q1) {
    for (int32_t q = q0 + 1; q < q1; ++q) {
        if (!d->eqlen[q]) return 0;
        if (d->dG[q] != d->dG[q0 + 1]) return 0;
    }
    return 1;
}
/* Longest run [q0, q1) with q1 <= end on which f, g are strided and h has a
 * shared offset array (the PSC I form; a BLAS run when also hstr[q0]). */
static int32_t extend_psc1(const fopd* d, int32_t q0, int32_t end) {
    int32_t q1 = q0 + 1;
    if (q1 >= end || !d->eqlen[q1] || !d->trans[q1]) return q1;
    /* the first link fixes the strides; every later link must repeat them */
    int64_t rf = d->dF[q1], rg = d->dG[q1], rh = d->dH[q1];
    ++q1;
    while (q1 < end && d->eqlen[q1] && d->trans[q1] && d->dF[q1] == rf && d->dG[q1] == rg &&
           d->dH[q1] == rh)
        ++q1;
    return q1;
}

typedef struct { int32_t type, q0, q1; } piece;

typedef struct {
    piece* v;
    int32_t n;
} plist;

static void push(plist* l, int32_t type, int32_t q0, int32_t q1) {
    l->v[l->n].type = type;
    l->v[l->n].q0 = q0;
    l->v[l->n].q1 = q1;
    l->n++;
}

/* Cost of one piece under Eq. 1 (R4). */
static int64_t piece_cost(const afun* a, const fopd* d, const piece* c, const int64_t* w) {
    int32_t m = c->q1 - c->q0;
    int64_t p = 0;
    for (int32_t q = c->q0; q < c->q1; ++q) p += a->len[q];
    int64_t sf = 0, sg = 0, sh = 0;
    if (c->type == T_PSC1) sh = a->len[c->q0];
    if (c->type == T_PSC2) {
        sf = run_F(d, c->q0, c->q1) ? 0 : m;
        sg = run_G(d, c->q0, c->q1) ? 0 : m;
        sh = p;
    }
    return ora_codelet_cost(p, sf, sg, sh, w[0], w[1], w[2]);
}

/* Positions of [a, b) not covered by BLAS / PSC I pieces become maximal
 * PSC II runs. */
static void leftovers_to_psc2(const uint8_t* cov, int32_t a, int32_t b, plist* out) {
    int32_t q = a;
    while (q < b) {
        if (cov[q - a]) { ++q; continue; }
        int32_t u = q;
        while (q < b && !cov[q - a]) ++q;
        push(out, T_PSC2, u, q);
    }
}

static void blas_first(const fopd* d, int32_t a, int32_t b, int allowed, uint8_t* cov, plist* out) {
    memset(cov, 0, (size_t)(b - a));
    int32_t q = a;
    while (q < b) {                              /* maximal BLAS runs */
        if (d->hstr[q]) {
            int32_t q1 = extend_psc1(d, q, b);
            push(out, T_BLAS, q, q1);
            memset(cov + (q - a), 1, (size_t)(q1 - q));
            q = q1;
        } else {
            ++q;
        }
    }
    if (allowed & ALLOW_PSC1) {                  /* PSC I runs in the gaps */
        q = a;
        while (q < b) {
            if (cov[q - a]) { ++q; continue; }
            int32_t v = q;
            while (v < b && !cov[v - a]) ++v;
            int32_t u = q;
            while (u < v) {
                int32_t u1 = extend_psc1(d, u, v);
                if (u1 - u >= 2) {
                    push(out, T_PSC1, u, u1);
                    memset(cov + (u - a), 1, (size_t)(u1 - u));
                    u = u1;
                } else {
                    ++u;
                }
            }
            q = v;
        }
    }
    leftovers_to_psc2(cov, a, b, out);
}

static void psc1_first(const fopd* d, int32_t a, int32_t b, int allowed, uint8_t* cov, plist* out) {
    memset(cov, 0, (size_t)(b - a));
    int32_t q = a;
    while (q < b) {
        int32_t q1 = extend_psc1(d, q, b);
        if (q1 - q >= 2) {
            int t = (d->hstr[q] && (allowed & ALLOW_BLAS)) ? T_BLAS : T_PSC1;
            push(out, t, q, q1);
            memset(cov + (q - a), 1, (size_t)(q1 - q));
            q = q1;
        } else {
            ++q;
        }
    }
    leftovers_to_psc2(cov, a, b, out);
}

static int cmp_piece(const void* x, const void* y) {
    const piece* p = (const piece*)x;
    const piece* q = (const piece*)y;
    return (p->q0 > q->q0) - (p->q0 < q->q0);
}

static void emit(const afun* a, const fopd* d, int64_t part, const piece* c, int64_t* rec) {
    int32_t m = c->q1 - c->q0;
    int32_t q0 = c->q0;
    int F = run_F(d, q0, c->q1), G = run_G(d, q0, c->q1);
    rec[0] = part;
    rec[1] = c->type;
    rec[2] = q0;
    rec[3] = m;
    rec[4] = (c->type == T_PSC2) ? -1 : a->len[q0];
    rec[5] = F;
    rec[6] = (F && m >= 2) ? d->dF[q0 + 1] : 0;
    rec[7] = G;
    rec[8] = (G && m >= 2) ? d->dG[q0 + 1] : 0;
    rec[9] = (c->type != T_PSC2 && a->len[q0] >= 1) ? a->Ai[a->cs[q0]] : 0;
    rec[10] = (c->type != T_PSC2 && m >= 2) ? d->dH[q0 + 1] : 0;
    rec[11] = (c->type == T_BLAS && a->len[q0] >= 2) ? d->sigma[q0] : 0;
}

/*
 * Algorithm 1 for K in {SpMV, SpTRSV} on the CSR pattern (Ap, Ai).
 * Outputs (caller-allocated, sizes n / n+1):
 *   perm[n]          partition sequence (identity for SpMV, level order for SpTRSV,
 *                    (block, level) order for SpTRSV with coarsen = R > 0, R14)
 *   level_ptr[n+1]   partition boundaries; *nparts partitions
 *   gs[n]            start of each position's points in the executor's value array
 * and a malloc'd array of canonical records (*out, *ncod records of NF int64).
 * weights = {w_op, w_cl, w_idx}.
 */
int ora_inspect(int kind, int32_t n, const int32_t* Ap, const int32_t* Ai, int32_t t,
                int allowed, const int64_t* weights, int32_t coarsen, int32_t* perm,
                int32_t* level_ptr, int32_t* nparts, int64_t* gs, int64_t** out, int64_t* ncod) {
    if (n < 0 || t < 1 || !(allowed & ALLOW_PSC2) || coarsen < 0) return ORA_ERR_ARG;
    *out = NULL;
    *ncod = 0;
    int32_t* len = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t* lev = NULL;
    if (!len || !cs) return ORA_ERR_OOM;

    /* computeAccessFunctions, findDependencies and partitionIterationSpace */
    if (kind == ORA_SPMV) {
        for (int32_t i = 0; i < n; ++i) perm[i] = i;
        level_ptr[0] = 0;
        if (n > 0) level_ptr[1] = n;
        *nparts = (n > 0) ? 1 : 0;
        for (int32_t q = 0; q < n; ++q) {
            len[q] = Ap[q + 1] - Ap[q];
            cs[q] = Ap[q];
            gs[q] = Ap[q];
        }
    } else if (kind == ORA_SPTRSV) {
        lev = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        if (!lev) return ORA_ERR_OOM;
        for (int32_t i = 0; i < n; ++i) {
            if (Ap[i + 1] <= Ap[i] || Ai[Ap[i + 1] - 1] != i) {
                free(lev); free(len); free(cs);
                return ORA_ERR_MISSING_DIAG;
            }
        }
        int32_t depth = ora_levels(n, Ap, Ai, lev);
        if (depth < 0) { free(lev); free(len); free(cs); return ORA_ERR_NOT_LOWER; }
        int rc;
        if (coarsen > 0) {
            rc = ora_coarse_order(n, lev, depth, coarsen, level_ptr, perm, nparts);   /* R14 */
        } else {
            rc = ora_level_order(n, lev, depth, level_ptr, perm);
            *nparts = depth;
        }
        if (rc) { free(lev); free(len); free(cs); return rc; }
        int64_t acc = 0;
        for (int32_t q = 0; q < n; ++q) {
            int32_t r = perm[q];
            len[q] = Ap[r + 1] - Ap[r] - 1;     /* off-diagonal points (R5) */
            cs[q] = Ap[r];
            gs[q] = acc;                        /* level-ordered value copy */
            acc += len[q];
        }
    } else {
        free(len); free(cs);
        return ORA_ERR_ARG;
    }

    afun a = {n, perm, gs, cs, len, Ai};
    size_t nn = (size_t)(n > 0 ? n : 1);
    fopd d;
    d.hstr = (uint8_t*)malloc(nn);
    d.eqlen = (uint8_t*)malloc(nn);
    d.trans = (uint8_t*)malloc(nn);
    d.sigma = (int64_t*)malloc(8 * nn);
    d.dF = (int64_t*)malloc(8 * nn);
    d.dG = (int64_t*)malloc(8 * nn);
    d.dH = (int64_t*)malloc(8 * nn);
    size_t tt = (size_t)t;
    piece* bufs[3];
    for (int s = 0; s < 3; ++s) bufs[s] = (piece*)malloc(sizeof(piece) * tt);
    uint8_t* cov = (uint8_t*)malloc(tt);
    int64_t cap = 1024, cnt = 0;
    int64_t* rec = (int64_t*)malloc(sizeof(int64_t) * NF * (size_t)cap);
    int rc = ORA_OK;
    if (!d.hstr || !d.eqlen || !d.trans || !d.sigma || !d.dF || !d.dG || !d.dH || !bufs[0] ||
        !bufs[1] || !bufs[2] || !cov || !rec) {
        rc = ORA_ERR_OOM;
        goto done;
    }

    for (int32_t p = 0; p < *nparts; ++p) {                 /* each partition p */
        int32_t pb = level_ptr[p], pe = level_ptr[p + 1];
        compute_fopd(&a, pb, pe, &d);                       /* ComputeFOPD */
        for (int32_t ra = pb; ra < pe; ra += t) {           /* GetConsecutiveIterations: regions */
            int32_t rb = (ra + t < pe) ? ra + t : pe;
            plist L[3] = {{bufs[0], 0}, {bufs[1], 0}, {bufs[2], 0}};
            int64_t C[3] = {-1, -1, -1};
            if (allowed & ALLOW_BLAS) blas_first(&d, ra, rb, allowed, cov, &L[0]);   /* BLAS_first */
            if (allowed & ALLOW_PSC1) psc1_first(&d, ra, rb, allowed, cov, &L[1]);   /* PSCI_first */
            push(&L[2], T_PSC2, ra, rb);                                            /* PSCII_first */
            int best = -1;                                                          /* min_cost */
            for (int s = 0; s < 3; ++s) {
                if (s == 0 && !(allowed & ALLOW_BLAS)) continue;
                if (s == 1 && !(allowed & ALLOW_PSC1)) continue;
                C[s] = 0;
                for (int32_t i = 0; i < L[s].n; ++i) C[s] += piece_cost(&a, &d, &L[s].v[i], weights);
                if (best < 0 || C[s] < C[best]) best = s;
            }
            qsort(L[best].v, (size_t)L[best].n, sizeof(piece), cmp_piece);
            for (int32_t i = 0; i < L[best].n; ++i) {                               /* cList.append */
                if (cnt == cap) {
                    cap *= 2;
                    int64_t* nr = (int64_t*)realloc(rec, sizeof(int64_t) * NF * (size_t)cap);
                    if (!nr) { rc = ORA_ERR_OOM; goto done; }
                    rec = nr;
                }
                emit(&a, &d, p, &L[best].v[i], rec + NF * cnt);
                ++cnt;
            }
        }
    }

done:
    free(d.hstr); free(d.eqlen); free(d.trans); free(d.sigma);
    free(d.dF); free(d.dG); free(d.dH);
    for (int s = 0; s < 3; ++s) free(bufs[s]);
    free(cov); free(len); free(cs); free(lev);
    if (rc) { free(rec); return rc; }
    *out = rec;
    *ncod = cnt;
    return ORA_OK;
}

void ora_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Plan validity: the expansion of every codelet through its access functions */
/* reproduces the CSR trace, each trace point exactly once.                   */
/* ------------------------------------------------------------------------ */

/* Returns 0 when valid, else a positive code naming the first failed check
 * and writes the offending record index to *bad.  Checks, for every record:
 *   - it lies inside one partition, positions covered exactly once overall;
 *   - BLAS / PSC I rows all have n points;
 *   - f strided: seq[q0+i0] == seq[q0] + rho*i0
 *   - g strided: gs[q0+i0] + i1 == gs[q0] + gamma*i0 + i1
 *   - BLAS h:   Ai[cs + i1] == h0 + delta*i0 + sigma*i1
 *   - PSC I h:  Ai[cs + i1] == h0 + delta*i0 + (Ai[cs(q0) + i1] - h0)
 *   - BLAS / PSC I must claim f and g strided. */
int ora_check_plan(int kind, int32_t n, const int32_t* Ap, const int32_t* Ai,
                   const int32_t* seq, const int32_t* level_ptr, int32_t nparts,
                   const int64_t* gs, const int64_t* rec, int64_t ncod, int64_t* bad) {
    *bad = -1;
    uint8_t* seen = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!seen) return 99;
    int rc = 0;
    for (int64_t c = 0; c < ncod && !rc; ++c) {
        const int64_t* r = rec + NF * c;
        int64_t part = r[0], type = r[1], q0 = r[2], m = r[3], nn = r[4];
        int64_t fs = r[5], rho = r[6], gst = r[7], gam = r[8], h0 = r[9], del = r[10], sig = r[11];
        if (part < 0 || part >= nparts || m < 1 || q0 < level_ptr[part] ||
            q0 + m > level_ptr[part + 1] || type < 0 || type > 2) { rc = 1; *bad = c; break; }
        if (type != T_PSC2 && (!fs || !gst)) { rc = 2; *bad = c; break; }
        for (int64_t i0 = 0; i0 < m && !rc; ++i0) {
            int64_t q = q0 + i0;
            if (seen[q]) { rc = 3; *bad = c; break; }
            seen[q] = 1;
            int32_t row = seq[q];
            int64_t cs = Ap[row];
            int64_t len = Ap[row + 1] - Ap[row] - (kind == ORA_SPTRSV ? 1 : 0);
            int64_t cs0 = Ap[seq[q0]];
            if (fs && (int64_t)row != (int64_t)seq[q0] + rho * i0) { rc = 4; *bad = c; break; }
            if (type != T_PSC2 && len != nn) { rc = 5; *bad = c; break; }
            if (gst) {
                int64_t len0 = Ap[seq[q0] + 1] - Ap[seq[q0]] - (kind == ORA_SPTRSV ? 1 : 0);
                if (len != len0 || gs[q] != gs[q0] + gam * i0) { rc = 6; *bad = c; break; }
            }
            if (type == T_BLAS) {
                for (int64_t i1 = 0; i1 < len; ++i1)
                    if ((int64_t)Ai[cs + i1] != h0 + del * i0 + sig * i1) { rc = 7; *bad = c; break; }
            } else if (type == T_PSC1) {
                for (int64_t i1 = 0; i1 < len; ++i1)
                    if ((int64_t)Ai[cs + i1] != h0 + del * i0 + ((int64_t)Ai[cs0 + i1] - h0)) {
                        rc = 8; *bad = c; break;
                    }
                if (len >= 1 && (int64_t)Ai[cs0] != h0) { rc = 8; *bad = c; break; }
            }
        }
    }
    if (!rc) {
        for (int32_t q = 0; q < n; ++q)
            if (!seen[q]) { rc = 9; *bad = q; break; }
    }
    free(seen);
    return rc;
}
