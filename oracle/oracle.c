/*
 * oracle.c -- plain, slow, obviously correct CPU FP64 reference for the numeric
 * phase of HYLU (Chen, "HYLU: Hybrid Parallel Sparse LU Factorization").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path never
 * calls it, and it shares no code, header or table with the CUDA library.
 *
 * Everything here follows the definitions one step at a time, with dense
 * work vectors and sorted sets, no blocking and no reordering:
 *   - scaled, permuted matrix  Ahat = Pr * Dr * A * Dc * Pc           (Sec. 2.1)
 *   - symbolic structure: row-by-row closure of the up-looking
 *     elimination, fixed before any numeric work                       (Sec. 2.1, 2.2)
 *   - supernodes: runs of consecutive rows with identical U structure (Sec. 2.2)
 *   - padded storage pattern (dense supernode diagonal blocks, full-width
 *     supernode segments in L) -- a reading, the paper gives no detail (Sec. 2.2)
 *   - symbolic flop count                                              (Sec. 2.1)
 *   - up-looking (transposed left-looking) numeric LU, row by row,
 *     largest-magnitude pivot inside a supernode's diagonal block,
 *     no pivoting for standalone rows, small-pivot perturbation        (Sec. 2.2, Fig. 1)
 *   - forward/backward substitution and its transpose                  (Sec. 2.3)
 *   - iterative refinement when a pivot was perturbed                  (Sec. 2.3)
 *
 * Conventions (also used by the tests):
 *   rowperm[i] = original row placed at row i, colperm[k] = original column
 *   placed at column k, dr/dc indexed by ORIGINAL row/column.
 *   Ahat(i,k) = dr[rowperm[i]] * A(rowperm[i], colperm[k]) * dc[colperm[k]].
 *   Ahat * Pi = L * U, L unit lower (Doolittle), Pi a column permutation that
 *   only exchanges columns inside a supernode's diagonal block; piv[p] is the
 *   column label that ends at position p.
 *   Stored factor row i (on the padded pattern, sorted column indices):
 *     index c below the start of row i's supernode -> L(i, position c)
 *     index c inside row i's own supernode block   -> position c
 *                                                     (L if c < i, U if c >= i)
 *     index c past the end of row i's supernode    -> U(i, label c)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int n;
    /* Ahat */
    int64_t *a_rp; int32_t *a_ci; double *a_v;
    /* unpadded symbolic pattern F */
    int64_t *f_rp; int32_t *f_ci;
    /* supernode partition */
    int nsn; int32_t *sn_start; int32_t *sn_of;
    /* padded pattern and factor values */
    int64_t *p_rp; int32_t *p_ci; double *p_v;
    int32_t *piv;
    double *udiag;
    double flops_unpadded, flops_padded;
    double tau;
    int nperturb;
} or_ctx;

static void *xmalloc(size_t s) { void *p = malloc(s ? s : 1); return p; }

or_ctx *or_new(int n) {
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->n = n;
    return c;
}

void or_free(or_ctx *c) {
    if (!c) return;
    free(c->a_rp); free(c->a_ci); free(c->a_v);
    free(c->f_rp); free(c->f_ci);
    free(c->sn_start); free(c->sn_of);
    free(c->p_rp); free(c->p_ci); free(c->p_v);
    free(c->piv); free(c->udiag);
    free(c);
}

/* ------------------------------------------------------------------ Ahat */
static void sort_pairs(int32_t *k, double *v, int64_t m) {
    /* insertion sort: rows are short and this is the oracle */
    for (int64_t a = 1; a < m; ++a) {
        int32_t kk = k[a]; double vv = v[a]; int64_t b = a - 1;
        while (b >= 0 && k[b] > kk) { k[b + 1] = k[b]; v[b + 1] = v[b]; --b; }
        k[b + 1] = kk; v[b + 1] = vv;
    }
}

/* Ahat = Pr * Dr * A * Dc * Pc (static pivoting + scaling, then the symmetric
 * fill-reducing permutation), Sec. 2.1.  Returns 0, or -1 on a bad input. */
int or_build_ahat(or_ctx *c, const int64_t *rp, const int32_t *ci, const double *v,
                  const int32_t *rowperm, const int32_t *colperm,
                  const double *dr, const double *dc) {
    int n = c->n;
    int32_t *qinv = (int32_t *)xmalloc(sizeof(int32_t) * n);
    for (int k = 0; k < n; ++k) qinv[k] = -1;
    for (int k = 0; k < n; ++k) {
        if (colperm[k] < 0 || colperm[k] >= n || qinv[colperm[k]] != -1) { free(qinv); return -1; }
        qinv[colperm[k]] = k;
    }
    int64_t nnz = rp[n];
    c->a_rp = (int64_t *)xmalloc(sizeof(int64_t) * (n + 1));
    c->a_ci = (int32_t *)xmalloc(sizeof(int32_t) * nnz);
    c->a_v = (double *)xmalloc(sizeof(double) * nnz);
    int64_t pos = 0;
    c->a_rp[0] = 0;
    for (int i = 0; i < n; ++i) {
        int r = rowperm[i];
        for (int64_t q = rp[r]; q < rp[r + 1]; ++q) {
            int oc = ci[q];
            c->a_ci[pos] = qinv[oc];
            c->a_v[pos] = dr[r] * v[q] * dc[oc];
            ++pos;
        }
        sort_pairs(c->a_ci + c->a_rp[i], c->a_v + c->a_rp[i], pos - c->a_rp[i]);
        c->a_rp[i + 1] = pos;
    }
    free(qinv);
    return 0;
}

/* ------------------------------------------------------------- symbolic */
/* binary min-heap of int32 */
typedef struct { int32_t *h; int64_t m, cap; } heap_t;
static void hpush(heap_t *H, int32_t x) {
    if (H->m == H->cap) { H->cap = H->cap ? 2 * H->cap : 64; H->h = (int32_t *)realloc(H->h, sizeof(int32_t) * H->cap); }
    int64_t i = H->m++;
    H->h[i] = x;
    while (i > 0) { int64_t p = (i - 1) / 2; if (H->h[p] <= H->h[i]) break; int32_t t = H->h[p]; H->h[p] = H->h[i]; H->h[i] = t; i = p; }
}
static int32_t hpop(heap_t *H) {
    int32_t top = H->h[0];
    H->h[0] = H->h[--H->m];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < H->m && H->h[l] < H->h[s]) s = l;
        if (r < H->m && H->h[r] < H->h[s]) s = r;
        if (s == i) break;
        int32_t t = H->h[s]; H->h[s] = H->h[i]; H->h[i] = t; i = s;
    }
    return top;
}
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Unpadded symbolic structure F (Sec. 2.1: the structure is fixed before the
 * numeric phase; Sec. 2.2: up-looking order).  Row i's structure is the
 * smallest set that holds Ahat(i,:) and i, and that holds U(k, >k) for every k
 * it holds with k < i.  The k < i are taken in ascending order from a heap. */
int or_symbolic(or_ctx *c) {
    int n = c->n;
    int32_t *mark = (int32_t *)xmalloc(sizeof(int32_t) * n);
    for (int j = 0; j < n; ++j) mark[j] = -1;
    int64_t cap = c->a_rp[n] * 2 + n + 16, nnz = 0;
    c->f_rp = (int64_t *)xmalloc(sizeof(int64_t) * (n + 1));
    c->f_ci = (int32_t *)xmalloc(sizeof(int32_t) * cap);
    int64_t *udiag_pos = (int64_t *)xmalloc(sizeof(int64_t) * n); /* index of the diagonal in F row */
    int32_t *upart = (int32_t *)xmalloc(sizeof(int32_t) * n);
    heap_t H = {0, 0, 0};
    c->f_rp[0] = 0;
    for (int i = 0; i < n; ++i) {
        int64_t nu = 0;
        mark[i] = i; upart[nu++] = i;
        for (int64_t q = c->a_rp[i]; q < c->a_rp[i + 1]; ++q) {
            int j = c->a_ci[q];
            if (mark[j] == i) continue;
            mark[j] = i;
            if (j < i) hpush(&H, j); else upart[nu++] = j;
        }
        int64_t row0 = nnz;
        while (H.m > 0) {
            int32_t k = hpop(&H);
            if (nnz + 1 > cap) { cap *= 2; c->f_ci = (int32_t *)realloc(c->f_ci, sizeof(int32_t) * cap); }
            c->f_ci[nnz++] = k;                       /* L(i,k), ascending */
            for (int64_t q = udiag_pos[k] + 1; q < c->f_rp[k + 1]; ++q) {
                int j = c->f_ci[q];                   /* j in U(k, >k) */
                if (mark[j] == i) continue;
                mark[j] = i;
                if (j < i) hpush(&H, j); else upart[nu++] = j;
            }
        }
        qsort(upart, (size_t)nu, sizeof(int32_t), cmp_i32);
        if (nnz + nu > cap) { while (nnz + nu > cap) cap *= 2; c->f_ci = (int32_t *)realloc(c->f_ci, sizeof(int32_t) * cap); }
        udiag_pos[i] = nnz;
        memcpy(c->f_ci + nnz, upart, sizeof(int32_t) * nu);
        nnz += nu;
        c->f_rp[i + 1] = nnz;
        (void)row0;
    }
    free(H.h); free(mark); free(udiag_pos); free(upart);
    return 0;
}

/* position of the diagonal inside row i of a sorted pattern */
static int64_t diag_index(const int64_t *rp, const int32_t *ci, int i) {
    for (int64_t q = rp[i]; q < rp[i + 1]; ++q) if (ci[q] == i) return q;
    return -1;
}

/* Supernodes (Sec. 2.2: consecutive rows with identical U structure).  Row
 * r+1 joins the supernode of row r iff U(r+1,:) equals U(r,:) without r and
 * the supernode holds fewer than sn_max rows. */
int or_supernodes(or_ctx *c, int sn_max) {
    int n = c->n;
    c->sn_start = (int32_t *)xmalloc(sizeof(int32_t) * (n + 1));
    c->sn_of = (int32_t *)xmalloc(sizeof(int32_t) * n);
    int ns = 0, cur_start = 0;
    c->sn_start[0] = 0;
    if (n == 0) {               /* no rows: the partition has no blocks */
        c->nsn = 0;
        return 0;
    }
    ns = 1;
    for (int r = 0; r + 1 < n; ++r) {
        int64_t dr = diag_index(c->f_rp, c->f_ci, r), dn = diag_index(c->f_rp, c->f_ci, r + 1);
        int64_t lr = c->f_rp[r + 1] - dr, ln = c->f_rp[r + 2] - dn;
        int same = (lr - 1 == ln);
        for (int64_t t = 0; same && t < ln; ++t)
            if (c->f_ci[dr + 1 + t] != c->f_ci[dn + t]) same = 0;
        if (!same || (r + 1 - cur_start) >= sn_max) {
            cur_start = r + 1;
            c->sn_start[ns++] = r + 1;
        }
    }
    c->sn_start[ns] = n;
    c->nsn = ns;
    for (int s = 0; s < ns; ++s)
        for (int i = c->sn_start[s]; i < c->sn_start[s + 1]; ++i) c->sn_of[i] = s;
    return ns;
}

/* Padded storage pattern (a reading of Sec. 2.2, "the data structure ... supports
 * the hybrid numerical kernels in a common way"):
 *   (i)   a supernode's diagonal block is stored dense;
 *   (ii)  a row that holds any L entry in a column of supernode S holds all
 *         columns of S.
 * Each row keeps its own L columns; U structure is left as it is.  Also
 * computes both flop counts (Sec. 2.1): every L(i,k) costs one division and
 * two flops per off-diagonal U(k,:) entry. */
int or_pad(or_ctx *c) {
    int n = c->n;
    char *in = (char *)calloc((size_t)n, 1);
    int32_t *lst = (int32_t *)xmalloc(sizeof(int32_t) * n);
    int64_t cap = c->f_rp[n] * 2 + 16, nnz = 0;
    c->p_rp = (int64_t *)xmalloc(sizeof(int64_t) * (n + 1));
    c->p_ci = (int32_t *)xmalloc(sizeof(int32_t) * cap);
    c->p_rp[0] = 0;
    int64_t *ulen = (int64_t *)xmalloc(sizeof(int64_t) * n);
    for (int i = 0; i < n; ++i) {
        int64_t d = diag_index(c->f_rp, c->f_ci, i);
        ulen[i] = c->f_rp[i + 1] - d;
    }
    for (int s = 0; s < c->nsn; ++s) {
        int r = c->sn_start[s], e = c->sn_start[s + 1] - 1;
        for (int i = r; i <= e; ++i) {
            int64_t nl = 0;
            for (int64_t q = c->f_rp[i]; q < c->f_rp[i + 1]; ++q) {
                int k = c->f_ci[q];
                if (k >= r) break;                          /* only columns before the block */
                int S = c->sn_of[k];
                for (int t = c->sn_start[S]; t < c->sn_start[S + 1]; ++t)   /* rule (ii) */
                    if (!in[t]) { in[t] = 1; lst[nl++] = t; }
            }
            qsort(lst, (size_t)nl, sizeof(int32_t), cmp_i32);
            int64_t d = diag_index(c->f_rp, c->f_ci, i);
            int64_t need = nl + (e - r + 1) + (c->f_rp[i + 1] - d);
            if (nnz + need > cap) { while (nnz + need > cap) cap *= 2; c->p_ci = (int32_t *)realloc(c->p_ci, sizeof(int32_t) * cap); }
            for (int64_t t = 0; t < nl; ++t) { c->p_ci[nnz++] = lst[t]; in[lst[t]] = 0; }
            for (int t = r; t <= e; ++t) c->p_ci[nnz++] = t;               /* rule (i) */
            for (int64_t q = d; q < c->f_rp[i + 1]; ++q)
                if (c->f_ci[q] > e) c->p_ci[nnz++] = c->f_ci[q];          /* tail of U */
            c->p_rp[i + 1] = nnz;
        }
    }
    /* flop counts */
    double fu = 0.0, fp = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int64_t q = c->f_rp[i]; q < c->f_rp[i + 1]; ++q) {
            int k = c->f_ci[q];
            if (k >= i) break;
            fu += 1.0 + 2.0 * (double)(ulen[k] - 1);
        }
        for (int64_t q = c->p_rp[i]; q < c->p_rp[i + 1]; ++q) {
            int k = c->p_ci[q];
            if (k >= i) break;
            fp += 1.0 + 2.0 * (double)(ulen[k] - 1);
        }
    }
    c->flops_unpadded = fu;
    c->flops_padded = fp;
    free(in); free(lst); free(ulen);
    return 0;
}

/* ------------------------------------------------------------- numeric */
static int64_t find_col(const int32_t *ci, int64_t s, int64_t e, int j) {
    for (int64_t q = s; q < e; ++q) if (ci[q] == j) return q;
    return -1;
}

/* Up-looking numeric LU on the padded pattern (Sec. 2.2, Fig. 1): row i takes
 * Ahat(i,:) into a dense work vector x (indexed by column label) and, for each
 * earlier position k it holds, in ascending order, sets l = x[label of k] / u_kk
 * and subtracts l * U(k, >k).  Inside a supernode the row then exchanges the
 * largest |x| of its diagonal block (first position on ties) to the diagonal;
 * standalone rows never pivot.  A pivot smaller than tau = tau_rel * max|Ahat|
 * becomes sign(pivot) * tau (sign(0) = +1) and is counted (Sec. 2.2).
 * Returns the number of perturbed pivots, or -1 if the pattern is not closed. */
int or_factor(or_ctx *c, double tau_rel) {
    int n = c->n;
    int64_t pn = c->p_rp[n];
    free(c->p_v); free(c->piv); free(c->udiag);
    c->p_v = (double *)calloc((size_t)pn, sizeof(double));
    c->piv = (int32_t *)xmalloc(sizeof(int32_t) * n);
    c->udiag = (double *)xmalloc(sizeof(double) * n);
    int32_t *pinv = (int32_t *)xmalloc(sizeof(int32_t) * n);   /* label -> position */
    for (int i = 0; i < n; ++i) { c->piv[i] = i; pinv[i] = i; }
    double amax = 0.0;
    for (int64_t q = 0; q < c->a_rp[n]; ++q) if (fabs(c->a_v[q]) > amax) amax = fabs(c->a_v[q]);
    double tau = tau_rel * amax;
    c->tau = tau;
    c->nperturb = 0;
    double *x = (double *)calloc((size_t)n, sizeof(double));
    int status = 0;
    for (int s = 0; s < c->nsn && status == 0; ++s) {
        int r = c->sn_start[s], e = c->sn_start[s + 1] - 1;
        for (int i = r; i <= e; ++i) {
            int64_t rs = c->p_rp[i], re = c->p_rp[i + 1];
            for (int64_t q = c->a_rp[i]; q < c->a_rp[i + 1]; ++q) {
                if (find_col(c->p_ci, rs, re, c->a_ci[q]) < 0) status = -1;
                x[c->a_ci[q]] = c->a_v[q];
            }
            /* sources in ascending position order */
            for (int64_t q = rs; q < re; ++q) {
                int k = c->p_ci[q];
                if (k >= i) break;
                int lab = c->piv[k];
                double l = x[lab] / c->udiag[k];
                x[lab] = l;                               /* L(i, position k) */
                int sk = c->sn_of[k], ek = c->sn_start[sk + 1] - 1;
                int64_t ks = c->p_rp[k], ke = c->p_rp[k + 1];
                for (int64_t t = ks; t < ke; ++t) {
                    int j = c->p_ci[t];
                    if (sk == s) {
                        /* source row inside this supernode: its block is kept by label
                         * until the supernode ends; U(k,.) = labels at positions > k */
                        if (j >= r && j <= e) {
                            if (pinv[j] > k) x[j] -= l * c->p_v[t];
                        } else if (j > e) {
                            x[j] -= l * c->p_v[t];
                        }
                    } else {
                        if (j <= k) continue;
                        if (j <= ek) x[c->piv[j]] -= l * c->p_v[t];  /* block, by position */
                        else x[j] -= l * c->p_v[t];                   /* tail, by label */
                    }
                }
            }
            if (e > r) {                                  /* supernode diagonal pivoting */
                int best = i; double bv = fabs(x[c->piv[i]]);
                for (int p = i + 1; p <= e; ++p) {
                    double a = fabs(x[c->piv[p]]);
                    if (a > bv) { bv = a; best = p; }
                }
                int t = c->piv[i]; c->piv[i] = c->piv[best]; c->piv[best] = t;
                pinv[c->piv[i]] = i; pinv[c->piv[best]] = best;
            }
            double u = x[c->piv[i]];
            if (fabs(u) < tau) { u = (u >= 0.0) ? tau : -tau; c->nperturb++; x[c->piv[i]] = u; }
            c->udiag[i] = u;
            /* store the row; the own block stays by label until the supernode ends */
            for (int64_t q = rs; q < re; ++q) {
                int j = c->p_ci[q];
                if (j < r) c->p_v[q] = x[c->piv[j]];      /* L by position (piv is final there) */
                else c->p_v[q] = x[j];
            }
            for (int64_t q = rs; q < re; ++q) {
                int j = c->p_ci[q];
                x[j] = 0.0;
                if (j < r) x[c->piv[j]] = 0.0;
            }
        }
        if (e > r) {                                      /* own block: labels -> positions */
            int w = e - r + 1;
            double *tmp = (double *)xmalloc(sizeof(double) * w);
            for (int i = r; i <= e; ++i) {
                int64_t b = find_col(c->p_ci, c->p_rp[i], c->p_rp[i + 1], r);
                for (int p = 0; p < w; ++p) tmp[p] = c->p_v[b + (c->piv[r + p] - r)];
                for (int p = 0; p < w; ++p) c->p_v[b + p] = tmp[p];
            }
            free(tmp);
        }
    }
    free(x); free(pinv);
    if (status) return -1;
    return c->nperturb;
}

/* ---------------------------------------------------------------- solves */
/* Solve A x = b for one right-hand side using the stored factors (Sec. 2.3):
 * bhat = Pr Dr b; L z = bhat; U w = z; xhat = Pi w; x = Dc Pc xhat. */
void or_solve(const or_ctx *c, const int32_t *rowperm, const int32_t *colperm,
              const double *dr, const double *dc, const double *b, double *x) {
    int n = c->n;
    double *z = (double *)xmalloc(sizeof(double) * n);
    double *w = (double *)xmalloc(sizeof(double) * n);
    int32_t *pinv = (int32_t *)xmalloc(sizeof(int32_t) * n);
    for (int p = 0; p < n; ++p) pinv[c->piv[p]] = p;
    for (int i = 0; i < n; ++i) z[i] = dr[rowperm[i]] * b[rowperm[i]];
    for (int i = 0; i < n; ++i) {                         /* forward, unit L */
        double s = z[i];
        for (int64_t q = c->p_rp[i]; q < c->p_rp[i + 1]; ++q) {
            int k = c->p_ci[q];
            if (k >= i) break;
            s -= c->p_v[q] * z[k];
        }
        z[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {                    /* backward, positions */
        int e = c->sn_start[c->sn_of[i] + 1] - 1;
        double s = z[i];
        for (int64_t q = c->p_rp[i]; q < c->p_rp[i + 1]; ++q) {
            int j = c->p_ci[q];
            if (j <= i) continue;
            int p = (j <= e) ? j : pinv[j];
            s -= c->p_v[q] * w[p];
        }
        w[i] = s / c->udiag[i];
    }
    for (int p = 0; p < n; ++p) z[c->piv[p]] = w[p];       /* xhat = Pi w */
    for (int k = 0; k < n; ++k) x[colperm[k]] = dc[colperm[k]] * z[k];
    free(z); free(w); free(pinv);
}

/* Solve A^T y = g with the same factors: ghat = Pc^T Dc g; U^T v = Pi^T ghat;
 * L^T yhat = v; y = Dr Pr^T yhat. */
void or_solve_transpose(const or_ctx *c, const int32_t *rowperm, const int32_t *colperm,
                        const double *dr, const double *dc, const double *g, double *y) {
    int n = c->n;
    double *h = (double *)xmalloc(sizeof(double) * n);
    double *v = (double *)xmalloc(sizeof(double) * n);
    int32_t *pinv = (int32_t *)xmalloc(sizeof(int32_t) * n);
    for (int p = 0; p < n; ++p) pinv[c->piv[p]] = p;
    double *gh = (double *)xmalloc(sizeof(double) * n);
    for (int k = 0; k < n; ++k) gh[k] = dc[colperm[k]] * g[colperm[k]];
    for (int p = 0; p < n; ++p) h[p] = gh[c->piv[p]];
    for (int i = 0; i < n; ++i) {                         /* U^T v = h, column sweep */
        int e = c->sn_start[c->sn_of[i] + 1] - 1;
        v[i] = h[i] / c->udiag[i];
        for (int64_t q = c->p_rp[i]; q < c->p_rp[i + 1]; ++q) {
            int j = c->p_ci[q];
            if (j <= i) continue;
            int p = (j <= e) ? j : pinv[j];
            h[p] -= c->p_v[q] * v[i];
        }
    }
    for (int i = n - 1; i >= 0; --i) {                    /* L^T yhat = v */
        for (int64_t q = c->p_rp[i]; q < c->p_rp[i + 1]; ++q) {
            int k = c->p_ci[q];
            if (k >= i) break;
            v[k] -= c->p_v[q] * v[i];
        }
    }
    for (int i = 0; i < n; ++i) y[rowperm[i]] = dr[rowperm[i]] * v[i];
    free(h); free(v); free(pinv); free(gh);
}

/* backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) on the
 * original A, and residual r = b - A x */
double or_backward_error(int n, const int64_t *rp, const int32_t *ci, const double *v,
                         const double *x, const double *b, double *r) {
    double anorm = 0.0, xn = 0.0, bn = 0.0, rn = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = b[i], ra = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) { s -= v[q] * x[ci[q]]; ra += fabs(v[q]); }
        if (r) r[i] = s;
        if (ra > anorm) anorm = ra;
        if (fabs(x[i]) > xn) xn = fabs(x[i]);
        if (fabs(b[i]) > bn) bn = fabs(b[i]);
        if (fabs(s) > rn) rn = fabs(s);
    }
    double den = anorm * xn + bn;
    return den > 0.0 ? rn / den : rn;
}

/* Solve with iterative refinement in FP64 on the original A (Sec. 2.3): runs
 * when a pivot was perturbed or when `force` is set; stops at backward error
 * <= tol, when the error fails to halve, or after maxit corrections.
 * Returns the number of corrections; *be_out gets the final backward error. */
int or_solve_refine(const or_ctx *c, const int64_t *rp, const int32_t *ci, const double *v,
                    const int32_t *rowperm, const int32_t *colperm,
                    const double *dr, const double *dc, const double *b, double *x,
                    double tol, int maxit, int force, double *be_out) {
    int n = c->n;
    double *r = (double *)xmalloc(sizeof(double) * n);
    double *d = (double *)xmalloc(sizeof(double) * n);
    or_solve(c, rowperm, colperm, dr, dc, b, x);
    double be = or_backward_error(n, rp, ci, v, x, b, r);
    int it = 0;
    if (c->nperturb > 0 || force) {
        while (be > tol && it < maxit) {
            or_solve(c, rowperm, colperm, dr, dc, r, d);
            for (int i = 0; i < n; ++i) x[i] += d[i];
            ++it;
            double nb = or_backward_error(n, rp, ci, v, x, b, r);
            int stalled = !(nb <= 0.5 * be);
            be = nb;
            if (stalled) break;
        }
    }
    if (be_out) *be_out = be;
    free(r); free(d);
    return it;
}

/* ------------------------------------------------------------- accessors */
int or_n(const or_ctx *c) { return c->n; }
int64_t or_f_nnz(const or_ctx *c) { return c->f_rp ? c->f_rp[c->n] : -1; }
int64_t or_p_nnz(const or_ctx *c) { return c->p_rp ? c->p_rp[c->n] : -1; }
int or_nsn(const or_ctx *c) { return c->nsn; }
int or_nperturb(const or_ctx *c) { return c->nperturb; }
double or_tau(const or_ctx *c) { return c->tau; }
double or_flops_unpadded(const or_ctx *c) { return c->flops_unpadded; }
double or_flops_padded(const or_ctx *c) { return c->flops_padded; }
void or_get_ahat(const or_ctx *c, int64_t *rp, int32_t *ci, double *v) {
    memcpy(rp, c->a_rp, sizeof(int64_t) * (c->n + 1));
    memcpy(ci, c->a_ci, sizeof(int32_t) * c->a_rp[c->n]);
    memcpy(v, c->a_v, sizeof(double) * c->a_rp[c->n]);
}
void or_get_f(const or_ctx *c, int64_t *rp, int32_t *ci) {
    memcpy(rp, c->f_rp, sizeof(int64_t) * (c->n + 1));
    memcpy(ci, c->f_ci, sizeof(int32_t) * c->f_rp[c->n]);
}
void or_get_sn(const or_ctx *c, int32_t *start) {
    memcpy(start, c->sn_start, sizeof(int32_t) * (c->nsn + 1));
}
void or_get_p(const or_ctx *c, int64_t *rp, int32_t *ci) {
    memcpy(rp, c->p_rp, sizeof(int64_t) * (c->n + 1));
    memcpy(ci, c->p_ci, sizeof(int32_t) * c->p_rp[c->n]);
}
void or_get_factor(const or_ctx *c, double *v, int32_t *piv, double *udiag) {
    memcpy(v, c->p_v, sizeof(double) * c->p_rp[c->n]);
    memcpy(piv, c->piv, sizeof(int32_t) * c->n);
    memcpy(udiag, c->udiag, sizeof(double) * c->n);
}
