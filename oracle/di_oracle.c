/*
 * di_oracle.c -- plain, sequential, FP64 CPU oracle for D-Iteration
 * (Hong, Huynh, Mathieu, "D-Iteration: diffusion approach for solving PageRank",
 * arXiv:1501.06350).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA path.  Every routine is written for obviousness, not speed: one thread,
 * no blocking, no reordering beyond what the cited definition states.
 *
 * Notation follows the paper: P is the n x n diffusion matrix with
 * P[i][j] = w(j,i) / sum_k w(j,k) for a link j -> i (Section 2.1, Eq. def-p),
 * so column j of P is the out-link row j of the out-CSR; F is the fluid vector
 * and H the history vector (Section 3.1).
 *
 * Parity status of each routine (what pins it is listed in the test-suite):
 *   or_canonical_csr     pinned (brute-force dictionary build on tiny inputs)
 *   or_transpose         pinned (brute force, and transpose of transpose)
 *   or_di_init/solve     pinned (dense direct solve, closed forms, invariant
 *                        Eq. HnFn, bound Eq. SL, Theorems 2 and 3)
 *   or_power_iteration   pinned (dense direct solve, contraction rate d)
 *   or_apply_batch       pinned (brute-force set semantics on tiny inputs)
 *   or_update_inject     pinned (Theorem update: resumed DI reaches the dense
 *                        solution of the new matrix)
 *   or_adjoint_jacobi    pinned (dense solve of (I - dP)^T lambda = g, the
 *                        duality g . x = (1 - d) lambda . Z, closed forms)
 *   or_grad_w            pinned (central finite differences of g . x(w) with
 *                        x from the dense solve)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_BAD_INPUT -1
#define OR_NO_MEMORY -2
#define OR_NOT_CONVERGED 1

/* ------------------------------------------------------------------------- */
/* Section 2.1, Eq. def-p: the link set E with weights w(j,i) > 0.            */
/* Input layout 0 = rows over sources (out-links), 1 = rows over targets.     */
/* Output: canonical out-CSR, each row sorted by target, duplicate links      */
/* merged by summing their weights in input order.                            */
/* Returns the merged link count, or OR_BAD_INPUT / OR_NO_MEMORY.             */
/* ------------------------------------------------------------------------- */
int64_t or_canonical_csr(int64_t n, int64_t nnz, const int64_t *ptr, const int32_t *idx,
                         const double *w, int layout, int64_t *out_ptr, int32_t *out_idx,
                         double *out_w)
{
    if (n < 1 || nnz < 0 || ptr[0] != 0 || ptr[n] != nnz) return OR_BAD_INPUT;
    for (int64_t r = 0; r < n; r++)
        if (ptr[r + 1] < ptr[r]) return OR_BAD_INPUT;
    for (int64_t e = 0; e < nnz; e++) {
        if (idx[e] < 0 || (int64_t)idx[e] >= n) return OR_BAD_INPUT;
        if (w && !(isfinite(w[e]) && w[e] > 0.0)) return OR_BAD_INPUT;
    }
    int64_t *src = malloc(sizeof(int64_t) * (nnz + 1));
    int64_t *dst = malloc(sizeof(int64_t) * (nnz + 1));
    int64_t *ord = malloc(sizeof(int64_t) * (nnz + 1));
    int64_t *tmp = malloc(sizeof(int64_t) * (nnz + 1));
    int64_t *cnt = calloc((size_t)n + 1, sizeof(int64_t));
    if (!src || !dst || !ord || !tmp || !cnt) {
        free(src); free(dst); free(ord); free(tmp); free(cnt);
        return OR_NO_MEMORY;
    }
    for (int64_t r = 0; r < n; r++)
        for (int64_t e = ptr[r]; e < ptr[r + 1]; e++) {
            if (layout == 0) { src[e] = r; dst[e] = idx[e]; }
            else             { src[e] = idx[e]; dst[e] = r; }
        }
    /* stable counting sort by target, then stable counting sort by source:
       the result is ordered by (source, target) with ties in input order */
    for (int64_t e = 0; e < nnz; e++) ord[e] = e;
    for (int pass = 0; pass < 2; pass++) {
        const int64_t *key = pass == 0 ? dst : src;
        memset(cnt, 0, sizeof(int64_t) * ((size_t)n + 1));
        for (int64_t e = 0; e < nnz; e++) cnt[key[ord[e]] + 1]++;
        for (int64_t r = 0; r < n; r++) cnt[r + 1] += cnt[r];
        for (int64_t e = 0; e < nnz; e++) tmp[cnt[key[ord[e]]]++] = ord[e];
        memcpy(ord, tmp, sizeof(int64_t) * nnz);
    }
    int64_t m = 0;
    for (int64_t r = 0; r <= n; r++) out_ptr[r] = 0;
    for (int64_t k = 0; k < nnz; k++) {
        int64_t e = ord[k];
        if (m > 0 && k > 0 && src[ord[k - 1]] == src[e] && dst[ord[k - 1]] == dst[e]) {
            if (out_w) out_w[m - 1] += w ? w[e] : 1.0;
            continue;
        }
        out_idx[m] = (int32_t)dst[e];
        if (out_w) out_w[m] = w ? w[e] : 1.0;
        out_ptr[src[e] + 1]++;
        m++;
    }
    for (int64_t r = 0; r < n; r++) out_ptr[r + 1] += out_ptr[r];
    free(src); free(dst); free(ord); free(tmp); free(cnt);
    return m;
}

/* In-link structure: for each target i the sources j of links j -> i in      */
/* ascending order (stable counting sort of a canonical out-CSR by target).   */
void or_transpose(int64_t n, const int64_t *ptr, const int32_t *idx, const double *w,
                  int64_t *tptr, int32_t *tidx, double *tw)
{
    int64_t nnz = ptr[n];
    for (int64_t r = 0; r <= n; r++) tptr[r] = 0;
    for (int64_t e = 0; e < nnz; e++) tptr[idx[e] + 1]++;
    for (int64_t r = 0; r < n; r++) tptr[r + 1] += tptr[r];
    int64_t *fill = malloc(sizeof(int64_t) * ((size_t)n + 1));
    memcpy(fill, tptr, sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t j = 0; j < n; j++)
        for (int64_t e = ptr[j]; e < ptr[j + 1]; e++) {
            int64_t pos = fill[idx[e]]++;
            tidx[pos] = (int32_t)j;
            if (tw) tw[pos] = w ? w[e] : 1.0;
        }
    free(fill);
}

/* Column sums of the link weights (Section 2.1, Eq. def-p): W_j = sum_k     */
/* w(j,k) added left to right in row order, or out(j) for unweighted graphs. */
static double *row_scale(int64_t n, const int64_t *ptr, const double *w)
{
    double *W = malloc(sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < n; j++) {
        if (!w) { W[j] = (double)(ptr[j + 1] - ptr[j]); continue; }
        W[j] = 0.0;
        for (int64_t k = ptr[j]; k < ptr[j + 1]; k++) W[j] += w[k];
    }
    return W;
}

/* Entry P[i][j] for the e-th link j -> i (Section 2.1, Eq. def-p):           */
/* w(j,i) / W_j, which is 1 / out(j) for unweighted graphs.                   */
static double p_entry(const double *W, const double *w, int64_t j, int64_t e)
{
    return (w ? w[e] : 1.0) / W[j];
}

/* Section 3.1: F_0 = (1 - d) Z, H_0 = 0.                                     */
void or_di_init(int64_t n, double d, const double *Z, double *F, double *H)
{
    double one_minus_d = 1.0 - d;
    for (int64_t i = 0; i < n; i++) {
        F[i] = one_minus_d * (Z ? Z[i] : 1.0 / (double)n);
        H[i] = 0.0;
    }
}

static double l1(int64_t n, const double *v)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += fabs(v[i]);
    return s;
}

typedef struct {
    double resid_l1;        /* |F|_1 at return (exact left-to-right sum)          */
    double l_dangling;      /* sum of H over dangling nodes (Section 3.3, l_k)    */
    int64_t diffusions;     /* number of elementary diffusions (Eq. defF steps)   */
    int64_t edge_pushes;    /* sum of out-degrees of the diffused nodes           */
    int64_t cycles;         /* passes of the round-robin cursor                   */
    int converged;
} or_info;

/* One elementary diffusion of node c (Section 3.1, Eq. defF and the H_k       */
/* recursion): H(c) += F(c); F += d F(c) P e_c - F(c) e_c.  Returns the change */
/* of |F|_1 so that the caller can keep a running norm.                        */
static double diffuse(const int64_t *ptr, const int32_t *idx, const double *w,
                      const double *W, double d, int64_t c, double *F, double *H)
{
    double f = F[c];
    double delta = -fabs(F[c]);
    H[c] += f;
    F[c] = 0.0;
    for (int64_t e = ptr[c]; e < ptr[c + 1]; e++) {
        int64_t i = idx[e];
        double before = fabs(F[i]);
        F[i] += d * f * p_entry(W, w, c, e);
        delta += fabs(F[i]) - before;
    }
    return delta;
}

/* ------------------------------------------------------------------------- */
/* D-Iteration on a given diffusion sequence (Section 3.1), with the two      */
/* schedulers of Section 3.4:                                                 */
/*   schedule 0 = DI-argmax: a round-robin cursor over 0..n-1 that skips a    */
/*                node unless |F(c)| is at least the average |F|_1 / n        */
/*                (ties included), zero-fluid nodes being skipped too;        */
/*   schedule 1 = DI-cyc: the identity permutation repeated.                  */
/* Stops when |F|_1 / (1 - d) <= tol (Theorem 1, Eq. SL), or after            */
/* max_diffusions steps.  F and H are in/out: pass them from or_di_init, or a */
/* state to resume from (Theorem update).  The running |F|_1 is recomputed    */
/* exactly at the end of each cursor pass and before any stop.                */
/* trace (nullable, max_diffusions entries): exact |F|_1 after each step.     */
/* ------------------------------------------------------------------------- */
int or_di_solve(int64_t n, const int64_t *ptr, const int32_t *idx, const double *w, double d,
                double *F, double *H, double tol, int64_t max_diffusions, int schedule,
                double *trace, or_info *info)
{
    if (n < 1 || !(d > 0.0 && d < 1.0) || !(tol > 0.0)) return OR_BAD_INPUT;
    double one_minus_d = 1.0 - d;
    double *W = row_scale(n, ptr, w);
    double S = l1(n, F);
    int64_t k = 0, pushes = 0, cycles = 0;
    int converged = S / one_minus_d <= tol;
    while (!converged && k < max_diffusions) {
        int checked = 0;
        int64_t took = 0;
        for (int64_t c = 0; c < n && !converged && k < max_diffusions; c++) {
            int take;
            if (schedule == 1) take = 1;
            else take = F[c] != 0.0 && fabs(F[c]) >= S / (double)n;
            if (!take) continue;
            S += diffuse(ptr, idx, w, W, d, c, F, H);
            pushes += ptr[c + 1] - ptr[c];
            if (trace) trace[k] = l1(n, F);
            k++;
            took++;
            if (S / one_minus_d <= tol && !checked) {
                S = l1(n, F);
                checked = 1;
                converged = S / one_minus_d <= tol;
            }
        }
        if (took == 0 && !converged && k < max_diffusions) {
            /* Rounding can make the computed average exceed every |F(c)| (all
               fluids equal).  The largest fluid is at least the exact average,
               so the exact test accepts it: take the first largest one. */
            int64_t best = 0;
            for (int64_t c = 1; c < n; c++)
                if (fabs(F[c]) > fabs(F[best])) best = c;
            S += diffuse(ptr, idx, w, W, d, best, F, H);
            pushes += ptr[best + 1] - ptr[best];
            if (trace) trace[k] = l1(n, F);
            k++;
        }
        cycles++;
        S = l1(n, F);
        converged = S / one_minus_d <= tol;
    }
    if (info) {
        double ld = 0.0;
        for (int64_t i = 0; i < n; i++)
            if (ptr[i + 1] == ptr[i]) ld += H[i];
        info->resid_l1 = l1(n, F);
        info->l_dangling = ld;
        info->diffusions = k;
        info->edge_pushes = pushes;
        info->cycles = cycles;
        info->converged = converged;
    }
    free(W);
    return converged ? OR_OK : OR_NOT_CONVERGED;
}

/* Section 2.2: x_{k+1} = d P x_k + (1 - d) Z starting from x_0 = (1 - d) Z,   */
/* until |x_{k+1} - x_k|_1 <= tol or max_iters.  P x is formed column by       */
/* column (out-link rows).  Returns the number of iterations performed.        */
int64_t or_power_iteration(int64_t n, const int64_t *ptr, const int32_t *idx, const double *w,
                           double d, const double *Z, double tol, int64_t max_iters, double *x)
{
    double *y = malloc(sizeof(double) * (size_t)n);
    double *W = row_scale(n, ptr, w);
    double one_minus_d = 1.0 - d;
    for (int64_t i = 0; i < n; i++) x[i] = one_minus_d * (Z ? Z[i] : 1.0 / (double)n);
    int64_t it = 0;
    while (it < max_iters) {
        for (int64_t i = 0; i < n; i++) y[i] = 0.0;
        for (int64_t j = 0; j < n; j++)
            for (int64_t e = ptr[j]; e < ptr[j + 1]; e++)
                y[idx[e]] += p_entry(W, w, j, e) * x[j];
        double change = 0.0;
        for (int64_t i = 0; i < n; i++) {
            double nx = d * y[i] + one_minus_d * (Z ? Z[i] : 1.0 / (double)n);
            change += fabs(nx - x[i]);
            x[i] = nx;
        }
        it++;
        if (change <= tol) break;
    }
    free(y);
    free(W);
    return it;
}

/* ------------------------------------------------------------------------- */
/* Link changes between P and P' (Section 3.5).  The batch is applied in      */
/* order to the canonical out-CSR: op +1 makes link src -> dst present with   */
/* weight wb (1 when wb is NULL), op -1 makes it absent (no-op if absent).    */
/* The output is canonical again.  Returns the new link count.                */
/* ------------------------------------------------------------------------- */
int64_t or_apply_batch(int64_t n, const int64_t *ptr, const int32_t *idx, const double *w,
                       int64_t m, const int32_t *bsrc, const int32_t *bdst, const double *wb,
                       const int8_t *op, int64_t *out_ptr, int32_t *out_idx, double *out_w)
{
    for (int64_t b = 0; b < m; b++) {
        if (bsrc[b] < 0 || bsrc[b] >= n || bdst[b] < 0 || bdst[b] >= n) return OR_BAD_INPUT;
        if (op[b] != 1 && op[b] != -1) return OR_BAD_INPUT;
        if (wb && op[b] == 1 && !(isfinite(wb[b]) && wb[b] > 0.0)) return OR_BAD_INPUT;
    }
    /* batch ordered by (src, dst), ties in batch order (two stable passes) */
    int64_t *ord = malloc(sizeof(int64_t) * (m + 1));
    int64_t *tmp = malloc(sizeof(int64_t) * (m + 1));
    int64_t *cnt = malloc(sizeof(int64_t) * ((size_t)n + 1));
    for (int64_t b = 0; b < m; b++) ord[b] = b;
    for (int pass = 0; pass < 2; pass++) {
        const int32_t *key = pass == 0 ? bdst : bsrc;
        memset(cnt, 0, sizeof(int64_t) * ((size_t)n + 1));
        for (int64_t b = 0; b < m; b++) cnt[key[ord[b]] + 1]++;
        for (int64_t r = 0; r < n; r++) cnt[r + 1] += cnt[r];
        for (int64_t b = 0; b < m; b++) tmp[cnt[key[ord[b]]]++] = ord[b];
        memcpy(ord, tmp, sizeof(int64_t) * m);
    }
    int64_t out = 0, b = 0;
    out_ptr[0] = 0;
    for (int64_t j = 0; j < n; j++) {
        int64_t e = ptr[j], ee = ptr[j + 1];
        while (e < ee || (b < m && bsrc[ord[b]] == j)) {
            int64_t t_old = e < ee ? idx[e] : INT64_MAX;
            int64_t t_b = (b < m && bsrc[ord[b]] == j) ? bdst[ord[b]] : INT64_MAX;
            if (t_old < t_b) {               /* untouched link */
                out_idx[out] = (int32_t)t_old;
                if (out_w) out_w[out] = w ? w[e] : 1.0;
                out++; e++;
                continue;
            }
            /* last batch entry for (j, t_b) decides */
            int64_t last = ord[b];
            while (b < m && bsrc[ord[b]] == j && bdst[ord[b]] == t_b) { last = ord[b]; b++; }
            if (t_old == t_b) e++;
            if (op[last] == 1) {
                out_idx[out] = (int32_t)t_b;
                if (out_w) out_w[out] = wb ? wb[last] : 1.0;
                out++;
            }
        }
        out_ptr[j + 1] = out;
    }
    free(ord); free(tmp); free(cnt);
    return out;
}

/* Theorem update (Section 3.5): F'_0 = F_{k0} + d (P' - P) H_{k0}.  Columns   */
/* j of P and P' that are equal contribute nothing and are skipped; for every */
/* other column the old entries are withdrawn and the new ones injected.      */
/* Returns the number of changed columns.                                     */
int64_t or_update_inject(int64_t n, const int64_t *ptr, const int32_t *idx, const double *w,
                         const int64_t *nptr, const int32_t *nidx, const double *nw, double d,
                         const double *H, double *F)
{
    int64_t changed = 0;
    double *W = row_scale(n, ptr, w);
    double *NW = row_scale(n, nptr, nw);
    for (int64_t j = 0; j < n; j++) {
        int64_t a = ptr[j], b = ptr[j + 1], na = nptr[j], nb = nptr[j + 1];
        int same = (b - a) == (nb - na);
        for (int64_t k = 0; same && k < b - a; k++) {
            if (idx[a + k] != nidx[na + k]) same = 0;
            else if (w && nw && w[a + k] != nw[na + k]) same = 0;
        }
        if (same) continue;
        changed++;
        for (int64_t e = a; e < b; e++) F[idx[e]] -= d * H[j] * p_entry(W, w, j, e);
        for (int64_t e = na; e < nb; e++) F[nidx[e]] += d * H[j] * p_entry(NW, nw, j, e);
    }
    free(W);
    free(NW);
    return changed;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the PageRank solve (not in the paper; the backward pass of      */
/* x = (1 - d)(I - d P)^-1 Z for a loss L = g . x).  lambda solves             */
/* (I - d P)^T lambda = g, i.e. lambda = g + d P^T lambda, whose Neumann       */
/* series sum_k d^k (P^T)^k g converges because every row of P^T sums to at    */
/* most 1 (the columns of P do, Section 2.1): |P^T v|_inf <= |v|_inf.          */
/* Plain Jacobi sweeps lambda_{k+1} = g + d P^T lambda_k from lambda_0 = g,    */
/* with (P^T lambda)_j = sum over links j -> i of P[i][j] lambda_i formed row  */
/* by row of the out-CSR.  |lambda - lambda_k|_inf <= d/(1-d) |lambda_k -      */
/* lambda_{k-1}|_inf, so the loop stops once that bound is at most tol.        */
/* Returns the number of sweeps, or OR_BAD_INPUT.                              */
/* ------------------------------------------------------------------------- */
int64_t or_adjoint_jacobi(int64_t n, const int64_t *ptr, const int32_t *idx, const double *w, double d,
                          const double *g, double tol, int64_t max_iters, double *lambda)
{
    if (n < 1 || !(d > 0.0 && d < 1.0) || !(tol > 0.0)) return OR_BAD_INPUT;
    double *W = row_scale(n, ptr, w);
    double *next = malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; i++) lambda[i] = g[i];
    int64_t it = 0;
    while (it < max_iters) {
        double change = 0.0;
        for (int64_t j = 0; j < n; j++) {
            double s = 0.0;
            for (int64_t e = ptr[j]; e < ptr[j + 1]; e++) s += p_entry(W, w, j, e) * lambda[idx[e]];
            next[j] = g[j] + d * s;
            double c = fabs(next[j] - lambda[j]);
            if (c > change) change = c;
        }
        memcpy(lambda, next, sizeof(double) * (size_t)n);
        it++;
        if (d / (1.0 - d) * change <= tol) break;
    }
    free(next);
    free(W);
    return it;
}

/* Gradient of L = g . x with respect to the link weights (not in the paper). */
/* With P[i][j] = w(j,i) / W_j (Section 2.1, Eq. def-p), W_j = sum_k w(j,k):  */
/*   dL/dP[a][b] = d lambda_a x_b, and dP[i][j]/dw(j,k) = [i = k]/W_j -       */
/*   w(j,i)/W_j^2, so dL/dw(j,k) = d x_j / W_j (lambda_k - (P^T lambda)_j).   */
/* grad has one entry per link of the canonical out-CSR, in its order; an     */
/* unweighted graph is treated as all weights 1.  dL/dZ = (1 - d) lambda.      */
void or_grad_w(int64_t n, const int64_t *ptr, const int32_t *idx, const double *w, double d,
               const double *x, const double *lambda, double *grad)
{
    double *W = row_scale(n, ptr, w);
    for (int64_t j = 0; j < n; j++) {
        if (ptr[j + 1] == ptr[j]) continue;
        double s = 0.0;
        for (int64_t e = ptr[j]; e < ptr[j + 1]; e++) s += p_entry(W, w, j, e) * lambda[idx[e]];
        for (int64_t e = ptr[j]; e < ptr[j + 1]; e++) grad[e] = d * x[j] / W[j] * (lambda[idx[e]] - s);
    }
    free(W);
}
