/*
 * oracle.c -- FP64 reference for E-A-HALS, written from the paper
 * (Ang & Gillis, arXiv 1805.06604).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the
 * benchmark's CPU-baseline leg.  It shares nothing with the CUDA library.
 *
 * Plain loops in double precision; the only freedom taken is the loop
 * nesting of sums whose order the paper does not fix.  Build with
 * -ffp-contract=off so that x86-64 and aarch64 give identical bits.
 *
 * Threads (OpenMP): only loops over independent outputs run in parallel --
 * columns of A = W^T X, rows of C = X H^T, entries of a Gram, columns of H
 * and rows of W in the sweeps and the exact NNLS, rows of the direct error
 * -- and every output keeps the sequential summation order, so the result
 * does not depend on the number of threads.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static double *orc_alloc(int64_t count)
{
    double *p = (double *)calloc((size_t)(count > 0 ? count : 1), sizeof(double));
    if (!p) abort();
    return p;
}

/* Remark 1: the constant term ||X||_F^2 = <X, X>. */
double orc_fro2(const orc_matrix *X)
{
    double s = 0.0;
    if (X->is_csr) {
        int64_t nnz = X->rowptr[X->m];
        for (int64_t p = 0; p < nnz; ++p) s += X->val[p] * X->val[p];
    } else {
        for (int64_t i = 0; i < X->m; ++i)
            for (int64_t j = 0; j < X->n; ++j) {
                double v = X->x[i * X->n + j];
                s += v * v;
            }
    }
    return s;
}

/* A(k,j) = sum_i W(i,k) X(i,j): the product W^T X of the HALS closed form
 * (Sec. 1).  Summed over i in increasing order. */
void orc_wtx(const orc_matrix *X, int r, const double *W, double *A)
{
    const int64_t m = X->m, n = X->n;
    memset(A, 0, sizeof(double) * (size_t)r * (size_t)n);
    if (X->is_csr) {
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = X->rowptr[i]; p < X->rowptr[i + 1]; ++p) {
                int64_t j = X->colidx[p];
                for (int k = 0; k < r; ++k) A[k * n + j] += W[i * r + k] * X->val[p];
            }
        return;
    }
    /* Dense: column blocks in parallel; each A(k,j) still sums over i in
     * increasing order. */
    const int64_t cb = 256;
    #pragma omp parallel for schedule(dynamic)
    for (int64_t j0 = 0; j0 < n; j0 += cb) {
        const int64_t j1 = j0 + cb < n ? j0 + cb : n;
        for (int64_t i = 0; i < m; ++i)
            for (int k = 0; k < r; ++k) {
                double w = W[i * r + k];
                for (int64_t j = j0; j < j1; ++j) A[k * n + j] += w * X->x[i * n + j];
            }
    }
}

/* C(i,k) = sum_j X(i,j) H(k,j): the product X H^T of Remark 1. */
void orc_xht(const orc_matrix *X, int r, const double *H, double *C)
{
    const int64_t m = X->m, n = X->n;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        for (int k = 0; k < r; ++k) {
            double s = 0.0;
            if (X->is_csr) {
                for (int64_t p = X->rowptr[i]; p < X->rowptr[i + 1]; ++p)
                    s += X->val[p] * H[k * n + X->colidx[p]];
            } else {
                for (int64_t j = 0; j < n; ++j) s += X->x[i * n + j] * H[k * n + j];
            }
            C[i * r + k] = s;
        }
    }
}

/* G(k,j) = W(:,k)^T W(:,j). */
void orc_gram_w(int64_t m, int r, const double *W, double *G)
{
    #pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < r; ++k)
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int64_t i = 0; i < m; ++i) s += W[i * r + k] * W[i * r + j];
            G[k * r + j] = s;
        }
}

/* D(k,j) = H(k,:) H(j,:)^T. */
void orc_gram_h(int64_t n, int r, const double *H, double *D)
{
    #pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < r; ++k)
        for (int j = 0; j < r; ++j) {
            double s = 0.0;
            for (int64_t c = 0; c < n; ++c) s += H[k * n + c] * H[j * n + c];
            D[k * r + j] = s;
        }
}

/* HALS closed form for row k of H (Sec. 1, second line of the display):
 *   H(k,:) = max(0, (W(:,k)^T X - sum_{j != k} (W(:,k)^T W(:,j)) H(j,:))
 *                    / ||W(:,k)||^2)
 * with A = W^T X and G = W^T W, so ||W(:,k)||^2 = G(k,k).  A zero
 * denominator (the paper does not treat it) leaves the row unchanged. */
static void hals_row_h_cols(int64_t n, int r, const double *A, const double *G,
                            double *H, int k, int64_t c0, int64_t c1)
{
    const double gkk = G[k * r + k];
    if (!(gkk > 0.0)) return;
    for (int64_t c = c0; c < c1; ++c) {
        double s = A[k * n + c];
        for (int j = 0; j < r; ++j) {
            if (j == k) continue;
            s -= G[k * r + j] * H[j * n + c];
        }
        double v = s / gkk;
        H[k * n + c] = v > 0.0 ? v : 0.0;
    }
}

void orc_hals_row_h(int64_t n, int r, const double *A, const double *G,
                    double *H, int k)
{
    hals_row_h_cols(n, r, A, G, H, k, 0, n);
}

/* The same closed form for column k of W, from the symmetry
 * ||X - WH|| = ||X^T - H^T W^T|| (Sec. 1):
 *   W(:,k) = max(0, (X H(k,:)^T - sum_{j != k} W(:,j) (H(j,:) H(k,:)^T))
 *                    / ||H(k,:)||^2)
 * with C = X H^T and D = H H^T. */
static void hals_col_w_rows(int r, const double *C, const double *D, double *W, int k,
                            int64_t i0, int64_t i1)
{
    const double dkk = D[k * r + k];
    if (!(dkk > 0.0)) return;
    for (int64_t i = i0; i < i1; ++i) {
        double s = C[i * r + k];
        for (int j = 0; j < r; ++j) {
            if (j == k) continue;
            s -= W[i * r + j] * D[j * r + k];
        }
        double v = s / dkk;
        W[i * r + k] = v > 0.0 ? v : 0.0;
    }
}

void orc_hals_col_w(int64_t m, int r, const double *C, const double *D,
                    double *W, int k)
{
    hals_col_w_rows(r, C, D, W, k, 0, m);
}

/* A-HALS: the rows of H are updated in cyclic order, and the whole pass is
 * repeated `sweeps` times reusing W^T W and W^T X (Sec. 1, second bullet).
 * A column of H only ever reads itself, A and G, so blocks of columns run
 * the whole sequence independently (in parallel); each column sees exactly
 * the sequential order of updates. */
void orc_hals_sweeps_h(int64_t n, int r, const double *A, const double *G,
                       double *H, int sweeps)
{
    const int64_t cb = 64;
    #pragma omp parallel for schedule(dynamic)
    for (int64_t c0 = 0; c0 < n; c0 += cb) {
        const int64_t c1 = c0 + cb < n ? c0 + cb : n;
        for (int l = 0; l < sweeps; ++l)
            for (int k = 0; k < r; ++k) hals_row_h_cols(n, r, A, G, H, k, c0, c1);
    }
}

void orc_hals_sweeps_w(int64_t m, int r, const double *C, const double *D,
                       double *W, int sweeps)
{
    const int64_t rb = 64;
    #pragma omp parallel for schedule(dynamic)
    for (int64_t i0 = 0; i0 < m; i0 += rb) {
        const int64_t i1 = i0 + rb < m ? i0 + rb : m;
        for (int l = 0; l < sweeps; ++l)
            for (int k = 0; k < r; ++k) hals_col_w_rows(r, C, D, W, k, i0, i1);
    }
}

/* The inner stopping rule of A-HALS (Gillis & Glineur 2012, cited in
 * Sec. 1): sweep after sweep, ||X^(l) - X^(l-1)||_F^2 is summed over all
 * coordinates (per column / row in index order, then the columns / rows in
 * order) and the loop stops after sweep l >= 2 once it is at most
 * delta^2 ||X^(1) - X^(0)||_F^2. */
static double sq_change(const double *a, const double *b, int64_t count)
{
    double s = 0.0;
    for (int64_t q = 0; q < count; ++q) {
        const double d = a[q] - b[q];
        s += d * d;
    }
    return s;
}

int orc_hals_sweeps_h_delta(int64_t n, int r, const double *A, const double *G,
                            double *H, int max_sweeps, double delta)
{
    double *prev = orc_alloc((int64_t)r * n), first = 0.0;
    int l = 0;
    while (l < max_sweeps) {
        memcpy(prev, H, sizeof(double) * (size_t)r * (size_t)n);
        orc_hals_sweeps_h(n, r, A, G, H, 1);
        ++l;
        const double d2 = sq_change(H, prev, (int64_t)r * n);
        if (l == 1) first = d2;
        else if (d2 <= delta * delta * first) break;
    }
    free(prev);
    return l;
}

int orc_hals_sweeps_w_delta(int64_t m, int r, const double *C, const double *D,
                            double *W, int max_sweeps, double delta)
{
    double *prev = orc_alloc(m * (int64_t)r), first = 0.0;
    int l = 0;
    while (l < max_sweeps) {
        memcpy(prev, W, sizeof(double) * (size_t)m * (size_t)r);
        orc_hals_sweeps_w(m, r, C, D, W, 1);
        ++l;
        const double d2 = sq_change(W, prev, m * (int64_t)r);
        if (l == 1) first = d2;
        else if (d2 <= delta * delta * first) break;
    }
    free(prev);
    return l;
}

/* Solves G_FF z = c for the free set F (Cholesky of the |F| x |F| block,
 * FP64).  F given as a list of nf indices.  Returns 0, or -1 when the block
 * is not positive definite. */
static int orc_solve_free(int r, const double *G, const double *c, const int *F, int nf,
                          double *z)
{
    double *L = orc_alloc((int64_t)nf * nf);
    for (int a = 0; a < nf; ++a) {
        for (int b = 0; b <= a; ++b) {
            double v = G[F[a] * r + F[b]];
            for (int q = 0; q < b; ++q) v -= L[a * nf + q] * L[b * nf + q];
            if (a == b) {
                if (!(v > 0.0)) {
                    free(L);
                    return -1;
                }
                L[a * nf + a] = sqrt(v);
            } else {
                L[a * nf + b] = v / L[b * nf + b];
            }
        }
    }
    for (int a = 0; a < nf; ++a) {           /* L y = c_F */
        double v = c[F[a]];
        for (int q = 0; q < a; ++q) v -= L[a * nf + q] * z[q];
        z[a] = v / L[a * nf + a];
    }
    for (int a = nf - 1; a >= 0; --a) {      /* L^T z = y */
        double v = z[a];
        for (int q = a + 1; q < nf; ++q) v -= L[q * nf + a] * z[q];
        z[a] = v / L[a * nf + a];
    }
    free(L);
    return 0;
}

/* Exact NNLS of the ANLS subproblems (Sec. 1, "solved exactly"):
 *   min_{x >= 0} 1/2 x^T G x - b^T x,  G = W^T W (r x r), b = W^T v,
 * i.e. min_{x >= 0} ||v - W x||^2, by block principal pivoting (Kim & Park,
 * the active-set-like method the paper uses): a free set F and its
 * complement, x_F = G_FF^{-1} b_F, x = 0 off F, y = G x - b (zero on F);
 * the infeasible indices {i in F: x_i < 0} and {i not in F: y_i < 0} all
 * change sides while their number keeps falling, with up to three further
 * full exchanges allowed, otherwise only the largest such index changes
 * side.  The KKT point (x >= 0, y >= 0, x_i y_i = 0) is the unique minimiser
 * when G is positive definite.  Comparisons use a tolerance of 1e-12 times
 * the scale of b and G (FP64 round-off at a degenerate optimum).  Indices
 * with G_ii = 0 (a zero column of W: the whole row of G is zero) do not
 * enter the problem and keep their value in x.  x holds the warm start on
 * entry (its support is the first free set) and the solution on return.
 * Returns the number of exchanges, or -1 when max_iter is reached or a free
 * block is singular (x is then the last iterate). */
int orc_nnls(int r, const double *G, const double *b, double *x, int max_iter)
{
    int *free_ = (int *)calloc((size_t)r, sizeof(int));
    int *act = (int *)calloc((size_t)r, sizeof(int));   /* index takes part */
    int *F = (int *)malloc(sizeof(int) * (size_t)(r > 0 ? r : 1));
    double *z = orc_alloc(r > 0 ? r : 1), *y = orc_alloc(r > 0 ? r : 1);
    double scale = 0.0;
    for (int i = 0; i < r; ++i) {
        act[i] = G[i * r + i] > 0.0;
        if (act[i]) free_[i] = x[i] > 0.0;
        if (fabs(b[i]) > scale) scale = fabs(b[i]);
        if (fabs(G[i * r + i]) > scale) scale = fabs(G[i * r + i]);
    }
    const double tol = 1e-12 * (scale > 0.0 ? scale : 1.0);
    int best = r + 1, alpha = 3, it = 0, status = -1;
    for (;;) {
        /* Solve on the free set; y on its complement. */
        int nf = 0;
        for (int i = 0; i < r; ++i)
            if (act[i] && free_[i]) F[nf++] = i;
        if (orc_solve_free(r, G, b, F, nf, z) != 0) break;
        for (int i = 0; i < r; ++i)
            if (act[i]) x[i] = 0.0;
        for (int a = 0; a < nf; ++a) x[F[a]] = z[a];
        for (int i = 0; i < r; ++i) {
            y[i] = 0.0;
            if (!act[i] || free_[i]) continue;
            double v = -b[i];
            for (int a = 0; a < nf; ++a) v += G[i * r + F[a]] * z[a];
            y[i] = v;
        }
        /* Infeasible indices. */
        int nv = 0, last = -1;
        for (int i = 0; i < r; ++i) {
            if (!act[i]) continue;
            const int bad = free_[i] ? (x[i] < -tol) : (y[i] < -tol);
            if (bad) {
                ++nv;
                last = i;
            }
        }
        if (nv == 0) {
            status = it;
            break;
        }
        if (it >= max_iter) break;
        ++it;
        if (nv < best) {
            best = nv;
            alpha = 3;
        } else if (alpha >= 1) {
            alpha -= 1;
        } else {
            free_[last] = !free_[last];   /* backup rule: the largest index only */
            continue;
        }
        for (int i = 0; i < r; ++i) {
            if (!act[i]) continue;
            const int bad = free_[i] ? (x[i] < -tol) : (y[i] < -tol);
            if (bad) free_[i] = !free_[i];
        }
    }
    /* Clamp the round-off negatives a converged free set may carry. */
    if (status >= 0)
        for (int i = 0; i < r; ++i)
            if (act[i] && x[i] < 0.0) x[i] = 0.0;
    free(free_);
    free(act);
    free(F);
    free(z);
    free(y);
    return status;
}

/* Exact subproblems of ANLS: every column of H (G = W^T W, b = A[:, j])
 * and every row of W (G = D, b = C[i, :]), warm-started from the values
 * held in H and W.  Returns the largest exchange count, -1 on failure. */
static int worse(int a, int b) { return (a < 0 || b < 0) ? -1 : (a > b ? a : b); }

int orc_nnls_h(int64_t n, int r, const double *A, const double *G, double *H)
{
    int worst = 0;
    #pragma omp parallel
    {
        double *b = orc_alloc(r), *x = orc_alloc(r);
        int mine = 0;
        #pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < n; ++j) {
            for (int k = 0; k < r; ++k) {
                b[k] = A[k * n + j];
                x[k] = H[k * n + j];
            }
            mine = worse(mine, orc_nnls(r, G, b, x, 100 * (r + 1)));
            for (int k = 0; k < r; ++k) H[k * n + j] = x[k];
        }
        #pragma omp critical
        worst = worse(worst, mine);
        free(b);
        free(x);
    }
    return worst;
}

int orc_nnls_w(int64_t m, int r, const double *C, const double *D, double *W)
{
    int worst = 0;
    #pragma omp parallel
    {
        int mine = 0;
        #pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < m; ++i)
            mine = worse(mine, orc_nnls(r, D, C + i * r, W + i * r, 100 * (r + 1)));
        #pragma omp critical
        worst = worse(worst, mine);
    }
    return worst;
}

/* Remark 1: ||X||^2 - 2 <W, X H^T> + <W^T W, H H^T>. */
double orc_err2_expanded(double fro2, int64_t m, int r, const double *W,
                         const double *C, const double *D)
{
    double cross = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int k = 0; k < r; ++k) cross += W[i * r + k] * C[i * r + k];
    double *G = orc_alloc((int64_t)r * r);
    orc_gram_w(m, r, W, G);
    double quad = 0.0;
    for (int k = 0; k < r; ++k)
        for (int j = 0; j < r; ++j) quad += G[k * r + j] * D[k * r + j];
    free(G);
    return fro2 - 2.0 * cross + quad;
}

/* sum_{i,j} (X(i,j) - (WH)(i,j))^2, every entry formed explicitly. */
double orc_err2_direct(const orc_matrix *X, int r, const double *W,
                       const double *H)
{
    const int64_t m = X->m, n = X->n;
    double *rows = orc_alloc(m);     /* sum over row i, j ascending */
    #pragma omp parallel
    {
        double *row = orc_alloc(n);
        #pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                double wh = 0.0;
                for (int k = 0; k < r; ++k) wh += W[i * r + k] * H[k * n + j];
                row[j] = -wh;
            }
            if (X->is_csr) {
                for (int64_t p = X->rowptr[i]; p < X->rowptr[i + 1]; ++p)
                    row[X->colidx[p]] += X->val[p];
            } else {
                for (int64_t j = 0; j < n; ++j) row[j] += X->x[i * n + j];
            }
            double t = 0.0;
            for (int64_t j = 0; j < n; ++j) t += row[j] * row[j];
            rows[i] = t;
        }
        free(row);
    }
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += rows[i];
    free(rows);
    return s;
}

/* The exact line-search step of Sec. 3 for the W-update: with
 * W_y(beta) = W_n + beta (W_n - W),
 *   beta* = <X - W_n H_y, (W_n - W) H_y> / ||(W_n - W) H_y||_F^2,
 * both inner products formed entry by entry over X (zeros of a CSR X
 * count).  0 when (W_n - W) H_y = 0. */
double orc_line_search_beta(const orc_matrix *X, int r, const double *W,
                            const double *Wn, const double *Hy)
{
    const int64_t m = X->m, n = X->n;
    double *nums = orc_alloc(m), *dens = orc_alloc(m);   /* per row, j ascending */
    #pragma omp parallel
    {
        double *res = orc_alloc(n), *dir = orc_alloc(n);
        #pragma omp for schedule(dynamic, 8)
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t j = 0; j < n; ++j) {
                double wh = 0.0, dh = 0.0;
                for (int k = 0; k < r; ++k) {
                    wh += Wn[i * r + k] * Hy[k * n + j];
                    dh += (Wn[i * r + k] - W[i * r + k]) * Hy[k * n + j];
                }
                res[j] = -wh;
                dir[j] = dh;
            }
            if (X->is_csr) {
                for (int64_t p = X->rowptr[i]; p < X->rowptr[i + 1]; ++p)
                    res[X->colidx[p]] += X->val[p];
            } else {
                for (int64_t j = 0; j < n; ++j) res[j] += X->x[i * n + j];
            }
            double a = 0.0, b = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                a += res[j] * dir[j];
                b += dir[j] * dir[j];
            }
            nums[i] = a;
            dens[i] = b;
        }
        free(res);
        free(dir);
    }
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        num += nums[i];
        den += dens[i];
    }
    free(nums);
    free(dens);
    return den > 0.0 ? num / den : 0.0;
}

void orc_sweep_counts(int64_t m, int64_t n, int64_t K, int r, double alpha,
                      int *lw, int *lh)
{
    double rho_w = 1.0 + ((double)K + (double)n * r) / ((double)m * (r + 1));
    double rho_h = 1.0 + ((double)K + (double)m * r) / ((double)n * (r + 1));
    *lw = (int)floor(1.0 + alpha * rho_w);
    *lh = (int)floor(1.0 + alpha * rho_h);
}

/* Algorithm 3.  On decrease: beta_{k+1} = min(beta_bar, gamma beta_k), then
 * beta_bar = min(1, gamma_bar beta_bar).  Otherwise: beta_{k+1} =
 * beta_k / eta and beta_bar = beta_{k-1}. */
void orc_beta_update(const orc_params *p, orc_scalars *s, int decreased)
{
    double next;
    if (decreased) {
        double grown = p->gamma * s->beta;
        next = grown < s->beta_bar ? grown : s->beta_bar;
        double bar = p->gamma_bar * s->beta_bar;
        s->beta_bar = bar < 1.0 ? bar : 1.0;
    } else {
        next = s->beta / p->eta;
        s->beta_bar = s->beta_prev;
    }
    s->beta_prev = s->beta;
    s->beta = next;
}

void orc_eahals_init(const orc_matrix *X, int r, const double *W,
                     const double *H, double *Wy, double *Hy,
                     const orc_params *p, orc_scalars *s)
{
    const int64_t m = X->m, n = X->n;
    memcpy(Wy, W, sizeof(double) * (size_t)(m * r));
    memcpy(Hy, H, sizeof(double) * (size_t)(r * n));
    double fro2 = orc_fro2(X);
    double *C = orc_alloc(m * r), *D = orc_alloc((int64_t)r * r);
    orc_xht(X, r, H, C);
    orc_gram_h(n, r, H, D);
    double e2 = orc_err2_expanded(fro2, m, r, W, C, D);
    free(C);
    free(D);
    double e0 = sqrt(e2 > 0.0 ? e2 : 0.0);
    s->beta = p->beta0;
    s->beta_bar = 1.0;
    s->beta_prev = p->beta0;
    s->e_last = e0;
    s->e_prev = e0;
    s->k = 0;
    s->lh_used = s->lw_used = 0;
}

/* One outer iteration of Algorithm 2 (steps 3 to 20) plus Algorithm 3. */
void orc_eahals_step(const orc_matrix *X, int r, double fro2, double *W,
                     double *H, double *Wy, double *Hy, const orc_params *p,
                     orc_scalars *s, int force, double *e_out,
                     double *beta_out, int *accepted_out, double *beta_star_out)
{
    const int64_t m = X->m, n = X->n;
    const double beta = s->beta;
    double *A = orc_alloc(r * n), *G = orc_alloc((int64_t)r * r);
    double *C = orc_alloc(m * r), *D = orc_alloc((int64_t)r * r);
    double *Hn = orc_alloc(r * n), *Wn = orc_alloc(m * r);
    double *Hw = orc_alloc(r * n);     /* the H that the W-update sees */
    double *Wy_new = orc_alloc(m * r), *Hy_new = orc_alloc(r * n);

    /* Step 3: H_n from NNLS on ||X - W_y H_n|| warm-started at H_y. */
    orc_wtx(X, r, Wy, A);
    orc_gram_w(m, r, Wy, G);
    memcpy(Hn, Hy, sizeof(double) * (size_t)(r * n));
    if (p->nnls_exact) orc_nnls_h(n, r, A, G, Hn);     /* E-ANLS: exact */
    else if (p->delta > 0.0) s->lh_used = orc_hals_sweeps_h_delta(n, r, A, G, Hn, p->lh, p->delta);
    else orc_hals_sweeps_h(n, r, A, G, Hn, p->lh);

    /* Steps 4-9: for hp >= 2, H_y = H_n + beta (H_n - H), projected when
     * hp = 3.  For hp = 1 the W-update uses H_n (H is extrapolated only
     * after it, as a warm start for the next H-update). */
    for (int64_t q = 0; q < r * n; ++q) {
        if (p->hp >= 2) {
            double v = Hn[q] + beta * (Hn[q] - H[q]);
            if (p->hp == 3) v = v > 0.0 ? v : 0.0;
            Hw[q] = v;
        } else {
            Hw[q] = Hn[q];
        }
    }

    /* Step 10: W_n from NNLS on ||X - W_n H_y|| warm-started at W_y. */
    orc_xht(X, r, Hw, C);
    orc_gram_h(n, r, Hw, D);
    memcpy(Wn, Wy, sizeof(double) * (size_t)(m * r));
    if (p->nnls_exact) orc_nnls_w(m, r, C, D, Wn);
    else if (p->delta > 0.0) s->lw_used = orc_hals_sweeps_w_delta(m, r, C, D, Wn, p->lw, p->delta);
    else orc_hals_sweeps_w(m, r, C, D, Wn, p->lw);

    /* The line-search step of Sec. 3 for this W-update (a diagnostic). */
    if (beta_star_out) *beta_star_out = orc_line_search_beta(X, r, W, Wn, Hw);

    /* Step 15 via Remark 1, reusing X H_y^T and H_y H_y^T of step 10. */
    double e2 = orc_err2_expanded(fro2, m, r, Wn, C, D);
    double e = sqrt(e2 > 0.0 ? e2 : 0.0);

    /* Step 11: W_y = W_n + beta (W_n - W); step 13 (hp = 1). */
    for (int64_t q = 0; q < m * r; ++q) {
        double v = Wn[q] + beta * (Wn[q] - W[q]);
        if (p->project_w) v = v > 0.0 ? v : 0.0;
        Wy_new[q] = v;
    }
    for (int64_t q = 0; q < r * n; ++q)
        Hy_new[q] = (p->hp == 1) ? Hn[q] + beta * (Hn[q] - H[q]) : Hw[q];

    /* Steps 16-20. */
    double ref = p->compare_prev ? s->e_prev : s->e_last;
    int accept = (force >= 0) ? (force != 0) : !(e > ref);
    if (accept) {
        memcpy(W, Wn, sizeof(double) * (size_t)(m * r));
        memcpy(H, Hn, sizeof(double) * (size_t)(r * n));
        memcpy(Wy, Wy_new, sizeof(double) * (size_t)(m * r));
        memcpy(Hy, Hy_new, sizeof(double) * (size_t)(r * n));
        s->e_last = e;
    } else {
        memcpy(Wy, W, sizeof(double) * (size_t)(m * r));
        memcpy(Hy, H, sizeof(double) * (size_t)(r * n));
    }
    s->e_prev = e;
    orc_beta_update(p, s, accept);
    s->k += 1;

    if (e_out) *e_out = e;
    if (beta_out) *beta_out = beta;
    if (accepted_out) *accepted_out = accept;
    free(A); free(G); free(C); free(D); free(Hn); free(Wn); free(Hw);
    free(Wy_new); free(Hy_new);
}

void orc_eahals_run(const orc_matrix *X, int r, double *W, double *H,
                    double *Wy, double *Hy, const orc_params *p,
                    orc_scalars *s, int iters, const int8_t *forced,
                    double *trace_e, double *trace_beta, uint8_t *trace_acc)
{
    double fro2 = orc_fro2(X);
    for (int it = 0; it < iters; ++it) {
        double e, b;
        int acc;
        orc_eahals_step(X, r, fro2, W, H, Wy, Hy, p, s,
                        forced ? forced[it] : -1, &e, &b, &acc, NULL);
        if (trace_e) trace_e[it] = e;
        if (trace_beta) trace_beta[it] = b;
        if (trace_acc) trace_acc[it] = (uint8_t)acc;
    }
}

void orc_ahals_run(const orc_matrix *X, int r, double *W, double *H,
                   int lw, int lh, int iters, double *trace_e)
{
    const int64_t m = X->m, n = X->n;
    double fro2 = orc_fro2(X);
    double *A = orc_alloc(r * n), *G = orc_alloc((int64_t)r * r);
    double *C = orc_alloc(m * r), *D = orc_alloc((int64_t)r * r);
    for (int it = 0; it < iters; ++it) {
        orc_wtx(X, r, W, A);
        orc_gram_w(m, r, W, G);
        orc_hals_sweeps_h(n, r, A, G, H, lh);
        orc_xht(X, r, H, C);
        orc_gram_h(n, r, H, D);
        orc_hals_sweeps_w(m, r, C, D, W, lw);
        if (trace_e) {
            double e2 = orc_err2_expanded(fro2, m, r, W, C, D);
            trace_e[it] = sqrt(e2 > 0.0 ? e2 : 0.0);
        }
    }
    free(A); free(G); free(C); free(D);
}
