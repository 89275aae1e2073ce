/*
 * oracle.h -- plain, slow FP64 CPU oracle for E-A-HALS (Ang & Gillis,
 * "Accelerating Nonnegative Matrix Factorization Algorithms using
 * Extrapolation", arXiv 1805.06604).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library under
 * paper_1805_06604_gb300/ includes, links or calls this code; only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg do.  It shares
 * no source, header, table or helper with the CUDA path.
 *
 * Every routine is a direct transcription of a definition in the paper, in
 * double precision, with plain loops and no blocking or reordering beyond
 * what the definition states.  Each function cites the passage it follows.
 *
 * Layouts (all row-major, all owned by the caller):
 *   X : m x n   dense (ld = n) or CSR (rowptr[m+1], colidx[nnz], val[nnz])
 *   W : m x r   W[i*r + k]
 *   H : r x n   H[k*n + j]
 *   A : r x n   A = W^T X
 *   C : m x r   C = X H^T
 *   G, D : r x r
 */
#ifndef EAHALS_ORACLE_H
#define EAHALS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int64_t m, n;
    int is_csr;               /* 0: dense row-major, 1: CSR            */
    const double *x;          /* dense values, m*n                      */
    const int64_t *rowptr;    /* CSR row pointers, m+1                  */
    const int32_t *colidx;    /* CSR column indices, nnz                */
    const double *val;        /* CSR values, nnz                        */
} orc_matrix;

typedef struct {
    int hp;                   /* Algorithm 2 variant, 1, 2 or 3          */
    double beta0;             /* Algorithm 3 initial beta                */
    double eta;               /* Algorithm 3 shrink factor               */
    double gamma;             /* Algorithm 3 growth factor of beta       */
    double gamma_bar;         /* Algorithm 3 growth factor of beta_bar   */
    int lw, lh;               /* inner HALS sweeps on W and on H         */
    int project_w;            /* 1: W_y = max(0, W_y) after extrapolation */
    int compare_prev;         /* 1: restart iff e(k) > e(k-1), e(k-1) the
                                 error the previous iteration computed,
                                 accepted or not (Alg. 2 step 16 as
                                 written); 0: iff e(k) exceeds the error
                                 of the last accepted iterate (option)   */
    int nnls_exact;           /* 1: solve both NNLS subproblems exactly
                                 (ANLS, Sec. 1; with extrapolation:
                                 E-ANLS) instead of lh / lw HALS sweeps  */
    double delta;             /* 0: exactly lh / lw sweeps; > 0: the
                                 A-HALS stopping rule (lh / lw as caps) */
} orc_params;

typedef struct {
    double beta;              /* beta_k used by the next iteration       */
    double beta_bar;          /* upper bound of Algorithm 3              */
    double beta_prev;         /* beta_{k-1}                              */
    double e_last;            /* error the next e(k) is compared with    */
    double e_prev;            /* e(k-1) as computed (accepted or not)    */
    int64_t k;                /* iterations done                         */
    int lh_used, lw_used;     /* sweeps the last iteration ran           */
} orc_scalars;

/* Threads used by the parallel loops (OpenMP; results do not depend on
 * it).  orc_set_threads(n <= 0) leaves the setting unchanged. */
void orc_set_threads(int n);
int orc_get_threads(void);

/* ||X||_F^2 (Remark 1). */
double orc_fro2(const orc_matrix *X);

/* A = W^T X, r x n (the W(:,k)^T X term of the HALS closed form, Sec. 1). */
void orc_wtx(const orc_matrix *X, int r, const double *W, double *A);

/* C = X H^T, m x r (the X H^T term of Remark 1). */
void orc_xht(const orc_matrix *X, int r, const double *H, double *C);

/* G = W^T W (r x r) and D = H H^T (r x r). */
void orc_gram_w(int64_t m, int r, const double *W, double *G);
void orc_gram_h(int64_t n, int r, const double *H, double *D);

/* One closed-form update of row k of H (Sec. 1, HALS):
 *   H(k,:) = max(0, (A(k,:) - sum_{j != k} G(k,j) H(j,:)) / G(k,k)).
 * Skipped (row unchanged) when G(k,k) == 0. */
void orc_hals_row_h(int64_t n, int r, const double *A, const double *G,
                    double *H, int k);

/* One closed-form update of column k of W (the symmetric update):
 *   W(:,k) = max(0, (C(:,k) - sum_{j != k} W(:,j) D(j,k)) / D(k,k)). */
void orc_hals_col_w(int64_t m, int r, const double *C, const double *D,
                    double *W, int k);

/* A-HALS inner loops: `sweeps` cyclic passes k = 0..r-1 (Sec. 1). */
void orc_hals_sweeps_h(int64_t n, int r, const double *A, const double *G,
                       double *H, int sweeps);
void orc_hals_sweeps_w(int64_t m, int r, const double *C, const double *D,
                       double *W, int sweeps);

/* A-HALS with the inner stopping rule of Gillis & Glineur (2012, the
 * A-HALS paper cited in Sec. 1): after sweep l >= 2 the loop stops once
 * ||H^(l) - H^(l-1)||_F <= delta ||H^(1) - H^(0)||_F; at most max_sweeps.
 * Returns the number of sweeps done. */
int orc_hals_sweeps_h_delta(int64_t n, int r, const double *A, const double *G,
                            double *H, int max_sweeps, double delta);
int orc_hals_sweeps_w_delta(int64_t m, int r, const double *C, const double *D,
                            double *W, int max_sweeps, double delta);

/* Exact NNLS, min_{x >= 0} 1/2 x^T G x - b^T x (G = W^T W, b = W^T v), by
 * block principal pivoting (the active-set-like method of Kim & Park that
 * the paper uses for ANLS, Sec. 1).  x: warm start in, solution out.
 * Indices with G_ii = 0 keep their value.  Returns the number of exchanges,
 * -1 if max_iter is reached or a free block is singular. */
int orc_nnls(int r, const double *G, const double *b, double *x, int max_iter);

/* ANLS subproblems solved exactly: every column of H (G, A = W^T X) and
 * every row of W (D, C = X H^T), warm-started from H / W. */
int orc_nnls_h(int64_t n, int r, const double *A, const double *G, double *H);
int orc_nnls_w(int64_t m, int r, const double *C, const double *D, double *W);

/* Remark 1: ||X - WH||^2 = ||X||^2 - 2<W, X H^T> + <W^T W, H H^T>,
 * with C = X H^T and D = H H^T given. */
double orc_err2_expanded(double fro2, int64_t m, int r, const double *W,
                         const double *C, const double *D);

/* ||X - WH||_F^2 computed entry by entry (O(mnr)); zeros of a CSR X count. */
double orc_err2_direct(const orc_matrix *X, int r, const double *W,
                       const double *H);

/* Inner sweep budget of A-HALS (Gillis & Glineur 2012, cited in Sec. 1):
 * rho_W = 1 + (K + n r) / (m (r + 1)),  L_W = floor(1 + alpha rho_W),
 * rho_H = 1 + (K + m r) / (n (r + 1)),  L_H = floor(1 + alpha rho_H),
 * K = number of stored entries of X. */
void orc_sweep_counts(int64_t m, int64_t n, int64_t K, int r, double alpha,
                      int *lw, int *lh);

/* Algorithm 3: beta update after iteration k; `decreased` is 1 when the
 * error decreased (the iterate was accepted). */
void orc_beta_update(const orc_params *p, orc_scalars *s, int decreased);

/* Algorithm 2, step 1: W_y = W, H_y = H, e(0) = ||X - WH||_F; Algorithm 3,
 * line 1: beta_bar = 1.  Fills *s. */
void orc_eahals_init(const orc_matrix *X, int r, const double *W,
                     const double *H, double *Wy, double *Hy,
                     const orc_params *p, orc_scalars *s);

/* One outer iteration of Algorithm 2 (steps 3-20) with Algorithm 3.
 * State (W, H, Wy, Hy, *s) is updated in place.  `force` < 0 lets the
 * error test decide; 0 / 1 forces restart / accept (decision replay).
 * Outputs e(k), the beta used, the decision and (when beta_star_out is
 * not NULL) the line-search step of Sec. 3 for this iteration's W-update
 * (orc_line_search_beta of W, W_n and the H_y the W-update used).
 * fro2 = ||X||_F^2. */
void orc_eahals_step(const orc_matrix *X, int r, double fro2, double *W,
                     double *H, double *Wy, double *Hy, const orc_params *p,
                     orc_scalars *s, int force, double *e_out,
                     double *beta_out, int *accepted_out, double *beta_star_out);

/* Sec. 3: beta* = argmin_beta ||X - (W_n + beta (W_n - W)) H_y||_F^2
 *       = <X - W_n H_y, (W_n - W) H_y> / ||(W_n - W) H_y||_F^2,
 * evaluated entry by entry (O(mnr)); 0 when (W_n - W) H_y = 0. */
double orc_line_search_beta(const orc_matrix *X, int r, const double *W,
                            const double *Wn, const double *Hy);

/* `iters` outer iterations; traces (length iters) may be NULL. */
void orc_eahals_run(const orc_matrix *X, int r, double *W, double *H,
                    double *Wy, double *Hy, const orc_params *p,
                    orc_scalars *s, int iters, const int8_t *forced,
                    double *trace_e, double *trace_beta,
                    uint8_t *trace_acc);

/* Un-extrapolated A-HALS (Algorithm 1 with HALS inner loops, H first then
 * W, matching the order of Algorithm 2): `iters` outer iterations. */
void orc_ahals_run(const orc_matrix *X, int r, double *W, double *H,
                   int lw, int lh, int iters, double *trace_e);

#ifdef __cplusplus
}
#endif
#endif
