/*
 * nmf.h -- C-ABI of the GB300 E-A-HALS library (libnmf_gb300.so).
 *
 * Solves  min ||X - WH||_F^2  s.t. W >= 0, H >= 0                 (Eq. 1)
 * with X in R^{m x n}, W in R^{m x r}, H in R^{r x n}, by the extrapolated
 * accelerated HALS method of Ang & Gillis, "Accelerating Nonnegative Matrix
 * Factorization Algorithms using Extrapolation" (arXiv 1805.06604):
 * Algorithm 2 (extrapolation with restarts, variants hp = 1, 2, 3), the beta
 * schedule of Algorithm 3, A-HALS inner loops built on the closed-form row
 * update of Sec. 1, and the cheap error of Remark 1.
 *
 * Conventions for every call:
 *  - Matrices are row-major FP32: X is m x n (leading dimension ld >= n) or
 *    CSR; W is m x r (W[i*r+k]); H is r x n (H[k*n+j]).
 *  - A pointer argument marked "host or device" is read according to the
 *    accompanying on_device / to_device flag.  The library never keeps or
 *    frees a caller's pointer: X, W0 and H0 are copied into library-owned
 *    device buffers during nmf_create.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work of a handle is enqueued on the stream given
 *    at creation; calls that return host data synchronise that stream.
 *  - Every call returns an nmf_status; no C++ exception crosses the ABI and
 *    no call exits the process.  nmf_last_error() gives a message for the
 *    last failing call on the calling thread.
 *  - The library runs only on sm_103a (GB300).  There is no CPU fallback:
 *    without a usable CUDA device, nmf_create returns NMF_ECUDA.
 */
#ifndef NMF_GB300_H
#define NMF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NMF_OK = 0,
    NMF_EINVAL = 1,      /* bad argument (shape, pointer, parameter range)   */
    NMF_ENOMEM = 2,      /* device or host allocation failed                  */
    NMF_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed       */
    NMF_ENONFINITE = 4,  /* NaN/Inf in the input or in the error e(k)         */
    NMF_ETIMEOUT = 5,    /* a bounded device-side wait expired                */
    NMF_ENOTSUP = 6      /* valid request outside this build (e.g. r > 128)  */
} nmf_status;

typedef enum { NMF_DENSE = 0, NMF_CSR = 1 } nmf_format;

/* Arithmetic of the two X products (W^T X and X H^T) and of the Gram
 * G = W_y^T W_y.  In the tensor-core modes G is formed on the tensor cores
 * from the same rounded factor W_y' as the product W_y'^T X; the Gram
 * D = H_y H_y^T stays an error-free accumulation on the CUDA cores in every
 * mode (Remark 1's error cancels ||X||^2 and needs D to ~2^-40).  Sweeps
 * and extrapolation are FP32 in every mode; the error terms are accumulated
 * in FP64 (Remark 1). */
typedef enum {
    NMF_PREC_FP32 = 0,   /* FP32 FMA on CUDA cores                            */
    NMF_PREC_TF32 = 1,   /* TF32 tensor cores (tcgen05), FP32 accumulate; the
                            library also keeps X^T (dense X only)             */
    NMF_PREC_BF16X3 = 2  /* split BF16 (hi/lo pairs of X, X^T and the factor),
                            three tcgen05 products, FP32 accumulate (dense X) */
} nmf_precision;

typedef struct {
    int32_t format;          /* nmf_format                                    */
    int32_t on_device;       /* 1: pointers below are device memory; 0: host  */
    int64_t m, n;            /* rows, columns                                 */
    int64_t ld;              /* dense: row stride in elements (>= n); 0 = n   */
    int64_t nnz;             /* CSR: number of stored entries                 */
    const float *values;     /* dense m x ld, or CSR values[nnz]              */
    const int64_t *rowptr;   /* CSR: m+1 offsets, rowptr[0] = 0, nondecreasing */
    const int32_t *colidx;   /* CSR: nnz column indices in [0, n)             */
} nmf_matrix;

typedef struct {
    int32_t hp;              /* Algorithm 2 variant: 1, 2 or 3 (default 3)    */
    double beta0;            /* Algorithm 3 initial beta, in [0, 1] (0.5).
                                beta0 = 0 gives un-extrapolated A-HALS (Sec. 2) */
    double eta;              /* shrink factor on restart (1.5)                */
    double gamma;            /* growth factor of beta (1.01)                  */
    double gamma_bar;        /* growth factor of beta_bar (1.005);
                                1 < gamma_bar < gamma < eta is required        */
    int32_t lw, lh;          /* inner HALS sweeps on W / on H; 0 = the A-HALS
                                budget floor(1 + alpha*rho) of Gillis & Glineur
                                (2012), computed by nmf_sweep_counts            */
    double alpha;            /* alpha of that budget (0.5)                    */
    int32_t project_w;       /* 1: W_y = max(0, W_y) after extrapolation (the
                                paper's Algorithm 2 does not project W_y; 0)  */
    int32_t compare_prev;    /* 1 (default): restart when e(k) > e(k-1), the
                                error the previous iteration computed, whether
                                it was accepted or not (Algorithm 2 step 16 as
                                written); 0: when e(k) exceeds the error of
                                the last accepted iterate (an option)          */
    int32_t precision;       /* nmf_precision (NMF_PREC_FP32)                 */
    int64_t trace_capacity;  /* initial device trace length (0 = 4096); grows */
    int32_t line_search_trace; /* 1: also record, every iteration, the exact
                                line-search step beta* of Sec. 3 for the
                                W-update (a diagnostic: one more r x r product
                                per row of W; nmf_get_line_search_trace); 0  */
    double delta;            /* A-HALS inner stopping rule (Gillis & Glineur
                                2012, cited in Sec. 1): 0 (default) runs
                                exactly lw / lh sweeps; delta > 0 stops the
                                loop after sweep l >= 2 once
                                ||X^(l) - X^(l-1)||_F <= delta ||X^(1) - X^(0)||_F,
                                lw / lh then being the caps (one launch per
                                sweep; nmf_info reports the sweeps run)       */
    int32_t exact_nnls;      /* 1: solve both NNLS subproblems exactly (ANLS,
                                Sec. 1 -- with extrapolation, E-ANLS) by block
                                principal pivoting, one warp per column of H /
                                row of W, instead of lh / lw HALS sweeps
                                (lw, lh, alpha unused; r <= 112); 0          */
} nmf_params;

typedef struct {
    int64_t k;               /* outer iterations done                         */
    double e_last;           /* error of the last accepted iterate            */
    double e_k;              /* e(k) of the last iteration (accepted or not)  */
    double fro2;             /* ||X||_F^2                                     */
    double relerr;           /* e_last / ||X||_F                              */
    double beta, beta_bar, beta_prev;  /* Algorithm 3 state for iteration k+1 */
    int32_t accepted;        /* decision of the last iteration                */
    int32_t lw, lh;          /* sweep budgets in use                          */
    int32_t device_status;   /* sticky device-side status (nmf_status)        */
    int32_t launches_per_iter; /* kernels one outer iteration launches        */
    int32_t lh_used, lw_used; /* sweeps on H / W in the last iteration (lh / lw
                                unless delta > 0)                              */
    int32_t exact_failed;    /* exact_nnls: 1 once an item's free block was not
                                positive definite or did not settle in
                                100 (r + 1) exchanges (the item then kept its
                                last iterate, as the paper's solver would)    */
} nmf_info;

typedef struct {
    int64_t iters;           /* iterations run by this call                   */
    double relerr;           /* ||X - W H||_F / ||X||_F of the returned pair
                                (W, H) at return (nmf_eval_error)             */
    double relerr_last;      /* e_last / ||X||_F at return: e(k) of the last
                                accepted iteration, ||X - W_n H_y||_F, which
                                for hp >= 2 is not the error of (W, H)        */
    double seconds;          /* wall time of the call                         */
    int32_t reached;         /* 1 when relerr <= target was observed          */
    int32_t timed_out;       /* 1 when max_seconds ended the call early       */
} nmf_result;

typedef struct nmf_handle nmf_handle;

/* Fills *p with the defaults above (the paper's final E-A-HALS settings,
 * Sec. 4.3.2: hp = 3, beta0 = 0.5, eta = 1.5, gamma = 1.01,
 * gamma_bar = 1.005). */
nmf_status nmf_params_default(nmf_params *p);

/* A-HALS inner-sweep budget (Gillis & Glineur 2012, cited in Sec. 1):
 * rho_W = 1 + (K + n r)/(m (r+1)), L_W = floor(1 + alpha rho_W);
 * rho_H = 1 + (K + m r)/(n (r+1)), L_H = floor(1 + alpha rho_H);
 * K = stored entries of X (m n if dense).  Pure host arithmetic. */
nmf_status nmf_sweep_counts(int64_t m, int64_t n, int64_t K, int32_t r,
                            double alpha, int32_t *lw, int32_t *lh);

/* Creates a solver: validates the inputs, copies X, W0 (m x r) and H0
 * (r x n) to the device (factors_on_device selects how W0/H0 are read),
 * computes ||X||_F^2 and e(0) = ||X - W0 H0||_F (Algorithm 2, step 1) and
 * sets W_y = W0, H_y = H0, beta = beta0, beta_bar = 1.
 * Errors: NMF_EINVAL for m, n, r < 1, a malformed CSR, hp outside {1,2,3},
 * parameters outside 0 <= beta0 <= 1 and 1 < gamma_bar < gamma < eta,
 * negative or non-finite W0/H0; NMF_ENONFINITE for NaN/Inf in X;
 * NMF_ENOTSUP for r > 128; NMF_ENOMEM / NMF_ECUDA from the device.
 * On failure *out is set to NULL and nothing is leaked. */
nmf_status nmf_create(nmf_handle **out, const nmf_matrix *X, int32_t r,
                      const float *W0, const float *H0,
                      int32_t factors_on_device, const nmf_params *p,
                      void *stream);

/* Enqueues `iters` outer iterations of Algorithm 2 (steps 3-20) with the
 * beta update of Algorithm 3 on the handle's stream.  The restart decisions
 * and the beta schedule run on the device.  With last == NULL there is no
 * host synchronisation and no device-to-host traffic; otherwise the call
 * synchronises the stream and fills *last as nmf_get_info does (e(k), the
 * beta used and the decision of the last iteration among them).
 * Errors: NMF_EINVAL for iters < 0; NMF_ECUDA from a launch. */
nmf_status nmf_step(nmf_handle *h, int32_t iters, nmf_info *last);

/* The error of the pair (W, H) the handle would return (the accepted
 * iterate, Algorithm 2 step 19): err = ||X - W H||_F and relerr =
 * err / ||X||_F, by Remark 1 (||X||^2 - 2<W, X H^T> + <W^T W, H H^T>, in
 * the residual form of e(k)) from a fresh product X H^T (FP32 with
 * compensated sums, in every precision mode) and H H^T accumulated
 * error-free.  e(k) itself is ||X - W_n H_y||_F (step 15), which differs
 * from this for hp >= 2.  Costs one pass over X; synchronises the stream.
 * Either output may be NULL.  Errors: NMF_ENONFINITE, NMF_ECUDA. */
nmf_status nmf_eval_error(nmf_handle *h, double *err, double *relerr);

/* Runs Algorithm 2 for up to max_iters iterations in chunks of
 * `check_every` (>= 1), the way the paper's experiments stop (Sec. 4: a
 * target error or a fixed time budget).  After each chunk it synchronises
 * and, when target_relerr > 0, evaluates the returned pair's relative
 * error (nmf_eval_error, one pass over X per check) and stops once it is
 * <= target_relerr; it also stops once max_seconds (> 0) of wall time have
 * passed (0 = no limit).  Fills *res when res != NULL.
 * Errors: NMF_EINVAL for max_iters < 0, check_every < 1, max_seconds < 0;
 * a sticky device status (e.g. NMF_ENONFINITE) is returned as such. */
nmf_status nmf_solve(nmf_handle *h, int64_t max_iters, double target_relerr,
                     double max_seconds, int32_t check_every, nmf_result *res);

/* Synchronises the stream and reports the scalar state of Algorithms 2
 * and 3 (e(k), e_last, beta, beta_bar, beta_{k-1}, the last decision). */
nmf_status nmf_get_info(nmf_handle *h, nmf_info *info);

/* Decision replay: iteration k (0-based count of iterations done) takes
 * the accept (1) / restart (0) decision accepted[k] instead of the test of
 * step 16 of Algorithm 2, for k < count (count = 0 clears it).  Everything
 * else -- e(k), both branches of Algorithm 3 -- runs unchanged, so a run
 * can follow another implementation's sequence of decisions (where e(k)
 * and e(k-1) are within round-off of each other, the two may take
 * different branches and then different paths of the non-convex problem).
 * A non-finite e(k) still restarts.  The array is copied; synchronises the
 * stream.  Errors: NMF_EINVAL, NMF_ENOMEM, NMF_ECUDA. */
nmf_status nmf_set_forced_decisions(nmf_handle *h, const uint8_t *accepted, int64_t count);

/* Copies the accepted iterate (W, H) -- the pair Algorithm 2 returns --
 * into W (m x r) and H (r x n), host or device per to_device.  Either
 * pointer may be NULL to skip it.  Synchronises the stream. */
nmf_status nmf_get_factors(nmf_handle *h, float *W, float *H,
                           int32_t to_device);

/* Copies the extrapolated pair (W_y, H_y) that the next iteration starts
 * from.  Same conventions as nmf_get_factors. */
nmf_status nmf_get_extrapolated(nmf_handle *h, float *Wy, float *Hy,
                                int32_t to_device);

/* Copies the per-iteration trace to host arrays of length `cap`: e(k), the
 * beta_k used by iteration k, and the accept (1) / restart (0) decision.
 * Any of the three pointers may be NULL.  *len receives min(k, cap).
 * Entry k is written by iteration k; after nmf_set_state moved k forward,
 * the entries of iterations this handle did not run are undefined. */
nmf_status nmf_get_trace(nmf_handle *h, double *e, double *beta,
                         uint8_t *accepted, int64_t cap, int64_t *len);

/* Sec. 3: beta*(k) = <X - W_n H_y, (W_n - W) H_y> / ||(W_n - W) H_y||_F^2,
 * the step that minimises ||X - (W_n + beta (W_n - W)) H_y||_F over beta
 * for iteration k's W-update (W the accepted iterate before it, W_n its
 * result, H_y the H it used), 0 when (W_n - W) H_y = 0.  Evaluated on the
 * device without another pass over X: the numerator is
 * -<W_n D - C, W_n - W> and the denominator sum_i (W_n - W)_i D
 * (W_n - W)_i^T with C = X H_y^T and D = H_y H_y^T of that iteration.
 * Copies min(iterations done, cap) values to host beta_star[]; *len gets
 * the count (entries of iterations this handle did not run, after
 * nmf_set_state, are undefined, as in nmf_get_trace).  NMF_ENOTSUP unless
 * the handle was created with line_search_trace = 1. */
nmf_status nmf_get_line_search_trace(nmf_handle *h, double *beta_star, int64_t cap,
                                     int64_t *len);

/* Full solver state for checkpoint/resume and for replaying a step from an
 * identical state: the pairs (W, H) and (W_y, H_y) of Algorithm 2 and the
 * scalars of Algorithm 3 (beta, beta_bar, beta_{k-1}) with e_last / e(k-1).
 * The four factor arrays are host or device per on_device; sizes as above.
 * nmf_get_state synchronises; any array may be NULL to skip it.
 * nmf_set_state needs all four; it resets the sticky device status. */
typedef struct {
    double beta, beta_bar, beta_prev;  /* Algorithm 3 */
    double e_last;           /* error the next e(k) is compared with          */
    double e_prev;           /* e(k-1) as computed                            */
    int64_t k;               /* iterations done                               */
} nmf_scalars;

nmf_status nmf_get_state(nmf_handle *h, nmf_scalars *s, float *W, float *H,
                         float *Wy, float *Hy, int32_t to_device);
nmf_status nmf_set_state(nmf_handle *h, const nmf_scalars *s, const float *W,
                         const float *H, const float *Wy, const float *Hy,
                         int32_t on_device);

/* Phases of one outer iteration, in launch order (nmf_profile_phases). */
typedef enum {
    NMF_PHASE_GRAM_W = 0,    /* G = W_y^T W_y                                 */
    NMF_PHASE_WTX = 1,       /* A = W_y^T X            (streams X)            */
    NMF_PHASE_HALS_H = 2,    /* H sweeps + extrapolate/project H (steps 3-9)  */
    NMF_PHASE_GRAM_H = 3,    /* D = H_y H_y^T                                 */
    NMF_PHASE_XHT = 4,       /* C = X H_y^T            (streams X)            */
    NMF_PHASE_HALS_W = 5,    /* W sweeps + e(k), restart decision, Alg. 3     */
    NMF_PHASE_FINALIZE = 6,  /* extrapolate W (and H for hp = 1), accept/restart */
    NMF_NUM_PHASES = 7
} nmf_phase;

/* Runs `iters` (>= 1) real outer iterations WITHOUT the CUDA graph, with a
 * CUDA event recorded on the handle's stream between consecutive phases,
 * and writes the mean device time of each phase in milliseconds to
 * ms[NMF_NUM_PHASES].  The iterations advance the solver exactly like
 * nmf_step.  Synchronises the stream. */
nmf_status nmf_profile_phases(nmf_handle *h, int32_t iters, double *ms);

/* out = P Q^T on the tensor cores, the product kernel of the TF32 and
 * BF16X3 precision modes (C = X H^T in the solver).  Device pointers: P is
 * M x K (row stride ldp), Q is q_rows x K (row stride ldq), out is
 * M x q_rows (row stride ldo), all FP32 row-major; ldp and ldq multiples of
 * 8; 1 <= q_rows <= 128.  precision is NMF_PREC_TF32 (operands read as
 * TF32) or NMF_PREC_BF16X3 (P and Q split into hi/lo BF16, three products,
 * FP32 accumulation).  Allocates its temporaries and synchronises `stream`.
 * Errors: NMF_EINVAL for bad shapes, NMF_ENOTSUP for other precisions,
 * NMF_ETIMEOUT when a bounded pipeline wait expired. */
nmf_status nmf_matmul_nt(const float *P, int64_t M, int64_t K, int64_t ldp, const float *Q,
                         int32_t q_rows, int64_t ldq, float *out, int64_t ldo,
                         int32_t precision, void *stream);

/* Failure detection (the paper has no counterpart): every wait inside the
 * tensor-core product kernel is bounded; when one runs out the kernel
 * records it, drains its own copies and MMAs, frees its tensor memory and
 * returns, and the call reports NMF_ETIMEOUT (nmf_matmul_nt) or the
 * handle's device_status becomes NMF_ETIMEOUT.  This hook lets a test make
 * one such wait run out on purpose without faulting anything: with
 * extra > 0, the last CTA of a tile shared by several CTAs waits, in its
 * final segment (no copy or MMA of it in flight), for `extra` partials that
 * never arrive, so the bounded wait (about 0.1 s) expires.  extra = 0
 * (the default) restores normal operation.  Applies to the current device;
 * launches already enqueued are not affected predictably, so set it between
 * synchronised calls.  A handle whose product timed out keeps stale tile
 * counters: destroy it.  Errors: NMF_EINVAL for extra < 0, NMF_ECUDA. */
nmf_status nmf_debug_set_fixup_stall(int32_t extra);

/* Releases every device and host resource of the handle (NULL is a no-op).
 * Synchronises the stream first. */
nmf_status nmf_destroy(nmf_handle *h);

/* ||X||_F^2 of a device matrix (m x n, row stride ld >= n, FP32), written to
 * the device double *out on `stream`, without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate at the point of use -- code whose device memory is owned
 * by another framework's allocator, or latency-critical loops where a
 * cudaMalloc could block.  Its partial sums live in a fixed 128 KiB
 * __device__ array inside the library, so: m*n is limited to 2^28 entries
 * (NMF_ENOTSUP beyond that); calls whose kernels overlap on the GPU race on
 * that array and must be serialised by the caller; the first call on each
 * device resolves the array's address (make it before any stream capture).
 * Inputs and output are the caller's device buffers.  Errors: NMF_EINVAL
 * for NULL pointers or bad shapes, NMF_ECUDA for launch failures. */
nmf_status nmf_fro2_noalloc(const float *X, int64_t m, int64_t n, int64_t ld,
                            double *out, void *stream);

/* ---- Batched solver: many independent problems of uneven size. ---------
 * Each instance is a full solver (as nmf_create).  One outer iteration of
 * every instance is captured into a single CUDA graph, in one of two forms:
 *  - grouped: one launch per phase of Algorithm 2 and kernel variant covers
 *    all instances (a device table gives every CTA its instance and its
 *    index within it), so an iteration of hundreds of instances is a few
 *    dozen launches; available when every instance is dense, FP32, without
 *    the delta rule and without exact NNLS;
 *  - chains: every instance's own kernels form a chain, and the chains are
 *    spread over B concurrent graph branches (longest first).
 * Both forms run each instance's kernels with the tiles, splits and CTAs of
 * its single solver, so results are bit-identical to nmf_step on that
 * instance.  The form, the branches, and the grouped form's columns of H
 * per sweep CTA are picked at creation by timing candidate graphs (the
 * tuning iterations are undone from a device snapshot).  All work goes on
 * `stream`. */
typedef struct nmf_batch nmf_batch;

/* A schedule of the batched graph. */
typedef struct nmf_batch_plan {
    int32_t grouped;           /* 1: grouped launches, 0: per-instance chains   */
    int32_t branches;          /* chains: concurrent branches (1..64); grouped:
                                  branches the launches of one phase are spread
                                  over (1..64)                                   */
    int32_t h_cols_per_cta;    /* grouped: columns of H per CTA of the H sweeps
                                  (1..32; 0 = the single solver's 32)            */
    int32_t launches_per_iter; /* out: kernel launches per outer iteration      */
    double ms_per_iter;        /* out: measured by the tuner (0 if set by hand) */
} nmf_batch_plan;

/* Xs[i], ranks[i], W0[i] (m_i x r_i), H0[i] (r_i x n_i) describe instance
 * i; p applies to all (sweep budgets computed per instance when 0).
 * Errors as nmf_create, reported with the failing instance index. */
nmf_status nmf_batch_create(nmf_batch **out, int32_t count, const nmf_matrix *Xs,
                            const int32_t *ranks, const float *const *W0,
                            const float *const *H0, int32_t factors_on_device,
                            const nmf_params *p, void *stream);
/* As nmf_batch_create, but instance i runs with its own parameters
 * params[i] (count entries; e.g. the grid of hp, beta0, eta, gamma and
 * gamma_bar values of the paper's sensitivity study, Sec. 4.2, run on the
 * same data in one graph).  params is borrowed during the call;
 * NMF_EINVAL when it is NULL, otherwise errors as nmf_batch_create. */
nmf_status nmf_batch_create_params(nmf_batch **out, int32_t count, const nmf_matrix *Xs,
                                   const int32_t *ranks, const float *const *W0,
                                   const float *const *H0, int32_t factors_on_device,
                                   const nmf_params *params, void *stream);
/* `iters` outer iterations of every instance: one graph launch each. */
nmf_status nmf_batch_step(nmf_batch *b, int32_t iters);
/* The same iterations as a per-instance launch loop (each instance's own
 * one-iteration graph, one after another): the baseline the batched graph
 * is measured against.  Results are identical to nmf_batch_step. */
nmf_status nmf_batch_step_loop(nmf_batch *b, int32_t iters);
nmf_status nmf_batch_get_info(nmf_batch *b, int32_t i, nmf_info *info);
nmf_status nmf_batch_get_factors(nmf_batch *b, int32_t i, float *W, float *H,
                                 int32_t to_device);
/* The autotuner's choice: branches and its measured ms per iteration. */
nmf_status nmf_batch_schedule(nmf_batch *b, int32_t *branches, double *ms_per_iter);
/* The schedule in use (all fields). */
nmf_status nmf_batch_get_plan(nmf_batch *b, nmf_batch_plan *plan);
/* Rebuilds the graph with the given schedule (grouped, branches,
 * h_cols_per_cta; the out fields are ignored).  Errors: NMF_EINVAL for NULL
 * or out-of-range fields, NMF_ENOTSUP for grouped when an instance is not
 * dense FP32 HALS, NMF_ECUDA for capture failures. */
nmf_status nmf_batch_set_plan(nmf_batch *b, const nmf_batch_plan *plan);
nmf_status nmf_batch_destroy(nmf_batch *b);

/* Message of the last failing call on this thread ("" if none). */
const char *nmf_last_error(void);

/* Library version string. */
const char *nmf_version(void);

#ifdef __cplusplus
}
#endif
#endif
