// capi.cu -- the extern "C" boundary of libnmf_gb300 (declared in
// include/nmf.h and include/nmf_ops.h).
//
// One outer iteration of Algorithm 2 (Ang & Gillis, arXiv 1805.06604) is
// the launch sequence
//   G = W_y^T W_y;  A = W_y^T X                        (inputs of step 3)
//   H_n = HALS sweeps from H_y; H_y' = H_n + beta (H_n - H) [hp >= 2]
//                                                       (steps 3-9, fused)
//   D = H_y' H_y'^T;  C = X H_y'^T                      (inputs of step 10)
//   W_n = HALS sweeps from W_y; e(k) by Remark 1; restart decision and
//   Algorithm 3 in the last CTA                         (steps 10, 15-20)
//   finalize: W_y = W_n + beta (W_n - W), H_y for hp = 1, accept/restart
//                                                       (steps 11-14, 17, 19)
// captured once into a CUDA graph and replayed by nmf_step.  Nothing in the
// loop reads back to the host.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <new>
#include <vector>

#include "common.cuh"
#include "nmf.h"

using namespace nmfg;

namespace {

thread_local char g_err[512] = "";

nmf_status fail(nmf_status s, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
nmf_status fail(nmf_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define NMF_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? NMF_ENOMEM : NMF_ECUDA,          \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                         \
    } while (0)

inline int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace

nmf_status nmfg::set_error(nmf_status s, const char *msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
    return s;
}

struct nmf_handle {
    cudaStream_t st = nullptr;          // caller's stream
    cudaStream_t cap = nullptr;         // private stream used for graph capture
    int64_t m = 0, n = 0, ld = 0, nnz = 0;
    int r = 0, rs = 0;
    int is_csr = 0;
    nmf_params p{};
    int lw = 0, lh = 0;
    // X
    float *X = nullptr;                          // dense m x ld
    int64_t *rowptr = nullptr;                   // CSR of X
    int32_t *colidx = nullptr;
    float *val = nullptr;
    int64_t *colptr = nullptr;                   // CSC of X (CSR of X^T)
    int32_t *rowidx = nullptr;
    float *cval = nullptr;
    int32_t *rowseg = nullptr, *colseg = nullptr;  // row (CSR) / column (CSC) of each entry
    float *Ht = nullptr;                         // n x rs transpose of H_y' (CSR path)
    float *carry = nullptr;                      // chunk partials of the CSR products
    // factors and products
    float *W = nullptr, *H = nullptr, *Wy = nullptr, *Hy = nullptr;
    float *Wn = nullptr, *Hn = nullptr, *Hw = nullptr;
    float *A = nullptr, *C = nullptr, *G = nullptr, *D = nullptr;
    float *C_lo = nullptr, *D_lo = nullptr;      // low parts for the Remark 1 terms
    float *G_lo = nullptr;                       // exact_nnls: low part of G
    // tensor-core precision modes
    int64_t ldm = 0;                             // m rounded up to 8
    float *Wt = nullptr;                          // W_y'^T (rs x ldm), TF32
    // W_y' (m x rs) and H_y' (r x ld): the factors as the tensor cores see
    // them, from which the Grams G and D are formed in those modes.
    float *Wq = nullptr, *Hq = nullptr;
    // Packed X for the tensor-core products: Pc for X H^T (P = X), Pa for
    // X^T W (P = X^T); the _lo arrays hold the BF16X3 low parts.
    void *Pc = nullptr, *Pc_lo = nullptr, *Pa = nullptr, *Pa_lo = nullptr;
    __nv_bfloat16 *Wth = nullptr, *Wtl = nullptr, *Hh = nullptr, *Hl = nullptr;
    unsigned int *tct_c = nullptr, *tct_a = nullptr;
    // Tensor-core Gram G = W_y'^T W_y': W_y'^T packed as P, its workspace
    // and tile tickets.
    void *Pg = nullptr, *Pg_lo = nullptr, *ws_g = nullptr;
    unsigned int *tct_g = nullptr;
    int *tc_err = nullptr;
    double *fro2 = nullptr;
    DevState *state = nullptr;
    ErrPartial *partials = nullptr;
    unsigned int *counter = nullptr;
    unsigned int *tickets = nullptr;             // split-K tickets of W^T X
    unsigned int *xtickets = nullptr;            // split-K tickets of X H^T
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int *flag = nullptr;
    // trace
    double *tr_e = nullptr, *tr_beta = nullptr;
    double *tr_bstar = nullptr;                  // line-search diagnostic (optional)
    unsigned char *tr_acc = nullptr;
    int64_t tr_cap = 0;
    unsigned char *forced = nullptr;             // decision replay (nmf_set_forced_decisions)
    int64_t forced_len = 0;
    double *eval = nullptr;                      // nmf_eval_error: e^2, e of (W, H)
    int *nnls_status = nullptr;                  // exact_nnls: an item did not settle
    // delta rule: per-sweep partials of ||change||^2 (first sweep, two
    // alternating buffers) and the stop flags, H side then W side.
    double *d2 = nullptr;
    int *stopped = nullptr;
    int np_h = 0, np_w = 0;
    int64_t k_enq = 0;                           // iterations enqueued so far
    // graph of one iteration
    cudaGraphExec_t exec = nullptr;
    DevState *h_state = nullptr;                 // pinned mirror for readback
    // The Grams run beside the X products in the iteration graph: their own
    // workspace, a side stream and the fork / join events of the capture.
    float *gws = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev[2] = {}, join_ev[2] = {};
};

namespace {

void free_handle(nmf_handle *h) {
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    void *ptrs[] = {h->X, h->rowptr, h->colidx, h->val, h->colptr, h->rowidx, h->cval, h->rowseg,
                    h->colseg, h->Ht,
                    h->carry,
                    h->W, h->H, h->Wy, h->Hy, h->Wn, h->Hn, h->Hw, h->A, h->C, h->G, h->D,
                    h->C_lo, h->D_lo, h->G_lo, h->Wt, h->Wq, h->Hq, h->Pc, h->Pc_lo, h->Pa, h->Pa_lo, h->Wth,
                    h->Wtl, h->Hh, h->Hl, h->tct_c, h->tct_a, h->tc_err, h->Pg, h->Pg_lo, h->ws_g, h->tct_g,
                    h->fro2, h->state, h->partials, h->counter, h->tickets, h->xtickets, h->ws, h->flag,
                    h->tr_e, h->tr_beta, h->tr_acc, h->tr_bstar, h->forced, h->eval, h->nnls_status, h->d2, h->stopped};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->side) cudaStreamDestroy(h->side);
    for (int i = 0; i < 2; ++i) {
        if (h->fork_ev[i]) cudaEventDestroy(h->fork_ev[i]);
        if (h->join_ev[i]) cudaEventDestroy(h->join_ev[i]);
    }
    if (h->gws) cudaFree(h->gws);
    delete h;
}

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    return e;
}

DevParams dev_params(const nmf_handle *h) {
    DevParams d;
    d.hp = h->p.hp;
    d.project_w = h->p.project_w;
    d.compare_prev = h->p.compare_prev;
    d.eta = h->p.eta;
    d.gamma = h->p.gamma;
    d.gamma_bar = h->p.gamma_bar;
    return d;
}

inline int round16(int r) { return (r + 15) / 16 * 16; }

// X products for the current layout and precision.
cudaError_t enqueue_wtx(nmf_handle *h, const float *Wsrc, cudaStream_t st) {
    if (h->is_csr)
        return launch_wtx_csc(h->colptr, h->rowidx, h->colseg, h->cval, h->n, h->nnz, h->r, h->rs,
                              Wsrc, h->A,
                              h->ld, h->carry, st);
    if (h->p.precision == NMF_PREC_FP32)
        return launch_wtx_f32(h->X, h->m, h->ld, h->ld, h->r, Wsrc, h->rs, h->A, h->ws,
                              h->tickets, st);
    // A^T = X^T W_y' on the tensor cores; W_y'^T was made by enqueue_prep_w.
    (void)Wsrc;
    TcOperands o{};
    if (h->p.precision == NMF_PREC_BF16X3) {
        o.Q = h->Wth;
        o.Q_lo = h->Wtl;
    } else {
        o.Q = h->Wt;
    }
    o.P = h->Pa;
    o.P_lo = h->Pa_lo;
    o.M = h->n;
    o.K = h->m;
    o.ldq = h->ldm;
    o.q_rows = h->r;
    o.N = round16(h->r);
    o.nvalid = h->r;
    return launch_tc_product(o, h->p.precision, true, h->A, h->ld, h->ws, h->tct_a, h->tc_err, st);
}

cudaError_t enqueue_xht(nmf_handle *h, const float *Hsrc, cudaStream_t st) {
    if (h->is_csr) {
        cudaError_t e = launch_transpose_h(Hsrc, h->r, h->n, h->ld, h->Ht, h->rs, st);
        if (e != cudaSuccess) return e;
        return launch_xht_csr(h->rowptr, h->colidx, h->rowseg, h->val, h->m, h->nnz, h->r, h->rs,
                              h->Ht, h->C,
                              h->carry, st);
    }
    if (h->p.precision == NMF_PREC_FP32)
        return launch_xht_f32(h->X, h->m, h->ld, h->r, Hsrc, h->ld, h->C, h->C_lo, h->rs, h->ws,
                              h->xtickets, st);
    // C = X H_y'^T on the tensor cores; H_y' was made by enqueue_prep_h.
    TcOperands o{};
    if (h->p.precision == NMF_PREC_BF16X3) {
        o.Q = h->Hh;
        o.Q_lo = h->Hl;
    } else {
        o.Q = h->Hq;
    }
    o.P = h->Pc;
    o.P_lo = h->Pc_lo;
    o.M = h->m;
    o.K = h->n;
    o.ldq = h->ld;
    o.q_rows = h->r;
    o.N = round16(h->r);
    o.nvalid = h->rs;
    return launch_tc_product(o, h->p.precision, false, h->C, h->rs, h->ws, h->tct_c, h->tc_err, st);
}

bool tc_mode(const nmf_handle *h) { return !h->is_csr && h->p.precision != NMF_PREC_FP32; }

// Tensor-core modes: the operand of the next product, made on st before the
// Gram of the same factor is forked off (both read it).  Returns the matrix
// the Gram is formed from: the factor itself, or its rounded copy.
cudaError_t enqueue_prep_w(nmf_handle *h, const float *Wsrc, cudaStream_t st, const float **gram_src) {
    *gram_src = Wsrc;
    if (!tc_mode(h)) return cudaSuccess;
    *gram_src = h->Wq;
    return launch_tc_prep_w(Wsrc, h->m, h->rs, h->rs, h->p.precision, h->Wq, h->Wt, h->Wth, h->Wtl,
                            h->ldm, st);
}

cudaError_t enqueue_prep_h(nmf_handle *h, const float *Hsrc, cudaStream_t st, const float **gram_src) {
    *gram_src = Hsrc;
    if (!tc_mode(h)) return cudaSuccess;
    *gram_src = h->Hq;
    return launch_tc_prep_h(Hsrc, h->r, h->ld, h->ld, h->p.precision, h->Hq, h->Hh, h->Hl, st);
}

// Tensor-core modes: G = W_y'^T W_y' on the tensor cores, from the same
// rounded factor as the product A = W_y'^T X (W_y'^T packed as P, the
// prepared W_y'^T as Q).  Launched without programmatic dependent launch:
// its P changes every iteration.  (D = H_y' H_y'^T stays an error-free
// accumulation on the CUDA cores: Remark 1's error needs it to ~2^-40.)
cudaError_t enqueue_tc_gram(nmf_handle *h, cudaStream_t st) {
    cudaError_t e = launch_tc_pack(h->Wq, h->m, h->r, h->rs, true, h->p.precision, h->Pg, h->Pg_lo,
                                   st);
    if (e != cudaSuccess) return e;
    TcOperands o{};
    if (h->p.precision == NMF_PREC_BF16X3) {
        o.Q = h->Wth;
        o.Q_lo = h->Wtl;
    } else {
        o.Q = h->Wt;
    }
    o.P = h->Pg;
    o.P_lo = h->Pg_lo;
    o.M = h->r;
    o.K = h->m;
    o.ldq = h->ldm;
    o.q_rows = h->r;
    o.N = round16(h->r);
    o.nvalid = h->r;
    o.no_pdl = 1;
    return launch_tc_product(o, h->p.precision, false, h->G, h->rs, h->ws_g, h->tct_g, h->tc_err,
                             st);
}

// One outer iteration of Algorithm 2, enqueued on st.  When ev != nullptr,
// ev[i] is recorded before phase i and ev[NMF_NUM_PHASES] after the last.
// With `overlap` (the single-instance graph), each Gram runs on the side
// stream beside the X product it is independent of (G = W_y^T W_y beside
// A = W_y^T X, D = H_y H_y^T beside C = X H_y^T); the next sweep waits for
// both.  Without it (per-phase profiling, batched graphs) all runs on st.
cudaError_t enqueue_iteration(nmf_handle *h, cudaStream_t st, cudaEvent_t *ev = nullptr,
                              bool overlap = false) {
    cudaError_t e;
    auto mark = [&](int i) -> cudaError_t {
        return ev ? cudaEventRecord(ev[i], st) : cudaSuccess;
    };
#define NMF_STEP(expr)                \
    do {                              \
        e = (expr);                   \
        if (e != cudaSuccess) return e; \
    } while (0)
    cudaStream_t gs = overlap ? h->side : st;
    // (Tensor-core modes: the operand preparation counts as the Gram phase.)
    NMF_STEP(mark(NMF_PHASE_GRAM_W));
    const float *Wg = nullptr;
    NMF_STEP(enqueue_prep_w(h, h->Wy, st, &Wg));
    if (overlap) {
        NMF_STEP(cudaEventRecord(h->fork_ev[0], st));
        NMF_STEP(cudaStreamWaitEvent(gs, h->fork_ev[0], 0));
    }
    if (tc_mode(h))
        NMF_STEP(enqueue_tc_gram(h, gs));
    else if (h->p.exact_nnls)
        NMF_STEP(launch_gram_rows_exact(Wg, h->m, h->rs, h->r, h->rs, h->G, h->G_lo, h->gws, gs));
    else
        NMF_STEP(launch_gram_rows(Wg, h->m, h->rs, h->r, h->rs, h->G, h->gws, gs));
    if (overlap) NMF_STEP(cudaEventRecord(h->join_ev[0], gs));
    NMF_STEP(mark(NMF_PHASE_WTX));
    NMF_STEP(enqueue_wtx(h, h->Wy, st));
    if (overlap) NMF_STEP(cudaStreamWaitEvent(st, h->join_ev[0], 0));
    NMF_STEP(mark(NMF_PHASE_HALS_H));
    HEpilogue hep{};
    hep.H_acc = h->H;
    hep.Hw = h->p.hp >= 2 ? h->Hw : nullptr;
    hep.state = h->state;
    hep.hp = h->p.hp;
    if (h->p.exact_nnls) {
        NMF_STEP(launch_nnls_h(h->n, h->ld, h->r, h->rs, h->A, h->G, h->Hy, h->Hn, hep,
                               h->nnls_status, st));
    } else if (h->p.delta > 0.0) {
        // The delta rule: one launch per sweep (each returns at once after
        // the rule has stopped the loop), then the extrapolation epilogue.
        NMF_STEP(cudaMemsetAsync(h->stopped, 0, sizeof(int), st));
        double *first = h->d2, *buf = h->d2 + h->np_h;
        for (int l = 1; l <= h->lh; ++l) {
            HEpilogue one{};
            one.stop.l = l;
            one.stop.delta2 = h->p.delta * h->p.delta;
            one.stop.d2_first = first;
            one.stop.d2_prev = l - 1 == 1 ? first : buf + ((l - 1) & 1) * h->np_h;
            one.stop.d2_out = l == 1 ? first : buf + (l & 1) * h->np_h;
            one.stop.nparts = h->np_h;
            one.stop.stopped = h->stopped;
            one.stop.used = &h->state->lh_used;
            NMF_STEP(launch_hals_h(h->n, h->ld, h->r, h->rs, h->A, h->G, l == 1 ? h->Hy : h->Hn,
                                   h->Hn, 1, one, st));
        }
        NMF_STEP(launch_hals_h(h->n, h->ld, h->r, h->rs, h->A, h->G, h->Hn, h->Hn, 0, hep, st));
    } else {
        NMF_STEP(launch_hals_h(h->n, h->ld, h->r, h->rs, h->A, h->G, h->Hy, h->Hn, h->lh, hep, st));
    }
    const float *Hused = h->p.hp >= 2 ? h->Hw : h->Hn;
    NMF_STEP(mark(NMF_PHASE_GRAM_H));
    const float *Hg = nullptr;
    NMF_STEP(enqueue_prep_h(h, Hused, st, &Hg));
    if (overlap) {
        NMF_STEP(cudaEventRecord(h->fork_ev[1], st));
        NMF_STEP(cudaStreamWaitEvent(gs, h->fork_ev[1], 0));
    }
    NMF_STEP(launch_gram_cols(Hg, h->n, h->ld, h->r, h->rs, h->D, h->D_lo, h->gws, gs));
    if (overlap) NMF_STEP(cudaEventRecord(h->join_ev[1], gs));
    NMF_STEP(mark(NMF_PHASE_XHT));
    NMF_STEP(enqueue_xht(h, Hused, st));
    if (overlap) NMF_STEP(cudaStreamWaitEvent(st, h->join_ev[1], 0));
    NMF_STEP(mark(NMF_PHASE_HALS_W));
    WEpilogue wep{};
    wep.C_lo = h->C_lo;
    wep.D_lo = h->D_lo;
    wep.partials = h->partials;
    wep.counter = h->counter;
    wep.state = h->state;
    wep.params = dev_params(h);
    wep.trace.e = h->tr_e;
    wep.trace.beta = h->tr_beta;
    wep.trace.acc = h->tr_acc;
    wep.trace.cap = h->tr_cap;
    wep.trace.bstar = h->tr_bstar;
    wep.trace.forced = h->forced;
    wep.trace.forced_len = h->forced_len;
    wep.W_prev = h->p.line_search_trace ? h->W : nullptr;
    if (h->p.exact_nnls) {
        NMF_STEP(launch_nnls_w(h->m, h->r, h->rs, h->C, h->D, h->Wy, h->Wn, wep, h->nnls_status,
                               st));
    } else if (h->p.delta > 0.0) {
        NMF_STEP(cudaMemsetAsync(h->stopped + 1, 0, sizeof(int), st));
        double *first = h->d2 + 3 * h->np_h, *buf = first + h->np_w;
        for (int l = 1; l <= h->lw; ++l) {
            WEpilogue one{};
            one.stop.l = l;
            one.stop.delta2 = h->p.delta * h->p.delta;
            one.stop.d2_first = first;
            one.stop.d2_prev = l - 1 == 1 ? first : buf + ((l - 1) & 1) * h->np_w;
            one.stop.d2_out = l == 1 ? first : buf + (l & 1) * h->np_w;
            one.stop.nparts = h->np_w;
            one.stop.stopped = h->stopped + 1;
            one.stop.used = &h->state->lw_used;
            NMF_STEP(launch_hals_w(h->m, h->r, h->rs, h->C, h->D, l == 1 ? h->Wy : h->Wn, h->Wn, 1,
                                   one, st));
        }
        NMF_STEP(launch_hals_w(h->m, h->r, h->rs, h->C, h->D, h->Wn, h->Wn, 0, wep, st));
    } else {
        NMF_STEP(launch_hals_w(h->m, h->r, h->rs, h->C, h->D, h->Wy, h->Wn, h->lw, wep, st));
    }
    NMF_STEP(mark(NMF_PHASE_FINALIZE));
    NMF_STEP(launch_finalize(h->m, h->rs, h->r, h->ld, h->W, h->H, h->Wy, h->Hy, h->Wn, h->Hn,
                             h->Hw, h->state, dev_params(h), st));
    NMF_STEP(mark(NMF_NUM_PHASES));
#undef NMF_STEP
    return cudaSuccess;
}

nmf_status build_graph(nmf_handle *h) {
    if (h->exec) {
        cudaGraphExecDestroy(h->exec);
        h->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    NMF_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_iteration(h, h->cap, nullptr, true);
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(NMF_ECUDA, "graph capture of one iteration failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&h->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(NMF_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return NMF_OK;
}

nmf_status ensure_trace(nmf_handle *h, int64_t need) {
    if (need <= h->tr_cap) return NMF_OK;
    int64_t cap = std::max<int64_t>(need, 2 * h->tr_cap);
    double *e = nullptr, *b = nullptr, *bs = nullptr;
    unsigned char *a = nullptr;
    NMF_CUDA(cudaStreamSynchronize(h->st));
    if (dalloc(&e, cap) != cudaSuccess || dalloc(&b, cap) != cudaSuccess ||
        dalloc(&a, cap) != cudaSuccess ||
        (h->p.line_search_trace && dalloc(&bs, cap) != cudaSuccess)) {
        cudaFree(e);
        cudaFree(b);
        cudaFree(a);
        cudaFree(bs);
        return fail(NMF_ENOMEM, "trace allocation of %lld entries failed", (long long)cap);
    }
    if (h->tr_cap > 0) {
        NMF_CUDA(cudaMemcpy(e, h->tr_e, sizeof(double) * h->tr_cap, cudaMemcpyDeviceToDevice));
        NMF_CUDA(cudaMemcpy(b, h->tr_beta, sizeof(double) * h->tr_cap, cudaMemcpyDeviceToDevice));
        NMF_CUDA(cudaMemcpy(a, h->tr_acc, h->tr_cap, cudaMemcpyDeviceToDevice));
        if (bs)
            NMF_CUDA(cudaMemcpy(bs, h->tr_bstar, sizeof(double) * h->tr_cap,
                                cudaMemcpyDeviceToDevice));
    }
    cudaFree(h->tr_e);
    cudaFree(h->tr_beta);
    cudaFree(h->tr_acc);
    cudaFree(h->tr_bstar);
    h->tr_e = e;
    h->tr_beta = b;
    h->tr_acc = a;
    h->tr_bstar = bs;
    h->tr_cap = cap;
    return build_graph(h);
}

cudaMemcpyKind kind_of(int src_dev, int dst_dev) {
    if (src_dev && dst_dev) return cudaMemcpyDeviceToDevice;
    if (src_dev) return cudaMemcpyDeviceToHost;
    if (dst_dev) return cudaMemcpyHostToDevice;
    return cudaMemcpyHostToHost;
}

nmf_status check_params(const nmf_params *p) {
    if (p->hp < 1 || p->hp > 3) return fail(NMF_EINVAL, "hp must be 1, 2 or 3 (got %d)", p->hp);
    if (p->line_search_trace != 0 && p->line_search_trace != 1)
        return fail(NMF_EINVAL, "line_search_trace must be 0 or 1 (got %d)", p->line_search_trace);
    if (!(p->beta0 >= 0.0 && p->beta0 <= 1.0))
        return fail(NMF_EINVAL, "beta0 must lie in [0, 1] (got %g)", p->beta0);
    if (!(1.0 < p->gamma_bar && p->gamma_bar < p->gamma && p->gamma < p->eta))
        return fail(NMF_EINVAL, "Algorithm 3 needs 1 < gamma_bar < gamma < eta (got %g, %g, %g)",
                    p->gamma_bar, p->gamma, p->eta);
    if (p->lw < 0 || p->lh < 0) return fail(NMF_EINVAL, "sweep counts must be >= 0");
    if (p->lw == 0 || p->lh == 0)
        if (!(p->alpha > 0.0)) return fail(NMF_EINVAL, "alpha must be > 0");
    if (!(p->delta >= 0.0) || !(p->delta < 1.0))
        return fail(NMF_EINVAL, "delta must lie in [0, 1) (got %g)", p->delta);
    if (p->exact_nnls != 0 && p->exact_nnls != 1)
        return fail(NMF_EINVAL, "exact_nnls must be 0 or 1 (got %d)", p->exact_nnls);
    if (p->precision < NMF_PREC_FP32 || p->precision > NMF_PREC_BF16X3)
        return fail(NMF_EINVAL, "unknown precision %d", p->precision);
    return NMF_OK;
}

// Host-side CSR validation and transpose (creation-time layout preparation).
nmf_status prepare_csr(const nmf_matrix *X, std::vector<int64_t> &rp, std::vector<int32_t> &ci,
                       std::vector<float> &v, std::vector<int64_t> &cp, std::vector<int32_t> &ri,
                       std::vector<float> &cv) {
    const int64_t m = X->m, n = X->n, nnz = X->nnz;
    rp.resize(m + 1);
    ci.resize(nnz);
    v.resize(nnz);
    cudaMemcpyKind k = X->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    NMF_CUDA(cudaMemcpy(rp.data(), X->rowptr, sizeof(int64_t) * (m + 1), k));
    if (nnz > 0) {
        NMF_CUDA(cudaMemcpy(ci.data(), X->colidx, sizeof(int32_t) * nnz, k));
        NMF_CUDA(cudaMemcpy(v.data(), X->values, sizeof(float) * nnz, k));
    }
    if (rp[0] != 0 || rp[m] != nnz) return fail(NMF_EINVAL, "CSR rowptr must run from 0 to nnz");
    for (int64_t i = 0; i < m; ++i)
        if (rp[i + 1] < rp[i]) return fail(NMF_EINVAL, "CSR rowptr decreases at row %lld", (long long)i);
    for (int64_t q = 0; q < nnz; ++q) {
        if (ci[q] < 0 || ci[q] >= n)
            return fail(NMF_EINVAL, "CSR column index %d out of [0, %lld)", ci[q], (long long)n);
        if (!std::isfinite(v[q])) return fail(NMF_ENONFINITE, "X holds a NaN or Inf");
    }
    // CSC by a stable counting sort on the column (rows stay ascending).
    cp.assign(n + 1, 0);
    for (int64_t q = 0; q < nnz; ++q) cp[ci[q] + 1]++;
    for (int64_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
    ri.resize(nnz);
    cv.resize(nnz);
    std::vector<int64_t> pos(cp.begin(), cp.end() - 1);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
            const int64_t d = pos[ci[q]]++;
            ri[d] = (int32_t)i;
            cv[d] = v[q];
        }
    return NMF_OK;
}

nmf_status check_factor_host(const float *p, int64_t count, const char *name) {
    for (int64_t q = 0; q < count; ++q)
        if (!(p[q] >= 0.0f) || !std::isfinite(p[q]))
            return fail(NMF_EINVAL, "%s must be finite and nonnegative (entry %lld is %g)", name,
                        (long long)q, (double)p[q]);
    return NMF_OK;
}

}  // namespace

extern "C" {

const char *nmf_last_error(void) { return g_err; }

const char *nmf_version(void) { return "nmf_gb300 0.1 (sm_103a)"; }

nmf_status nmf_params_default(nmf_params *p) {
    if (!p) return fail(NMF_EINVAL, "params pointer is NULL");
    memset(p, 0, sizeof(*p));
    p->hp = 3;
    p->beta0 = 0.5;
    p->eta = 1.5;
    p->gamma = 1.01;
    p->gamma_bar = 1.005;
    p->lw = 0;
    p->lh = 0;
    p->alpha = 0.5;
    p->project_w = 0;
    p->compare_prev = 1;
    p->precision = NMF_PREC_FP32;
    p->trace_capacity = 4096;
    p->line_search_trace = 0;
    return NMF_OK;
}

nmf_status nmf_sweep_counts(int64_t m, int64_t n, int64_t K, int32_t r, double alpha,
                            int32_t *lw, int32_t *lh) {
    if (m < 1 || n < 1 || r < 1 || K < 0 || !(alpha > 0.0) || !lw || !lh)
        return fail(NMF_EINVAL, "nmf_sweep_counts: bad arguments");
    const double rho_w = 1.0 + ((double)K + (double)n * r) / ((double)m * (r + 1));
    const double rho_h = 1.0 + ((double)K + (double)m * r) / ((double)n * (r + 1));
    *lw = (int32_t)floor(1.0 + alpha * rho_w);
    *lh = (int32_t)floor(1.0 + alpha * rho_h);
    return NMF_OK;
}

nmf_status nmf_create(nmf_handle **out, const nmf_matrix *X, int32_t r, const float *W0,
                      const float *H0, int32_t factors_on_device, const nmf_params *pin,
                      void *stream) {
    if (!out) return fail(NMF_EINVAL, "out pointer is NULL");
    *out = nullptr;
    if (!X || !W0 || !H0) return fail(NMF_EINVAL, "X, W0 and H0 are required");
    if (X->m < 1 || X->n < 1 || r < 1) return fail(NMF_EINVAL, "m, n and r must be >= 1");
    if (r > kMaxRank) return fail(NMF_ENOTSUP, "r = %d exceeds the build cap %d", r, kMaxRank);
    if (pin && pin->exact_nnls == 1 && r > 112)
        return fail(NMF_ENOTSUP, "exact_nnls supports r <= 112 (got %d)", r);
    if (X->format != NMF_DENSE && X->format != NMF_CSR)
        return fail(NMF_EINVAL, "unknown matrix format %d", X->format);
    if (!X->values) return fail(NMF_EINVAL, "X values pointer is NULL");
    if (X->format == NMF_CSR && (!X->rowptr || (X->nnz > 0 && !X->colidx) || X->nnz < 0))
        return fail(NMF_EINVAL, "CSR X needs rowptr, colidx and nnz >= 0");
    if (X->format == NMF_DENSE && X->ld != 0 && X->ld < X->n)
        return fail(NMF_EINVAL, "dense ld must be >= n");
    nmf_params p;
    if (pin) p = *pin;
    else nmf_params_default(&p);
    nmf_status s = check_params(&p);
    if (s != NMF_OK) return s;

    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        return fail(NMF_ECUDA, "no CUDA device is available (this library has no CPU path)");
    }

    if (p.precision != NMF_PREC_FP32) {
        if (X->format == NMF_CSR)
            return fail(NMF_ENOTSUP, "tensor-core precisions need a dense X");
        if (!tc_available())
            return fail(NMF_ENOTSUP, "the tensor-map driver entry point is unavailable");
    }
    nmf_handle *h = new (std::nothrow) nmf_handle();
    if (!h) return fail(NMF_ENOMEM, "host allocation failed");
    h->st = static_cast<cudaStream_t>(stream);
    h->m = X->m;
    h->n = X->n;
    h->r = r;
    h->rs = (int)round_up(r, 8);
    h->ld = round_up(X->n, 8);
    h->ldm = round_up(X->m, 8);
    h->is_csr = X->format == NMF_CSR;
    h->nnz = h->is_csr ? X->nnz : X->m * X->n;
    h->p = p;
    int32_t lw = p.lw, lh = p.lh;
    if (lw == 0 || lh == 0) {
        int32_t aw, ah;
        nmf_sweep_counts(h->m, h->n, h->nnz, r, p.alpha, &aw, &ah);
        if (lw == 0) lw = aw;
        if (lh == 0) lh = ah;
    }
    h->lw = lw;
    h->lh = lh;

#define NMF_TRY(expr)                         \
    do {                                      \
        nmf_status s_ = (expr);               \
        if (s_ != NMF_OK) {                   \
            free_handle(h);                   \
            return s_;                        \
        }                                     \
    } while (0)
#define NMF_TRYC(call) NMF_TRY([&]() -> nmf_status { NMF_CUDA(call); return NMF_OK; }())

    const int64_t m = h->m, n = h->n, ld = h->ld, rs = h->rs;
    NMF_TRYC(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    NMF_TRYC(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        NMF_TRYC(cudaEventCreateWithFlags(&h->fork_ev[i], cudaEventDisableTiming));
        NMF_TRYC(cudaEventCreateWithFlags(&h->join_ev[i], cudaEventDisableTiming));
    }
    NMF_TRYC(cudaMalloc(&h->gws, std::max(gram_ws_bytes(m, (int)rs), gram_ws_bytes(n, (int)rs))));
    NMF_TRYC(dalloc(&h->W, m * rs));
    NMF_TRYC(dalloc(&h->Wy, m * rs));
    NMF_TRYC(dalloc(&h->Wn, m * rs));
    NMF_TRYC(dalloc(&h->C, m * rs));
    NMF_TRYC(dalloc(&h->C_lo, m * rs));
    NMF_TRYC(dalloc(&h->H, r * ld));
    NMF_TRYC(dalloc(&h->Hy, r * ld));
    NMF_TRYC(dalloc(&h->Hn, r * ld));
    NMF_TRYC(dalloc(&h->Hw, r * ld));
    NMF_TRYC(dalloc(&h->A, r * ld));
    NMF_TRYC(dalloc(&h->G, rs * rs));
    NMF_TRYC(dalloc(&h->D, rs * rs));
    NMF_TRYC(dalloc(&h->D_lo, rs * rs));
    NMF_TRYC(dalloc(&h->G_lo, rs * rs));
    NMF_TRYC(dalloc(&h->fro2, 1));
    NMF_TRYC(dalloc(&h->eval, 2));
    NMF_TRYC(dalloc(&h->nnls_status, 1));
    h->np_h = hals_h_num_ctas(n, r);
    h->np_w = hals_w_num_ctas(m, r);
    NMF_TRYC(dalloc(&h->d2, 3 * (size_t)(h->np_h + h->np_w)));
    NMF_TRYC(dalloc(&h->stopped, 2));
    NMF_TRYC(cudaMemsetAsync(h->nnls_status, 0, sizeof(int), h->st));
    NMF_TRYC(dalloc(&h->state, 1));
    NMF_TRYC(dalloc(&h->flag, 1));
    const int npart = std::max({hals_w_num_ctas(m, r), err_rows_num_ctas(m), anls_num_ctas(m)});
    NMF_TRYC(dalloc(&h->partials, npart));
    NMF_TRYC(dalloc(&h->counter, 1));
    NMF_TRYC(dalloc(&h->tickets, wtx_num_tickets(ld)));
    NMF_TRYC(dalloc(&h->xtickets, xht_num_tickets(m)));
    NMF_TRYC(cudaHostAlloc((void **)&h->h_state, sizeof(DevState), cudaHostAllocDefault));
    size_t ws = std::max(gram_ws_bytes(m, (int)rs), gram_ws_bytes(n, (int)rs));
    ws = std::max(ws, fro2_ws_bytes(m * ld));
    if (!h->is_csr) ws = std::max({ws, wtx_ws_bytes(m, ld, r), xht_ws_bytes(m, ld, r)});
    if (p.precision != NMF_PREC_FP32)
        ws = std::max({ws, tc_ws_bytes(m, n, round16(r), p.precision),
                       tc_ws_bytes(n, m, round16(r), p.precision)});
    h->ws_bytes = ws;
    NMF_TRYC(cudaMalloc(&h->ws, ws));

    cudaStream_t st = h->st;
    for (void *q : {(void *)h->W, (void *)h->Wy, (void *)h->Wn, (void *)h->C, (void *)h->C_lo})
        NMF_TRYC(cudaMemsetAsync(q, 0, sizeof(float) * m * rs, st));
    for (void *q : {(void *)h->H, (void *)h->Hy, (void *)h->Hn, (void *)h->Hw, (void *)h->A})
        NMF_TRYC(cudaMemsetAsync(q, 0, sizeof(float) * r * ld, st));
    NMF_TRYC(cudaMemsetAsync(h->G, 0, sizeof(float) * rs * rs, st));
    NMF_TRYC(cudaMemsetAsync(h->D, 0, sizeof(float) * rs * rs, st));
    NMF_TRYC(cudaMemsetAsync(h->D_lo, 0, sizeof(float) * rs * rs, st));
    NMF_TRYC(cudaMemsetAsync(h->counter, 0, sizeof(unsigned int), st));
    NMF_TRYC(cudaMemsetAsync(h->tickets, 0, sizeof(unsigned int) * wtx_num_tickets(ld), st));
    NMF_TRYC(cudaMemsetAsync(h->xtickets, 0, sizeof(unsigned int) * xht_num_tickets(m), st));
    NMF_TRYC(cudaMemsetAsync(h->flag, 0, sizeof(int), st));
    NMF_TRYC(cudaMemsetAsync(h->state, 0, sizeof(DevState), st));

    // Factors: validate on the host (copying device inputs down), then pack.
    {
        std::vector<float> w(m * r), hh(r * n);
        cudaMemcpyKind kd = factors_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        NMF_TRYC(cudaMemcpy(w.data(), W0, sizeof(float) * m * r, kd));
        NMF_TRYC(cudaMemcpy(hh.data(), H0, sizeof(float) * r * n, kd));
        NMF_TRY(check_factor_host(w.data(), m * r, "W0"));
        NMF_TRY(check_factor_host(hh.data(), r * n, "H0"));
        NMF_TRYC(cudaMemcpy2DAsync(h->W, sizeof(float) * rs, w.data(), sizeof(float) * r,
                                   sizeof(float) * r, m, cudaMemcpyHostToDevice, st));
        NMF_TRYC(cudaMemcpy2DAsync(h->H, sizeof(float) * ld, hh.data(), sizeof(float) * n,
                                   sizeof(float) * n, r, cudaMemcpyHostToDevice, st));
        NMF_TRYC(cudaStreamSynchronize(st));
    }
    NMF_TRYC(cudaMemcpyAsync(h->Wy, h->W, sizeof(float) * m * rs, cudaMemcpyDeviceToDevice, st));
    NMF_TRYC(cudaMemcpyAsync(h->Hy, h->H, sizeof(float) * r * ld, cudaMemcpyDeviceToDevice, st));

    // X.
    if (h->is_csr) {
        std::vector<int64_t> rp, cp;
        std::vector<int32_t> ci, ri;
        std::vector<float> v, cv;
        NMF_TRY(prepare_csr(X, rp, ci, v, cp, ri, cv));
        const int64_t nnz = h->nnz;
        NMF_TRYC(dalloc(&h->rowptr, m + 1));
        NMF_TRYC(dalloc(&h->colidx, nnz));
        NMF_TRYC(dalloc(&h->val, nnz));
        NMF_TRYC(dalloc(&h->colptr, n + 1));
        NMF_TRYC(dalloc(&h->rowidx, nnz));
        NMF_TRYC(dalloc(&h->cval, nnz));
        NMF_TRYC(dalloc(&h->rowseg, nnz));
        NMF_TRYC(dalloc(&h->colseg, nnz));
        NMF_TRYC(dalloc(&h->Ht, n * rs));
        NMF_TRYC(dalloc(&h->carry, csr_carry_floats(nnz, (int)rs)));
        NMF_TRYC(cudaMemsetAsync(h->Ht, 0, sizeof(float) * n * rs, st));
        NMF_TRYC(cudaMemcpyAsync(h->rowptr, rp.data(), sizeof(int64_t) * (m + 1),
                                 cudaMemcpyHostToDevice, st));
        NMF_TRYC(cudaMemcpyAsync(h->colptr, cp.data(), sizeof(int64_t) * (n + 1),
                                 cudaMemcpyHostToDevice, st));
        if (nnz > 0) {
            NMF_TRYC(cudaMemcpyAsync(h->colidx, ci.data(), sizeof(int32_t) * nnz,
                                     cudaMemcpyHostToDevice, st));
            NMF_TRYC(cudaMemcpyAsync(h->val, v.data(), sizeof(float) * nnz,
                                     cudaMemcpyHostToDevice, st));
            NMF_TRYC(cudaMemcpyAsync(h->rowidx, ri.data(), sizeof(int32_t) * nnz,
                                     cudaMemcpyHostToDevice, st));
            NMF_TRYC(cudaMemcpyAsync(h->cval, cv.data(), sizeof(float) * nnz,
                                     cudaMemcpyHostToDevice, st));
            std::vector<int32_t> rsg(nnz), csg(nnz);
            for (int64_t i = 0; i < m; ++i)
                for (int64_t q = rp[i]; q < rp[i + 1]; ++q) rsg[q] = (int32_t)i;
            for (int64_t j = 0; j < n; ++j)
                for (int64_t q = cp[j]; q < cp[j + 1]; ++q) csg[q] = (int32_t)j;
            NMF_TRYC(cudaMemcpyAsync(h->rowseg, rsg.data(), sizeof(int32_t) * nnz,
                                     cudaMemcpyHostToDevice, st));
            NMF_TRYC(cudaMemcpyAsync(h->colseg, csg.data(), sizeof(int32_t) * nnz,
                                     cudaMemcpyHostToDevice, st));
            NMF_TRYC(cudaStreamSynchronize(st));     // rsg, csg leave scope
        }
        NMF_TRYC(cudaStreamSynchronize(st));
        NMF_TRYC(launch_fro2(h->val, 1, nnz, nnz, h->fro2, h->ws, st));
    } else {
        const int64_t xld = X->ld ? X->ld : n;
        NMF_TRYC(dalloc(&h->X, m * ld));
        NMF_TRYC(cudaMemsetAsync(h->X, 0, sizeof(float) * m * ld, st));
        NMF_TRYC(cudaMemcpy2DAsync(h->X, sizeof(float) * ld, X->values, sizeof(float) * xld,
                                   sizeof(float) * n, m,
                                   X->on_device ? cudaMemcpyDeviceToDevice
                                                : cudaMemcpyHostToDevice,
                                   st));
        NMF_TRYC(launch_nonfinite_scan(h->X, m * ld, h->flag, st));
        int bad = 0;
        NMF_TRYC(cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        NMF_TRYC(cudaStreamSynchronize(st));
        if (bad) {
            free_handle(h);
            return fail(NMF_ENONFINITE, "X holds a NaN or Inf");
        }
        NMF_TRYC(launch_fro2(h->X, m, ld, ld, h->fro2, h->ws, st));
        if (p.precision != NMF_PREC_FP32) {
            // Packed copies of X (for X H^T) and X^T (for X^T W), made once.
            const bool bf = p.precision == NMF_PREC_BF16X3;
            const size_t bc = tc_packed_bytes(m, n, p.precision);
            const size_t ba = tc_packed_bytes(n, m, p.precision);
            NMF_TRYC(cudaMalloc(&h->Pc, bc));
            NMF_TRYC(cudaMalloc(&h->Pa, ba));
            if (bf) {
                NMF_TRYC(cudaMalloc(&h->Pc_lo, bc));
                NMF_TRYC(cudaMalloc(&h->Pa_lo, ba));
            }
            NMF_TRYC(launch_tc_pack(h->X, m, n, ld, false, p.precision, h->Pc, h->Pc_lo, st));
            NMF_TRYC(launch_tc_pack(h->X, m, n, ld, true, p.precision, h->Pa, h->Pa_lo, st));
            NMF_TRYC(dalloc(&h->Wt, rs * h->ldm));
            NMF_TRYC(cudaMemsetAsync(h->Wt, 0, sizeof(float) * rs * h->ldm, st));
            NMF_TRYC(dalloc(&h->Wq, m * rs));
            NMF_TRYC(cudaMemsetAsync(h->Wq, 0, sizeof(float) * m * rs, st));
            NMF_TRYC(dalloc(&h->Hq, r * ld));
            NMF_TRYC(cudaMemsetAsync(h->Hq, 0, sizeof(float) * r * ld, st));
            NMF_TRYC(dalloc(&h->tct_c, tc_num_tickets(m)));
            NMF_TRYC(dalloc(&h->tct_a, tc_num_tickets(n)));
            NMF_TRYC(dalloc(&h->tc_err, 1));
            {
                const size_t bg = tc_packed_bytes(r, m, p.precision);
                NMF_TRYC(cudaMalloc(&h->Pg, bg));
                if (p.precision == NMF_PREC_BF16X3) NMF_TRYC(cudaMalloc(&h->Pg_lo, bg));
                NMF_TRYC(cudaMalloc(&h->ws_g, tc_ws_bytes(r, m, round16(r), p.precision)));
                NMF_TRYC(dalloc(&h->tct_g, tc_num_tickets(r)));
                NMF_TRYC(cudaMemsetAsync(h->tct_g, 0, sizeof(unsigned int) * tc_num_tickets(r), st));
            }
            NMF_TRYC(cudaMemsetAsync(h->tct_c, 0, sizeof(unsigned int) * tc_num_tickets(m), st));
            NMF_TRYC(cudaMemsetAsync(h->tct_a, 0, sizeof(unsigned int) * tc_num_tickets(n), st));
            NMF_TRYC(cudaMemsetAsync(h->tc_err, 0, sizeof(int), st));
            if (p.precision == NMF_PREC_BF16X3) {
                NMF_TRYC(dalloc(&h->Wth, rs * h->ldm));
                NMF_TRYC(dalloc(&h->Wtl, rs * h->ldm));
                NMF_TRYC(dalloc(&h->Hh, r * ld));
                NMF_TRYC(dalloc(&h->Hl, r * ld));
                NMF_TRYC(cudaMemsetAsync(h->Wth, 0, sizeof(__nv_bfloat16) * rs * h->ldm, st));
                NMF_TRYC(cudaMemsetAsync(h->Wtl, 0, sizeof(__nv_bfloat16) * rs * h->ldm, st));
                NMF_TRYC(cudaMemsetAsync(h->Hh, 0, sizeof(__nv_bfloat16) * r * ld, st));
                NMF_TRYC(cudaMemsetAsync(h->Hl, 0, sizeof(__nv_bfloat16) * r * ld, st));
            }
        }
    }

    // e(0) = ||X - W H||_F via Remark 1 (Algorithm 2 step 1).
    const float *H0g = nullptr;
    NMF_TRYC(enqueue_prep_h(h, h->H, st, &H0g));
    NMF_TRYC(launch_gram_cols(H0g, n, ld, r, (int)rs, h->D, h->D_lo, h->ws, st));
    NMF_TRYC(enqueue_xht(h, h->H, st));
    NMF_TRYC(launch_init_state(m, r, (int)rs, h->W, h->C, h->C_lo, h->D, h->D_lo, h->fro2,
                               h->state, p.beta0, h->partials, st));
    NMF_TRYC(cudaStreamSynchronize(st));

    int64_t cap = p.trace_capacity > 0 ? p.trace_capacity : 4096;
    NMF_TRY(ensure_trace(h, cap));
    NMF_TRYC(cudaStreamSynchronize(st));
#undef NMF_TRYC
#undef NMF_TRY
    *out = h;
    g_err[0] = 0;
    return NMF_OK;
}

nmf_status nmf_step(nmf_handle *h, int32_t iters, nmf_info *last) {
    if (!h) return fail(NMF_EINVAL, "handle is NULL");
    if (iters < 0) return fail(NMF_EINVAL, "iters must be >= 0");
    nmf_status s = ensure_trace(h, h->k_enq + iters);
    if (s != NMF_OK) return s;
    for (int32_t i = 0; i < iters; ++i) NMF_CUDA(cudaGraphLaunch(h->exec, h->st));
    h->k_enq += iters;
    if (last) return nmf_get_info(h, last);
    return NMF_OK;
}

nmf_status nmf_get_info(nmf_handle *h, nmf_info *info) {
    if (!h || !info) return fail(NMF_EINVAL, "handle and info are required");
    NMF_CUDA(cudaMemcpyAsync(h->h_state, h->state, sizeof(DevState), cudaMemcpyDeviceToHost, h->st));
    NMF_CUDA(cudaStreamSynchronize(h->st));
    const DevState &d = *h->h_state;
    info->k = d.k;
    info->e_last = d.e_last;
    info->e_k = d.e_k;
    info->fro2 = d.fro2;
    info->relerr = d.fro2 > 0.0 ? d.e_last / sqrt(d.fro2) : 0.0;
    info->beta = d.beta;
    info->beta_bar = d.beta_bar;
    info->beta_prev = d.beta_prev;
    info->accepted = d.accepted;
    info->lw = h->lw;
    info->lh = h->lh;
    info->device_status = d.status;
    // dense: gram W (2) + W^T X (1) + H sweeps (1) + gram H (2) + X H^T (1) +
    // W sweeps (1) + finalize (1); CSR: each product is 2 kernels (+ a
    // memset) and X H^T adds the H transpose.
    info->launches_per_iter = h->is_csr ? 12 : 9;
    info->lh_used = h->p.delta > 0.0 ? d.lh_used : (h->p.exact_nnls ? 0 : h->lh);
    info->lw_used = h->p.delta > 0.0 ? d.lw_used : (h->p.exact_nnls ? 0 : h->lw);
    // Tensor-core modes: + the W_y' and H_y' operand preparations.
    if (tc_mode(h)) info->launches_per_iter = 11;
    if (h->p.delta > 0.0 && !h->p.exact_nnls) info->launches_per_iter += h->lh + h->lw;
    {
        int e = 0;
        NMF_CUDA(cudaMemcpy(&e, h->nnls_status, sizeof(int), cudaMemcpyDeviceToHost));
        info->exact_failed = e;
    }
    if (h->tc_err) {
        int e = 0;
        NMF_CUDA(cudaMemcpy(&e, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e && info->device_status == 0) info->device_status = (int32_t)NMF_ETIMEOUT;
    }
    return NMF_OK;
}

nmf_status nmf_eval_error(nmf_handle *h, double *err, double *relerr) {
    if (!h) return fail(NMF_EINVAL, "handle is NULL");
    cudaStream_t st = h->st;
    // C, C_lo, D and D_lo are rebuilt by every iteration before they are
    // read, so they serve as scratch here.  FP32 compensated products in
    // every precision mode: the yardstick is the same for all of them.
    NMF_CUDA(launch_gram_cols(h->H, h->n, h->ld, h->r, h->rs, h->D, h->D_lo, h->ws, st));
    if (h->is_csr) {
        NMF_CUDA(enqueue_xht(h, h->H, st));
    } else {
        NMF_CUDA(launch_xht_f32(h->X, h->m, h->ld, h->r, h->H, h->ld, h->C, h->C_lo, h->rs,
                                h->ws, h->xtickets, st));
    }
    NMF_CUDA(launch_err_rows(h->m, h->r, h->rs, h->W, h->C, h->C_lo, h->D, h->D_lo, h->partials,
                             st));
    NMF_CUDA(launch_pair_error(h->m, h->fro2, h->partials, h->eval, st));
    double out[2] = {0.0, 0.0}, f2 = 0.0;
    NMF_CUDA(cudaMemcpyAsync(out, h->eval, sizeof(out), cudaMemcpyDeviceToHost, st));
    NMF_CUDA(cudaMemcpyAsync(&f2, h->fro2, sizeof(double), cudaMemcpyDeviceToHost, st));
    NMF_CUDA(cudaStreamSynchronize(st));
    if (!std::isfinite(out[0])) return fail(NMF_ENONFINITE, "the error of (W, H) is not finite");
    if (err) *err = out[1];
    if (relerr) *relerr = f2 > 0.0 ? out[1] / sqrt(f2) : 0.0;
    return NMF_OK;
}

nmf_status nmf_solve(nmf_handle *h, int64_t max_iters, double target_relerr, double max_seconds,
                     int32_t check_every, nmf_result *res) {
    if (!h) return fail(NMF_EINVAL, "handle is NULL");
    if (max_iters < 0 || check_every < 1 || !(max_seconds >= 0.0))
        return fail(NMF_EINVAL, "bad max_iters / check_every / max_seconds");
    auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    int64_t done = 0;
    int reached = 0, timed_out = 0;
    double rel = -1.0;
    nmf_info info{};
    nmf_status s;
    while (done < max_iters) {
        const int32_t chunk = (int32_t)std::min<int64_t>(check_every, max_iters - done);
        s = nmf_step(h, chunk, &info);
        if (s != NMF_OK) return s;
        done += chunk;
        if (info.device_status != 0)
            return fail((nmf_status)info.device_status, "device reported status %d after %lld iterations",
                        info.device_status, (long long)info.k);
        if (target_relerr > 0.0) {
            s = nmf_eval_error(h, nullptr, &rel);
            if (s != NMF_OK) return s;
            if (rel <= target_relerr) {
                reached = 1;
                break;
            }
        }
        if (max_seconds > 0.0 && elapsed() >= max_seconds) {
            timed_out = done < max_iters;
            break;
        }
    }
    if (rel < 0.0) {
        s = nmf_eval_error(h, nullptr, &rel);
        if (s != NMF_OK) return s;
    }
    s = nmf_get_info(h, &info);
    if (s != NMF_OK) return s;
    if (res) {
        res->iters = done;
        res->relerr = rel;
        res->relerr_last = info.relerr;
        res->seconds = elapsed();
        res->reached = reached;
        res->timed_out = timed_out;
    }
    return NMF_OK;
}

nmf_status nmf_set_forced_decisions(nmf_handle *h, const uint8_t *accepted, int64_t count) {
    if (!h || count < 0 || (count > 0 && !accepted))
        return fail(NMF_EINVAL, "nmf_set_forced_decisions: bad arguments");
    NMF_CUDA(cudaStreamSynchronize(h->st));
    unsigned char *d = nullptr;
    if (count > 0) {
        NMF_CUDA(cudaMalloc(&d, (size_t)count));
        cudaError_t e = cudaMemcpy(d, accepted, (size_t)count, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return fail(NMF_ECUDA, "nmf_set_forced_decisions: %s", cudaGetErrorString(e));
        }
    }
    if (h->forced) cudaFree(h->forced);
    h->forced = d;
    h->forced_len = count;
    return build_graph(h);        // the decision kernel takes the array by value
}

static nmf_status copy_w_out(nmf_handle *h, const float *src, float *dst, int to_device) {
    NMF_CUDA(cudaMemcpy2DAsync(dst, sizeof(float) * h->r, src, sizeof(float) * h->rs,
                               sizeof(float) * h->r, h->m, kind_of(1, to_device), h->st));
    return NMF_OK;
}
static nmf_status copy_h_out(nmf_handle *h, const float *src, float *dst, int to_device) {
    NMF_CUDA(cudaMemcpy2DAsync(dst, sizeof(float) * h->n, src, sizeof(float) * h->ld,
                               sizeof(float) * h->n, h->r, kind_of(1, to_device), h->st));
    return NMF_OK;
}
static nmf_status copy_w_in(nmf_handle *h, const float *src, float *dst, int on_device) {
    NMF_CUDA(cudaMemcpy2DAsync(dst, sizeof(float) * h->rs, src, sizeof(float) * h->r,
                               sizeof(float) * h->r, h->m, kind_of(on_device, 1), h->st));
    return NMF_OK;
}
static nmf_status copy_h_in(nmf_handle *h, const float *src, float *dst, int on_device) {
    NMF_CUDA(cudaMemcpy2DAsync(dst, sizeof(float) * h->ld, src, sizeof(float) * h->n,
                               sizeof(float) * h->n, h->r, kind_of(on_device, 1), h->st));
    return NMF_OK;
}

nmf_status nmf_get_factors(nmf_handle *h, float *W, float *H, int32_t to_device) {
    if (!h) return fail(NMF_EINVAL, "handle is NULL");
    nmf_status s;
    if (W && (s = copy_w_out(h, h->W, W, to_device)) != NMF_OK) return s;
    if (H && (s = copy_h_out(h, h->H, H, to_device)) != NMF_OK) return s;
    NMF_CUDA(cudaStreamSynchronize(h->st));
    return NMF_OK;
}

nmf_status nmf_get_extrapolated(nmf_handle *h, float *Wy, float *Hy, int32_t to_device) {
    if (!h) return fail(NMF_EINVAL, "handle is NULL");
    nmf_status s;
    if (Wy && (s = copy_w_out(h, h->Wy, Wy, to_device)) != NMF_OK) return s;
    if (Hy && (s = copy_h_out(h, h->Hy, Hy, to_device)) != NMF_OK) return s;
    NMF_CUDA(cudaStreamSynchronize(h->st));
    return NMF_OK;
}

nmf_status nmf_get_trace(nmf_handle *h, double *e, double *beta, uint8_t *accepted, int64_t cap,
                         int64_t *len) {
    if (!h || cap < 0) return fail(NMF_EINVAL, "bad arguments");
    nmf_info info;
    nmf_status s = nmf_get_info(h, &info);
    if (s != NMF_OK) return s;
    int64_t n = std::min<int64_t>(std::min<int64_t>(info.k, h->tr_cap), cap);
    if (n > 0) {
        if (e) NMF_CUDA(cudaMemcpy(e, h->tr_e, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (beta) NMF_CUDA(cudaMemcpy(beta, h->tr_beta, sizeof(double) * n, cudaMemcpyDeviceToHost));
        if (accepted) NMF_CUDA(cudaMemcpy(accepted, h->tr_acc, n, cudaMemcpyDeviceToHost));
    }
    if (len) *len = n;
    return NMF_OK;
}

nmf_status nmf_get_line_search_trace(nmf_handle *h, double *beta_star, int64_t cap, int64_t *len) {
    if (!h || cap < 0) return fail(NMF_EINVAL, "bad arguments");
    if (!h->p.line_search_trace)
        return fail(NMF_ENOTSUP, "the handle was created without line_search_trace = 1");
    nmf_info info;
    nmf_status s = nmf_get_info(h, &info);
    if (s != NMF_OK) return s;
    int64_t n = std::min<int64_t>(std::min<int64_t>(info.k, h->tr_cap), cap);
    if (n > 0 && beta_star)
        NMF_CUDA(cudaMemcpy(beta_star, h->tr_bstar, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (len) *len = n;
    return NMF_OK;
}

nmf_status nmf_get_state(nmf_handle *h, nmf_scalars *s, float *W, float *H, float *Wy, float *Hy,
                         int32_t to_device) {
    if (!h) return fail(NMF_EINVAL, "handle is NULL");
    nmf_status st;
    if (W && (st = copy_w_out(h, h->W, W, to_device)) != NMF_OK) return st;
    if (H && (st = copy_h_out(h, h->H, H, to_device)) != NMF_OK) return st;
    if (Wy && (st = copy_w_out(h, h->Wy, Wy, to_device)) != NMF_OK) return st;
    if (Hy && (st = copy_h_out(h, h->Hy, Hy, to_device)) != NMF_OK) return st;
    NMF_CUDA(cudaMemcpyAsync(h->h_state, h->state, sizeof(DevState), cudaMemcpyDeviceToHost, h->st));
    NMF_CUDA(cudaStreamSynchronize(h->st));
    if (s) {
        s->beta = h->h_state->beta;
        s->beta_bar = h->h_state->beta_bar;
        s->beta_prev = h->h_state->beta_prev;
        s->e_last = h->h_state->e_last;
        s->e_prev = h->h_state->e_prev;
        s->k = h->h_state->k;
    }
    return NMF_OK;
}

nmf_status nmf_set_state(nmf_handle *h, const nmf_scalars *s, const float *W, const float *H,
                         const float *Wy, const float *Hy, int32_t on_device) {
    if (!h || !s || !W || !H || !Wy || !Hy) return fail(NMF_EINVAL, "all arguments are required");
    if (s->k < 0) return fail(NMF_EINVAL, "k must be >= 0");
    nmf_status st;
    if ((st = copy_w_in(h, W, h->W, on_device)) != NMF_OK) return st;
    if ((st = copy_h_in(h, H, h->H, on_device)) != NMF_OK) return st;
    if ((st = copy_w_in(h, Wy, h->Wy, on_device)) != NMF_OK) return st;
    if ((st = copy_h_in(h, Hy, h->Hy, on_device)) != NMF_OK) return st;
    NMF_CUDA(cudaMemcpyAsync(h->h_state, h->state, sizeof(DevState), cudaMemcpyDeviceToHost, h->st));
    NMF_CUDA(cudaStreamSynchronize(h->st));
    DevState d = *h->h_state;
    d.beta = s->beta;
    d.beta_bar = s->beta_bar;
    d.beta_prev = s->beta_prev;
    d.e_last = s->e_last;
    d.e_prev = s->e_prev;
    d.k = s->k;
    d.status = 0;
    *h->h_state = d;
    NMF_CUDA(cudaMemcpyAsync(h->state, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, h->st));
    NMF_CUDA(cudaStreamSynchronize(h->st));
    h->k_enq = s->k;
    return ensure_trace(h, h->k_enq + 1);
}

nmf_status nmf_profile_phases(nmf_handle *h, int32_t iters, double *ms) {
    if (!h || !ms || iters < 1) return fail(NMF_EINVAL, "handle, ms and iters >= 1 are required");
    nmf_status s = ensure_trace(h, h->k_enq + iters);
    if (s != NMF_OK) return s;
    cudaEvent_t ev[NMF_NUM_PHASES + 1] = {};
    for (int i = 0; i <= NMF_NUM_PHASES; ++i) {
        cudaError_t e = cudaEventCreate(&ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
            return fail(NMF_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
        }
    }
    double acc[NMF_NUM_PHASES] = {};
    nmf_status out = NMF_OK;
    for (int32_t it = 0; it < iters && out == NMF_OK; ++it) {
        cudaError_t e = enqueue_iteration(h, h->st, ev);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[NMF_NUM_PHASES]);
        if (e != cudaSuccess) {
            out = fail(NMF_ECUDA, "profiled iteration failed: %s", cudaGetErrorString(e));
            break;
        }
        h->k_enq += 1;
        for (int i = 0; i < NMF_NUM_PHASES; ++i) {
            float t = 0.0f;
            cudaEventElapsedTime(&t, ev[i], ev[i + 1]);
            acc[i] += t;
        }
    }
    for (int i = 0; i <= NMF_NUM_PHASES; ++i) cudaEventDestroy(ev[i]);
    if (out != NMF_OK) return out;
    for (int i = 0; i < NMF_NUM_PHASES; ++i) ms[i] = acc[i] / iters;
    return NMF_OK;
}

nmf_status nmf_matmul_nt(const float *P, int64_t M, int64_t K, int64_t ldp, const float *Q,
                         int32_t q_rows, int64_t ldq, float *out, int64_t ldo, int32_t precision,
                         void *stream) {
    if (!P || !Q || !out || M < 1 || K < 1 || q_rows < 1 || q_rows > kMaxRank || ldp < K ||
        ldq < K || ldo < q_rows || ldp % 8 || ldq % 8)
        return fail(NMF_EINVAL, "nmf_matmul_nt: bad pointers or shapes (ld must be multiples of 8)");
    if (precision != NMF_PREC_TF32 && precision != NMF_PREC_BF16X3)
        return fail(NMF_ENOTSUP, "nmf_matmul_nt runs the tensor-core precisions only");
    if (!tc_available()) return fail(NMF_ENOTSUP, "the tensor-map driver entry point is unavailable");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int N = round16(q_rows);
    void *ws = nullptr;
    unsigned int *tickets = nullptr;
    int *err = nullptr;
    void *ph = nullptr, *pl = nullptr;
    __nv_bfloat16 *qh = nullptr, *ql = nullptr;
    float *qf = nullptr;
    auto cleanup = [&]() {
        cudaFree(qf);
        cudaFree(ws);
        cudaFree(tickets);
        cudaFree(err);
        cudaFree(ph);
        cudaFree(pl);
        cudaFree(qh);
        cudaFree(ql);
    };
    const size_t wsb = tc_ws_bytes(M, K, N, precision);
    cudaError_t e = cudaMalloc(&ws, wsb);
    if (e == cudaSuccess) e = cudaMalloc(&tickets, sizeof(unsigned int) * tc_num_tickets(M));
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(tickets, 0, sizeof(unsigned int) * tc_num_tickets(M), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    TcOperands o{};
    o.M = M;
    o.K = K;
    o.ldq = ldq;
    o.q_rows = q_rows;
    o.N = N;
    o.nvalid = q_rows;
    const bool bf = precision == NMF_PREC_BF16X3;
    const size_t pb = tc_packed_bytes(M, K, precision);
    if (e == cudaSuccess) e = cudaMalloc(&ph, pb);
    if (e == cudaSuccess && bf) e = cudaMalloc(&pl, pb);
    if (e == cudaSuccess) e = launch_tc_pack(P, M, K, ldp, false, precision, ph, pl, st);
    // Q as the tensor cores see it (nearest TF32 values, or the hi/lo pair).
    if (e == cudaSuccess) e = cudaMalloc(&qf, sizeof(float) * q_rows * ldq);
    if (e == cudaSuccess && bf) {
        e = cudaMalloc(&qh, sizeof(__nv_bfloat16) * q_rows * ldq);
        if (e == cudaSuccess) e = cudaMalloc(&ql, sizeof(__nv_bfloat16) * q_rows * ldq);
    }
    if (e == cudaSuccess) e = launch_tc_prep_h(Q, q_rows, K, ldq, precision, qf, qh, ql, st);
    o.Q = bf ? static_cast<const void *>(qh) : static_cast<const void *>(qf);
    o.Q_lo = ql;
    o.P = ph;
    o.P_lo = pl;
    if (e == cudaSuccess) e = launch_tc_product(o, precision, false, out, ldo, ws, tickets, err, st);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? NMF_ENOMEM : NMF_ECUDA, "nmf_matmul_nt: %s",
                    cudaGetErrorString(e));
    if (flag) return fail(NMF_ETIMEOUT, "nmf_matmul_nt: a bounded tensor-core pipeline wait expired");
    return NMF_OK;
}

nmf_status nmf_debug_set_fixup_stall(int32_t extra) {
    if (extra < 0) return fail(NMF_EINVAL, "nmf_debug_set_fixup_stall: extra must be >= 0");
    NMF_CUDA(tc_set_fixup_stall(extra));
    return NMF_OK;
}

nmf_status nmf_destroy(nmf_handle *h) {
    if (!h) return NMF_OK;
    cudaStreamSynchronize(h->st);
    free_handle(h);
    return NMF_OK;
}


// --------------------------------------------------------------------------
// Batched solver: one CUDA graph per outer iteration holding the kernels of
// every instance, split into `branches` independent chains (each a capture
// stream forked from and joined to the graph's origin), so the GPU runs the
// instances of different branches concurrently.  An autotuner picks the
// number of branches and a longest-first assignment of instances to branches
// by timing candidate graphs on a snapshot of the state, which it restores.
// --------------------------------------------------------------------------
}  // extern "C"

struct nmf_batch {
    cudaStream_t st = nullptr;                  // caller's stream
    std::vector<nmf_handle *> h;
    std::vector<cudaStream_t> br;               // capture streams
    cudaGraphExec_t exec = nullptr;
    void *tables = nullptr;                     // device tables of a grouped graph
    nmf_batch_plan plan{};                      // schedule of `exec`
    int64_t k_enq = 0;
};

namespace {

void free_batch(nmf_batch *b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->tables) cudaFree(b->tables);
    for (auto *h : b->h) free_handle(h);
    for (auto s : b->br) cudaStreamDestroy(s);
    delete b;
}

double est_cost(const nmf_handle *h) {
    const double m = (double)h->m, n = (double)h->n, r = (double)h->r;
    return 4.0 * m * n * r + 2.0 * r * r * (h->lh * n + h->lw * m);
}

// Longest-first: instances sorted by decreasing cost, each to the least
// loaded branch.
std::vector<std::vector<int>> assign(const nmf_batch *b, int branches) {
    std::vector<int> idx(b->h.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
    std::sort(idx.begin(), idx.end(),
              [&](int x, int y) { return est_cost(b->h[x]) > est_cost(b->h[y]); });
    std::vector<std::vector<int>> out(branches);
    std::vector<double> load(branches, 0.0);
    for (int i : idx) {
        const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        out[j].push_back(i);
        load[j] += est_cost(b->h[i]);
    }
    return out;
}

nmf_status build_chains_graph(nmf_batch *b, int branches, cudaGraphExec_t *exec) {
    *exec = nullptr;
    const auto groups = assign(b, branches);
    cudaStream_t origin = b->br[0];
    cudaGraph_t g = nullptr;
    std::vector<cudaEvent_t> evs;
    auto mk = [&]() {
        cudaEvent_t e;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        evs.push_back(e);
        return e;
    };
    cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaEvent_t fork = mk();
        e = cudaEventRecord(fork, origin);
        for (int j = 1; j < branches && e == cudaSuccess; ++j)
            e = cudaStreamWaitEvent(b->br[j], fork, 0);
        for (int j = 0; j < branches && e == cudaSuccess; ++j)
            for (int i : groups[j]) {
                e = enqueue_iteration(b->h[i], b->br[j]);
                if (e != cudaSuccess) break;
            }
        for (int j = 1; j < branches && e == cudaSuccess; ++j) {
            cudaEvent_t join = mk();
            e = cudaEventRecord(join, b->br[j]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, join, 0);
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(origin, &g);
    for (auto ev : evs) cudaEventDestroy(ev);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return fail(NMF_ECUDA, "batch graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(NMF_ECUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
    return NMF_OK;
}


// ---------------------------------------------------------------- grouped
// One outer iteration of all instances as a few grouped launches, phase by
// phase of Algorithm 2: [Gram of W_y | A = W_y^T X] -> H sweeps -> [Gram of
// H_y | C = X H_y^T] -> W sweeps with the error and the decision ->
// finalize.  Within a phase, the launches of the different kernel variants
// (instances of different r) are independent and may run on concurrent
// branches.  Every instance gets exactly the CTAs of its single launch.
bool batch_groupable(const nmf_batch *b) {
    for (auto *h : b->h)
        if (h->is_csr || h->p.precision != NMF_PREC_FP32 || h->p.delta > 0.0 || h->p.exact_nnls ||
            hals_w_group_key(h->m, h->r) < 0)
            return false;
    return true;
}

enum GKind { kGramPartial, kGramReduce, kWtx, kSweepH, kXht, kHalsW, kFinalize };
struct GLaunch {
    GKind kind;
    int key;
    size_t items, begin;        // byte offsets into the device tables
    int nitems;
    int64_t ctas;
    int max_r;
};

struct GStaging {
    std::vector<unsigned char> host;
    size_t add(const void *p, size_t bytes) {
        const size_t off = (host.size() + 15) / 16 * 16;
        host.resize(off + bytes);
        memcpy(host.data() + off, p, bytes);
        return off;
    }
};

// Items of one kernel variant (key) in instance order of decreasing cost,
// so that the largest instances' CTAs are dispatched first.
template <typename Item>
GLaunch stage_group(GStaging &sg, GKind kind, int key, const std::vector<Item> &items,
                    const std::vector<int64_t> &ctas, int max_r) {
    std::vector<int64_t> begin(items.size() + 1, 0);
    for (size_t i = 0; i < items.size(); ++i) begin[i + 1] = begin[i] + ctas[i];
    GLaunch L{};
    L.kind = kind;
    L.key = key;
    L.items = sg.add(items.data(), sizeof(Item) * items.size());
    L.begin = sg.add(begin.data(), sizeof(int64_t) * begin.size());
    L.nitems = (int)items.size();
    L.ctas = begin.back();
    L.max_r = max_r;
    return L;
}

cudaError_t run_glaunch(const GLaunch &L, const unsigned char *dev, cudaStream_t st) {
    const int64_t *begin = reinterpret_cast<const int64_t *>(dev + L.begin);
    const void *items = dev + L.items;
    switch (L.kind) {
        case kGramPartial:
            return launch_gram_partial_grouped(L.key, static_cast<const GramItem *>(items), begin,
                                               L.nitems, L.ctas, st);
        case kGramReduce:
            return launch_gram_reduce_grouped((L.key & 1) != 0,
                                              static_cast<const GramItem *>(items), begin,
                                              L.nitems, L.ctas, st);
        case kWtx:
            return launch_wtx_grouped(L.key, static_cast<const WtxItem *>(items), begin, L.nitems,
                                      L.ctas, st);
        case kSweepH:
            return launch_sweep_h_grouped(static_cast<const SweepItem *>(items), begin, L.nitems,
                                          L.ctas, L.max_r, st);
        case kXht:
            return launch_xht_grouped(L.key, static_cast<const XhtItem *>(items), begin, L.nitems,
                                      L.ctas, st);
        case kHalsW:
            return launch_hals_w_grouped(L.key, static_cast<const HalsWItem *>(items), begin,
                                         L.nitems, L.ctas, st);
        case kFinalize:
            return launch_finalize_grouped(static_cast<const FinalizeItem *>(items), begin,
                                           L.nitems, L.ctas, st);
    }
    return cudaErrorInvalidValue;
}

using GChain = std::vector<GLaunch>;        // launches in order on one branch
using GPhase = std::vector<GChain>;         // independent chains

// Groups the instances by key (in order of decreasing cost) and stages one
// launch -- or a partial + reduce chain for the Grams -- per key.
template <typename Item, typename Plan>
void stage_phase(GStaging &sg, GPhase &ph, const nmf_batch *b, const std::vector<int> &order,
                 GKind kind, Plan plan) {
    std::vector<int> keys;
    std::vector<std::vector<Item>> items;
    std::vector<std::vector<int64_t>> ctas, ctas2;
    std::vector<int> max_r;
    for (int i : order) {
        Item it{};
        int64_t c = 0, c2 = 0;
        const int key = plan(b->h[i], &it, &c, &c2);
        size_t g = std::find(keys.begin(), keys.end(), key) - keys.begin();
        if (g == keys.size()) {
            keys.push_back(key);
            items.push_back(std::vector<Item>());
            ctas.push_back(std::vector<int64_t>());
            ctas2.push_back(std::vector<int64_t>());
            max_r.push_back(0);
        }
        items[g].push_back(it);
        ctas[g].push_back(c);
        ctas2[g].push_back(c2);
        max_r[g] = std::max(max_r[g], b->h[i]->r);
    }
    for (size_t g = 0; g < keys.size(); ++g) {
        GChain ch;
        ch.push_back(stage_group(sg, kind, keys[g], items[g], ctas[g], max_r[g]));
        if (kind == kGramPartial) {
            GLaunch red = stage_group(sg, kGramReduce, keys[g], items[g], ctas2[g],
                                      max_r[g]);
            ch.push_back(red);
        }
        ph.push_back(ch);
    }
}

nmf_status build_grouped_graph(nmf_batch *b, int branches, int h_cols, cudaGraphExec_t *exec,
                               void **tables, int *launches) {
    *exec = nullptr;
    *tables = nullptr;
    std::vector<int> order(b->h.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return est_cost(b->h[x]) > est_cost(b->h[y]); });
    GStaging sg;
    std::vector<GPhase> phases(5);
    cudaError_t ce = cudaSuccess;
    auto keep = [&](cudaError_t e) {
        if (e != cudaSuccess && ce == cudaSuccess) ce = e;
    };
    // Phase 1: G = W_y^T W_y (FP32 Gram) beside A = W_y^T X.
    stage_phase<GramItem>(sg, phases[0], b, order, kGramPartial,
                          [&](nmf_handle *h, GramItem *it, int64_t *c, int64_t *c2) {
                              plan_gram_item(h->Wy, h->m, h->rs, h->r, h->rs, h->G, nullptr,
                                             h->gws, it, c, c2);
                              return gram_group_key(h->r, true, false);
                          });
    stage_phase<WtxItem>(sg, phases[0], b, order, kWtx,
                         [&](nmf_handle *h, WtxItem *it, int64_t *c, int64_t *) {
                             keep(plan_wtx_item(h->X, h->m, h->ld, h->ld, h->r, h->Wy, h->rs,
                                                h->A, h->ws, h->tickets, it, c));
                             return wtx_group_key(h->rs);
                         });
    // Phase 2: the H sweeps with the fused extrapolation of H (steps 3-9).
    stage_phase<SweepItem>(sg, phases[1], b, order, kSweepH,
                           [&](nmf_handle *h, SweepItem *it, int64_t *c, int64_t *) {
                               HEpilogue hep{};
                               hep.H_acc = h->H;
                               hep.Hw = h->p.hp >= 2 ? h->Hw : nullptr;
                               hep.state = h->state;
                               hep.hp = h->p.hp;
                               plan_sweep_h_item(h->n, h->ld, h->r, h->rs, h->A, h->G, h->Hy,
                                                 h->Hn, h->lh, hep, h_cols, it, c);
                               return 0;
                           });
    // Phase 3: D = H_y H_y^T (error-free) beside C = X H_y^T.
    stage_phase<GramItem>(sg, phases[2], b, order, kGramPartial,
                          [&](nmf_handle *h, GramItem *it, int64_t *c, int64_t *c2) {
                              const float *Hu = h->p.hp >= 2 ? h->Hw : h->Hn;
                              plan_gram_item(Hu, h->n, h->ld, h->r, h->rs, h->D, h->D_lo, h->gws,
                                             it, c, c2);
                              return gram_group_key(h->r, false, true);
                          });
    stage_phase<XhtItem>(sg, phases[2], b, order, kXht,
                         [&](nmf_handle *h, XhtItem *it, int64_t *c, int64_t *) {
                             const float *Hu = h->p.hp >= 2 ? h->Hw : h->Hn;
                             keep(plan_xht_item(h->X, h->m, h->ld, h->r, Hu, h->ld, h->C, h->C_lo,
                                                h->rs, h->ws, h->xtickets, it, c));
                             return xht_group_key(h->m, h->r);
                         });
    // Phase 4: the W sweeps, Remark 1's error, the decision (steps 10, 15-20).
    stage_phase<HalsWItem>(sg, phases[3], b, order, kHalsW,
                           [&](nmf_handle *h, HalsWItem *it, int64_t *c, int64_t *) {
                               WEpilogue wep{};
                               wep.C_lo = h->C_lo;
                               wep.D_lo = h->D_lo;
                               wep.partials = h->partials;
                               wep.counter = h->counter;
                               wep.state = h->state;
                               wep.params = dev_params(h);
                               wep.trace.e = h->tr_e;
                               wep.trace.beta = h->tr_beta;
                               wep.trace.acc = h->tr_acc;
                               wep.trace.cap = h->tr_cap;
                               wep.trace.bstar = h->tr_bstar;
                               wep.trace.forced = h->forced;
                               wep.trace.forced_len = h->forced_len;
                               wep.W_prev = h->p.line_search_trace ? h->W : nullptr;
                               plan_hals_w_item(h->m, h->r, h->rs, h->C, h->D, h->Wy, h->Wn,
                                                h->lw, wep, it, c);
                               return hals_w_group_key(h->m, h->r);
                           });
    // Phase 5: extrapolation of W (and of H for hp = 1), accept/restart copies.
    stage_phase<FinalizeItem>(sg, phases[4], b, order, kFinalize,
                              [&](nmf_handle *h, FinalizeItem *it, int64_t *c, int64_t *) {
                                  plan_finalize_item(h->m, h->rs, h->r, h->ld, h->W, h->H, h->Wy,
                                                     h->Hy, h->Wn, h->Hn, h->Hw, h->state,
                                                     dev_params(h), it, c);
                                  return 0;
                              });
    if (ce != cudaSuccess) return fail(NMF_ECUDA, "grouped plan: %s", cudaGetErrorString(ce));

    void *dev = nullptr;
    NMF_CUDA(cudaMalloc(&dev, std::max<size_t>(sg.host.size(), 16)));
    cudaError_t e = cudaMemcpy(dev, sg.host.data(), sg.host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        return fail(NMF_ECUDA, "grouped tables: %s", cudaGetErrorString(e));
    }
    const unsigned char *d = static_cast<const unsigned char *>(dev);
    cudaStream_t origin = b->br[0];
    const int nb = std::max(1, std::min(branches, (int)b->br.size()));
    cudaGraph_t g = nullptr;
    std::vector<cudaEvent_t> evs;
    auto mk = [&]() {
        cudaEvent_t ev;
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        evs.push_back(ev);
        return ev;
    };
    int count = 0;
    e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    for (const GPhase &ph : phases) {
        if (e != cudaSuccess) break;
        const int used = std::min<int>(nb, (int)ph.size());
        if (used > 1) {
            cudaEvent_t fork = mk();
            e = cudaEventRecord(fork, origin);
            for (int j = 1; j < used && e == cudaSuccess; ++j)
                e = cudaStreamWaitEvent(b->br[j], fork, 0);
        }
        for (size_t c = 0; c < ph.size() && e == cudaSuccess; ++c)
            for (const GLaunch &L : ph[c]) {
                e = run_glaunch(L, d, b->br[c % used]);
                ++count;
                if (e != cudaSuccess) break;
            }
        for (int j = 1; j < used && e == cudaSuccess; ++j) {
            cudaEvent_t join = mk();
            e = cudaEventRecord(join, b->br[j]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, join, 0);
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(origin, &g);
    for (auto ev : evs) cudaEventDestroy(ev);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        cudaFree(dev);
        return fail(NMF_ECUDA, "grouped graph capture failed: %s",
                    cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaFree(dev);
        return fail(NMF_ECUDA, "grouped graph instantiate: %s", cudaGetErrorString(e));
    }
    *tables = dev;
    *launches = count;
    return NMF_OK;
}

// Builds the graph of a schedule; on success it replaces b's graph.
nmf_status build_batch_graph(nmf_batch *b, const nmf_batch_plan &pl) {
    cudaGraphExec_t ex = nullptr;
    void *tab = nullptr;
    int launches = 0;
    nmf_status s;
    if (pl.grouped) {
        s = build_grouped_graph(b, pl.branches, pl.h_cols_per_cta, &ex, &tab, &launches);
    } else {
        s = build_chains_graph(b, pl.branches, &ex);
        launches = 0;
        for (auto *h : b->h) launches += h->is_csr ? 12 : (tc_mode(h) ? 11 : 9);
    }
    if (s != NMF_OK) return s;
    NMF_CUDA(cudaStreamSynchronize(b->st));          // the old graph may still run
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->tables) cudaFree(b->tables);
    b->exec = ex;
    b->tables = tab;
    b->plan = pl;
    b->plan.launches_per_iter = launches;
    return NMF_OK;
}

// Device-side snapshot of every instance's iterate and scalar state.
struct Snapshot {
    std::vector<void *> bufs;
    ~Snapshot() {
        for (void *p : bufs) cudaFree(p);
    }
};

nmf_status snapshot(nmf_batch *b, Snapshot &sn, bool restore) {
    size_t q = 0;
    for (auto *h : b->h) {
        struct Item {
            void *p;
            size_t bytes;
        } items[] = {{h->W, sizeof(float) * h->m * h->rs},  {h->Wy, sizeof(float) * h->m * h->rs},
                     {h->H, sizeof(float) * h->r * h->ld},  {h->Hy, sizeof(float) * h->r * h->ld},
                     {h->state, sizeof(DevState)}};
        for (auto &it : items) {
            if (!restore) {
                void *d = nullptr;
                NMF_CUDA(cudaMalloc(&d, it.bytes));
                sn.bufs.push_back(d);
                NMF_CUDA(cudaMemcpyAsync(d, it.p, it.bytes, cudaMemcpyDeviceToDevice, b->st));
            } else {
                NMF_CUDA(cudaMemcpyAsync(it.p, sn.bufs[q++], it.bytes, cudaMemcpyDeviceToDevice,
                                         b->st));
            }
        }
    }
    NMF_CUDA(cudaStreamSynchronize(b->st));
    return NMF_OK;
}

nmf_status batch_ensure_trace(nmf_batch *b, int64_t need) {
    bool grown = false;
    for (auto *h : b->h)
        if (need > h->tr_cap) {
            nmf_status s = ensure_trace(h, need);
            if (s != NMF_OK) return s;
            grown = true;
        }
    if (grown && b->exec) {
        nmf_status s = build_batch_graph(b, b->plan);
        if (s != NMF_OK) return s;
    }
    return NMF_OK;
}

// Times `iters` graph launches of a candidate schedule (after one warm-up).
nmf_status time_plan(nmf_batch *b, const nmf_batch_plan &pl, cudaEvent_t e0, cudaEvent_t e1,
                     double *ms) {
    cudaGraphExec_t ex = nullptr;
    void *tab = nullptr;
    int launches = 0;
    nmf_status s = pl.grouped ? build_grouped_graph(b, pl.branches, pl.h_cols_per_cta, &ex, &tab,
                                                    &launches)
                              : build_chains_graph(b, pl.branches, &ex);
    if (s != NMF_OK) return s;
    cudaGraphLaunch(ex, b->st);                 // warm
    cudaEventRecord(e0, b->st);
    for (int it = 0; it < 3; ++it) cudaGraphLaunch(ex, b->st);
    cudaEventRecord(e1, b->st);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaGraphExecDestroy(ex);
    if (tab) cudaFree(tab);
    if (e != cudaSuccess) return fail(NMF_ECUDA, "autotune run failed: %s", cudaGetErrorString(e));
    *ms = t / 3.0;
    return NMF_OK;
}

// Candidate schedules: chains over 1..64 branches; grouped launches (when
// every instance allows them) with the launches of a phase on one or on
// several branches, and 32 or 16 columns of H per sweep CTA.  The fastest
// measured one is kept.
nmf_status autotune(nmf_batch *b) {
    const int count = (int)b->h.size();
    std::vector<nmf_batch_plan> cands;
    for (int c : {1, 2, 4, 8, 16, 32, 64})
        if (c <= count && c <= (int)b->br.size()) cands.push_back(nmf_batch_plan{0, c, 0, 0, 0.0});
    if (batch_groupable(b))
        for (int c : {1, 16})
            for (int cols : {32, 16})
                if (c <= (int)b->br.size()) cands.push_back(nmf_batch_plan{1, c, cols, 0, 0.0});
    nmf_status s = batch_ensure_trace(b, b->k_enq + 4 * (int64_t)cands.size() + 8);
    if (s != NMF_OK) return s;
    Snapshot sn;
    s = snapshot(b, sn, false);
    if (s != NMF_OK) return s;
    cudaEvent_t e0, e1;
    NMF_CUDA(cudaEventCreate(&e0));
    NMF_CUDA(cudaEventCreate(&e1));
    double best = 1e30;
    nmf_batch_plan best_pl = cands.front();
    for (const auto &pl : cands) {
        double ms = 0.0;
        s = time_plan(b, pl, e0, e1, &ms);
        if (s != NMF_OK) break;
        if (ms < best) {
            best = ms;
            best_pl = pl;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != NMF_OK) return s;
    s = snapshot(b, sn, true);                      // undo the tuning iterations
    if (s != NMF_OK) return s;
    s = build_batch_graph(b, best_pl);
    if (s != NMF_OK) return s;
    b->plan.ms_per_iter = best;
    return NMF_OK;
}

}  // namespace

extern "C" {

namespace {

// Instance i takes parameters p[i * p_stride] (p_stride 0: one set for all).
nmf_status batch_create(nmf_batch **out, int32_t count, const nmf_matrix *Xs,
                        const int32_t *ranks, const float *const *W0, const float *const *H0,
                        int32_t factors_on_device, const nmf_params *p, size_t p_stride,
                        void *stream) {
    if (!out) return fail(NMF_EINVAL, "out pointer is NULL");
    *out = nullptr;
    if (count < 1 || !Xs || !ranks || !W0 || !H0)
        return fail(NMF_EINVAL, "nmf_batch_create: count >= 1 and all arrays are required");
    nmf_batch *b = new (std::nothrow) nmf_batch();
    if (!b) return fail(NMF_ENOMEM, "host allocation failed");
    b->st = static_cast<cudaStream_t>(stream);
    for (int32_t i = 0; i < count; ++i) {
        nmf_handle *h = nullptr;
        const nmf_params *pi = p ? p + (size_t)i * p_stride : nullptr;
        nmf_status s = nmf_create(&h, &Xs[i], ranks[i], W0[i], H0[i], factors_on_device, pi, stream);
        if (s != NMF_OK) {
            free_batch(b);
            char msg[600];
            snprintf(msg, sizeof(msg), "instance %d: %s", (int)i, g_err);
            return fail(s, "%s", msg);
        }
        b->h.push_back(h);
    }
    const int nbr = std::min<int>(64, count);
    for (int j = 0; j < nbr; ++j) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            free_batch(b);
            return fail(NMF_ECUDA, "stream creation failed");
        }
        b->br.push_back(s);
    }
    nmf_status s = autotune(b);
    if (s != NMF_OK) {
        free_batch(b);
        return s;
    }
    *out = b;
    return NMF_OK;
}

}  // namespace

nmf_status nmf_batch_create(nmf_batch **out, int32_t count, const nmf_matrix *Xs,
                            const int32_t *ranks, const float *const *W0, const float *const *H0,
                            int32_t factors_on_device, const nmf_params *p, void *stream) {
    return batch_create(out, count, Xs, ranks, W0, H0, factors_on_device, p, 0, stream);
}

nmf_status nmf_batch_create_params(nmf_batch **out, int32_t count, const nmf_matrix *Xs,
                                   const int32_t *ranks, const float *const *W0,
                                   const float *const *H0, int32_t factors_on_device,
                                   const nmf_params *params, void *stream) {
    if (!params) return fail(NMF_EINVAL, "nmf_batch_create_params: params (count entries) is NULL");
    return batch_create(out, count, Xs, ranks, W0, H0, factors_on_device, params, 1, stream);
}

nmf_status nmf_batch_step(nmf_batch *b, int32_t iters) {
    if (!b || iters < 0) return fail(NMF_EINVAL, "bad arguments");
    nmf_status s = batch_ensure_trace(b, b->k_enq + iters);
    if (s != NMF_OK) return s;
    for (int32_t i = 0; i < iters; ++i) NMF_CUDA(cudaGraphLaunch(b->exec, b->st));
    b->k_enq += iters;
    for (auto *h : b->h) h->k_enq = b->k_enq;
    return NMF_OK;
}

nmf_status nmf_batch_step_loop(nmf_batch *b, int32_t iters) {
    if (!b || iters < 0) return fail(NMF_EINVAL, "bad arguments");
    nmf_status s = batch_ensure_trace(b, b->k_enq + iters);
    if (s != NMF_OK) return s;
    for (int32_t it = 0; it < iters; ++it)
        for (auto *h : b->h) NMF_CUDA(cudaGraphLaunch(h->exec, b->st));
    b->k_enq += iters;
    for (auto *h : b->h) h->k_enq = b->k_enq;
    return NMF_OK;
}

nmf_status nmf_batch_get_info(nmf_batch *b, int32_t i, nmf_info *info) {
    if (!b || i < 0 || i >= (int32_t)b->h.size()) return fail(NMF_EINVAL, "bad instance index");
    NMF_CUDA(cudaStreamSynchronize(b->st));
    return nmf_get_info(b->h[i], info);
}

nmf_status nmf_batch_get_factors(nmf_batch *b, int32_t i, float *W, float *H, int32_t to_device) {
    if (!b || i < 0 || i >= (int32_t)b->h.size()) return fail(NMF_EINVAL, "bad instance index");
    NMF_CUDA(cudaStreamSynchronize(b->st));
    return nmf_get_factors(b->h[i], W, H, to_device);
}

nmf_status nmf_batch_schedule(nmf_batch *b, int32_t *branches, double *ms_per_iter) {
    if (!b) return fail(NMF_EINVAL, "batch is NULL");
    if (branches) *branches = b->plan.branches;
    if (ms_per_iter) *ms_per_iter = b->plan.ms_per_iter;
    return NMF_OK;
}

nmf_status nmf_batch_get_plan(nmf_batch *b, nmf_batch_plan *plan) {
    if (!b || !plan) return fail(NMF_EINVAL, "batch or plan is NULL");
    *plan = b->plan;
    return NMF_OK;
}

nmf_status nmf_batch_set_plan(nmf_batch *b, const nmf_batch_plan *plan) {
    if (!b || !plan) return fail(NMF_EINVAL, "batch or plan is NULL");
    nmf_batch_plan pl = *plan;
    if ((pl.grouped != 0 && pl.grouped != 1) || pl.branches < 1 || pl.branches > 64 ||
        pl.h_cols_per_cta < 0 || pl.h_cols_per_cta > 32)
        return fail(NMF_EINVAL, "plan fields out of range");
    if (pl.grouped && !batch_groupable(b))
        return fail(NMF_ENOTSUP, "grouped launches need dense FP32 HALS instances");
    pl.branches = std::min<int>(pl.branches, (int)b->br.size());
    pl.ms_per_iter = 0.0;
    return build_batch_graph(b, pl);
}

nmf_status nmf_batch_destroy(nmf_batch *b) {
    if (!b) return NMF_OK;
    cudaStreamSynchronize(b->st);
    free_batch(b);
    return NMF_OK;
}

}  // extern "C"
