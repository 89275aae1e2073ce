// common.cuh -- internal definitions shared by the CUDA translation units of
// libnmf_gb300 (never included by the oracle or by callers).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nmf.h"

namespace nmfg {

constexpr int kMaxRank = 128;      // build cap on r (nmf_create: NMF_ENOTSUP above)
constexpr int kNumSMs = 152;       // GB300: 2 dies x 76 SMs

// Device-resident scalar state of Algorithms 2 and 3.  Written only by the
// single thread that takes the restart decision; read by every kernel of the
// next iteration.
struct DevState {
    double beta;          // beta_k for the iteration about to run
    double beta_bar;      // Algorithm 3 upper bound
    double beta_prev;     // beta_{k-1}
    double e_last;        // error the next e(k) is compared with
    double e_prev;        // e(k-1) as computed
    double fro2;          // ||X||_F^2
    double e_k;           // e(k) of the last iteration
    double beta_used;     // beta_k of the last iteration (the extrapolation step)
    long long k;          // iterations done
    int accepted;         // decision of the last iteration
    int status;           // sticky nmf_status raised on the device
    int lh_used, lw_used; // inner sweeps the last iteration ran (delta rule)
};

// Parameters the device logic needs (copied by value into kernel args).
struct DevParams {
    int hp;
    int project_w;
    int compare_prev;
    double eta, gamma, gamma_bar;
};

// Trace written by the decision thread.
struct DevTrace {
    double *e;
    double *beta;
    unsigned char *acc;
    double *bstar;        // line-search step of Sec. 3 per iteration, or null
    long long cap;
    const unsigned char *forced;  // decision replay: iteration k takes forced[k]
    long long forced_len;         // (for k < forced_len) instead of the test
};

// Error reduction partials of one W-sweep launch (Remark 1 in residual
// form, ||X - W H||^2 = ||X||^2 - cross + quad): cross = <W_n, C>,
// quad = <W_n, W_n D - C>, accumulated per CTA in FP64.
struct ErrPartial {
    double cross;
    double quad;
    double bnum;          // line-search diagnostic: -<W_n D - C, W_n - W>
    double bden;          //                         <(W_n - W) D, W_n - W>
};

}  // namespace nmfg

// ----------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files, used by capi.cu).
// Every launcher returns the cudaError_t of its launches.
//
// Internal layouts (the library's own copies, zero padded):
//   X : m x ld   row-major, ld = n rounded up to a multiple of 8
//   W, W_y, W_n, C : m x rs row-major, rs = r rounded up to a multiple of 8
//   H, H_y, H_n, H_w, A : r x ld row-major
//   G, D : rs x rs
// ----------------------------------------------------------------------------
namespace nmfg {

// ||X||_F^2 in FP64 over rows x cols entries with row stride ld.
size_t fro2_ws_bytes(int64_t count);
cudaError_t launch_fro2(const float *vals, int64_t rows, int64_t cols, int64_t ld,
                        double *out, void *ws, cudaStream_t st);

// G = M^T M for M (N x ldm, r used columns) -- the Gram of W -- or
// G = M M^T for M (r x ldm, N used columns) -- the Gram of H.  G is rs x rs.
size_t gram_ws_bytes(int64_t N, int rs);
cudaError_t launch_gram_rows(const float *M, int64_t N, int64_t ldm, int r, int rs, float *G,
                             void *ws, cudaStream_t st);
// Error-free Gram of W (G + G_lo, G the exactly rounded FP32 value): the
// exact NNLS solves need G to FP32 accuracy, not the ~sqrt(32) u of the
// blocked FP32 sums that the few HALS sweeps tolerate.
cudaError_t launch_gram_rows_exact(const float *M, int64_t N, int64_t ldm, int r, int rs,
                                   float *G, float *G_lo, void *ws, cudaStream_t st);
// The Gram of H is accumulated error-free and returned as G + G_lo.
cudaError_t launch_gram_cols(const float *M, int64_t N, int64_t ldm, int r, int rs, float *G,
                             float *G_lo, void *ws, cudaStream_t st);

// Dense products, FP32 on CUDA cores.  A = W^T X (r x ld), C = X H^T (m x rs).
// The split-K of A needs ws (partial tiles) and wtx_num_tickets() zeroed
// counters, which the kernel leaves at zero.
size_t wtx_ws_bytes(int64_t m, int64_t ld, int r);
int64_t wtx_num_tickets(int64_t ld);
cudaError_t launch_wtx_f32(const float *X, int64_t m, int64_t lda, int64_t ldx, int r,
                           const float *W, int rs, float *A, void *ws, unsigned int *tickets,
                           cudaStream_t st);
size_t xht_ws_bytes(int64_t m, int64_t ldx, int r);
int64_t xht_num_tickets(int64_t m);
cudaError_t launch_xht_f32(const float *X, int64_t m, int64_t ldx, int r, const float *H,
                           int64_t ldh, float *C, float *C_lo, int rs, void *ws,
                           unsigned int *tickets, cudaStream_t st);

// ---------------------------------------------------------------------------
// Grouped launches (the batched solver): one launch runs one kernel variant
// over many independent problems.  Each problem is an item of a device
// table holding its own arguments and CTA count; CTA b of the launch serves
// the item i with begin[i] <= b < begin[i + 1], as its CTA b - begin[i].  An
// item thus runs exactly the CTAs, tiles and splits of its own single
// launch, and computes the same values bit for bit.
// ---------------------------------------------------------------------------
// The item of this CTA of a grouped launch (binary search of the prefix
// sums) and the CTA's index within the item.
__device__ __forceinline__ int group_item(const int64_t *__restrict__ begin, int nitems,
                                          int64_t &local) {
    const int64_t b = blockIdx.x;
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(begin + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    local = b - __ldg(begin + lo);
    return lo;
}

struct WtxItem {
    const float *X;
    int64_t m, ldx;
    int r;
    const float *W;
    float *A;
    int64_t lda, rows_per_split;
    float *part;
    unsigned int *tickets;
    int64_t tiles;
    int nsplit;
};
struct XhtItem {
    const float *X;
    int64_t m, ldx;
    int r;
    const float *H;
    int64_t ldh;
    float *C, *C_lo;
    int rs;
    int64_t cols_per_split;
    float *part;
    unsigned int *tickets;
    int64_t tiles;
    int nsplit;
};
// A Gram (launch_gram_rows / launch_gram_cols): partial launch, then reduce.
struct GramItem {
    const float *M;
    int64_t N, ldm;
    int r, rs;
    int64_t chunk;
    float *part, *part_lo;
    int nparts;
    float *G, *G_lo;
};
struct FinalizeItem {
    int64_t nw, nh;
    float *W, *H, *Wy, *Hy;
    const float *Wn, *Hn, *Hw;
    const DevState *state;
    DevParams p;
};
// Item setup: the variant key (items of one key share a launch), the item's
// arguments and its CTA count(s).
int gram_group_key(int r, bool rows, bool exact);
void plan_gram_item(const float *M, int64_t N, int64_t ldm, int r, int rs, float *G,
                    float *G_lo, void *ws, GramItem *it, int64_t *ctas_partial,
                    int64_t *ctas_reduce);
cudaError_t launch_gram_partial_grouped(int key, const GramItem *items, const int64_t *begin,
                                        int nitems, int64_t ctas, cudaStream_t st);
cudaError_t launch_gram_reduce_grouped(bool exact, const GramItem *items, const int64_t *begin,
                                       int nitems, int64_t ctas, cudaStream_t st);
void plan_finalize_item(int64_t m, int rs, int r, int64_t ldh, float *W, float *H, float *Wy,
                        float *Hy, const float *Wn, const float *Hn, const float *Hw,
                        const DevState *state, DevParams p, FinalizeItem *it, int64_t *ctas);
cudaError_t launch_finalize_grouped(const FinalizeItem *items, const int64_t *begin, int nitems,
                                    int64_t ctas, cudaStream_t st);
int wtx_group_key(int rs);
cudaError_t plan_wtx_item(const float *X, int64_t m, int64_t lda, int64_t ldx, int r,
                          const float *W, int rs, float *A, void *ws, unsigned int *tickets,
                          WtxItem *it, int64_t *ctas);
cudaError_t launch_wtx_grouped(int key, const WtxItem *items, const int64_t *begin, int nitems,
                               int64_t ctas, cudaStream_t st);
int xht_group_key(int64_t m, int r);
cudaError_t plan_xht_item(const float *X, int64_t m, int64_t ldx, int r, const float *H,
                          int64_t ldh, float *C, float *C_lo, int rs, void *ws,
                          unsigned int *tickets, XhtItem *it, int64_t *ctas);
cudaError_t launch_xht_grouped(int key, const XhtItem *items, const int64_t *begin, int nitems,
                               int64_t ctas, cudaStream_t st);

// The early stop of A-HALS's inner loop (Gillis & Glineur 2012): sweep l
// runs only while the previous one still moved the iterate by more than
// delta times the first one, ||X^(l-1) - X^(l-2)||_F > delta ||X^(1) - X^(0)||_F.
// In that mode every sweep is one launch (sweeps = 1, l = 1, 2, ...); each
// sums ||change||^2 over its CTA into d2_out[CTA], and launch l >= 3 first
// compares the totals of sweeps l-1 and 1 (every CTA adds the partials in
// the same fixed order, so all take the same decision) and, once the rule
// holds, sets *stopped and every later launch returns at once.
struct SweepStop {
    int l;                    // 1-based sweep of this launch; 0: rule off
    double delta2;            // delta^2
    const double *d2_first;   // partials of sweep 1
    const double *d2_prev;    // partials of sweep l-1
    double *d2_out;           // partials of this sweep, one per CTA
    int nparts;               // CTAs per launch
    int *stopped;             // 1 once the rule has stopped the loop
    int *used;                // sweeps done this iteration
};

// HALS sweeps.  H side: columns of H independent given A and G.  W side:
// rows of W independent given C and D.
struct HEpilogue {            // optional fused work after the H sweeps
    const float *H_acc;       // accepted H (for the extrapolation)
    float *Hw;                // where to write the H_y used by the W-update, or null
    const DevState *state;    // beta_k
    int hp;
    SweepStop stop;
};
struct WEpilogue {            // optional fused work after the W sweeps
    const float *C_lo;        // low parts of C = X H^T and D = H H^T (error terms)
    const float *D_lo;
    ErrPartial *partials;     // one per CTA, or null (no error terms)
    unsigned int *counter;    // last-CTA ticket (zero between launches)
    DevState *state;          // decision + Algorithm 3, or null
    DevParams params;
    DevTrace trace;
    const float *W_prev;      // the accepted W (line-search diagnostic), or null
    SweepStop stop;
};
// Grouped sweeps (see the grouped launches above).  H side: the blocked
// kernel; W side: the lane-pipelined kernel, whose variant key is (T, S).
struct SweepItem {
    int64_t items;
    int r;
    int64_t ld;
    int nt;
    const float *A, *G;
    int rs;
    const float *Xin;
    float *Xout;
    int sweeps;
    HEpilogue hep;
};
struct HalsWItem {
    int64_t items;
    int r;
    int64_t ld;
    const float *A, *G;
    int rs;
    const float *Xin;
    float *Xout;
    int sweeps;
    WEpilogue wep;
    int64_t nblk;            // CTAs of the item (its error partials)
};
void plan_sweep_h_item(int64_t n, int64_t ldh, int r, int rs, const float *A, const float *G,
                       const float *H_in, float *H_out, int sweeps, const HEpilogue &ep, int nt,
                       SweepItem *it, int64_t *ctas);
cudaError_t launch_sweep_h_grouped(const SweepItem *items, const int64_t *begin, int nitems,
                                   int64_t ctas, int max_r, cudaStream_t st);
int hals_w_group_key(int64_t m, int r);      // -1: no grouped variant
void plan_hals_w_item(int64_t m, int r, int rs, const float *C, const float *D,
                      const float *W_in, float *W_out, int sweeps, const WEpilogue &ep,
                      HalsWItem *it, int64_t *ctas);
cudaError_t launch_hals_w_grouped(int key, const HalsWItem *items, const int64_t *begin,
                                  int nitems, int64_t ctas, cudaStream_t st);
cudaError_t launch_hals_h(int64_t n, int64_t ldh, int r, int rs, const float *A,
                          const float *G, const float *H_in, float *H_out, int sweeps,
                          const HEpilogue &ep, cudaStream_t st);
cudaError_t launch_hals_w(int64_t m, int r, int rs, const float *C, const float *D,
                          const float *W_in, float *W_out, int sweeps, const WEpilogue &ep,
                          cudaStream_t st);
int hals_w_num_ctas(int64_t m, int r);
int hals_h_num_ctas(int64_t n, int r);

// Exact NNLS subproblems (anls.cu), the block solvers of ANLS / E-ANLS:
// same operands and epilogues as the sweeps; *status is set to 1 when an
// item's free block was not positive definite or it did not settle (that
// item keeps its last iterate).
int anls_num_ctas(int64_t items);
cudaError_t launch_nnls_h(int64_t n, int64_t ldh, int r, int rs, const float *A, const float *G,
                          const float *H_in, float *H_out, const HEpilogue &ep, int *status,
                          cudaStream_t st);
cudaError_t launch_nnls_w(int64_t m, int r, int rs, const float *C, const float *D,
                          const float *W_in, float *W_out, const WEpilogue &ep, int *status,
                          cudaStream_t st);

// Algorithm 2 steps 11-20 after the decision: extrapolation, projection and
// accept/restart copies, W side and H side.
cudaError_t launch_finalize(int64_t m, int rs, int r, int64_t ldh, float *W, float *H,
                            float *Wy, float *Hy, const float *Wn, const float *Hn,
                            const float *Hw, const DevState *state, DevParams p,
                            cudaStream_t st);

// Remark 1 error terms of (W, C = X H^T, D = H H^T) given as hi + lo pairs,
// one partial per CTA.
int err_rows_num_ctas(int64_t m);
cudaError_t launch_err_rows(int64_t m, int r, int rs, const float *W, const float *C,
                            const float *C_lo, const float *D, const float *D_lo,
                            ErrPartial *part, cudaStream_t st);

// e^2 and e of a pair from the launch_err_rows partials (out[0], out[1]).
cudaError_t launch_pair_error(int64_t m, const double *fro2, const ErrPartial *partials,
                              double *out, cudaStream_t st);

// e(0) (Algorithm 2 step 1) and the initial Algorithm 3 values.
cudaError_t launch_init_state(int64_t m, int r, int rs, const float *W, const float *C,
                              const float *C_lo, const float *D, const float *D_lo,
                              const double *fro2, DevState *state, double beta0,
                              ErrPartial *partials, cudaStream_t st);

// Sparse X (csr.cu): C = X H^T from CSR with Ht = H^T (n x rs); A = W^T X
// from the CSC copy; H (r x ldh) -> Ht.  `carry` holds csr_carry_floats()
// floats of per-chunk partials.
size_t csr_carry_floats(int64_t nnz, int rs);
// rowseg / colseg: the row (CSR) or column (CSC) of every stored entry.
cudaError_t launch_xht_csr(const int64_t *rowptr, const int32_t *colidx, const int32_t *rowseg,
                           const float *val, int64_t m, int64_t nnz, int r, int rs,
                           const float *Ht, float *C, float *carry, cudaStream_t st);
cudaError_t launch_wtx_csc(const int64_t *colptr, const int32_t *rowidx, const int32_t *colseg,
                           const float *val, int64_t n, int64_t nnz, int r, int rs,
                           const float *W, float *A, int64_t lda, float *carry, cudaStream_t st);
cudaError_t launch_transpose_h(const float *H, int r, int64_t n, int64_t ldh, float *Ht, int rs,
                               cudaStream_t st);

// Tensor-core products (tc_products.cu): out = P Q^T, P (M x K) and Q
// (q_rows x K) K-major in FP32 (TF32 mode) or as BF16 hi/lo pairs (BF16X3
// mode); N = q_rows rounded up to 16 (<= 128); nvalid columns are written.
// transposed_out writes out[col * out_ld + row].
// out = P Q^T on the tensor cores.  P (M x K) is given packed (launch_tc_pack;
// P_lo is the BF16X3 low part), Q (q_rows x K, row stride ldq) row-major
// (FP32 for TF32, BF16 hi/lo for BF16X3); N = q_rows rounded up to 16.
struct TcOperands {
    const void *P, *P_lo, *Q, *Q_lo;
    int64_t M, K, ldq;
    int q_rows, N, nvalid;
    int no_pdl;         // 1: plain launch.  With programmatic dependent launch
                        // the kernel streams P before its predecessor ends,
                        // which is only right when P is constant (packed X).
};
size_t tc_packed_bytes(int64_t M, int64_t K, int precision);
cudaError_t launch_tc_pack(const float *x, int64_t rows, int64_t cols, int64_t ld, bool transposed,
                           int precision, void *out_hi, void *out_lo, cudaStream_t st);
size_t tc_ws_bytes(int64_t M, int64_t K, int N, int precision);
int64_t tc_num_tickets(int64_t M);
bool tc_available();
// Failure-detection hook: the last CTA of a shared tile waits, in its final
// segment, for `extra` partials that never come (see tc_products.cu).
cudaError_t tc_set_fixup_stall(int extra);
cudaError_t launch_tc_product(const TcOperands &o, int precision, bool transposed_out, float *out,
                              int64_t out_ld, void *ws, unsigned int *tickets, int *err_flag,
                              cudaStream_t st);
// The factor operands as the tensor cores see them (TF32: nearest TF32
// value; BF16X3: hi + lo), so that products and Grams use one matrix.
// H_y (rows x cols, row stride ld): q (and hi / lo) in the same layout.
// W_y (rows x cols, row stride ld_in): q in the same layout, plus the
// transposed operand (cols x rows, stride ld_t): qt for TF32, ht / lt for
// BF16X3.
cudaError_t launch_tc_prep_h(const float *H, int64_t rows, int64_t cols, int64_t ld,
                             int precision, float *q, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                             cudaStream_t st);
cudaError_t launch_tc_prep_w(const float *W, int64_t rows, int64_t cols, int64_t ld_in,
                             int precision, float *q, float *qt, __nv_bfloat16 *ht,
                             __nv_bfloat16 *lt, int64_t ld_t, cudaStream_t st);

// Records `msg` as the calling thread's nmf_last_error() and returns s.
nmf_status set_error(nmf_status s, const char *msg);

// Sets *flag to 1 when v[0..count) holds a NaN or an Inf.
cudaError_t launch_nonfinite_scan(const float *v, int64_t count, int *flag, cudaStream_t st);

}  // namespace nmfg
