// decide.cuh -- the restart decision of Algorithm 2 (steps 16-20) and the
// beta schedule of Algorithm 3 (Ang & Gillis, arXiv 1805.06604), taken on
// the device by one thread of the W-sweep kernel's last CTA once e(k) is
// known (Remark 1), so no iteration reads anything back to the host.
#pragma once
#include <math.h>

#include "common.cuh"

namespace nmfg {

// Double-float accumulation (hi + lo in FP32) of sums of x * (a + a_lo), the
// per-row error terms of Remark 1: FP32 error-free steps (rounded
// intrinsics, so nothing is contracted) instead of FP64 arithmetic, whose
// pipe on this GPU is a small fraction of the FP32 one.  Over a row of r
// terms the result is exact to about r 2^-48 relative.
struct DFAcc {
    float h = 0.0f, l = 0.0f;
};
__device__ __forceinline__ void df_add_prod(DFAcc &acc, float x, float a, float a_lo) {
    const float p = __fmul_rn(x, a);
    const float pe = __fmaf_rn(x, a, -p);                      // x a = p + pe exactly
    const float t = __fadd_rn(acc.h, p);
    const float bb = __fsub_rn(t, acc.h);
    const float e = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    acc.l = __fadd_rn(acc.l, __fadd_rn(e, __fmaf_rn(x, a_lo, pe)));
    acc.h = t;
}
__device__ __forceinline__ double df_value(const DFAcc &acc) {
    return (double)acc.h + (double)acc.l;
}

// Algorithm 3 and steps 16-20 of Algorithm 2, run by one thread.
__device__ __forceinline__ void decide_and_update_beta(DevState *s, const DevParams &p, const DevTrace &t,
                                       double cross, double quad, double bnum, double bden) {
    // Remark 1 in residual form: ||X||^2 - <W_n, C> + <W_n, W_n D - C>.
    const double e2 = s->fro2 - cross + quad;
    const double e = sqrt(e2 > 0.0 ? e2 : 0.0);
    const int finite = isfinite(e2) ? 1 : 0;
    if (!finite) s->status = (int)NMF_ENONFINITE;
    const double ref = p.compare_prev ? s->e_prev : s->e_last;
    const long long k = s->k;
    int acc = finite && !(e > ref);                                   // restart only if e(k) > ref
    if (t.forced != nullptr && k < t.forced_len) acc = finite && t.forced[k] != 0;
    if (k < t.cap) {
        t.e[k] = e;
        t.beta[k] = s->beta;
        t.acc[k] = (unsigned char)acc;
        // Sec. 3's line-search step for this W-update (diagnostic only).
        if (t.bstar) t.bstar[k] = bden > 0.0 ? bnum / bden : 0.0;
    }
    s->beta_used = s->beta;
    s->e_k = e;
    s->accepted = acc;
    if (acc) s->e_last = e;
    s->e_prev = e;
    double next;
    if (acc) {
        const double grown = p.gamma * s->beta;
        next = grown < s->beta_bar ? grown : s->beta_bar;
        const double bar = p.gamma_bar * s->beta_bar;
        s->beta_bar = bar < 1.0 ? bar : 1.0;
    } else {
        next = s->beta / p.eta;
        s->beta_bar = s->beta_prev;
    }
    s->beta_prev = s->beta;
    s->beta = next;
    s->k = k + 1;
}

// Sum of p[0..n) in a fixed order by the whole CTA (blockDim.x a multiple
// of 32, <= 1024): thread t adds p[t], p[t + blockDim], ... in order, the
// warps combine by a fixed butterfly, and warp sums are added in warp order.
// Every CTA that calls it on the same data gets the same bits.
__device__ __forceinline__ double cta_sum_fixed(const double *p, int n, double *sh32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (threadIdx.x % 32 == 0) sh32[threadIdx.x / 32] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += sh32[w];
    __syncthreads();
    return s;
}

// The early-stop test at the start of sweep launch l (see SweepStop):
// true when this launch must not sweep.  Uniform across the CTA.  bid: the
// CTA's index in its launch.
__device__ __forceinline__ bool sweep_stopped(const SweepStop &st, double *sh32, int64_t bid) {
    if (st.l <= 0) return false;
    if (*(volatile int *)st.stopped) return true;
    if (st.l < 3) return false;
    const double prev = cta_sum_fixed(st.d2_prev, st.nparts, sh32);
    const double first = cta_sum_fixed(st.d2_first, st.nparts, sh32);
    if (prev <= st.delta2 * first) {
        if (threadIdx.x == 0 && bid == 0) *st.stopped = 1;
        return true;
    }
    return false;
}

// The sum of squared changes of this CTA's items after sweep l, and the
// sweep count.  v is the thread's own partial.
__device__ __forceinline__ void sweep_record(const SweepStop &st, double v, double *sh32,
                                             int64_t bid) {
    if (st.l <= 0) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (threadIdx.x % 32 == 0) sh32[threadIdx.x / 32] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += sh32[w];
        st.d2_out[bid] = s;
        if (bid == 0) *st.used = st.l;
    }
}

}  // namespace nmfg
