// hals_impl.cuh -- A-HALS inner loops (Sec. 1 of Ang & Gillis, arXiv 1805.06604).
//
// H side: for every column j of H independently, `sweeps` cyclic passes of
//   H(k,j) <- max(0, (A(k,j) - sum_{i != k} G(k,i) H(i,j)) / G(k,k)),
// k = 0..r-1, with A = W_y^T X and G = W_y^T W_y.  W side: the same update
// on every row of W with C = X H_y^T and D = H_y H_y^T.
//
// Work decomposition.  One "item" (a column of H or a row of W) belongs to
// T consecutive lanes; lane t stores coordinates j = s*T + t, s < S, so the
// item is padded to RP = S*T coordinates (padding coordinates have a zero
// Gram row and column and never change).  Every update is the dot-product
// form above -- recomputed from the current iterate, so no running gradient
// accumulates rounding across sweeps.  The sum over i != k is split:
//
//   s_k = [a_k - sum_{i not in E_k} G(k,i) x_i]  -  sum_{d=1..D} G(k,k-d) x_{k-d}
//          \_______ P_k: partial dots ________/     \____ chain terms ______/
//
// with E_k = {k-D, ..., k-1, k} (indices mod RP, D = T).  P_k only reads
// coordinates that were final D steps earlier, so each lane computes its
// share of P_k D updates ahead and the T shares are combined by a butterfly
// of shuffles that is off the critical path.  Every lane then evaluates the
// chain terms itself (all but the newest one during the previous update),
// so the new x_k is available in all T lanes without a broadcast; only its
// owner stores it.  A zero G(k,k) leaves x_k unchanged (the paper does not treat
// it; the whole k-th Gram row is then zero, so x_k enters no other update).
//
// Fused epilogues.  H side: H_y = H_n + beta (H_n - H) (projected for
// hp = 3), Algorithm 2 steps 4-9.  W side: per-row FP64 terms of Remark 1,
// <W_n, C> and <W_n^T W_n, D> = sum_i w_i . (D w_i), reduced per CTA; the
// last CTA to finish sums the CTA partials in a fixed order, forms e(k),
// takes the restart decision of steps 16-20 and applies Algorithm 3.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <utility>

#include "common.cuh"
#include "decide.cuh"

namespace nmfg {
namespace {

constexpr int kThreads = 128;                    // largest CTA (launches use 32..128)

// Layout of one item's coordinates in global memory.
//   kColumn: element k of item j at base[k * ld + j]   (columns of H)
//   kRow:    element k of item i at base[i * ld + k]   (rows of W)
enum ItemLayout { kColumn = 0, kRow = 1 };

template <int L>
__device__ __forceinline__ int64_t elem_index(int64_t item, int k, int64_t ld) {
    return L == kColumn ? (int64_t)k * ld + item : item * ld + k;
}

// Shared-memory vector load.  The sweep loop reads the Gram through a base
// pointer offset by (sweep index * hoist_guard), where hoist_guard is a kernel
// argument that is always 0: the compiler cannot prove the loads loop
// invariant, so it does not hoist S*S*T Gram values into registers across
// sweeps, yet it is free to schedule every load early within a sweep.
__device__ __forceinline__ float4 lds4(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-lane share of P_kk: the owner adds a_kk; every lane subtracts
// G(kk, j) x_j over its coordinates j = s*T + t outside E_kk.  With D = T,
// E_kk \ {kk} = {g, ..., g+T-1} (g = kk - T mod RP) holds exactly one
// coordinate of every lane, in slot g/T (lanes t >= g%T) or slot g/T + 1
// (lanes t < g%T); kk itself sits in slot g/T + 1 of lane g%T.  `gv` is the
// lane's slice of Gram row kk (prefetched).  The slot of coordinate g-1,
// written by the update just before, is accumulated last.
template <int T, int S, int KK>
__device__ __forceinline__ float partial_dot(const float (&gv)[S], int t, const float (&x)[S],
                                             const float (&a)[S]) {
    constexpr int RP = S * T;
    constexpr int G0 = (KK - T + RP) % RP;
    constexpr int SA = G0 / T;                 // first candidate slot
    constexpr int SB = (SA + 1) % S;           // second candidate slot
    constexpr int GR = G0 % T;
    constexpr int SL = ((G0 - 1 + RP) % RP) / T;   // slot of the newest coordinate
    float p[4] = {(t == KK % T) ? a[KK / T] : 0.0f, 0.0f, 0.0f, 0.0f};
    auto term = [&](int s) {
        float &acc = p[s & 3];
        if (s == SA) {
            if (t < GR) acc = fmaf(-gv[s], x[s], acc);      // slot SA excluded for t >= GR
        } else if (s == SB) {
            if (t > GR) acc = fmaf(-gv[s], x[s], acc);      // slot SB excluded for t <= GR
        } else {
            acc = fmaf(-gv[s], x[s], acc);
        }
    };
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (s != SL) term(s);
    term(SL);
    return (p[0] + p[1]) + (p[2] + p[3]);
}

// Lane t's slice of Gram row k (S values, 16-byte aligned, SP >= S).
template <int S, int SP>
__device__ __forceinline__ void load_slice(float (&gv)[S], const float *row) {
#pragma unroll
    for (int q = 0; q < (S + 3) / 4; ++q) {
        const float4 v = lds4(row + 4 * q);
        if (4 * q + 0 < S) gv[4 * q + 0] = v.x;
        if (4 * q + 1 < S) gv[4 * q + 1] = v.y;
        if (4 * q + 2 < S) gv[4 * q + 2] = v.z;
        if (4 * q + 3 < S) gv[4 * q + 3] = v.w;
    }
}

template <int T>
__device__ __forceinline__ float group_allreduce(float p) {
#pragma unroll
    for (int o = 1; o < T; o <<= 1) p += __shfl_xor_sync(0xffffffffu, p, o, T);
    return p;
}

template <int T, int S, int LAYOUT>
__device__ __forceinline__ void
hals_body(int64_t items, int r, int64_t ld,
          const float *__restrict__ Aglob,     // right-hand side a (A or C)
          const float *__restrict__ Gglob,     // Gram (G or D), rs x rs
          int rs,
          const float *Xin, float *Xout, int sweeps,     // may alias (one sweep in place)
          int hoist_guard, const HEpilogue &hep, const WEpilogue &wep,
          int64_t bid, int64_t nblk) {     // CTA index and count of the launch (or item)
    constexpr int RP = S * T;                    // padded item length
    constexpr int D = T;                         // lookahead depth
    constexpr int PF = 2;                        // prefetch distance (updates)
    // Per-lane slice stride: 16-byte aligned and an odd number of 16-byte
    // units, so the T slices a warp reads in one phase fall in distinct banks.
    constexpr int SP = 4 * ((S + 3) / 4) + (((S + 3) / 4) % 2 == 0 ? 4 : 0);
    constexpr int ROW = T * SP;                  // one permuted Gram row
    static_assert(S >= 2, "the lookahead needs RP >= 2T");
    extern __shared__ __align__(16) float smem[];
    float *Grow = smem;                          // [RP][T][SP]: Grow[k][t][s] = G(k, s*T+t)
    float *Band = smem + RP * ROW;               // [RP][16]: G(k,k-1..k-D), 1/G(k,k)
    float *Glo = Band + RP * 16;                 // W side with error terms: low part of D
    __shared__ double red_cross[kThreads / 32], red_quad[kThreads / 32];
    __shared__ double red_bnum[kThreads / 32], red_bden[kThreads / 32];
    __shared__ bool am_last;
    __shared__ double sh32[32];
    const bool err_terms = LAYOUT == kRow && wep.partials != nullptr;
    const SweepStop &stop = LAYOUT == kRow ? wep.stop : hep.stop;
    if (sweep_stopped(stop, sh32, bid)) return;          // A-HALS early stop (delta rule)
    // A programmatically dependent successor (the tensor-core X product)
    // may start streaming X now; it waits for this grid before reading H_y.
    asm volatile("griddepcontrol.launch_dependents;");

    for (int idx = threadIdx.x; idx < RP * ROW; idx += blockDim.x) {
        const int k = idx / ROW, rem = idx % ROW;
        const int tt = rem / SP, s = rem % SP;
        const int i = s * T + tt;
        Grow[idx] = (k < r && s < S && i < r) ? Gglob[k * rs + i] : 0.0f;
    }
    if (err_terms) {
        for (int idx = threadIdx.x; idx < RP * ROW; idx += blockDim.x) {
            const int k = idx / ROW, rem = idx % ROW;
            const int tt = rem / SP, s = rem % SP;
            const int i = s * T + tt;
            Glo[idx] = (k < r && s < S && i < r) ? wep.D_lo[k * rs + i] : 0.0f;
        }
    }
    for (int idx = threadIdx.x; idx < RP * 16; idx += blockDim.x) {
        const int k = idx / 16, c = idx % 16;
        float v = 0.0f;
        if (k < r) {
            if (c < D) {
                const int i = (k - 1 - c + RP) % RP;
                v = i < r ? Gglob[k * rs + i] : 0.0f;
            } else if (c == D) {
                const float d = Gglob[k * rs + k];
                v = d > 0.0f ? 1.0f / d : 0.0f;
            }
        }
        Band[idx] = v;
    }
    __syncthreads();

    const int t = threadIdx.x % T;
    const int64_t item = bid * (blockDim.x / T) + threadIdx.x / T;
    const bool valid = item < items;
    const unsigned gmask = 0xffffffffu;

    float x[S], a[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int k = s * T + t;
        const bool in = valid && k < r;
        x[s] = in ? Xin[elem_index<LAYOUT>(item, k, ld)] : 0.0f;
        a[s] = in ? Aglob[elem_index<LAYOUT>(item, k, ld)] : 0.0f;
    }

    // Pipeline state.  hist[k % D]: the newest values x_{k-1..k-D}
    // (replicated in the group).  P[k % D]: reduced P_k.  The butterfly that
    // combines the T lane shares of a partial takes one exchange per update,
    // and each shuffle's result is used one update after it was issued.
    // Update k+1's sum without its newest term, c, is formed during update k
    // from values that are already final, so the loop-carried path of an
    // update is one fused multiply-add, one multiply and one max whatever T.
    // Band rows and Gram slices are prefetched PF updates ahead.
    constexpr int NST = (T == 8) ? 3 : (T == 4 ? 2 : 1);   // butterfly stages = log2(T)
    // v[j]: a partial after j exchanges; sh[j]: its partner's value, read by
    // a shuffle issued one update earlier.
    float P[D], hist[D], v[NST], sh[NST];
#pragma unroll
    for (int d = 1; d <= D; ++d) {
        const int j = RP - d;                       // "previous sweep" coordinates
        hist[j % D] = __shfl_sync(gmask, x[j / T], j % T, T);
    }
    // Prologue: complete P_0 .. P_{D-NST-1}; P_{D-j} (j = 1..NST) enters the
    // pipeline as if its raw share had been computed j updates ago.
    [&]<int... J>(std::integer_sequence<int, J...>) {
        (
            [&] {
                constexpr int kk = J;
                float gs[S];
                load_slice<S, SP>(gs, Grow + kk * ROW + t * SP);
                float p = partial_dot<T, S, kk>(gs, t, x, a);
                if constexpr (kk < D - NST) {
                    P[kk % D] = group_allreduce<T>(p);        // complete
                } else {
                    constexpr int j = D - kk;                 // 1..NST
#pragma unroll
                    for (int e = 0; e + 1 < j; ++e) p += __shfl_xor_sync(gmask, p, 1 << e, T);
                    v[j - 1] = p;
                    sh[j - 1] = __shfl_xor_sync(gmask, p, 1 << (j - 1), T);
                }
            }(),
            ...);
    }(std::make_integer_sequence<int, D>{});
    // Band values are read as warp-wide broadcast scalars (one wavefront each).
    // bq[i] and gq[i] hold the band row of update k+i and the Gram slice of
    // the partial computed at update k+i, at the start of update k.
    float bq[PF][D + 1], gq[PF][S];
#pragma unroll
    for (int i = 0; i < PF; ++i) {
#pragma unroll
        for (int d = 0; d <= D; ++d) bq[i][d] = Band[(i % RP) * 16 + d];
        load_slice<S, SP>(gq[i], Grow + ((D + i) % RP) * ROW + t * SP);
    }
    float c = P[0];                                 // update 0 without its newest term
#pragma unroll
    for (int d = D; d >= 2; --d) c = fmaf(-bq[0][d - 1], hist[(RP - d) % D], c);

#pragma unroll 1
    for (int l = 0; l < sweeps; ++l) {
        const float *Gl = Grow + l * hoist_guard;   // == Grow (see lds4)
        const float *Bl = Band + l * hoist_guard;
        // One sweep: RP updates, fully unrolled via a compile-time index.
        [&]<int... K>(std::integer_sequence<int, K...>) {
            (
                [&] {
                    constexpr int k = K;
                    constexpr int kk = (k + D) % RP;          // partial computed now
                    // The body is ordered so that every long-latency result
                    // (shuffle, shared load) is consumed as late as possible
                    // in the update, or in a later one.
                    // (1) Update k: the newest chain term, scale, clamp.
                    const float s_k = fmaf(-bq[0][0], hist[(k - 1 + RP) % D], c);
                    const float inv = bq[0][D];
                    const float h = fmaxf(s_k * inv, 0.0f);
                    if (t == k % T && inv > 0.0f) x[k / T] = h;
                    hist[k % D] = h;
                    // (2) Butterfly of earlier partials, one exchange per
                    // update: the partial of update k+D-NST completes; the
                    // others take the shuffle issued last update and issue
                    // the next one.
                    P[(k + D - NST) % D] = v[NST - 1] + sh[NST - 1];
#pragma unroll
                    for (int j = NST - 1; j >= 1; --j) {
                        v[j] = v[j - 1] + sh[j - 1];
                        sh[j] = __shfl_xor_sync(gmask, v[j], 1 << j, T);
                    }
                    // (3) Update k+1 without its newest term (x_k is not used).
                    {
                        float cn = P[(k + 1) % D];
#pragma unroll
                        for (int d = D; d >= 2; --d)
                            cn = fmaf(-bq[1][d - 1], hist[(k + 1 - d + RP) % D], cn);
                        c = cn;
                    }
                    // (4) Rotate the prefetch rings and issue the loads of
                    // update k+PF.
                    float gcur[S];
#pragma unroll
                    for (int s2 = 0; s2 < S; ++s2) gcur[s2] = gq[0][s2];
#pragma unroll
                    for (int i = 0; i + 1 < PF; ++i) {
#pragma unroll
                        for (int d = 0; d <= D; ++d) bq[i][d] = bq[i + 1][d];
#pragma unroll
                        for (int s2 = 0; s2 < S; ++s2) gq[i][s2] = gq[i + 1][s2];
                    }
                    {
                        const float *band = Bl + ((k + PF) % RP) * 16;
#pragma unroll
                        for (int d = 0; d <= D; ++d) bq[PF - 1][d] = band[d];
                    }
                    load_slice<S, SP>(gq[PF - 1], Gl + ((kk + PF) % RP) * ROW + t * SP);
                    // (5) Raw share of the partial of update k + D, and the
                    // first exchange (consumed next update).
                    v[0] = partial_dot<T, S, kk>(gcur, t, x, a);
                    sh[0] = __shfl_xor_sync(gmask, v[0], 1, T);
                }(),
                ...);
        }(std::make_integer_sequence<int, RP>{});
    }

    // Keeps the compiler from moving the stores into the sweep loop.
    asm volatile("" ::: "memory");
    double moved = 0.0;                                  // ||change||^2 (delta rule)
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int k = s * T + t;
        if (valid && k < r) {
            const int64_t q = elem_index<LAYOUT>(item, k, ld);
            if (stop.l > 0) {
                const double dx = (double)x[s] - (double)Xin[q];
                moved = fma(dx, dx, moved);
            }
            Xout[q] = x[s];
        }
    }
    sweep_record(stop, moved, sh32, bid);

    if constexpr (LAYOUT == kColumn) {
        // Algorithm 2 steps 4-9: H_y = H_n + beta (H_n - H), projected if hp = 3.
        if (hep.Hw != nullptr) {
            const float beta = (float)hep.state->beta;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int k = s * T + t;
                if (valid && k < r) {
                    const int64_t q = elem_index<LAYOUT>(item, k, ld);
                    float w = fmaf(beta, x[s] - hep.H_acc[q], x[s]);
                    if (hep.hp == 3) w = fmaxf(w, 0.0f);
                    hep.Hw[q] = w;
                }
            }
        }
    }

    if (err_terms) {
        // Remark 1 for this row, in the residual form
        //   ||x - w H||^2 contribution = -<w, c> + <w, R>,  R = D w - c,
        // which equals -2<w, c> + w.(D w) exactly.  Near convergence R is
        // small, so only <w, c> cancels against ||X||^2: it is summed in
        // FP64 from c = C + C_lo, and R is evaluated with error-free
        // products and sums from D + D_lo (both accurate to about 2^-40).
        float hi[S], lo[S], clo[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int k = s * T + t;
            clo[s] = (valid && k < r) ? wep.C_lo[elem_index<LAYOUT>(item, k, ld)] : 0.0f;
            hi[s] = -a[s];
            lo[s] = -clo[s];
        }
#pragma unroll 1
        for (int j = 0; j < RP; ++j) {
            const float wj = __shfl_sync(gmask, x[j / T], j % T, T);
            const float *row_hi = Grow + j * ROW + t * SP;   // D(j, s*T+t) = D(s*T+t, j)
            const float *row_lo = Glo + j * ROW + t * SP;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const float dh = row_hi[s], dl = row_lo[s];
                const float p = dh * wj;
                const float pe = fmaf(dh, wj, -p);
                const float sum = hi[s] + p, bb = sum - hi[s];
                lo[s] += ((hi[s] - (sum - bb)) + (p - bb)) + pe + dl * wj;
                hi[s] = sum;
            }
        }
        DFAcc cacc, qacc;
        if (valid) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                df_add_prod(cacc, x[s], a[s], clo[s]);
                df_add_prod(qacc, x[s], hi[s], lo[s]);
            }
        }
        double cross = df_value(cacc), quad = df_value(qacc);
        // Line-search diagnostic (Sec. 3): with the direction
        // dW = W_n - W (W the accepted iterate), beta* = num / den where
        //   num = <X - W_n H_y, dW H_y> = -<W_n D - C, dW>,
        //   den = ||dW H_y||^2 = sum_i dW_i D dW_i^T.
        double bnum = 0.0, bden = 0.0;
        if (wep.W_prev != nullptr) {
            float dl[S], dd[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int k = s * T + t;
                dl[s] = (valid && k < r) ? x[s] - wep.W_prev[elem_index<LAYOUT>(item, k, ld)]
                                         : 0.0f;
                bnum = fma(-(double)dl[s], (double)hi[s] + (double)lo[s], bnum);
                dd[s] = 0.0f;
            }
#pragma unroll 1
            for (int j = 0; j < RP; ++j) {
                const float dj = __shfl_sync(gmask, dl[j / T], j % T, T);
                const float *row_hi = Grow + j * ROW + t * SP;
#pragma unroll
                for (int s = 0; s < S; ++s) dd[s] = fmaf(row_hi[s], dj, dd[s]);
            }
#pragma unroll
            for (int s = 0; s < S; ++s) bden = fma((double)dl[s], (double)dd[s], bden);
        }
        cross = warp_sum_d(cross);
        quad = warp_sum_d(quad);
        bnum = warp_sum_d(bnum);
        bden = warp_sum_d(bden);
        const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
        if (lane == 0) {
            red_cross[warp] = cross;
            red_quad[warp] = quad;
            red_bnum[warp] = bnum;
            red_bden[warp] = bden;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double c = 0.0, qd = 0.0, bn = 0.0, bd = 0.0;
            for (int w = 0; w < (int)blockDim.x / 32; ++w) {
                c += red_cross[w];
                qd += red_quad[w];
                bn += red_bnum[w];
                bd += red_bden[w];
            }
            wep.partials[bid].cross = c;
            wep.partials[bid].quad = qd;
            wep.partials[bid].bnum = bn;
            wep.partials[bid].bden = bd;
            __threadfence();
            const unsigned int done = atomicAdd(wep.counter, 1u);
            am_last = (done == (unsigned int)(nblk - 1));
        }
        __syncthreads();
        if (am_last) {
            // Fixed-order sum of the CTA partials (deterministic).
            __threadfence();
            double c = 0.0, qd = 0.0, bn = 0.0, bd = 0.0;
            for (int b = threadIdx.x; b < (int)nblk; b += blockDim.x) {
                const volatile ErrPartial *pp = wep.partials + b;
                c += pp->cross;
                qd += pp->quad;
                bn += pp->bnum;
                bd += pp->bden;
            }
            c = warp_sum_d(c);
            qd = warp_sum_d(qd);
            bn = warp_sum_d(bn);
            bd = warp_sum_d(bd);
            if (lane == 0) {
                red_cross[warp] = c;
                red_quad[warp] = qd;
                red_bnum[warp] = bn;
                red_bden[warp] = bd;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double cs = 0.0, qs = 0.0, bns = 0.0, bds = 0.0;
                for (int w = 0; w < (int)blockDim.x / 32; ++w) {
                    cs += red_cross[w];
                    qs += red_quad[w];
                    bns += red_bnum[w];
                    bds += red_bden[w];
                }
                *wep.counter = 0u;
                if (wep.state != nullptr)
                    decide_and_update_beta(wep.state, wep.params, wep.trace, cs, qs, bns, bds);
            }
        }
    }
}

template <int T, int S, int LAYOUT>
__global__ void __launch_bounds__(kThreads, 1)
hals_kernel(int64_t items, int r, int64_t ld, const float *__restrict__ Aglob,
            const float *__restrict__ Gglob, int rs, const float *Xin, float *Xout, int sweeps,
            int hoist_guard, HEpilogue hep, WEpilogue wep) {
    hals_body<T, S, LAYOUT>(items, r, ld, Aglob, Gglob, rs, Xin, Xout, sweeps, hoist_guard, hep,
                            wep, blockIdx.x, gridDim.x);
}
// W side of many problems in one launch (hoist_guard: 0, as above).
template <int T, int S>
__global__ void __launch_bounds__(kThreads, 1)
hals_w_grouped(const HalsWItem *__restrict__ table, const int64_t *__restrict__ begin,
               int nitems, int hoist_guard) {
    int64_t local;
    const HalsWItem &it = table[group_item(begin, nitems, local)];
    const HEpilogue none{};
    hals_body<T, S, kRow>(it.items, it.r, it.ld, it.A, it.G, it.rs, it.Xin, it.Xout, it.sweeps,
                          hoist_guard, none, it.wep, local, it.nblk);
}

}  // namespace

// Launches the sweep kernel for T lanes per item and S slots per lane.
// Instantiated in hals_inst_*.cu so that the variants compile in parallel.
template <int T, int S, int LAYOUT>
cudaError_t hals_launch(int64_t items, int r, int64_t ld, const float *A, const float *G, int rs,
                        const float *Xin, float *Xout, int sweeps, const HEpilogue &hep,
                        const WEpilogue &wep, int cta_threads, cudaStream_t st) {
    constexpr int RP = S * T;
    constexpr int SP = 4 * ((S + 3) / 4) + (((S + 3) / 4) % 2 == 0 ? 4 : 0);
    const size_t smem = sizeof(float) * (size_t)(RP * T * SP * (LAYOUT == 1 ? 2 : 1) + RP * 16);
    auto kern = hals_kernel<T, S, LAYOUT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (cta_threads < 32 || cta_threads > kThreads || cta_threads % 32) return cudaErrorInvalidValue;
    const int64_t per_cta = cta_threads / T;
    const unsigned grid = (unsigned)((items + per_cta - 1) / per_cta);
    if (grid == 0) return cudaSuccess;
    kern<<<grid, cta_threads, smem, st>>>(items, r, ld, A, G, rs, Xin, Xout, sweeps, 0, hep, wep);
    return cudaGetLastError();
}

// A grouped launch of the W side (all items share T, S and the CTA size).
template <int T, int S>
cudaError_t hals_w_launch_grouped(const HalsWItem *items, const int64_t *begin, int nitems,
                                  int64_t ctas, int cta_threads, cudaStream_t st) {
    constexpr int RP = S * T;
    constexpr int SP = 4 * ((S + 3) / 4) + (((S + 3) / 4) % 2 == 0 ? 4 : 0);
    const size_t smem = sizeof(float) * (size_t)(RP * T * SP * 2 + RP * 16);
    auto kern = hals_w_grouped<T, S>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (cta_threads < 32 || cta_threads > kThreads || cta_threads % 32) return cudaErrorInvalidValue;
    if (nitems < 1 || ctas < 1) return cudaSuccess;
    kern<<<(unsigned)ctas, cta_threads, smem, st>>>(items, begin, nitems, 0);
    return cudaGetLastError();
}

}  // namespace nmfg

#define NMF_HALS_INSTANTIATE_ONE(TV, SV, LV)                                                    \
    template cudaError_t nmfg::hals_launch<TV, SV, LV>(                                         \
        int64_t, int, int64_t, const float *, const float *, int, const float *, float *, int,  \
        const nmfg::HEpilogue &, const nmfg::WEpilogue &, int, cudaStream_t);
// The W side (rows of W, item layout kRow): single and grouped launches.
#define NMF_HALS_INSTANTIATE_ROWS(TV, SV)                                                   \
    NMF_HALS_INSTANTIATE_ONE(TV, SV, 1)                                                     \
    template cudaError_t nmfg::hals_w_launch_grouped<TV, SV>(                               \
        const nmfg::HalsWItem *, const int64_t *, int, int64_t, int, cudaStream_t);
