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
// short chain (D fused multiply-adds, one multiply, one max) itself, so the
// new x_k is available in all T lanes without a broadcast; only its owner
// stores it.  A zero G(k,k) leaves x_k unchanged (the paper does not treat
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

namespace nmfg {
namespace {

constexpr int kThreads = 128;

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

// Algorithm 3 and steps 16-20 of Algorithm 2, run by one thread.
__device__ void decide_and_update_beta(DevState *s, const DevParams &p, const DevTrace &t,
                                       double cross, double quad) {
    const double e2 = s->fro2 - 2.0 * cross + quad;                 // Remark 1
    const double e = sqrt(e2 > 0.0 ? e2 : 0.0);
    const int finite = isfinite(e2) ? 1 : 0;
    if (!finite) s->status = (int)NMF_ENONFINITE;
    const double ref = p.compare_prev ? s->e_prev : s->e_last;
    const int acc = finite && !(e > ref);                             // restart only if e(k) > ref
    const long long k = s->k;
    if (k < t.cap) {
        t.e[k] = e;
        t.beta[k] = s->beta;
        t.acc[k] = (unsigned char)acc;
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

// Per-lane share of P_kk: the owner adds a_kk; every lane subtracts
// G(kk, j) x_j over its coordinates j = s*T + t outside E_kk.  With D = T,
// E_kk \ {kk} = {g, ..., g+T-1} (g = kk - T mod RP) holds exactly one
// coordinate of every lane, in slot g/T (lanes t >= g%T) or slot g/T + 1
// (lanes t < g%T); kk itself sits in slot g/T + 1 of lane g%T.
template <int T, int S, int SP, int KK>
__device__ __forceinline__ float partial_dot(const float *Grow, int t, const float (&x)[S],
                                             const float (&a)[S]) {
    constexpr int RP = S * T;
    constexpr int G0 = (KK - T + RP) % RP;
    constexpr int SA = G0 / T;                 // first candidate slot
    constexpr int SB = (SA + 1) % S;           // second candidate slot
    constexpr int GR = G0 % T;
    const float *row = Grow + KK * (T * SP) + t * SP;
    // Two accumulators halve the dependent FMA chain.
    float p0 = (t == KK % T) ? a[KK / T] : 0.0f, p1 = 0.0f;
#pragma unroll
    for (int q = 0; q < SP / 4; ++q) {
        const float4 v = lds4(row + 4 * q);
        const float gv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int s = 4 * q + u;
            if (s >= S) continue;
            float &p = (s & 1) ? p1 : p0;
            if (s == SA) {
                if (t < GR) p = fmaf(-gv[u], x[s], p);      // slot SA excluded for t >= GR
            } else if (s == SB) {
                if (t > GR) p = fmaf(-gv[u], x[s], p);      // slot SB excluded for t <= GR
            } else {
                p = fmaf(-gv[u], x[s], p);
            }
        }
    }
    return p0 + p1;
}

template <int T>
__device__ __forceinline__ float group_allreduce(float p) {
#pragma unroll
    for (int o = 1; o < T; o <<= 1) p += __shfl_xor_sync(0xffffffffu, p, o, T);
    return p;
}

template <int T, int S, int LAYOUT>
__global__ void __launch_bounds__(kThreads)
hals_kernel(int64_t items, int r, int64_t ld,
            const float *__restrict__ Aglob,     // right-hand side a (A or C)
            const float *__restrict__ Gglob,     // Gram (G or D), rs x rs
            int rs,
            const float *__restrict__ Xin, float *__restrict__ Xout, int sweeps,
            int hoist_guard, HEpilogue hep, WEpilogue wep) {
    constexpr int RP = S * T;                    // padded item length
    constexpr int D = T;                         // lookahead depth
    constexpr int SP = 4 * ((S + 3) / 4);        // per-lane slice, 16-byte aligned
    constexpr int ROW = T * SP;                  // one permuted Gram row
    static_assert(S >= 2, "the lookahead needs RP >= 2T");
    extern __shared__ __align__(16) float smem[];
    float *Grow = smem;                          // [RP][T][SP]: Grow[k][t][s] = G(k, s*T+t)
    float *Band = smem + RP * ROW;               // [RP][8]: G(k,k-1..k-D), 1/G(k,k)
    __shared__ double red_cross[kThreads / 32], red_quad[kThreads / 32];
    __shared__ bool am_last;

    for (int idx = threadIdx.x; idx < RP * ROW; idx += blockDim.x) {
        const int k = idx / ROW, rem = idx % ROW;
        const int tt = rem / SP, s = rem % SP;
        const int i = s * T + tt;
        Grow[idx] = (k < r && s < S && i < r) ? Gglob[k * rs + i] : 0.0f;
    }
    for (int idx = threadIdx.x; idx < RP * 8; idx += blockDim.x) {
        const int k = idx / 8, c = idx % 8;
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
    const int64_t item = (int64_t)blockIdx.x * (kThreads / T) + threadIdx.x / T;
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

    // Pipeline state: P[k % D] = P_k for the next D updates, hist[k % D] =
    // the newest values x_{k-1..k-D} (replicated in the group).
    float P[D], hist[D];
#pragma unroll
    for (int d = 1; d <= D; ++d) {
        const int j = RP - d;                       // "previous sweep" coordinates
        hist[j % D] = __shfl_sync(gmask, x[j / T], j % T, T);
    }
    // Prologue: P_0 .. P_{D-1} from the initial iterate.
#define NMF_PROLOGUE(KK) \
    if (KK < D) P[KK % D] = group_allreduce<T>(partial_dot<T, S, SP, KK % RP>(Grow, t, x, a));
    NMF_PROLOGUE(0) NMF_PROLOGUE(1) NMF_PROLOGUE(2) NMF_PROLOGUE(3)
#undef NMF_PROLOGUE

#pragma unroll 1
    for (int l = 0; l < sweeps; ++l) {
        const float *Gl = Grow + l * hoist_guard;   // == Grow (see lds4)
        const float *Bl = Band + l * hoist_guard;
        // One sweep: RP updates, fully unrolled via a compile-time index.
        [&]<int... K>(std::integer_sequence<int, K...>) {
            (
                [&] {
                    constexpr int k = K;
                    // Chain of update k.
                    const float *band = Bl + k * 8;
                    const float4 b0 = lds4(band);
                    const float4 b1 = lds4(band + 4);
                    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                    float s_k = P[k % D];
#pragma unroll
                    for (int d = D; d >= 1; --d)
                        s_k = fmaf(-bv[d - 1], hist[(k - d + RP) % D], s_k);
                    const float inv = bv[D];
                    const float h = fmaxf(s_k * inv, 0.0f);
                    if (t == k % T && inv > 0.0f) x[k / T] = h;
                    hist[k % D] = h;
                    // Partial dots of update k + D (coordinates final before k).
                    constexpr int kk = (k + D) % RP;
                    P[kk % D] = group_allreduce<T>(partial_dot<T, S, SP, kk>(Gl, t, x, a));
                }(),
                ...);
        }(std::make_integer_sequence<int, RP>{});
    }

    // Keeps the compiler from moving the stores into the sweep loop.
    asm volatile("" ::: "memory");
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int k = s * T + t;
        if (valid && k < r) Xout[elem_index<LAYOUT>(item, k, ld)] = x[s];
    }

    if constexpr (LAYOUT == kColumn) {
        // Algorithm 2 steps 4-9: H_y = H_n + beta (H_n - H), projected if hp = 3.
        if (hep.Hw != nullptr) {
            const float beta = (float)hep.state->beta;
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int k = s * T + t;
                if (valid && k < r) {
                    const int64_t q = elem_index<LAYOUT>(item, k, ld);
                    float v = fmaf(beta, x[s] - hep.H_acc[q], x[s]);
                    if (hep.hp == 3) v = fmaxf(v, 0.0f);
                    hep.Hw[q] = v;
                }
            }
        }
    }

    if (LAYOUT == kRow && wep.partials != nullptr) {
        // Remark 1 terms of this row: <w, c> and w . (D w), D w recomputed
        // from the final w.
        float dw[S];
#pragma unroll
        for (int s = 0; s < S; ++s) dw[s] = 0.0f;
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const float wj = __shfl_sync(gmask, x[j / T], j % T, T);
            const float *row = Grow + j * ROW + t * SP;      // D(j, s*T+t) = D(s*T+t, j)
#pragma unroll
            for (int q = 0; q < SP / 4; ++q) {
                const float4 v = lds4(row + 4 * q);
                const float gv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (4 * q + u < S) dw[4 * q + u] = fmaf(gv[u], wj, dw[4 * q + u]);
            }
        }
        double cross = 0.0, quad = 0.0;
        if (valid) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                cross = fma((double)x[s], (double)a[s], cross);
                quad = fma((double)x[s], (double)dw[s], quad);
            }
        }
        cross = warp_sum_d(cross);
        quad = warp_sum_d(quad);
        const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
        if (lane == 0) {
            red_cross[warp] = cross;
            red_quad[warp] = quad;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double c = 0.0, qd = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) {
                c += red_cross[w];
                qd += red_quad[w];
            }
            wep.partials[blockIdx.x].cross = c;
            wep.partials[blockIdx.x].quad = qd;
            __threadfence();
            const unsigned int done = atomicAdd(wep.counter, 1u);
            am_last = (done == gridDim.x - 1);
        }
        __syncthreads();
        if (am_last) {
            // Fixed-order sum of the CTA partials (deterministic).
            __threadfence();
            double c = 0.0, qd = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
                const volatile ErrPartial *pp = wep.partials + b;
                c += pp->cross;
                qd += pp->quad;
            }
            c = warp_sum_d(c);
            qd = warp_sum_d(qd);
            if (lane == 0) {
                red_cross[warp] = c;
                red_quad[warp] = qd;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double cs = 0.0, qs = 0.0;
                for (int w = 0; w < kThreads / 32; ++w) {
                    cs += red_cross[w];
                    qs += red_quad[w];
                }
                *wep.counter = 0u;
                if (wep.state != nullptr)
                    decide_and_update_beta(wep.state, wep.params, wep.trace, cs, qs);
            }
        }
    }
}

}  // namespace

// Launches the sweep kernel for T lanes per item and S slots per lane.
// Instantiated in hals_inst_*.cu so that the variants compile in parallel.
template <int T, int S, int LAYOUT>
cudaError_t hals_launch(int64_t items, int r, int64_t ld, const float *A, const float *G, int rs,
                        const float *Xin, float *Xout, int sweeps, const HEpilogue &hep,
                        const WEpilogue &wep, cudaStream_t st) {
    constexpr int RP = S * T;
    constexpr int SP = 4 * ((S + 3) / 4);
    const size_t smem = sizeof(float) * (size_t)(RP * T * SP + RP * 8);
    auto kern = hals_kernel<T, S, LAYOUT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t per_cta = kThreads / T;
    const unsigned grid = (unsigned)((items + per_cta - 1) / per_cta);
    if (grid == 0) return cudaSuccess;
    kern<<<grid, kThreads, smem, st>>>(items, r, ld, A, G, rs, Xin, Xout, sweeps, 0, hep, wep);
    return cudaGetLastError();
}

}  // namespace nmfg

#define NMF_HALS_INSTANTIATE(TV, SV)                                                            \
    template cudaError_t nmfg::hals_launch<TV, SV, 0>(int64_t, int, int64_t, const float *,     \
                                                      const float *, int, const float *,        \
                                                      float *, int, const nmfg::HEpilogue &,    \
                                                      const nmfg::WEpilogue &, cudaStream_t);   \
    template cudaError_t nmfg::hals_launch<TV, SV, 1>(int64_t, int, int64_t, const float *,     \
                                                      const float *, int, const float *,        \
                                                      float *, int, const nmfg::HEpilogue &,    \
                                                      const nmfg::WEpilogue &, cudaStream_t);
