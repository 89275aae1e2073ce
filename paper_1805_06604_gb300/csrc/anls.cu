// anls.cu -- the NNLS subproblems of ANLS solved exactly (Sec. 1 of Ang &
// Gillis, arXiv 1805.06604: "ANLS ... solves the NNLS subproblems exactly",
// with the active-set-like method of Kim & Park), for E-ANLS: Algorithm 2
// with exact block updates.
//
// H side: for every column j of H, min_{x >= 0} 1/2 x^T G x - b^T x with
// G = W_y^T W_y and b = (W_y^T X)(:, j), warm-started at H_y(:, j).  W side:
// every row of W with G = D = H_y H_y^T and b = (X H_y^T)(i, :).
//
// Block principal pivoting, one warp per item.  Free set F (the support of
// the warm start, among coordinates with G_ii > 0), x_F = G_FF^{-1} b_F by a
// Cholesky factorisation of G_FF in the warp's shared memory (packed lower
// triangle, FP32), x = 0 off F, y = G x - b off F.  Infeasible coordinates
// -- x_i < -tol on F, y_i < -tol off F -- all change sides while their
// number keeps falling, with three more full exchanges allowed when it does
// not; after that only the largest infeasible index changes side.  The KKT
// point (x >= 0, y >= 0, x_i y_i = 0) is the unique minimiser when G is
// positive definite.  Coordinates with G_ii = 0 keep their value (the whole
// Gram row is zero).  tol = 1e-6 times the largest |b_i| or G_ii of the
// item: FP32 round-off at a degenerate optimum (the FP64 oracle uses 1e-12);
// a free coordinate counts as infeasible when G_ii x_i < -tol, i.e. in the
// units of y (the oracle tests x_i itself: at 1e-12 the two agree, while in
// FP32 an unscaled test would clamp values up to tol / 1 instead of
// tol / G_ii).
// Negative round-off left on a converged free set is clamped to zero.  An
// item whose free block is not positive definite, or that does not settle
// in 100 (r + 1) exchanges, keeps its last iterate and raises a status.
//
// The fused epilogues are those of the HALS sweeps: H_y = H_n + beta
// (H_n - H) (projected for hp = 3) on the H side; Remark 1's error terms,
// the restart decision and Algorithm 3 on the W side.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "decide.cuh"

namespace nmfg {
namespace {

constexpr int kAnlsWarps = 4;
constexpr int kAnlsThreads = 32 * kAnlsWarps;
constexpr int kSlots = kMaxRank / 32;          // coordinates per lane (r <= 128)
constexpr float kTolRel = 1e-6f;

enum ItemLayout { kColumn = 0, kRow = 1 };

template <int L>
__device__ __forceinline__ int64_t elem_index(int64_t item, int k, int64_t ld) {
    return L == kColumn ? (int64_t)k * ld + item : item * ld + k;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__host__ __device__ __forceinline__ int tri(int a) { return a * (a + 1) / 2; }   // row a of packed L

// Per-warp scratch (floats unless noted): L packed (r (r+1) / 2), z, rhs,
// x, b (r each), F (r ints).
struct WarpScratch {
    float *L, *z, *x, *b, *rr;
    int *F;
};

__host__ __device__ inline int warp_scratch_floats(int r) {
    return (tri(r) + 3) / 4 * 4 + 5 * ((r + 3) / 4 * 4);
}

template <int LAYOUT, bool ERR>
__global__ void __launch_bounds__(kAnlsThreads)
nnls_kernel(int64_t items, int r, int64_t ld,
            const float *__restrict__ Bglob,     // right-hand sides b (A or C)
            const float *__restrict__ Gglob,     // Gram (G or D), rs x rs
            int rs, const float *__restrict__ Xin, float *__restrict__ Xout,
            HEpilogue hep, WEpilogue wep, int *__restrict__ status) {
    asm volatile("griddepcontrol.launch_dependents;");
    extern __shared__ __align__(16) float smem[];
    const int rq = (r + 3) / 4 * 4;
    float *Gs = smem;                                   // r x rq
    float *Glo = Gs + r * rq;                           // W side: low part of D
    float *wbase = Glo + (ERR ? r * rq : 0);
    const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
    for (int e = tid; e < r * rq; e += kAnlsThreads) {
        const int k = e / rq, i = e % rq;
        Gs[e] = i < r ? Gglob[k * rs + i] : 0.0f;
        if (ERR) Glo[e] = i < r ? wep.D_lo[k * rs + i] : 0.0f;
    }
    __syncthreads();
    WarpScratch ws;
    {
        float *p = wbase + warp * warp_scratch_floats(r);
        ws.L = p;
        p += (tri(r) + 3) / 4 * 4;
        ws.z = p;
        p += rq;
        ws.x = p;
        p += rq;
        ws.b = p;
        p += rq;
        ws.rr = p;
        p += rq;
        ws.F = reinterpret_cast<int *>(p);
    }
    const unsigned full = 0xffffffffu;
    const int max_iter = 100 * (r + 1);
    DFAcc cacc, qacc;                      // Remark 1 terms (double-float FP32)
    double bnum = 0.0, bden = 0.0;
    int bad_status = 0;

    for (int64_t item = (int64_t)blockIdx.x * kAnlsWarps + warp; item < items;
         item += (int64_t)gridDim.x * kAnlsWarps) {
        // Lane l holds coordinates l, l + 32, l + 64, l + 96.
        bool act[kSlots], fr[kSlots];
        float scale = 0.0f;
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const int i = lane + 32 * s;
            act[s] = fr[s] = false;
            if (i < r) {
                const int64_t q = elem_index<LAYOUT>(item, i, ld);
                const float bi = Bglob[q], xi = Xin[q], gii = Gs[i * rq + i];
                ws.b[i] = bi;
                ws.x[i] = xi;
                act[s] = gii > 0.0f;
                fr[s] = act[s] && xi > 0.0f;
                scale = fmaxf(scale, fmaxf(fabsf(bi), fabsf(gii)));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) scale = fmaxf(scale, __shfl_xor_sync(full, scale, o));
        const float tol = kTolRel * (scale > 0.0f ? scale : 1.0f);
        __syncwarp();
        int best = r + 1, alpha = 3, it = 0, ok = 0;
        for (;;) {
            // Free list F (ascending) by ballots.
            int nf = 0;
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                const bool in = act[s] && fr[s];
                const unsigned bal = __ballot_sync(full, in);
                if (in) ws.F[nf + __popc(bal & ((1u << lane) - 1u))] = lane + 32 * s;
                nf += __popc(bal);
            }
            __syncwarp();
            // L = G_FF (packed lower), then Cholesky in place.
            for (int e = lane; e < tri(nf); e += 32) {
                int a = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
                while (tri(a + 1) <= e) ++a;
                while (tri(a) > e) --a;
                const int c = e - tri(a);
                ws.L[e] = Gs[ws.F[a] * rq + ws.F[c]];
            }
            __syncwarp();
            // Left-looking: column c from the finished columns before it,
            // the diagonal by a warp sum over row c, the rows below one per
            // lane (a dot product each), so a column is one parallel step.
            bool pd = true;
            for (int c = 0; c < nf; ++c) {
                float part = 0.0f;
                for (int k = lane; k < c; k += 32) {
                    const float v = ws.L[tri(c) + k];
                    part = fmaf(v, v, part);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(full, part, o);
                part = __shfl_sync(full, part, 0);          // one value for the whole warp
                const float d = ws.L[tri(c) + c] - part;
                if (!(d > 0.0f)) {
                    pd = false;
                    break;
                }
                const float lc = sqrtf(d), ilc = 1.0f / lc;
                const float *lrow = ws.L + tri(c);
                for (int i = c + 1 + lane; i < nf; i += 32) {
                    const float *irow = ws.L + tri(i);
                    float sdot = irow[c];
                    for (int k = 0; k < c; ++k) sdot = fmaf(-irow[k], lrow[k], sdot);
                    ws.L[tri(i) + c] = sdot * ilc;
                }
                __syncwarp();
                if (lane == 0) ws.L[tri(c) + c] = lc;
                __syncwarp();
            }
            if (!pd) break;
            // L L^T v = v in place (column-oriented triangular solves).
            auto chol_solve = [&](float *v) {
                for (int c = 0; c < nf; ++c) {
                    const float vc = v[c] / ws.L[tri(c) + c];
                    __syncwarp();
                    if (lane == 0) v[c] = vc;
                    for (int i = c + 1 + lane; i < nf; i += 32) v[i] -= ws.L[tri(i) + c] * vc;
                    __syncwarp();
                }
                for (int c = nf - 1; c >= 0; --c) {
                    const float vc = v[c] / ws.L[tri(c) + c];
                    __syncwarp();
                    if (lane == 0) v[c] = vc;
                    for (int i = lane; i < c; i += 32) v[i] -= ws.L[tri(c) + i] * vc;
                    __syncwarp();
                }
            };
            // x_F = G_FF^{-1} b_F, then one step of iterative refinement
            // with the residual b_F - G_FF x_F (the FP32 factorisation's
            // error grows with |F|; the refined solution's is set by the
            // residual, about kappa u).
            for (int a = lane; a < nf; a += 32) ws.z[a] = ws.b[ws.F[a]];
            __syncwarp();
            chol_solve(ws.z);
            for (int a = lane; a < nf; a += 32) {
                const float *grow = Gs + ws.F[a] * rq;
                float rho = ws.b[ws.F[a]];
                for (int c = 0; c < nf; ++c) rho = fmaf(-grow[ws.F[c]], ws.z[c], rho);
                ws.rr[a] = rho;
            }
            __syncwarp();
            chol_solve(ws.rr);
            for (int a = lane; a < nf; a += 32) ws.z[a] += ws.rr[a];
            __syncwarp();
            // x on F, 0 on the bound set; y = G x - b on the bound set.
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                const int i = lane + 32 * s;
                if (i < r && act[s] && !fr[s]) ws.x[i] = 0.0f;
            }
            for (int a = lane; a < nf; a += 32) ws.x[ws.F[a]] = ws.z[a];
            __syncwarp();
            int nv = 0, last = -1;
            bool bad[kSlots];
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                const int i = lane + 32 * s;
                bad[s] = false;
                if (i < r && act[s]) {
                    if (fr[s]) {
                        // In gradient units, like y: G_ii x_i is the change
                        // of y_i that x_i accounts for.
                        bad[s] = Gs[i * rq + i] * ws.x[i] < -tol;
                    } else {
                        float y = -ws.b[i];
                        for (int a = 0; a < nf; ++a) y = fmaf(Gs[i * rq + ws.F[a]], ws.z[a], y);
                        bad[s] = y < -tol;
                    }
                }
                const unsigned bal = __ballot_sync(full, bad[s]);
                nv += __popc(bal);
                if (bal) last = 32 * s + 31 - __clz(bal);
            }
            if (nv == 0) {
                ok = 1;
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
                // Backup rule: only the largest infeasible index changes side.
#pragma unroll
                for (int s = 0; s < kSlots; ++s)
                    if (lane + 32 * s == last) fr[s] = !fr[s];
                __syncwarp();
                continue;
            }
#pragma unroll
            for (int s = 0; s < kSlots; ++s)
                if (bad[s]) fr[s] = !fr[s];
            __syncwarp();
        }
        if (!ok) bad_status = 1;
        // Clamp the round-off negatives a converged free set may carry.
        float xv[kSlots];
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
            const int i = lane + 32 * s;
            xv[s] = 0.0f;
            if (i < r) {
                float v = ws.x[i];
                if (ok && act[s] && v < 0.0f) v = 0.0f;
                xv[s] = v;
                const int64_t q = elem_index<LAYOUT>(item, i, ld);
                Xout[q] = v;
                if (LAYOUT == kColumn && hep.Hw != nullptr) {
                    // Algorithm 2 steps 4-9: H_y = H_n + beta (H_n - H), projected if hp = 3.
                    const float beta = (float)hep.state->beta;
                    float w = fmaf(beta, v - hep.H_acc[q], v);
                    if (hep.hp == 3) w = fmaxf(w, 0.0f);
                    hep.Hw[q] = w;
                }
            }
        }
        if constexpr (ERR) {
            // Remark 1 for this row in the residual form (as the sweep
            // kernels): -<w, c> + <w, D w - c>, D w - c with error-free
            // products and sums from D + D_lo and C + C_lo.
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                const int i = lane + 32 * s;
                if (i < r) ws.x[i] = xv[s];
            }
            __syncwarp();
            const bool ls = wep.W_prev != nullptr;
            if (ls) {
                for (int i = lane; i < r; i += 32)
                    ws.z[i] = ws.x[i] - wep.W_prev[elem_index<LAYOUT>(item, i, ld)];
                __syncwarp();
            }
#pragma unroll
            for (int s = 0; s < kSlots; ++s) {
                const int k = lane + 32 * s;
                if (k >= r) continue;
                const int64_t q = elem_index<LAYOUT>(item, k, ld);
                const float c = Bglob[q], clo = wep.C_lo[q];
                float hi = -c, lo = -clo, dd = 0.0f;
                for (int i = 0; i < r; ++i) {
                    const float dh = Gs[k * rq + i], dl = Glo[k * rq + i], wv = ws.x[i];
                    const float pp = dh * wv;
                    const float pe = fmaf(dh, wv, -pp);
                    const float sum = hi + pp, bb = sum - hi;
                    lo += ((hi - (sum - bb)) + (pp - bb)) + pe + dl * wv;
                    hi = sum;
                    if (ls) dd = fmaf(dh, ws.z[i], dd);
                }
                df_add_prod(cacc, xv[s], c, clo);
                df_add_prod(qacc, xv[s], hi, lo);
                if (ls) {
                    // Line-search diagnostic of Sec. 3 (see hals_impl.cuh).
                    const float dk = ws.z[k];
                    bnum = fma(-(double)dk, (double)hi + (double)lo, bnum);
                    bden = fma((double)dk, (double)dd, bden);
                }
            }
        }
        __syncwarp();
    }
    if (bad_status && lane == 0) atomicExch(status, 1);

    if constexpr (ERR) {
        __shared__ double red[4][kAnlsWarps];
        __shared__ bool am_last;
        double cross = warp_sum_d(df_value(cacc));
        double quad = warp_sum_d(df_value(qacc));
        bnum = warp_sum_d(bnum);
        bden = warp_sum_d(bden);
        if (lane == 0) {
            red[0][warp] = cross;
            red[1][warp] = quad;
            red[2][warp] = bnum;
            red[3][warp] = bden;
        }
        __syncthreads();
        if (tid == 0) {
            double cs = 0.0, qs = 0.0, bn = 0.0, bd = 0.0;
            for (int w = 0; w < kAnlsWarps; ++w) {
                cs += red[0][w];
                qs += red[1][w];
                bn += red[2][w];
                bd += red[3][w];
            }
            wep.partials[blockIdx.x].cross = cs;
            wep.partials[blockIdx.x].quad = qs;
            wep.partials[blockIdx.x].bnum = bn;
            wep.partials[blockIdx.x].bden = bd;
            __threadfence();
            const unsigned int done = atomicAdd(wep.counter, 1u);
            am_last = (done == gridDim.x - 1);
        }
        __syncthreads();
        if (am_last) {
            __threadfence();
            double c = 0.0, qd = 0.0, bn = 0.0, bd = 0.0;
            for (int b = tid; b < (int)gridDim.x; b += kAnlsThreads) {
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
            __syncthreads();
            if (lane == 0) {
                red[0][warp] = c;
                red[1][warp] = qd;
                red[2][warp] = bn;
                red[3][warp] = bd;
            }
            __syncthreads();
            if (tid == 0) {
                double cs = 0.0, qs = 0.0, bns = 0.0, bds = 0.0;
                for (int w = 0; w < kAnlsWarps; ++w) {
                    cs += red[0][w];
                    qs += red[1][w];
                    bns += red[2][w];
                    bds += red[3][w];
                }
                *wep.counter = 0u;
                if (wep.state != nullptr)
                    decide_and_update_beta(wep.state, wep.params, wep.trace, cs, qs, bns, bds);
            }
        }
    }
}

size_t anls_smem_bytes(int r, bool err) {
    const int rq = (r + 3) / 4 * 4;
    return sizeof(float) * ((size_t)r * rq * (err ? 2 : 1) +
                            (size_t)kAnlsWarps * warp_scratch_floats(r));
}

template <int LAYOUT, bool ERR>
cudaError_t anls_launch(int64_t items, int r, int64_t ld, const float *B, const float *G, int rs,
                        const float *Xin, float *Xout, const HEpilogue &hep, const WEpilogue &wep,
                        int *status, cudaStream_t st) {
    const size_t smem = anls_smem_bytes(r, ERR);
    auto kern = nnls_kernel<LAYOUT, ERR>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)anls_num_ctas(items);
    kern<<<grid, kAnlsThreads, smem, st>>>(items, r, ld, B, G, rs, Xin, Xout, hep, wep, status);
    return cudaGetLastError();
}

}  // namespace

// Grid of the exact solver: one warp per item while that fills at most
// eight CTAs per SM, then a grid-stride loop.
int anls_num_ctas(int64_t items) {
    const int64_t want = (items + kAnlsWarps - 1) / kAnlsWarps;
    const int64_t cap = 8LL * kNumSMs;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

cudaError_t launch_nnls_h(int64_t n, int64_t ldh, int r, int rs, const float *A, const float *G,
                          const float *H_in, float *H_out, const HEpilogue &ep, int *status,
                          cudaStream_t st) {
    WEpilogue none{};
    return anls_launch<kColumn, false>(n, r, ldh, A, G, rs, H_in, H_out, ep, none, status, st);
}

cudaError_t launch_nnls_w(int64_t m, int r, int rs, const float *C, const float *D,
                          const float *W_in, float *W_out, const WEpilogue &ep, int *status,
                          cudaStream_t st) {
    HEpilogue none{};
    if (ep.partials == nullptr) return cudaErrorInvalidValue;
    return anls_launch<kRow, true>(m, r, rs, C, D, rs, W_in, W_out, none, ep, status, st);
}

}  // namespace nmfg
